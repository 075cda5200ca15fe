// Device kernels of the KKT library (sm_103a, FP64).
//
// On GB300 the FP64 pipe delivers about 1.2 TFLOP/s for the whole GPU, so
// the supernodal factorisation and the triangular solves are bound by DFMA
// issue, not by HBM.  The kernels therefore (i) never spend FP64 work on
// padding beyond the supernode panels, (ii) keep a panel in shared memory
// while it is factorised, and (iii) leave all index arithmetic to the
// integer pipes.
#pragma once
#include <cooperative_groups.h>
#include <cstdint>
#include <cuda_runtime.h>
#include <math_constants.h>

#include "fp64_lean.cuh"
#include "sparse_dot.cuh"

namespace kktgb {

constexpr int kThreads = 256;

// Bounds-check builds (compiled with -DKKT_BOUNDS_CHECK=1): every index read
// from a precomputed map -- assembly slots, supernodes of level and task
// lists, update segments, the target column and relative row of every Schur
// update, the row indices of the solves -- is tested against the extent it
// must lie in before it is used; a failed test records the first error code
// in a device word (read back by kkt_factor / kkt_solve as KKT_ERR_INTERNAL)
// and the access is skipped.  No trap, no assert.  In ordinary builds
// kkt_in() is the constant true and the tests compile away.
#ifndef KKT_BOUNDS_CHECK
#define KKT_BOUNDS_CHECK 0
#endif
enum {
    kBcSlot = 1,       // assembly slot outside the panel storage
    kBcSupernode = 2,  // level / task list entry outside 0 .. ns-1
    kBcSegment = 3,    // update segment target not an ancestor index
    kBcColumn = 4,     // Schur update column outside the target supernode
    kBcRelRow = 5,     // relative row outside the target supernode's rows
    kBcSolveRow = 6    // solve row index outside 0 .. n-1
};
__device__ __forceinline__ bool kkt_in(int* berr, bool ok, int code) {
#if KKT_BOUNDS_CHECK
    if (!ok && berr) atomicCAS(berr, 0, code);
    return ok;
#else
    (void)berr;
    (void)ok;
    (void)code;
    return true;
#endif
}

// Kernels that run inside the graph of one CG iteration take `active`: when
// it points to 0 (CG has converged) they return at once, so iterations
// enqueued after convergence do nothing.  NULL means always active.
#define KKT_RETURN_IF_INACTIVE(active) \
    do {                               \
        if ((active) && *(active) == 0) return; \
    } while (0)
constexpr int kSubtreeThreads = 64;   // CTA size of the small-subtree kernels
constexpr int kChunkRows = 512;   // rows per reduction chunk (one CTA each)

// Supernode plan (device pointers).  Panel of supernode s: column-major,
// rows(s) x cols(s), leading dimension sn_r[s], at Lx + sn_lptr[s].
struct Plan {
    const int* sn_f;          // first column
    const int* sn_c;          // number of columns
    const int* sn_r;          // number of rows (incl. the diagonal block)
    const long long* sn_lptr; // panel offset
    const int* sn_rptr;       // offset of rows(s) in rows
    const int* rows;          // row structures (permuted labels)
    const int* seg_ptr;       // update segments of s: [seg_ptr[s], seg_ptr[s+1])
    const int* seg_t;         // target supernode
    const int* seg_a;         // first below-row (0-based among below rows)
    const int* seg_b;         // one past the last below-row of the segment
    const long long* seg_map; // offset in relmap of positions of below rows a..rb-1
    const int* relmap;        // positions of rows in the target's rows(t)
    const unsigned long long* rmask;   // structural mask of every panel row
    int* berr;                // bounds-check error word (bounds-check builds)
    int ns, n;                // supernodes, columns
    long long panel;          // panel entries
    const int* sn_inst;       // batches: instance of every supernode
    const int* inst_on;       // batches: per-instance switch of the factorisation (NULL: all on)
};

// A batch instance switched off keeps its panels as the assembly leaves them
// and takes no factorisation work (the batched IPM switches off members that
// take no step; their right-hand sides are zero, so their solves give zero
// whatever the panels hold).
__device__ __forceinline__ bool sn_on(const Plan& P, int s) {
    return !P.inst_on || __ldg(P.inst_on + P.sn_inst[s]) != 0;
}

// ------------------------------------------------------------- assembly
// Js = J scaled row-wise by sqrt(D) (D > 0 in both schemes), so that every
// J^T D J product of the assembly is one FMA: D_r J_ra J_rb = Js_a Js_b.
// One thread per row of J (CSR): one square root per row, not per entry.
__global__ void scale_rows_sqrt_kernel(int m, const int* __restrict__ jp,
                                       const double* __restrict__ J, const double* __restrict__ D,
                                       double Dconst, double* __restrict__ Js) {
    const double sc = sqrt(Dconst);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
        const double sr = D ? sqrt(D[r]) : sc;
        for (int q = jp[r]; q < jp[r + 1]; ++q) Js[q] = J[q] * sr;
    }
}

// One thread per stored entry of the lower triangle of P K P^T: sums its
// sources (W entries, diagonal Sigma_x + delta_x, products Js_a Js_b, in that
// order within a slot) and writes the panel slot.  Source encoding: b == -1 -> W[a];
// b == -2 -> sigma[a] + delta_x (dvec[a] when a per-variable vector is
// given); b >= 0 -> Js[a] * Js[b].
template <typename T>
__global__ void assemble_kernel(long long nk, const long long* __restrict__ slot,
                                const long long* __restrict__ sptr,
                                const int2* __restrict__ src, const double* __restrict__ W,
                                const double* __restrict__ Js, const double* __restrict__ sigma,
                                double delta_x, const double* __restrict__ dvec,
                                T* __restrict__ Lx, long long nslot, int* berr) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nk;
         e += (long long)gridDim.x * blockDim.x) {
        // the first source initialises the sum (no FP64 add of a zero; the
        // same values as accumulating from 0)
        const long long q0 = sptr[e], q1 = sptr[e + 1];
        double v = 0.0;
        if (q0 < q1) {
            const int2 s = src[q0];
            if (s.y == -1) v = W[s.x];
            else if (s.y == -2) v = sigma[s.x] + (dvec ? dvec[s.x] : delta_x);
            else v = Js[s.x] * Js[s.y];
        }
        // A slot's sources come grouped (W entries, then the diagonal, then
        // the J products), so three loops, each of one instruction type:
        // lanes of a warp with different sources no longer step through all
        // three branch bodies per source.
        long long q = q0 + 1;
        int2 s = q < q1 ? src[q] : make_int2(0, 0);
        while (q < q1 && s.y == -1) {
            v += W[s.x];
            if (++q < q1) s = src[q];
        }
        if (q < q1 && s.y == -2) {
            v += sigma[s.x] + (dvec ? dvec[s.x] : delta_x);
            if (++q < q1) s = src[q];
        }
        while (q < q1) {   // products (any other source is still summed correctly)
            if (s.y >= 0) v = fma(Js[s.x], Js[s.y], v);
            else if (s.y == -1) v += W[s.x];
            else v += sigma[s.x] + (dvec ? dvec[s.x] : delta_x);
            if (++q < q1) s = src[q];
        }
        const long long sl = slot[e];
        if (kkt_in(berr, sl >= 0 && sl < nslot, kBcSlot)) Lx[sl] = (T)v;
    }
}

// ------------------------------------------------------------- factor
// On GB300 a warp-wide DFMA occupies an SM sub-partition's FP64 pipe for the
// same time whether 1 or 32 lanes are active, and four warps per SM already
// saturate the pipe.  The panel kernels are therefore written densely and
// lane-packed: every FP64 instruction carries 32 useful lanes except at the
// tails of flattened index spaces.  Panels are dense column-major blocks of
// rows(s) x cols(s) (explicit zeros of relaxed supernodes included).

// Integer quotient q = e / len and remainder for small non-negative values
// (e < 2^22), through a float reciprocal with a one-step correction.
__device__ __forceinline__ void fast_divmod(int e, int len, float rcp, int& q, int& rem) {
    q = __float2int_rz(((float)e + 0.5f) * rcp);
    rem = e - q * len;
    if (rem < 0) { --q; rem += len; }
    else if (rem >= len) { ++q; rem -= len; }
}

// The pivot is a column-sequential chain, and on GB300 every FP64
// instruction on it holds the sub-partition's FP64 unit for 64 cycles, so it
// is kept short: range tests on the bit pattern (integer unit), and the
// reciprocal square root from the single-precision estimate y0 (relative
// error below 2^-21, the conversions done on the bit patterns) refined by
// one third-order step of the Householder family: with r = 1 - d y0^2,
// 1/sqrt(d) = y0 (1 - r)^(-1/2) = y0 (1 + r/2 + 3r^2/8 + O(r^3)),
// truncation below 2^-60 -- five FP64 operations.
__device__ __forceinline__ double rsqrt_householder(double d) {
    if (!lean_range(d)) return 1.0 / sqrt(d);
    const double y0 = f64_of(rsqrtf(f32_of(d)));   // conversions on the integer units
    const double t = d * y0;
    const double r = fma(-t, y0, 1.0);
    const double p = fma(0.375, r, 0.5);
    return fma(y0 * r, p, y0);
}

__device__ __forceinline__ double pivot_rsqrt(double d) { return rsqrt_householder(d); }
__device__ __forceinline__ float pivot_rsqrt(float d) { return 1.0f / sqrtf(d); }

constexpr long long kBitsInf = 0x7ff0000000000000LL;

// positive, finite (and nonzero): a usable pivot
__device__ __forceinline__ bool pivot_ok(double d) {
    const long long b = __double_as_longlong(d);
    return b > 0 && b < kBitsInf;
}
__device__ __forceinline__ bool pivot_ok(float d) {
    const int b = __float_as_int(d);
    return b > 0 && b < 0x7f800000;
}

// Where a non-positive pivot is reported: atomic minimum of the failing
// column into word[0], or into word[inst] when col_inst maps every (permuted)
// column to its instance of a block-diagonal batch.
struct FailSink {
    int* word;
    const int* col_inst;
    __device__ __forceinline__ void report(int col) const {
        atomicMin(word + (col_inst ? col_inst[col] : 0), col);
    }
};

// Pivot of column j: failure check and the reciprocal 1/L_jj, stored for the
// solves.  L_jj itself is never read again (the trailing updates use the
// scaled column below it, the solves a unit diagonal and the reciprocals),
// so the diagonal slot is left as it is.
template <typename T>
__device__ __forceinline__ T take_pivot(T* A, int r, int f, int j, FailSink fail,
                                             T* dinv) {
    T d = A[j + (long long)j * r];
    if (!pivot_ok(d)) {
        fail.report(f + j);
        d = 1.0;
    }
    const T inv = pivot_rsqrt(d);
    dinv[f + j] = inv;
    return inv;
}

// Right-looking Cholesky of the first c columns of a panel A (lda = r, rows
// [0, nrows)): for each column j, (1) scale rows j+1.. by 1/L_jj, (2) update
// the trailing rectangle rows [j+1, nrows) x cols [j+1, c) (entries above the
// diagonal are skipped), with the thread that finishes (j+1, j+1) taking the
// next pivot.  Two barriers per column.
template <typename T>
__device__ __forceinline__ void panel_factor(T* A, int f, int c, int r, int nrows, FailSink fail,
                                             T* dinv) {
    __shared__ T s_inv[2];
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) s_inv[0] = take_pivot(A, r, f, 0, fail, dinv);
    __syncthreads();
    for (int j = 0; j < c; ++j) {
        const T inv = s_inv[j & 1];
        T* colj = A + (long long)j * r;
        for (int i = j + 1 + tid; i < nrows; i += nt) colj[i] *= inv;
        __syncthreads();
        const int len = nrows - j - 1, ncol = c - j - 1;
        if (ncol > 0) {
            const float rcp = 1.0f / (float)len;
            const int total = ncol * len;
            for (int e = tid; e < total; e += nt) {
                int q, rem;
                fast_divmod(e, len, rcp, q, rem);
                const int kk = j + 1 + q, ii = j + 1 + rem;
                if (ii < kk) continue;
                T* p = A + ii + (long long)kk * r;
                const T v = fma(-colj[ii], colj[kk], *p);
                if (ii == j + 1 && kk == j + 1) {
                    *p = v;
                    s_inv[(j + 1) & 1] = take_pivot(A, r, f, j + 1, fail, dinv);
                } else {
                    *p = v;
                }
            }
        }
        __syncthreads();
    }
}

// Segment lookup for update column jj (below-row index) of supernode s.
// With bounds checks it also returns false (and records the error) when the
// target or the column it names lies outside the tree; rt = rows of the
// target, for the caller's check of the relative row.
__device__ __forceinline__ bool update_target(const Plan& P, int s, int c, int jj, long long& base,
                                              const int*& rm, int& a, int& rt) {
    const int sp0 = P.seg_ptr[s], sp1 = P.seg_ptr[s + 1];
    int k = sp0;
    while (k < sp1 - 1 && jj >= P.seg_b[k]) ++k;
    const int t = P.seg_t[k];
    if (!kkt_in(P.berr, sp1 > sp0 && t > s && t < P.ns, kBcSegment)) return false;
    a = P.seg_a[k];
    const int row = P.rows[P.sn_rptr[s] + c + jj];
    rt = P.sn_r[t];
    if (!kkt_in(P.berr, row >= P.sn_f[t] && row < P.sn_f[t] + P.sn_c[t], kBcColumn)) return false;
    base = P.sn_lptr[t] + (long long)(row - P.sn_f[t]) * rt;
    rm = P.relmap + P.seg_map[k];
    return true;
}

// SYRK of the rows below the diagonal block, L21 L21^T, over the packed
// lower triangle: thread -> outputs p = p0 + tid, p0 + tid + nt, ... < p1
// with p = ii (ii + 1) / 2 + jj (row by row, jj <= ii), so every lane of a
// warp has an output (8 x 4 tiles leave the lanes above the diagonal idle, a
// third of them when rb is small).  The pair is decoded with an FP32 square
// root and an integer correction; each output is a c-term FMA chain over
// L21 (row i at A21[i], column stride ld), scattered into its ancestor.
template <typename T>
__device__ __forceinline__ void syrk_pairs(const Plan& P, int s, int c, const T* A21, int ld, int p0,
                                           int p1, T* Lx) {
    for (int p = p0 + (int)threadIdx.x; p < p1; p += blockDim.x) {
        int ii = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
        while (ii * (ii + 1) / 2 > p) --ii;
        while ((ii + 1) * (ii + 2) / 2 <= p) ++ii;
        const int jj = p - ii * (ii + 1) / 2;
        const T* ai = A21 + ii;
        const T* aj = A21 + jj;
        T sum = 0.0;
        for (int k = 0; k < c; ++k) sum = fma(ai[(long long)k * ld], aj[(long long)k * ld], sum);
        long long base;
        const int* rm;
        int a, rt;
        if (!update_target(P, s, c, jj, base, rm, a, rt)) continue;
        const int q = rm[ii - a];
        if (kkt_in(P.berr, q >= 0 && q < rt, kBcRelRow)) atomicAdd(Lx + base + q, -sum);
    }
}

template <typename T>
__device__ __forceinline__ void syrk_packed(const Plan& P, int s, int c, int r, const T* A, T* Lx) {
    const int rb = r - c;
    syrk_pairs(P, s, c, A + c, r, 0, rb * (rb + 1) / 2, Lx);
}

// One CTA per supernode (levels with many supernodes): the whole panel in
// shared memory when it fits, dense right-looking factorisation, then the
// SYRK tiles of the rows below the diagonal block.
template <typename T>
__global__ void __launch_bounds__(kThreads)
factor_level_kernel(Plan P, const int* __restrict__ lvl_sn, T* __restrict__ Lx,
                    FailSink fail, long long smem_elems, T* __restrict__ dinv) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int s = lvl_sn[blockIdx.x];
    if (!kkt_in(P.berr, s >= 0 && s < P.ns, kBcSupernode)) return;
    if (!sn_on(P, s)) return;
    const int f = P.sn_f[s], c = P.sn_c[s], r = P.sn_r[s];
    const long long lp = P.sn_lptr[s];
    const int tid = threadIdx.x, nt = blockDim.x;
    const bool in_smem = (long long)r * c <= smem_elems;
    T* A = in_smem ? sm : Lx + lp;
    if (in_smem) {
        const T* g = Lx + lp;
        for (long long e = tid; e < (long long)r * c; e += nt) A[e] = g[e];
        __syncthreads();
    }
    panel_factor(A, f, c, r, r, fail, dinv);
    if (in_smem) {   // written back normalised (Lhat = L diag(dinv)); the SYRK below reads the smem copy
        T* g = Lx + lp;
        for (long long e = tid; e < (long long)r * c; e += nt) g[e] = A[e] * dinv[f + (int)(e / r)];
    }
    if (r > c) syrk_packed(P, s, c, r, A, Lx);
}

// Levels with few supernodes run in three launches spread over many CTAs:
// (1) POTRF of each diagonal block, (2) TRSM of the rows below, one row per
// warp, (3) SYRK tiles, one tile per warp.
// Cholesky of a square c x c block (c <= 64) in shared memory.  The trailing
// update runs over the lower triangle only, through a table of its (row,
// column) pairs ordered by column descending: the pairs still active at step
// j (column > j) are then the first (c-1-j)(c-j)/2 entries, so every lane of
// every FP64 warp instruction has work.
template <typename T>
__device__ __forceinline__ void square_factor(T* A, int f, int c, FailSink fail, T* dinv) {
    __shared__ T s_inv[2];
    __shared__ short2 tab[64 * 63 / 2];
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < c * c; e += nt) {
        const int ii = e % c, kk = e / c;
        if (kk >= 1 && ii >= kk) tab[(c - 1 - kk) * (c - kk) / 2 + (ii - kk)] = make_short2((short)ii, (short)kk);
    }
    if (tid == 0) s_inv[0] = take_pivot(A, c, f, 0, fail, dinv);
    __syncthreads();
    for (int j = 0; j < c; ++j) {
        const T inv = s_inv[j & 1];
        T* colj = A + (long long)j * c;
        for (int i = j + 1 + tid; i < c; i += nt) colj[i] *= inv;
        __syncthreads();
        const int active = (c - 1 - j) * (c - j) / 2;
        for (int e = tid; e < active; e += nt) {
            const short2 pr = tab[e];
            const int ii = pr.x, kk = pr.y;
            T* p = A + ii + kk * c;
            *p = fma(-colj[ii], colj[kk], *p);
            if (ii == j + 1 && kk == j + 1) s_inv[(j + 1) & 1] = take_pivot(A, c, f, j + 1, fail, dinv);
        }
        __syncthreads();
    }
}

// Cholesky of a square c x c block, c <= 64, with look-ahead: warp 0 holds
// the critical path (lanes = rows, two per lane when c > 32): at step j it
// applies column j to column j + 1, takes the pivot (every lane computes the
// same reciprocal square root, so the broadcast costs one shuffle), scales
// and publishes column j + 1, while warps 1-3 apply column j to the columns
// beyond j + 1 (pairs from the column-descending table, active pairs a
// prefix).  One barrier per column; warps 4 and up only join the barriers,
// so no update instruction competes with warp 0 for its sub-partition's FP64
// unit.  Every entry receives the updates of columns 0, 1, ... in order with
// the same FMAs as square_factor, so the result is the same.
template <typename T>
__device__ __forceinline__ void square_factor_lookahead(T* A, int f, int c, FailSink fail, T* dinv) {
    __shared__ short2 tab[64 * 63 / 2];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool two = c > 32;   // a second row per lane of warp 0 (uniform)
    for (int e = tid; e < c * c; e += blockDim.x) {
        const int ii = e % c, kk = e / c;
        if (kk >= 1 && ii >= kk) tab[(c - 1 - kk) * (c - kk) / 2 + (ii - kk)] = make_short2((short)ii, (short)kk);
    }
    if (warp == 0) {   // column 0
        const T a = lane < c ? A[lane] : T(0.0);
        T d = __shfl_sync(0xffffffffu, a, 0);
        if (!pivot_ok(d)) {
            if (lane == 0) fail.report(f);
            d = 1.0;
        }
        const T inv = pivot_rsqrt(d);
        if (lane == 0) dinv[f] = inv;
        if (lane > 0 && lane < c) A[lane] = a * inv;
        if (two && lane + 32 < c) A[lane + 32] *= inv;
    }
    __syncthreads();
    for (int j = 0; j + 1 < c; ++j) {
        const T* colj = A + j * c;
        if (warp == 0) {
            T* col1 = A + (j + 1) * c;
            const T cj1 = colj[j + 1];
            const bool below = lane > j && lane < c;
            T a = below ? col1[lane] : T(0.0);
            a = fma(-(below ? colj[lane] : T(0.0)), cj1, a);
            T a2 = T(0.0);
            if (two) {
                const bool below2 = lane + 32 > j && lane + 32 < c;
                a2 = below2 ? col1[lane + 32] : T(0.0);
                a2 = fma(-(below2 ? colj[lane + 32] : T(0.0)), cj1, a2);
            }
            T d = j + 1 < 32 ? __shfl_sync(0xffffffffu, a, j + 1) : __shfl_sync(0xffffffffu, a2, j + 1 - 32);
            if (!pivot_ok(d)) {
                if (lane == 0) fail.report(f + j + 1);
                d = 1.0;
            }
            const T inv = pivot_rsqrt(d);
            if (lane == 0) dinv[f + j + 1] = inv;
            if (lane > j + 1 && lane < c) col1[lane] = a * inv;
            if (two && lane + 32 > j + 1 && lane + 32 < c) col1[lane + 32] = a2 * inv;
        } else if (warp < 4) {
            const int active = (c - 2 - j) * (c - 1 - j) / 2;
            for (int e = tid - 32; e < active; e += 96) {
                const short2 pr = tab[e];
                T* p = A + pr.x + pr.y * c;
                *p = fma(-colj[pr.x], colj[pr.y], *p);
            }
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
potrf_diag_kernel(Plan P, const int* __restrict__ lvl_sn, T* __restrict__ Lx,
                  FailSink fail, T* __restrict__ dinv) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int s = lvl_sn[blockIdx.x];
    if (!kkt_in(P.berr, s >= 0 && s < P.ns, kBcSupernode)) return;
    if (!sn_on(P, s)) return;
    const int f = P.sn_f[s], c = P.sn_c[s], r = P.sn_r[s];
    T* g = Lx + P.sn_lptr[s];
    for (int e = threadIdx.x; e < c * c; e += blockDim.x) sm[e] = g[(e % c) + (long long)(e / c) * r];
    __syncthreads();
    if (c <= 64) square_factor_lookahead(sm, f, c, fail, dinv);
    else square_factor(sm, f, c, fail, dinv);
    // the unused upper triangle receives the transpose of L11 diag(dinv)
    // (column-scaled by the reciprocal pivots), once, for the TRSM CTAs
    for (int e = threadIdx.x; e < c * c; e += blockDim.x) {
        const int row = e % c, col = e / c;
        if (row > col) sm[col + row * c] = sm[e] * dinv[f + col];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < c * c; e += blockDim.x) g[(e % c) + (long long)(e / c) * r] = sm[e];
}

// Warp substitutions with two values per lane (rows lane and lane + 32 of a
// block of c <= 64 columns).  A warp FP64 instruction costs the same issue
// slot whatever the number of active lanes, so the loops are split where a
// half has no work: columns < 32 update both halves (the upper half only
// when c > 32), columns >= 32 only the upper half; blocks of <= 32 columns
// never touch the upper half.
// Unit lower triangular: z := Lhat11^{-1} z, Lhat11(x, j) = D[x + j * ldd].
template <typename T>
__device__ __forceinline__ void warp_lower_solve(const T* D, int ldd, int c, int lane, T& z0, T& z1) {
    const int c0 = min(c, 32);
    if (c <= 32) {
        for (int j = 0; j < c0; ++j) {
            const T zj = __shfl_sync(0xffffffffu, z0, j);
            if (lane > j && lane < c) z0 = fma(-D[lane + j * ldd], zj, z0);
        }
        return;
    }
    for (int j = 0; j < 32; ++j) {
        const T zj = __shfl_sync(0xffffffffu, z0, j);
        if (lane > j) z0 = fma(-D[lane + j * ldd], zj, z0);
        if (lane + 32 < c) z1 = fma(-D[lane + 32 + j * ldd], zj, z1);
    }
    for (int j = 32; j < c; ++j) {
        const T zj = __shfl_sync(0xffffffffu, z1, j - 32);
        if (lane + 32 > j && lane + 32 < c) z1 = fma(-D[lane + 32 + j * ldd], zj, z1);
    }
}

// Unit upper triangular with the transpose of Lhat11: t := Lhat11^{-T} t,
// Lhat11(j, x) = D[j + x * ldd].
template <typename T>
__device__ __forceinline__ void warp_upper_solve(const T* D, int ldd, int c, int lane, T& t0, T& t1) {
    if (c > 32) {
        for (int j = c - 1; j >= 32; --j) {
            const T wj = __shfl_sync(0xffffffffu, t1, j - 32);
            t0 = fma(-D[j + lane * ldd], wj, t0);
            if (lane + 32 < j) t1 = fma(-D[j + (lane + 32) * ldd], wj, t1);
        }
    }
    for (int j = min(c, 32) - 1; j >= 0; --j) {
        const T wj = __shfl_sync(0xffffffffu, t0, j);
        if (lane < j) t0 = fma(-D[j + lane * ldd], wj, t0);
    }
}

constexpr int kTrsmWarps = 8;   // rows per TRSM CTA (one per warp)

// X L11^T = A21: task = (supernode, first below-row); warp w solves row
// task.y + w with lanes over the columns (two per lane).  The columns of L11
// come pre-scaled by the reciprocal pivots (the diagonal-block kernel leaves
// them transposed in the upper triangle), so a step is one shuffle and one
// FMA: a_l -= a_k (L_lk / L_kk); the final x_k = a_k / L_kk is one multiply.
template <typename T>
__global__ void __launch_bounds__(32 * kTrsmWarps)
trsm_rows_kernel(Plan P, const int2* __restrict__ tasks, T* __restrict__ Lx,
                 const T* __restrict__ dinv) {
    __shared__ T D[64 * 64];
    const int2 task = tasks[blockIdx.x];
    const int s = task.x;
    if (!kkt_in(P.berr, s >= 0 && s < P.ns, kBcSupernode)) return;
    if (!sn_on(P, s)) return;
    const int f = P.sn_f[s], c = P.sn_c[s], r = P.sn_r[s];
    T* g = Lx + P.sn_lptr[s];
    for (int e = threadIdx.x; e < c * c; e += blockDim.x)   // L11(row, col) dinv(col), row > col,
        D[e] = g[e / c + (long long)(e % c) * r];            // stored transposed above the diagonal
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = task.y + warp;
    if (i >= r - c) return;
    T* row = g + c + i;                       // element k at row[k * r]
    T a0 = lane < c ? row[(long long)lane * r] : 0.0;
    T a1 = lane + 32 < c ? row[(long long)(lane + 32) * r] : 0.0;
    warp_lower_solve(D, c, c, lane, a0, a1);   // a := a Lhat11^{-T} in row form
    if (lane < c) row[(long long)lane * r] = a0 * dinv[f + lane];
    if (lane + 32 < c) row[(long long)(lane + 32) * r] = a1 * dinv[f + lane + 32];
}

// SYRK of a split level: task = (supernode, first pair, end pair) of the
// packed lower triangle of L21 L21^T.  The CTA first copies L21 (rows c.. of
// the panel, rb x c) into shared memory with coalesced loads when `stage` is
// set (one memory latency instead of one per FMA pair), then computes one
// output per thread as in the fused kernels.
template <typename T>
__global__ void __launch_bounds__(kThreads)
syrk_stage_kernel(Plan P, const int4* __restrict__ tasks, T* __restrict__ Lx, int stage) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* S = reinterpret_cast<T*>(smem_raw);
    const int4 t = tasks[blockIdx.x];
    const int s = t.x;
    if (!kkt_in(P.berr, s >= 0 && s < P.ns, kBcSupernode)) return;
    if (!sn_on(P, s)) return;
    const int c = P.sn_c[s], r = P.sn_r[s], rb = r - c;
    const T* g = Lx + P.sn_lptr[s];
    if (stage) {
        for (int e = threadIdx.x; e < rb * c; e += blockDim.x) {
            const int i = e % rb, k = e / rb;
            S[e] = g[c + i + (long long)k * r];
        }
        __syncthreads();
        syrk_pairs(P, s, c, (const T*)S, rb, t.y, t.z, Lx);
    } else {
        syrk_pairs(P, s, c, g + c, r, t.y, t.z, Lx);
    }
}

// The small top levels of the tree (a few supernodes each) in one launch per
// level instead of three: a thread-block cluster of kClusterCtas CTAs per
// supernode.  (1) CTA 0 factorises the diagonal block as potrf_diag_kernel;
// (2) after a cluster barrier every warp of the cluster solves rows of L21
// as trsm_rows_kernel; (3) after a second barrier each CTA stages L21 and
// computes its share of the packed SYRK pairs.  Cluster barriers are
// hardware barriers with release / acquire semantics at cluster scope, and
// data written by another CTA of the cluster is read through L2.
constexpr int kClusterCtas = 8;

template <typename T>
__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(kThreads)
narrow_level_cluster_kernel(Plan P, const int* __restrict__ lvl_sn, T* __restrict__ Lx, FailSink fail,
                            T* __restrict__ dinv) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int rank = (int)cluster.block_rank();
    const int s = lvl_sn[blockIdx.x / kClusterCtas];
    if (!kkt_in(P.berr, s >= 0 && s < P.ns, kBcSupernode)) return;   // the whole cluster returns together
    if (!sn_on(P, s)) return;   // switched-off instance: the whole cluster returns together
    const int f = P.sn_f[s], c = P.sn_c[s], r = P.sn_r[s], rb = r - c;
    T* g = Lx + P.sn_lptr[s];
    const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    // (1) diagonal block
    if (rank == 0) {
        for (int e = tid; e < c * c; e += nt) sm[e] = g[(e % c) + (long long)(e / c) * r];
        __syncthreads();
        if (c <= 64) square_factor_lookahead(sm, f, c, fail, dinv);
        else square_factor(sm, f, c, fail, dinv);
        for (int e = tid; e < c * c; e += nt) {   // transpose of L11 diag(dinv) above the diagonal
            const int row = e % c, col = e / c;
            if (row > col) sm[col + row * c] = sm[e] * dinv[f + col];
        }
        __syncthreads();
        for (int e = tid; e < c * c; e += nt) g[(e % c) + (long long)(e / c) * r] = sm[e];
    }
    cluster.sync();
    // (2) rows below the diagonal block
    for (int e = tid; e < c * c; e += nt) sm[e] = __ldcg(g + e / c + (long long)(e % c) * r);
    __syncthreads();
    const T di0 = lane < c ? __ldcg(dinv + f + lane) : T(0.0);
    const T di1 = lane + 32 < c ? __ldcg(dinv + f + lane + 32) : T(0.0);
    for (int i = rank * nw + warp; i < rb; i += kClusterCtas * nw) {
        T* row = g + c + i;
        T a0 = lane < c ? row[(long long)lane * r] : T(0.0);
        T a1 = lane + 32 < c ? row[(long long)(lane + 32) * r] : T(0.0);
        warp_lower_solve(sm, c, c, lane, a0, a1);
        if (lane < c) row[(long long)lane * r] = a0 * di0;
        if (lane + 32 < c) row[(long long)(lane + 32) * r] = a1 * di1;
    }
    cluster.sync();
    // (3) SYRK share of this CTA
    const int np = rb * (rb + 1) / 2;
    const int p0 = (int)((long long)np * rank / kClusterCtas);
    const int p1 = (int)((long long)np * (rank + 1) / kClusterCtas);
    for (int e = tid; e < rb * c; e += nt) sm[e] = __ldcg(g + c + e % rb + (long long)(e / rb) * r);
    __syncthreads();
    syrk_pairs(P, s, c, (const T*)sm, rb, p0, p1, Lx);
}

// After the factorisation: Lhat = L diag(1/l) (unit diagonal; the reciprocal
// pivots stay in dinv).  The triangular solves then substitute without
// divisions: L z = b is Lhat u = b with z = u / l, and L^T w = z is
// Lhat^T w = u / l^2.  One CTA per supernode.
template <typename T>
__global__ void __launch_bounds__(kThreads)
normalize_panels_kernel(Plan P, const int* __restrict__ list, int count, T* __restrict__ Lx,
                        const T* __restrict__ dinv) {
    for (int q = blockIdx.x; q < count; q += gridDim.x) {
        const int s = list[q];
        if (!kkt_in(P.berr, s >= 0 && s < P.ns, kBcSupernode)) continue;
        if (!sn_on(P, s)) continue;
        const int f = P.sn_f[s], c = P.sn_c[s], r = P.sn_r[s];
        T* A = Lx + P.sn_lptr[s];
        for (int e = threadIdx.x; e < r * c; e += blockDim.x) A[e] *= dinv[f + e / r];
    }
}

// ------------------------------------------------------------- solves
// x[rows below] -= Lhat21 u: lanes over 32 consecutive rows (coalesced
// loads), the warps given to a row block split its columns, and their partial
// sums meet in shared memory.  Each thread's column loads are issued in
// batches of eight, so a batch costs one memory latency and the dependent
// FMA chain per thread is c / (warps per row block) long, not c.  A has the
// leading dimension ld: r in global memory, a padded stride when staged.
template <typename T>
__device__ __forceinline__ void scatter_below(const T* __restrict__ A, int c, int r, int ld,
                                              const T* __restrict__ u, const int* __restrict__ rows,
                                              T* __restrict__ x, T (*part)[32], int* berr, int n) {
    const int tid = threadIdx.x, nw = blockDim.x >> 5, warp = tid >> 5, lane = tid & 31;
    const int rb = r - c;
    for (int i0 = 0; i0 < rb; i0 += 32 * nw) {
        const int nrb = min(nw, (rb - i0 + 31) >> 5);   // row blocks in this pass
        const int wpr = nw / nrb;                        // warps per row block
        const int blk = warp % nrb, q = warp / nrb;
        const int i = i0 + 32 * blk + lane;
        T sum = 0.0;
        if (q < wpr && i < rb) {
            const T* a = A + c + i;
            for (int k0 = q; k0 < c; k0 += 8 * wpr) {
                T v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int k = k0 + j * wpr;
                    v[j] = k < c ? a[(long long)k * ld] : T(0.0);
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int k = k0 + j * wpr;
                    if (k < c) sum = fma(v[j], u[k], sum);
                }
            }
        }
        part[warp][lane] = sum;
        __syncthreads();
        if (tid < 32 * nrb && i0 + tid < rb) {
            const int b = tid >> 5;
            T t = part[b][lane];
            for (int qq = 1; qq < wpr; ++qq) t += part[b + qq * nrb][lane];
            const int rw = rows[c + i0 + tid];
            if (kkt_in(berr, rw >= 0 && rw < n, kBcSolveRow)) atomicAdd(x + rw, -t);
        }
        __syncthreads();
    }
}

// Forward substitution L z = b, one CTA per supernode of a level: the
// diagonal block in shared memory, one warp substitutes with shuffles
// (unit diagonal; the reciprocal pivots are applied in the backward pass),
// then all warps form Lhat21 u and scatter it.
template <typename T, bool kDynD>
__global__ void __launch_bounds__(kThreads)
forward_level_kernel(Plan P, const int* __restrict__ lvl_sn, const T* __restrict__ Lx,
                     const T* __restrict__ dinv, T* __restrict__ x,
    const int* __restrict__ active) {
    KKT_RETURN_IF_INACTIVE(active);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T Dst[kDynD ? 1 : 64 * 64];
    T* D = kDynD ? reinterpret_cast<T*>(smem_raw) : Dst;   // c x c
    __shared__ T z[64];
    __shared__ T part[kThreads / 32][32];
    const int s = lvl_sn[blockIdx.x];
    if (!kkt_in(P.berr, s >= 0 && s < P.ns, kBcSupernode)) return;
    const int f = P.sn_f[s], c = P.sn_c[s], r = P.sn_r[s];
    const T* A = Lx + P.sn_lptr[s];
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < c * c; e += nt) D[e] = A[(e % c) + (long long)(e / c) * r];
    __syncthreads();
    if (tid < 32) {
        const int lane = tid;
        T z0 = lane < c ? x[f + lane] : 0.0;
        T z1 = lane + 32 < c ? x[f + lane + 32] : 0.0;
        warp_lower_solve(D, c, c, lane, z0, z1);   // unit lower triangular (normalised factor)
        if (lane < c) { z[lane] = z0; x[f + lane] = z0; }
        if (lane + 32 < c) { z[lane + 32] = z1; x[f + lane + 32] = z1; }
    }
    __syncthreads();
    scatter_below(A, c, r, r, z, P.rows + P.sn_rptr[s], x, part, P.berr, P.n);
}

// Backward substitution L^T w = z, one CTA per supernode of a level
// (levels visited top-down): t_k = z_k - L21(:,k)^T w_below with lanes over
// the columns k and warps over row blocks, then one warp substitutes with
// the diagonal block.
template <typename T, bool kStageXb, bool kDynD>
__global__ void __launch_bounds__(kThreads)
backward_level_kernel(Plan P, const int* __restrict__ lvl_sn, const T* __restrict__ Lx,
                      const T* __restrict__ dinv, T* __restrict__ x, int dsz,
    const int* __restrict__ active) {
    KKT_RETURN_IF_INACTIVE(active);
    __shared__ T part[kThreads / 32][64];
    __shared__ T Dst[kDynD ? 1 : 64 * 64];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* D = kDynD ? reinterpret_cast<T*>(smem_raw) : Dst;   // c x c (dsz = the level's widest c squared)
    T* xb = reinterpret_cast<T*>(smem_raw) + (kDynD ? dsz : 0);   // x of the rows below, when staged
    const int s = lvl_sn[blockIdx.x];
    if (!kkt_in(P.berr, s >= 0 && s < P.ns, kBcSupernode)) return;
    const int f = P.sn_f[s], c = P.sn_c[s], r = P.sn_r[s];
    const T* A = Lx + P.sn_lptr[s];
    const int* rows = P.rows + P.sn_rptr[s];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    const int rb = r - c;
    for (int e = tid; e < c * c; e += nt) D[e] = A[(e % c) + (long long)(e / c) * r];
    if (kStageXb)
        for (int i = tid; i < rb; i += nt) {
            const int rw = rows[c + i];
            xb[i] = kkt_in(P.berr, rw >= 0 && rw < P.n, kBcSolveRow) ? x[rw] : T(0.0);
        }
    __syncthreads();
    // warp w sums rows i = w, w + nw, ... for columns k = lane, lane + 32
    {
        T s0 = 0.0, s1 = 0.0;
        if (c > 32) {
            for (int i = warp; i < rb; i += nw) {
                const int rw = rows[c + i];
                const T xv = kStageXb ? xb[i] : (kkt_in(P.berr, rw >= 0 && rw < P.n, kBcSolveRow) ? x[rw] : T(0.0));
                s0 = fma(A[c + i + (long long)lane * r], xv, s0);
                if (lane + 32 < c) s1 = fma(A[c + i + (long long)(lane + 32) * r], xv, s1);
            }
        } else if (lane < c) {
            for (int i = warp; i < rb; i += nw)
                s0 = fma(A[c + i + (long long)lane * r],
                         kStageXb ? xb[i]
                                  : (kkt_in(P.berr, rows[c + i] >= 0 && rows[c + i] < P.n, kBcSolveRow) ? x[rows[c + i]]
                                                                                                 : T(0.0)),
                         s0);
        }
        part[warp][lane] = s0;
        part[warp][lane + 32] = s1;
    }
    __syncthreads();
    if (tid < 32) {
        // L^T w = z with L = Lhat diag(l): Lhat^T w = z / l = u / l^2
        T t0 = 0.0, t1 = 0.0;
        if (lane < c) {
            t0 = part[0][lane];
            for (int w = 1; w < nw; ++w) t0 += part[w][lane];
            const T di = dinv[f + lane];
            t0 = fma(x[f + lane] * di, di, -t0);
        }
        if (lane + 32 < c) {   // second half only for supernodes wider than a warp
            t1 = part[0][lane + 32];
            for (int w = 1; w < nw; ++w) t1 += part[w][lane + 32];
            const T di = dinv[f + lane + 32];
            t1 = fma(x[f + lane + 32] * di, di, -t1);
        }
        warp_upper_solve(D, c, c, lane, t0, t1);   // unit upper triangular
        if (lane < c) x[f + lane] = t0;
        if (lane + 32 < c) x[f + lane + 32] = t1;
    }
}

// ------------------------------------------------------------- staged levels
// Programmatic dependent launch: a level kernel lets the next one start at
// once (launch_dependents), so the next level's CTAs load what does not
// depend on x (the panel, its row indices, the pivots) while this level
// still runs; grid_dependency_wait then blocks until the previous grid has
// completed and its writes are visible.  Without the launch attribute the
// wait returns at once and the trigger does nothing.
__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Leading dimension of a panel staged in shared memory: odd, so the lanes of
// a column-strided access (lane = column) fall in different banks.
__host__ __device__ __forceinline__ int staged_ld(int r) { return r | 1; }

// Copy the r x c panel A (leading dimension r) to S (leading dimension ld).
template <typename T>
__device__ __forceinline__ void stage_panel(const T* __restrict__ A, int c, int r, int ld, T* __restrict__ S) {
    const int tid = threadIdx.x, nt = blockDim.x, rc = r * c;
    for (int e0 = tid; e0 < rc; e0 += 4 * nt) {
        T v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = e0 + u * nt;
            v[u] = e < rc ? A[e] : T(0.0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = e0 + u * nt;
            if (e < rc) S[(e % r) + (e / r) * ld] = v[u];
        }
    }
}

// Forward substitution of supernode s once its panel is staged in S (leading
// dimension ld) and every contribution to x[f, f + c) has arrived: the warp
// substitution, then Lhat21 u scattered into the rows below.
template <typename T>
__device__ __forceinline__ void forward_staged_supernode(const Plan& P, int s, const T* S, int ld,
                                                         T* __restrict__ x, T* z, T (*part)[32]) {
    const int f = P.sn_f[s], c = P.sn_c[s], r = P.sn_r[s];
    const int tid = threadIdx.x;
    if (tid < 32) {
        const int lane = tid;
        T z0 = lane < c ? __ldcg(x + f + lane) : T(0.0);
        T z1 = lane + 32 < c ? __ldcg(x + f + lane + 32) : T(0.0);
        warp_lower_solve(S, ld, c, lane, z0, z1);   // unit lower triangular (normalised factor)
        if (lane < c) { z[lane] = z0; x[f + lane] = z0; }
        if (lane + 32 < c) { z[lane + 32] = z1; x[f + lane + 32] = z1; }
    }
    __syncthreads();
    scatter_below(S, c, r, ld, z, P.rows + P.sn_rptr[s], x, part, P.berr, P.n);
}

// Forward substitution of one level with the panel staged in shared memory
// before the wait on the previous level; after the wait it costs the warp
// substitution and Lhat21 u.  Same arithmetic as forward_level_kernel.
template <typename T>
__global__ void __launch_bounds__(kThreads)
forward_level_staged_kernel(Plan P, const int* __restrict__ lvl_sn, const T* __restrict__ Lx,
                            T* __restrict__ x, const int* __restrict__ active) {
    pdl_launch_dependents();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* S = reinterpret_cast<T*>(smem_raw);   // panel, leading dimension staged_ld(r)
    __shared__ T z[64];
    __shared__ T part[kThreads / 32][32];
    const int s = lvl_sn[blockIdx.x];
    const bool ok = kkt_in(P.berr, s >= 0 && s < P.ns, kBcSupernode);
    const int c = ok ? P.sn_c[s] : 0, r = ok ? P.sn_r[s] : 0;
    const int ld = staged_ld(r);
    if (ok) stage_panel(Lx + P.sn_lptr[s], c, r, ld, S);
    grid_dependency_wait();
    KKT_RETURN_IF_INACTIVE(active);
    if (!ok) return;
    __syncthreads();
    forward_staged_supernode(P, s, S, ld, x, z, part);
}

// Backward substitution of supernode s, the part that does not depend on x:
// the panel staged in S (leading dimension ld), the row indices below in rix
// (-1 where a bounds check failed) and the first warp's reciprocal pivots.
template <typename T>
__device__ __forceinline__ void backward_stage_supernode(const Plan& P, int s, const T* __restrict__ Lx,
                                                         const T* __restrict__ dinv, T* S, int ld, int* rix,
                                                         T& di0, T& di1) {
    const int f = P.sn_f[s], c = P.sn_c[s], r = P.sn_r[s], rb = r - c;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    stage_panel(Lx + P.sn_lptr[s], c, r, ld, S);
    const int* rows = P.rows + P.sn_rptr[s] + c;
    for (int i = tid; i < rb; i += nt) {
        const int rw = rows[i];
        rix[i] = kkt_in(P.berr, rw >= 0 && rw < P.n, kBcSolveRow) ? rw : -1;
    }
    if (tid < 32) {
        di0 = lane < c ? dinv[f + lane] : T(0.0);
        di1 = lane + 32 < c ? dinv[f + lane + 32] : T(0.0);
    }
}

// Backward substitution of a staged supernode once x of its rows below is
// final (the caller has synchronised the CTA after staging): xb gathers
// those values, t = u / l^2 - L21^T w, then the warp substitution with the
// diagonal block.  Supernodes of <= 32 columns sum L21^T w with a warp
// instruction over 32 / cp rows (lane = row group, column k < cp).
template <typename T>
__device__ __forceinline__ void backward_staged_supernode(const Plan& P, int s, const T* S, int ld, T* xb,
                                                          const int* rix, T di0, T di1, T* __restrict__ x,
                                                          T (*part)[64]) {
    const int f = P.sn_f[s], c = P.sn_c[s], r = P.sn_r[s], rb = r - c;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    for (int i = tid; i < rb; i += nt) xb[i] = rix[i] >= 0 ? __ldcg(x + rix[i]) : T(0.0);
    __syncthreads();
    if (c <= 32) {
        const int cp = c == 1 ? 1 : 1 << (32 - __clz(c - 1));
        const int k = lane & (cp - 1), G = 32 / cp;
        T s0 = 0.0;
        if (k < c)
            for (int i = warp * G + lane / cp; i < rb; i += nw * G) s0 = fma(S[c + i + k * ld], xb[i], s0);
        for (int off = cp; off < 32; off <<= 1) s0 += __shfl_xor_sync(0xffffffffu, s0, off);
        if (lane < cp) part[warp][lane] = s0;
    } else {
        T s0 = 0.0, s1 = 0.0;
        for (int i = warp; i < rb; i += nw) {
            const T xv = xb[i];
            s0 = fma(S[c + i + lane * ld], xv, s0);
            if (lane + 32 < c) s1 = fma(S[c + i + (lane + 32) * ld], xv, s1);
        }
        part[warp][lane] = s0;
        part[warp][lane + 32] = s1;
    }
    __syncthreads();
    if (tid < 32) {
        // L^T w = z with L = Lhat diag(l): Lhat^T w = z / l = u / l^2
        T t0 = 0.0, t1 = 0.0;
        if (lane < c) {
            t0 = part[0][lane];
            for (int w = 1; w < nw; ++w) t0 += part[w][lane];
            t0 = fma(__ldcg(x + f + lane) * di0, di0, -t0);
        }
        if (lane + 32 < c) {
            t1 = part[0][lane + 32];
            for (int w = 1; w < nw; ++w) t1 += part[w][lane + 32];
            t1 = fma(__ldcg(x + f + lane + 32) * di1, di1, -t1);
        }
        warp_upper_solve(S, ld, c, lane, t0, t1);   // unit upper triangular
        if (lane < c) x[f + lane] = t0;
        if (lane + 32 < c) x[f + lane + 32] = t1;
    }
}

// Backward substitution of one level, staged like the forward kernel (the
// panel, the row indices below and the reciprocal pivots before the wait).
// Shared memory: panel (arc elements), then x of the rows below (mrb), then
// their indices (mrb ints).
template <typename T>
__global__ void __launch_bounds__(kThreads)
backward_level_staged_kernel(Plan P, const int* __restrict__ lvl_sn, const T* __restrict__ Lx,
                             const T* __restrict__ dinv, T* __restrict__ x, int arc, int mrb,
                             const int* __restrict__ active) {
    pdl_launch_dependents();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* S = reinterpret_cast<T*>(smem_raw);
    T* xb = S + arc;
    int* rix = reinterpret_cast<int*>(xb + mrb);
    __shared__ T part[kThreads / 32][64];
    const int s = lvl_sn[blockIdx.x];
    const bool ok = kkt_in(P.berr, s >= 0 && s < P.ns, kBcSupernode);
    const int r = ok ? P.sn_r[s] : 0;
    const int ld = staged_ld(r);
    T di0 = 0.0, di1 = 0.0;
    if (ok) backward_stage_supernode(P, s, Lx, dinv, S, ld, rix, di0, di1);
    grid_dependency_wait();
    KKT_RETURN_IF_INACTIVE(active);
    if (!ok) return;
    __syncthreads();
    backward_staged_supernode(P, s, S, ld, xb, rix, di0, di1, x, part);
}

// ------------------------------------------------------------- subtrees
// Small subtrees of the supernodal tree (task = its supernodes in
// postorder) are processed by one CTA each, without per-level launches.
// Values that earlier supernodes of the same task updated through atomics
// are read with ld.global.cg (L2), never from a possibly stale L1 line.
template <typename T>
__global__ void __launch_bounds__(kSubtreeThreads)
factor_subtree_kernel(Plan P, const int* __restrict__ task_ptr, const int* __restrict__ task_sn,
                      T* __restrict__ Lx, FailSink fail, T* __restrict__ dinv) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int q = task_ptr[blockIdx.x]; q < task_ptr[blockIdx.x + 1]; ++q) {
        const int s = task_sn[q];
        if (!kkt_in(P.berr, s >= 0 && s < P.ns, kBcSupernode)) continue;   // uniform over the CTA
        if (!sn_on(P, s)) continue;   // uniform over the CTA
        const int f = P.sn_f[s], c = P.sn_c[s], r = P.sn_r[s];
        T* g = Lx + P.sn_lptr[s];
        for (int e = tid; e < r * c; e += nt) sm[e] = __ldcg(g + e);
        __syncthreads();
        panel_factor(sm, f, c, r, r, fail, dinv);
        // written back normalised (Lhat = L diag(dinv)); the SYRK below reads the smem copy
        for (int e = tid; e < r * c; e += nt) g[e] = sm[e] * dinv[f + e / r];
        if (r > c) syrk_packed(P, s, c, r, sm, Lx);
        __threadfence();
        __syncthreads();
    }
}

// The columns of a subtree task form one range [lo, lo + w) (a subtree is
// contiguous in postorder), and during a triangular solve only the task's
// own supernodes write into it: the task keeps that slice of x in shared
// memory (xs), updates inside the task are plain shared-memory adds in the
// order the supernodes come, and only the rows above the task go to global
// memory (atomics in the forward pass, reads in the backward pass).  No
// device-wide fence between the task's supernodes; the slice is written
// back at the end.  Returns w (0: the task list failed a bounds check).
__device__ __forceinline__ int task_range(const Plan& P, const int* __restrict__ task_sn, int q0, int q1,
                                          int& lo) {
    if (q1 <= q0) return 0;
    const int sa = task_sn[q0], sb = task_sn[q1 - 1];
    if (!kkt_in(P.berr, sa >= 0 && sa < P.ns && sb >= 0 && sb < P.ns, kBcSupernode)) return 0;
    lo = P.sn_f[sa];
    return P.sn_f[sb] + P.sn_c[sb] - lo;
}

// Forward substitution over the supernodes task_sn[q0 .. q1) of one subtree
// task, in postorder (D: shared memory for the c x c diagonal block, xs:
// for the task's slice of x).
template <typename T>
__device__ __forceinline__ void forward_subtree_task(const Plan& P, const int* __restrict__ task_sn, int q0,
                                                     int q1, const T* __restrict__ Lx, T* __restrict__ x, T* D,
                                                     T* z, T* xs) {
    const int tid = threadIdx.x, nt = blockDim.x;
    int lo = 0;
    const int w = task_range(P, task_sn, q0, q1, lo);
    if (w == 0) return;
    for (int e = tid; e < w; e += nt) xs[e] = __ldcg(x + lo + e);
    for (int q = q0; q < q1; ++q) {
        const int s = task_sn[q];
        if (!kkt_in(P.berr, s >= 0 && s < P.ns, kBcSupernode)) continue;   // uniform over the CTA
        const int f = P.sn_f[s], c = P.sn_c[s], r = P.sn_r[s];
        const T* A = Lx + P.sn_lptr[s];
        for (int e = tid; e < c * c; e += nt) D[e] = A[(e % c) + (long long)(e / c) * r];
        __syncthreads();
        if (tid < 32) {
            const int lane = tid;
            T* xf = xs + (f - lo);
            T z0 = lane < c ? xf[lane] : T(0.0);
            T z1 = lane + 32 < c ? xf[lane + 32] : T(0.0);
            warp_lower_solve(D, c, c, lane, z0, z1);   // unit lower triangular (normalised factor)
            if (lane < c) { z[lane] = z0; xf[lane] = z0; }
            if (lane + 32 < c) { z[lane + 32] = z1; xf[lane + 32] = z1; }
        }
        __syncthreads();
        const int* rows = P.rows + P.sn_rptr[s];
        for (int i = tid; i < r - c; i += nt) {
            T sum = 0.0;
            for (int k = 0; k < c; ++k) sum = fma(A[c + i + (long long)k * r], z[k], sum);
            const int rw = rows[c + i];
            if (rw >= lo && rw < lo + w)
                xs[rw - lo] -= sum;   // rows of one supernode are distinct: no two threads meet
            else if (kkt_in(P.berr, rw >= 0 && rw < P.n, kBcSolveRow))
                atomicAdd(x + rw, -sum);
        }
        __syncthreads();
    }
    for (int e = tid; e < w; e += nt) x[lo + e] = xs[e];
}

// Forward substitution over a subtree task (supernodes in postorder).
// Shared memory: the widest diagonal block (dsz elements), then the slice.
template <typename T>
__global__ void __launch_bounds__(kSubtreeThreads)
forward_subtree_kernel(Plan P, const int* __restrict__ task_ptr, const int* __restrict__ task_sn,
                       const T* __restrict__ Lx, const T* __restrict__ dinv,
                       T* __restrict__ x, int dsz,
    const int* __restrict__ active) {
    pdl_launch_dependents();   // the first staged level may stage its panels during the last wave
    KKT_RETURN_IF_INACTIVE(active);
    __shared__ T z[64];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* D = reinterpret_cast<T*>(smem_raw);   // diagonal block of the current supernode
    forward_subtree_task(P, task_sn, task_ptr[blockIdx.x], task_ptr[blockIdx.x + 1], Lx, x, D, z, D + dsz);
}

// Backward substitution over the supernodes task_sn[q0 .. q1) of one subtree
// task, in reverse postorder (dyn: shared memory for the diagonal block and
// x of the rows below; xs: the task's slice of x; part: one row of 64 per
// warp).
template <typename T>
__device__ __forceinline__ void backward_subtree_task(const Plan& P, const int* __restrict__ task_sn, int q0,
                                                      int q1, const T* __restrict__ Lx,
                                                      const T* __restrict__ dinv, T* __restrict__ x, T* dyn,
                                                      T (*part)[64], T* xs) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    int lo = 0;
    const int w = task_range(P, task_sn, q0, q1, lo);
    if (w == 0) return;
    for (int e = tid; e < w; e += nt) xs[e] = __ldcg(x + lo + e);
    for (int q = q1 - 1; q >= q0; --q) {
        const int s = task_sn[q];
        if (!kkt_in(P.berr, s >= 0 && s < P.ns, kBcSupernode)) continue;   // uniform over the CTA
        const int f = P.sn_f[s], c = P.sn_c[s], r = P.sn_r[s];
        const T* A = Lx + P.sn_lptr[s];
        const int* rows = P.rows + P.sn_rptr[s];
        const int rb = r - c;
        T* D = dyn;
        T* xb = dyn + c * c;
        T* xf = xs + (f - lo);
        for (int e = tid; e < c * c; e += nt) D[e] = A[(e % c) + (long long)(e / c) * r];
        for (int i = tid; i < rb; i += nt) {
            const int rw = rows[c + i];
            xb[i] = rw >= lo && rw < lo + w ? xs[rw - lo]
                    : kkt_in(P.berr, rw >= 0 && rw < P.n, kBcSolveRow) ? __ldcg(x + rw) : T(0.0);
        }
        __syncthreads();
        if (c <= 32) {
            // narrow supernode: a warp instruction covers 32 / cp rows (lane =
            // row group g, column k < cp), so few FP64 issue slots go to idle
            // lanes; the row groups are summed with butterfly shuffles
            const int cp = c == 1 ? 1 : 1 << (32 - __clz(c - 1));
            const int k = lane & (cp - 1), G = 32 / cp;
            T s0 = 0.0;
            if (k < c)
                for (int i = warp * G + lane / cp; i < rb; i += nw * G)
                    s0 = fma(A[c + i + (long long)k * r], xb[i], s0);
            for (int off = cp; off < 32; off <<= 1) s0 += __shfl_xor_sync(0xffffffffu, s0, off);
            if (lane < cp) part[warp][lane] = s0;
            __syncthreads();
            if (tid < 32) {
                T t0 = 0.0, t1 = 0.0;
                if (lane < c) {
                    t0 = part[0][lane];
                    for (int w2 = 1; w2 < nw; ++w2) t0 += part[w2][lane];
                    const T di = dinv[f + lane];
                    t0 = fma(xf[lane] * di, di, -t0);   // u / l^2 - L21^T w
                }
                warp_upper_solve(D, c, c, lane, t0, t1);
                if (lane < c) xf[lane] = t0;
            }
            __syncthreads();
            continue;
        }
        T s0 = 0.0, s1 = 0.0;
        for (int i = warp; i < rb; i += nw) {
            const T xv = xb[i];
            s0 = fma(A[c + i + (long long)lane * r], xv, s0);
            if (lane + 32 < c) s1 = fma(A[c + i + (long long)(lane + 32) * r], xv, s1);
        }
        part[warp][lane] = s0;
        part[warp][lane + 32] = s1;
        __syncthreads();
        if (tid < 32) {
            T t0 = 0.0, t1 = 0.0;
            for (int w2 = 0; w2 < nw; ++w2) { t0 += part[w2][lane]; t1 += part[w2][lane + 32]; }
            // L^T w = z with L = Lhat diag(l): Lhat^T w = z / l = u / l^2
            const T di0 = lane < c ? dinv[f + lane] : 0.0;
            const T di1 = lane + 32 < c ? dinv[f + lane + 32] : 0.0;
            t0 = lane < c ? xf[lane] * di0 * di0 - t0 : 0.0;
            t1 = lane + 32 < c ? xf[lane + 32] * di1 * di1 - t1 : 0.0;
            warp_upper_solve(D, c, c, lane, t0, t1);   // unit upper triangular
            if (lane < c) xf[lane] = t0;
            if (lane + 32 < c) xf[lane + 32] = t1;
        }
        __syncthreads();
    }
    for (int e = tid; e < w; e += nt) x[lo + e] = xs[e];
}

// Backward substitution over a subtree task (supernodes in reverse postorder).
template <typename T>
__global__ void __launch_bounds__(kSubtreeThreads)
backward_subtree_kernel(Plan P, const int* __restrict__ task_ptr, const int* __restrict__ task_sn,
                        const T* __restrict__ Lx, const T* __restrict__ dinv,
                        T* __restrict__ x, int dsz,
    const int* __restrict__ active) {
    KKT_RETURN_IF_INACTIVE(active);
    __shared__ T part[kSubtreeThreads / 32][64];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* dyn = reinterpret_cast<T*>(smem_raw);   // [diagonal block | x of the rows below] (dsz), then the slice
    backward_subtree_task(P, task_sn, task_ptr[blockIdx.x], task_ptr[blockIdx.x + 1], Lx, dinv, x, dyn, part,
                          dyn + dsz);
}

// ------------------------------------------------------------- dataflow solves
// One launch per direction for the whole triangular solve.  The work items
// are the subtree tasks and the supernodes of the levels, listed in a
// topological order of the tree (tasks, then the levels bottom-up).  CTAs
// take items by ticket (an atomic counter): a CTA with ticket i only waits
// for items with smaller tickets, which CTAs already running hold, so every
// wait ends however many CTAs are resident.  A level supernode stages its
// panel before it waits, so the wait overlaps the loads; it then waits on
// one word in L2:
//   forward:  cnt[i] counts the items below it whose contributions to x are
//             in (their atomics fenced before the count), until nchild[i];
//             the waiter re-arms it to zero for the next solve;
//   backward: done[up] holds the epoch of the solve in which its parent
//             finished (x of the parent's columns final); the epoch is the
//             solve count, advanced by the last CTA to leave.
// The waits are bounded (one second by the global timer, and at most
// kFlowSpinLimit polls with backoff): a wait that gives up records 1 in the
// mapped host word herr and goes on, so the kernel always completes and the
// host reports the failure (its x is then invalid).
struct Flow {
    const int* item;     // forward order: >= 0 supernode of the levels, < 0 subtree task -(b + 1)
    const int* up;       // index of the item the item's forward result feeds (its parent), -1: none
    const int* nchild;   // forward: items feeding each item
    int* cnt;            // forward arrival counters (zero between solves)
    unsigned* done;      // backward: epoch at which each level supernode finished
    unsigned* ctrl;      // [0] next ticket, [1] CTAs that left, [2] epoch of the last backward solve
    int* herr;           // mapped host word: a wait gave up
    int first, nitems;   // the items [first, nitems) take part (first > 0: the subtree tasks run
                         // in their own launches, before the forward and after the backward)
    int task_xs_fwd, task_xs_bwd;   // shared-memory offset (elements) of a task's slice of x
};
constexpr int kFlowThreads = 128;
constexpr int kFlowSpinLimit = 1 << 24;
constexpr unsigned long long kFlowWaitNs = 1000000000ull;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const void* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// One thread waits until *p == want (bounded, see above).
__device__ __forceinline__ void flow_wait(const void* p, unsigned want, int* herr) {
    const unsigned long long t0 = global_ns();
    for (int it = 0;; ++it) {
        if (ld_acquire_gpu(p) == want) break;
        if (it >= kFlowSpinLimit || global_ns() - t0 > kFlowWaitNs) {
            *(volatile int*)herr = 1;
            break;
        }
        __nanosleep(it < 64 ? 32 : 256);
    }
    __threadfence();
}

// Ticket of the calling CTA's next item (all threads receive it).
__device__ __forceinline__ int flow_ticket(const Flow& F, int* s_ticket) {
    if (threadIdx.x == 0) *s_ticket = (int)atomicAdd(F.ctrl, 1u);
    __syncthreads();
    return *s_ticket;
}

// The last CTA to leave resets the ticket counters (and publishes the epoch).
__device__ __forceinline__ void flow_leave(const Flow& F, bool backward, unsigned epoch) {
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(F.ctrl + 1, 1u) == gridDim.x - 1) {
            F.ctrl[0] = 0;
            F.ctrl[1] = 0;
            if (backward) F.ctrl[2] = epoch;
        }
    }
}

// L z = b on the permuted vector x.  Dynamic shared memory: the widest staged
// panel (staged_ld(r) x c) or subtree diagonal block.
template <typename T>
__global__ void __launch_bounds__(kFlowThreads)
forward_flow_kernel(Plan P, Flow F, const int* __restrict__ task_ptr, const int* __restrict__ task_sn,
                    const T* __restrict__ Lx, T* __restrict__ x, const int* __restrict__ active) {
    KKT_RETURN_IF_INACTIVE(active);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* S = reinterpret_cast<T*>(smem_raw);
    __shared__ T z[64];
    __shared__ T part[kFlowThreads / 32][32];
    __shared__ int s_ticket;
    const int tid = threadIdx.x;
    while (true) {
        const int i = F.first + flow_ticket(F, &s_ticket);
        if (i >= F.nitems) break;
        const int it = F.item[i];
        if (it < 0) {
            const int b = -it - 1;
            forward_subtree_task(P, task_sn, task_ptr[b], task_ptr[b + 1], Lx, x, S, z, S + F.task_xs_fwd);
        } else if (kkt_in(P.berr, it < P.ns, kBcSupernode)) {
            const int c = P.sn_c[it], r = P.sn_r[it], ld = staged_ld(r);
            stage_panel(Lx + P.sn_lptr[it], c, r, ld, S);
            if (tid == 0 && F.nchild[i] > 0) {
                flow_wait(F.cnt + i, (unsigned)F.nchild[i], F.herr);
                F.cnt[i] = 0;
            }
            __syncthreads();
            forward_staged_supernode(P, it, S, ld, x, z, part);
        }
        __threadfence();
        __syncthreads();
        if (tid == 0 && F.up[i] >= 0) {
            __threadfence();
            atomicAdd(F.cnt + F.up[i], 1);
        }
    }
    flow_leave(F, false, 0u);
}

// L^T w = z in place, items in the reverse order.  Dynamic shared memory:
// the widest staged panel with x and the indices of its rows below, or the
// widest subtree diagonal block with its rows below.
template <typename T>
__global__ void __launch_bounds__(kFlowThreads)
backward_flow_kernel(Plan P, Flow F, const int* __restrict__ task_ptr, const int* __restrict__ task_sn,
                     const T* __restrict__ Lx, const T* __restrict__ dinv, T* __restrict__ x,
                     const int* __restrict__ active) {
    KKT_RETURN_IF_INACTIVE(active);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* S = reinterpret_cast<T*>(smem_raw);
    __shared__ T part[kFlowThreads / 32][64];
    __shared__ int s_ticket;
    const int tid = threadIdx.x;
    const unsigned epoch = *(volatile unsigned*)(F.ctrl + 2) + 1u;
    while (true) {
        const int i = F.nitems - 1 - flow_ticket(F, &s_ticket);
        if (i < F.first) break;
        const int it = F.item[i], up = F.up[i];
        if (it < 0) {
            const int b = -it - 1;
            if (tid == 0 && up >= 0) flow_wait(F.done + up, epoch, F.herr);
            __syncthreads();
            backward_subtree_task(P, task_sn, task_ptr[b], task_ptr[b + 1], Lx, dinv, x, S, part,
                                  S + F.task_xs_bwd);
        } else if (kkt_in(P.berr, it < P.ns, kBcSupernode)) {
            const int c = P.sn_c[it], r = P.sn_r[it], ld = staged_ld(r);
            T* xb = S + (size_t)ld * c;
            int* rix = reinterpret_cast<int*>(xb + (r - c));
            T di0 = 0.0, di1 = 0.0;
            backward_stage_supernode(P, it, Lx, dinv, S, ld, rix, di0, di1);
            if (tid == 0 && up >= 0) flow_wait(F.done + up, epoch, F.herr);
            __syncthreads();
            backward_staged_supernode(P, it, S, ld, xb, rix, di0, di1, x, part);
            __threadfence();
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                st_release_gpu(F.done + i, epoch);
            }
        }
        __syncthreads();
    }
    flow_leave(F, true, epoch);
}

template <typename Tin, typename Tout>
__global__ void gather_kernel(int n, const int* __restrict__ idx, const Tin* __restrict__ in,
                              Tout* __restrict__ out,
    const int* __restrict__ active) {
    KKT_RETURN_IF_INACTIVE(active);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = (Tout)in[idx[i]];
}

template <typename Tin, typename Tout>
__global__ void scatter_kernel(int n, const int* __restrict__ idx, const Tin* __restrict__ in,
                               Tout* __restrict__ out,
    const int* __restrict__ active) {
    KKT_RETURN_IF_INACTIVE(active);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[idx[i]] = (Tout)in[i];
}

// ------------------------------------------------------------- sparse BLAS
// (J^T (Dscale o a_y))_i over the column i of J (Dscale NULL -> Dconst):
// entries in batches -- index loads, then value loads, then the FMAs
__device__ __forceinline__ double jt_row_dot(int i, const int* __restrict__ jt_ptr,
                                             const int* __restrict__ jt_row, const int* __restrict__ jt_idx,
                                             const double* __restrict__ J, const double* __restrict__ ay,
                                             const double* __restrict__ Dscale, double Dconst) {
    double s = 0.0;
    const int q0 = jt_ptr[i], q1 = jt_ptr[i + 1];
    for (int q = q0; q < q1; q += kGatherBatch) {
        int ri[kGatherBatch], ii[kGatherBatch];
#pragma unroll
        for (int u = 0; u < kGatherBatch; ++u) {
            const bool ok = q + u < q1;
            ri[u] = ok ? jt_row[q + u] : 0;
            ii[u] = ok ? jt_idx[q + u] : 0;
        }
        double jv[kGatherBatch], dv[kGatherBatch], yv[kGatherBatch];
#pragma unroll
        for (int u = 0; u < kGatherBatch; ++u) {
            const bool ok = q + u < q1;
            jv[u] = ok ? J[ii[u]] : 0.0;
            dv[u] = ok && Dscale ? Dscale[ri[u]] : Dconst;
            yv[u] = ok ? ay[ri[u]] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kGatherBatch; ++u)
            if (q + u < q1) s = fma(jv[u] * dv[u], yv[u], s);
    }
    return s;
}

// out_x = a_x + alpha * J^T (Dscale o a_y)    (Dscale NULL -> Dconst)
__global__ void jt_axpy_kernel(int n, const int* __restrict__ jt_ptr, const int* __restrict__ jt_row,
                               const int* __restrict__ jt_idx, const double* __restrict__ J,
                               const double* __restrict__ ax, const double* __restrict__ ay,
                               const double* __restrict__ Dscale, double Dconst, double alpha,
                               double* __restrict__ out,
    const int* __restrict__ active) {
    KKT_RETURN_IF_INACTIVE(active);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = (ax ? ax[i] : 0.0) + alpha * jt_row_dot(i, jt_ptr, jt_row, jt_idx, J, ay, Dscale, Dconst);
}

// The CG iteration's J^T p written straight into the permuted vector of the
// solves: xp[i] = (J^T p)_{perm[i]} (the values jt_axpy_kernel and a gather
// would give, without the intermediate vector and the extra launch).
template <typename T>
__global__ void jt_gather_kernel(int n, const int* __restrict__ perm, const int* __restrict__ jt_ptr,
                                 const int* __restrict__ jt_row, const int* __restrict__ jt_idx,
                                 const double* __restrict__ J, const double* __restrict__ p,
                                 T* __restrict__ xp, const int* __restrict__ active) {
    KKT_RETURN_IF_INACTIVE(active);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        xp[i] = (T)(0.0 + 1.0 * jt_row_dot(perm[i], jt_ptr, jt_row, jt_idx, J, p, nullptr, 1.0));
}

// ... and J K^{-1} J^T p read from the permuted solution: out_r = (J x)_r
// with x_v = xp[iperm[v]] (the values a scatter and j_apply_kernel would
// give, in the same order).
template <typename T>
__global__ void j_apply_perm_kernel(int m, const int* __restrict__ j_ptr, const int* __restrict__ j_col,
                                    const double* __restrict__ J, const int* __restrict__ iperm,
                                    const T* __restrict__ xp, double* __restrict__ out,
                                    const int* __restrict__ active) {
    KKT_RETURN_IF_INACTIVE(active);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
        const int q0 = j_ptr[r], q1 = j_ptr[r + 1];
        double s = 0.0;
        for (int q = q0; q < q1; q += kGatherBatch) {
            int ic[kGatherBatch];
            double a[kGatherBatch];
#pragma unroll
            for (int u = 0; u < kGatherBatch; ++u) {
                const bool ok = q + u < q1;
                ic[u] = ok ? iperm[j_col[q + u]] : 0;
                a[u] = ok ? J[q + u] : 0.0;
            }
            double b[kGatherBatch];
#pragma unroll
            for (int u = 0; u < kGatherBatch; ++u) b[u] = q + u < q1 ? (double)xp[ic[u]] : 0.0;
#pragma unroll
            for (int u = 0; u < kGatherBatch; ++u)
                if (q + u < q1) s = fma(a[u], b[u], s);
        }
        out[r] = 1.0 * s;
    }
}

// out_y = Dscale o (J x - b_y)   (Dscale NULL -> Dconst; b_y NULL -> 0)
__global__ void j_apply_kernel(int m, const int* __restrict__ j_ptr, const int* __restrict__ j_col,
                               const double* __restrict__ J, const double* __restrict__ x,
                               const double* __restrict__ by, const double* __restrict__ Dscale,
                               double Dconst, double* __restrict__ out,
    const int* __restrict__ active) {
    KKT_RETURN_IF_INACTIVE(active);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
        double s = gather_dot_direct(j_ptr[r], j_ptr[r + 1], j_col, J, x, 0.0);
        if (by) s -= by[r];
        out[r] = (Dscale ? Dscale[r] : Dconst) * s;
    }
}

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long*>(addr), __double_as_longlong(v));
}

// block maximum of values >= 0, on the bit patterns (integer units)
__device__ __forceinline__ double block_max(double v) {
    __shared__ long long red[kThreads / 32];
    long long b = __double_as_longlong(v);
    for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_down_sync(0xffffffffu, b, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = b;
    __syncthreads();
    if (w == 0) {
        b = lane < (int)(blockDim.x >> 5) ? red[lane] : 0LL;
        for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_down_sync(0xffffffffu, b, o));
    }
    return __longlong_as_double(b);
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// ------------------------------------------------------------- segmented
// Reductions and vector updates run over chunks: contiguous row ranges of one
// instance of a block-diagonal batch (a single system is a batch of one).
// Chunk = {lo, hi, inst, -}; one CTA per chunk, so every reduction result
// belongs to one instance and the order of additions is fixed.
// Rows of the "xy" space are the n primal rows followed by the m dual rows.

// Residual of the original system: r = b - K_orig v, with
//   K_orig = [[W + diag(sigma + delta_x), J^T], [J, -diag(C)]]
// (delta_x per variable when dvec is given) and the max-norms of r, v, b
// accumulated into red[3 inst + 0..2].
__global__ void __launch_bounds__(kThreads)
residual_kernel(const int4* __restrict__ chunks, int n, const int* __restrict__ wf_ptr,
                const int* __restrict__ wf_col, const int* __restrict__ wf_idx,
                const double* __restrict__ W, const int* __restrict__ j_ptr,
                const int* __restrict__ j_col, const int* __restrict__ jt_ptr,
                const int* __restrict__ jt_row, const int* __restrict__ jt_idx,
                const double* __restrict__ J, const double* __restrict__ sigma, double delta_x,
                const double* __restrict__ dvec, const double* __restrict__ C,
                const double* __restrict__ bx, const double* __restrict__ by,
                const double* __restrict__ vx, const double* __restrict__ vy,
                double* __restrict__ rx, double* __restrict__ ry, double* __restrict__ red) {
    const int4 ch = chunks[blockIdx.x];
    double mr = 0.0, mv = 0.0, mb = 0.0;
    for (int i = ch.x + threadIdx.x; i < ch.y; i += blockDim.x) {
        if (i < n) {
            double s = (sigma[i] + (dvec ? dvec[i] : delta_x)) * vx[i];
            s = gather_dot(wf_ptr[i], wf_ptr[i + 1], wf_idx, wf_col, W, vx, s);
            s = gather_dot(jt_ptr[i], jt_ptr[i + 1], jt_idx, jt_row, J, vy, s);
            double r = bx[i] - s;
            rx[i] = r;
            mr = max_abs(mr, r);   // max-norms on the integer units
            mv = max_abs(mv, vx[i]);
            mb = max_abs(mb, bx[i]);
        } else {
            int k = i - n;
            double s = C ? -C[k] * vy[k] : 0.0;
            s = gather_dot_direct(j_ptr[k], j_ptr[k + 1], j_col, J, vx, s);
            double r = by[k] - s;
            ry[k] = r;
            mr = max_abs(mr, r);
            mv = max_abs(mv, vy[k]);
            mb = max_abs(mb, by[k]);
        }
    }
    mr = block_max(mr);
    mv = block_max(mv);
    mb = block_max(mb);
    if (threadIdx.x == 0) {
        atomic_max_nonneg(red + 3 * ch.z + 0, mr);
        atomic_max_nonneg(red + 3 * ch.z + 1, mv);
        atomic_max_nonneg(red + 3 * ch.z + 2, mb);
    }
}

// ||K_orig||_inf (row sums of |K_orig|) per instance into knorm[inst].
__global__ void __launch_bounds__(kThreads)
knorm_kernel(const int4* __restrict__ chunks, int n, const int* __restrict__ wf_ptr,
             const int* __restrict__ wf_col, const int* __restrict__ wf_idx,
             const double* __restrict__ W, const int* __restrict__ j_ptr,
             const int* __restrict__ jt_ptr, const int* __restrict__ jt_idx,
             const double* __restrict__ J, const double* __restrict__ sigma, double delta_x,
             const double* __restrict__ dvec, const double* __restrict__ C,
             double* __restrict__ knorm) {
    const int4 ch = chunks[blockIdx.x];
    double mx = 0.0;
    for (int i = ch.x + threadIdx.x; i < ch.y; i += blockDim.x) {
        double s = 0.0;
        if (i < n) {
            double d = sigma[i] + (dvec ? dvec[i] : delta_x);
            for (int q = wf_ptr[i]; q < wf_ptr[i + 1]; ++q) {
                if (wf_col[q] == i) d += W[wf_idx[q]];
                else s += fabs(W[wf_idx[q]]);
            }
            s += fabs(d);
            for (int q = jt_ptr[i]; q < jt_ptr[i + 1]; ++q) s += fabs(J[jt_idx[q]]);
        } else {
            int k = i - n;
            for (int q = j_ptr[k]; q < j_ptr[k + 1]; ++q) s += fabs(J[q]);
            if (C) s += fabs(C[k]);
        }
        mx = max_nonneg(mx, s);
    }
    mx = block_max(mx);
    if (threadIdx.x == 0) atomic_max_nonneg(knorm + ch.z, mx);
}

// (ux, uy) += (dx, dy) on the rows of instances with act[inst] != 0
__global__ void __launch_bounds__(kThreads)
seg_axpy_kernel(const int4* __restrict__ chunks, int n, const int* __restrict__ act,
                const double* __restrict__ dx, const double* __restrict__ dy,
                double* __restrict__ ux, double* __restrict__ uy) {
    const int4 ch = chunks[blockIdx.x];
    if (!act[ch.z]) return;
    for (int i = ch.x + threadIdx.x; i < ch.y; i += blockDim.x) {
        if (i < n) ux[i] += dx[i];
        else uy[i - n] += dy[i - n];
    }
}

__global__ void recip_kernel(int n, const double* __restrict__ x, double* __restrict__ y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        y[i] = 1.0 / x[i];
}

__global__ void fill_kernel(int n, double v, double* __restrict__ y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = v;
}

// out[i] = val[inst of i]: per-variable delta_x of a batch (x-space chunks)
__global__ void expand_kernel(const int4* __restrict__ chunks, const double* __restrict__ val,
                              double* __restrict__ out) {
    const int4 ch = chunks[blockIdx.x];
    const double v = val[ch.z];
    for (int i = ch.x + threadIdx.x; i < ch.y; i += blockDim.x) out[i] = v;
}

// ---- per-instance CG on S_gamma (HyKKT, Eq. schurcomp), dual-space chunks.
// cgs[4 inst + {0: rr, 1: rr_new, 2: p^T S p, 3: stop}], cgi[2 inst + {0:
// active, 1: iterations}]; any[0] = some instance still active (guards the
// graph-captured iteration), any[1] unused.

// Deterministic dot products: per-chunk partial sums, then per instance the
// partials of its chunks added in chunk order by one warp.
__global__ void __launch_bounds__(kThreads)
seg_dot_partial_kernel(const int4* __restrict__ chunks, const double* __restrict__ a,
                       const double* __restrict__ b, double* __restrict__ part,
                       const int* __restrict__ active) {
    KKT_RETURN_IF_INACTIVE(active);
    const int4 ch = chunks[blockIdx.x];
    double s = 0.0;
    for (int i = ch.x + threadIdx.x; i < ch.y; i += blockDim.x) s += a[i] * b[i];
    s = block_sum(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads)
seg_dot_final_kernel(int nb, const int* __restrict__ inst_chunk_ptr, const double* __restrict__ part,
                     double* __restrict__ cgs, int slot, const int* __restrict__ active) {
    KKT_RETURN_IF_INACTIVE(active);
    const int inst = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (inst >= nb) return;
    double s = 0.0;
    for (int q = inst_chunk_ptr[inst] + lane; q < inst_chunk_ptr[inst + 1]; q += 32) s += part[q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) cgs[4 * inst + slot] = s;
}

// x += alpha p; r -= alpha q  with alpha = rr / pSp of the chunk's instance
__global__ void __launch_bounds__(kThreads)
cg_update_xr_kernel(const int4* __restrict__ chunks, const double* __restrict__ cgs,
                    const int* __restrict__ cgi, const double* __restrict__ p,
                    const double* __restrict__ q, double* __restrict__ x, double* __restrict__ r,
                    const int* __restrict__ active) {
    KKT_RETURN_IF_INACTIVE(active);
    const int4 ch = chunks[blockIdx.x];
    if (!cgi[2 * ch.z]) return;
    const double alpha = cgs[4 * ch.z + 0] / cgs[4 * ch.z + 2];
    for (int i = ch.x + threadIdx.x; i < ch.y; i += blockDim.x) {
        x[i] += alpha * p[i];
        r[i] -= alpha * q[i];
    }
}

// p = r + beta p  with beta = rr_new / rr
__global__ void __launch_bounds__(kThreads)
cg_update_p_kernel(const int4* __restrict__ chunks, const double* __restrict__ cgs,
                   const int* __restrict__ cgi, const double* __restrict__ r, double* __restrict__ p,
                   const int* __restrict__ active) {
    KKT_RETURN_IF_INACTIVE(active);
    const int4 ch = chunks[blockIdx.x];
    if (!cgi[2 * ch.z]) return;
    const double beta = cgs[4 * ch.z + 1] / cgs[4 * ch.z + 0];
    for (int i = ch.x + threadIdx.x; i < ch.y; i += blockDim.x) p[i] = r[i] + beta * p[i];
}

__device__ __forceinline__ int block_or(int v) {
    return __syncthreads_or(v);
}

// Start: stop = tol sqrt(rr0); an instance is active when act[inst] (its
// refinement still runs), sqrt(rr0) > stop and max_cg > 0.  One CTA.
__global__ void __launch_bounds__(kThreads)
cg_init_kernel(int nb, double* __restrict__ cgs, int* __restrict__ cgi, const int* __restrict__ act,
               double tol, int max_cg, int* __restrict__ any) {
    int mine = 0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const double rr = cgs[4 * i + 0];
        const double stop = tol * sqrt(rr);
        cgs[4 * i + 3] = stop;
        const int a = (act[i] && sqrt(rr) > stop && max_cg > 0) ? 1 : 0;
        cgi[2 * i] = a;
        cgi[2 * i + 1] = 0;
        mine |= a;
    }
    mine = block_or(mine);
    if (threadIdx.x == 0) {
        any[0] = mine;
        any[1] = 0;
    }
}

// After each iteration: rr <- rr_new, iterations + 1, active while
// sqrt(rr) > stop and iterations < max_cg.  One CTA.
__global__ void __launch_bounds__(kThreads)
cg_check_kernel(int nb, double* __restrict__ cgs, int* __restrict__ cgi, int max_cg,
                int* __restrict__ any) {
    if (any[0] == 0) return;
    int mine = 0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        if (!cgi[2 * i]) continue;
        const double rr = cgs[4 * i + 1];
        cgs[4 * i + 0] = rr;
        const int it = cgi[2 * i + 1] + 1;
        cgi[2 * i + 1] = it;
        const int a = (sqrt(rr) > cgs[4 * i + 3] && it < max_cg) ? 1 : 0;
        cgi[2 * i] = a;
        mine |= a;
    }
    mine = block_or(mine);
    if (threadIdx.x == 0) any[0] = mine;
}

// ---- the one-graph step (kkt_factor_solve): refinement and CG loops as
// conditional WHILE nodes whose conditions these kernels set.
// Per instance rst[4 i + {0: state, 1: stalled sweeps, 2: sweeps, 3: CG
// iterations}], reta[2 i + {0: eta, 1: previous eta}]; ctl[0] = index of
// the next sweep.
constexpr int kRefineRunning = 1;

// Before the first sweep: instances with a factor run, the others report
// not-SPD (code nspd); the loop runs if any instance does.  One CTA.
__global__ void __launch_bounds__(kThreads)
refine_init_kernel(int nb, const int* __restrict__ fail, int nofail, int nspd, int* __restrict__ act,
                   int* __restrict__ rst, double* __restrict__ reta, int* __restrict__ ctl,
                   cudaGraphConditionalHandle loop) {
    int mine = 0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const int run = fail[i] == nofail ? 1 : 0;
        rst[4 * i + 0] = run ? kRefineRunning : nspd;
        rst[4 * i + 1] = 0;
        rst[4 * i + 2] = 0;
        rst[4 * i + 3] = 0;
        reta[2 * i + 0] = CUDART_INF;
        reta[2 * i + 1] = CUDART_INF;
        act[i] = run;
        mine |= run;
    }
    mine = block_or(mine);
    if (threadIdx.x == 0) {
        ctl[0] = 0;
        cudaGraphSetConditional(loop, mine ? 1u : 0u);
    }
}

// After sweep k = ctl[0]: the backward error of every running instance,
// eta = ||r||_inf / (||K||_inf ||v||_inf + ||b||_inf) from the residual
// maxima red[3 i + {r, v, b}], then the stopping rules (tol: KKT_OK, two
// successive sweeps above 0.9 of the previous eta: code stall); the loop
// continues while an instance runs and k + 1 <= max_refine.  One CTA.
__global__ void __launch_bounds__(kThreads)
refine_update_kernel(int nb, const double* __restrict__ red, const double* __restrict__ knorm, double tol,
                     int max_refine, int ok_code, int stall_code, int* __restrict__ act, int* __restrict__ rst,
                     double* __restrict__ reta, int* __restrict__ ctl, cudaGraphConditionalHandle loop) {
    const int k = ctl[0];
    int mine = 0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        if (rst[4 * i] != kRefineRunning) continue;
        const double rmax = red[3 * i], vmax = red[3 * i + 1], bmax = red[3 * i + 2];
        const double den = knorm[i] * vmax + bmax;
        const double e = den > 0 ? rmax / den : (rmax > 0 ? CUDART_INF : 0.0);
        int state = kRefineRunning;
        rst[4 * i + 2] = k;
        if (e <= tol) {
            state = ok_code;
        } else if (k > 0 && e > 0.9 * reta[2 * i + 1]) {
            if (++rst[4 * i + 1] >= 2) state = stall_code;
        } else {
            rst[4 * i + 1] = 0;
        }
        rst[4 * i] = state;
        reta[2 * i + 1] = e;
        reta[2 * i] = e;
        act[i] = state == kRefineRunning ? 1 : 0;
        mine |= act[i];
    }
    mine = block_or(mine);
    if (threadIdx.x == 0) {
        ctl[0] = k + 1;
        cudaGraphSetConditional(loop, (mine && k + 1 <= max_refine) ? 1u : 0u);
    }
}

// CG loop condition: some instance's CG still runs (flag any[0] of
// cg_init_kernel / cg_check_kernel); count[0] += inc counts the iterations
// the loop ran.
__global__ void cg_cond_kernel(const int* __restrict__ any, cudaGraphConditionalHandle loop,
                               int* __restrict__ count, int inc) {
    if (threadIdx.x == 0) {
        count[0] += inc;
        cudaGraphSetConditional(loop, any[0] ? 1u : 0u);
    }
}

// After an inner HyKKT solve: add every instance's CG iterations.
__global__ void cg_count_kernel(int nb, const int* __restrict__ cgi, int* __restrict__ rst) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x)
        rst[4 * i + 3] += cgi[2 * i + 1];
}

}  // namespace kktgb

// defined before df64.cuh, like the kernels above, so that fma and the
// shuffles of T = double / float resolve to the CUDA built-ins
#include "fused_factor.cuh"
