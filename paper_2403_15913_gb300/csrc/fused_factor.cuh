// Fused factorisation of a tree level whose supernodes have at most 32
// columns and at most 128 rows below the diagonal block (in the tray column
// every level above the subtree tasks: the wide levels of small
// separators and the top levels, one stage's compositions each).
//
// One launch per level instead of three (diagonal block, rows below, Schur
// update), and a pivot chain about half as long.  The numbers are those of
// the Cholesky factor: written as P K P^T = Lhat D Lhat^T with Lhat unit
// lower triangular and D = diag(d_j), L = Lhat D^(1/2), the panel stores Lhat
// and dinv[j] = 1/sqrt(d_j), exactly as the other factor kernels.
//
// Right-looking LDL^T with a one-column look-ahead, on the panel U (rows x
// columns, in shared memory) of unnormalised Schur values:
//   step j:  d_j = U[j][j] is final;  r_j = 1/d_j;
//            Lhat[i][j] = U[i][j] r_j                       (rows i > j)
//            U[i][l] -= U[i][j] Lhat[l][j]    for j < l <= i (the update
//            of L L^T by column j: L[i][j] L[l][j] = U[i][j] U[l][j] r_j).
// Warp 0 carries only the chain from r_j to r_{j+1}: the update of column
// j+1 of the diagonal block, the new pivot d_{j+1} and its reciprocal (an
// FP32 seed and one third-order step), where a Cholesky pivot also needs a
// square root and the scaling of the column.  The other
// warps apply column j to the columns beyond j + 1 (lower triangle of the
// diagonal block, through a table of its pairs ordered by column descending,
// so the active pairs are a prefix) and to the rows below the diagonal
// block; with kReserve the warps that share warp 0's sub-partition stay out
// of the way, so no worker instruction queues in front of the chain on that
// sub-partition's FP64 unit.
//
// After the last column: dinv, the normalised panel, and the Schur update
// of the rows below, Lhat21 U21^T = L21 L21^T over the packed lower
// triangle, scattered into the ancestors with atomics.  Wide levels run one
// CTA per supernode (factor_fused_kernel); levels with fewer supernodes than
// SMs run a thread-block cluster per supernode that splits the rows below
// and the Schur pairs among its CTAs (factor_fused_cluster_kernel).
#pragma once

namespace kktgb {

constexpr int kFusedMaxC = 32;
constexpr int kFusedMaxRb = 128;
constexpr int kFusedThreads = 256;
constexpr int kFusedClusterMax = 8;   // CTAs per supernode (portable cluster size)

template <typename T>
__device__ __forceinline__ T chain_rcp(T d);
template <>
__device__ __forceinline__ double chain_rcp<double>(double d) { return rcp_pos(d); }
template <>
__device__ __forceinline__ float chain_rcp<float>(float d) { return 1.0f / d; }

// named barrier 1: warp 0 arrives when the normalised column is published,
// the worker warps wait for it
__device__ __forceinline__ void bar_arrive(int id, int count) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Schur update over packed pairs p in [p0, p1): A(ii, :) . B(jj, :) with
// A = Lhat21 (column stride lda), B = U21 (column stride ldb), scattered as
// in syrk_pairs.  The c-term sum runs as two interleaved chains (even and
// odd k), halving its dependent FMA latency without idle lanes.
template <typename T>
__device__ __forceinline__ void syrk_pairs_ldl(const Plan& P, int s, int c, const T* A, int lda,
                                               const T* B, int ldb, int p0, int p1, T* Lx) {
    for (int p = p0 + (int)threadIdx.x; p < p1; p += blockDim.x) {
        int ii = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
        while (ii * (ii + 1) / 2 > p) --ii;
        while ((ii + 1) * (ii + 2) / 2 <= p) ++ii;
        const int jj = p - ii * (ii + 1) / 2;
        const T* ai = A + ii;
        const T* bj = B + jj;
        T s0 = 0.0, s1 = 0.0;
        int k = 0;
        for (; k + 1 < c; k += 2) {
            s0 = fma(ai[k * lda], bj[k * ldb], s0);
            s1 = fma(ai[(k + 1) * lda], bj[(k + 1) * ldb], s1);
        }
        if (k < c) s0 = fma(ai[k * lda], bj[k * ldb], s0);
        long long base;
        const int* rm;
        int a, rt;
        if (!update_target(P, s, c, jj, base, rm, a, rt)) continue;
        const int q = rm[ii - a];
        if (kkt_in(P.berr, q >= 0 && q < rt, kBcRelRow)) atomicAdd(Lx + base + q, -(s0 + s1));
    }
}

// The factorisation of one panel (diagonal block + nr rows below, in
// shared memory U, ld = ru) by the chain warp and the worker warps; returns
// with every column final (unnormalised) and rr[] = 1/d_j.
template <typename T, bool kReserve>
__device__ __forceinline__ void fused_panel(T* U, int ru, int c, int nr, int f, FailSink fail, T* rr,
                                            T (*lh)[kFusedMaxC], const short2* tab) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // workers: every warp but 0 (and, with kReserve, but those sharing
    // warp 0's sub-partition); wid / nw = index and count of worker threads
    const bool worker = warp != 0 && !(kReserve && (warp & 3) == 0);
    const int nworkers = kReserve ? (kFusedThreads / 32 - kFusedThreads / 128) : (kFusedThreads / 32 - 1);
    const int wrank = kReserve ? warp - 1 - (warp >> 2) : warp - 1;
    const int wid = wrank * 32 + lane, nw = nworkers * 32;
    // warp 0's registers: cur = column j of the diagonal block (lane = row),
    // rj = 1/d_j, and, prepared a step ahead, b = U[j+1][j], sq = b^2 and
    // pc = cur * b, so that r_{j+1} depends on r_j through four FP64 FMAs:
    // d_{j+1} = U[j+1][j+1] - sq r_j and the three of the reciprocal
    T cur = T(0.0), rj = T(0.0), sq = T(0.0), pc = T(0.0);
    if (warp == 0) {
        cur = lane < c ? U[lane] : T(0.0);
        const T d0 = __shfl_sync(0xffffffffu, cur, 0);
        const bool ok = pivot_ok(d0);
        if (!ok && lane == 0) fail.report(f);
        rj = chain_rcp(ok ? d0 : T(1.0));
        if (lane == 0) rr[0] = rj;
        const T b = __shfl_sync(0xffffffffu, cur, c > 1 ? 1 : 0);
        sq = b * b;
        pc = cur * b;
    }
    __syncthreads();
    const float rcp = nr > 0 ? 1.0f / (float)nr : 0.0f;
    for (int j = 0; j < c; ++j) {
        const T* colj = U + j * ru;
        if (warp == 0) {
            if (j + 1 < c) {
                T* col1 = U + (j + 1) * ru;
                const T a = col1[j + 1];
                const T nxt = lane > j + 1 && lane < c ? col1[lane] : T(0.0);
                const T dd = fma(-sq, rj, a);                 // pivot of column j+1
                const T lhv = cur * rj;                       // Lhat[.][j] for the workers
                if (lane > j && lane < c) lh[j & 1][lane] = lhv;
                bar_arrive(1, 32 + nw);
                const T upd = fma(-pc, rj, nxt);              // column j+1 by column j
                const bool ok = pivot_ok(dd);
                if (!ok && lane == 0) fail.report(f + j + 1);
                const T rn = chain_rcp(ok ? dd : T(1.0));
                __syncwarp();
                if (lane > j + 1 && lane < c) col1[lane] = upd;
                if (lane == 0) {
                    col1[j + 1] = dd;
                    rr[j + 1] = rn;
                }
                const T bn = __shfl_sync(0xffffffffu, upd, j + 2 < c ? j + 2 : 0);
                sq = bn * bn;
                pc = upd * bn;
                cur = upd;
                rj = rn;
            } else {
                if (lane > j && lane < c) lh[j & 1][lane] = cur * rj;
                bar_arrive(1, 32 + nw);
            }
        } else if (worker) {
            bar_sync(1, 32 + nw);
            const T* Lc = lh[j & 1];
            // diagonal block, columns j+2 .. c-1 (pairs with column >= j+2)
            const int npair = (c - 2 - j) * (c - 1 - j) / 2;
            for (int e = wid; e < npair; e += nw) {
                const short2 pr = tab[e];
                T* p = U + pr.x + pr.y * ru;
                *p = fma(-colj[pr.x], Lc[pr.y], *p);
            }
            // rows below, columns j+1 .. c-1
            const int ncol = c - 1 - j;
            if (ncol > 0 && nr > 0) {
                for (int e = wid; e < ncol * nr; e += nw) {
                    int q, i;
                    fast_divmod(e, nr, rcp, q, i);
                    const int kk = j + 1 + q, ii = c + i;
                    T* p = U + ii + kk * ru;
                    *p = fma(-colj[ii], Lc[kk], *p);
                }
            }
        }
        __syncthreads();
    }
}

template <typename T>
__device__ __forceinline__ void fused_tab(short2* tab, int c) {
    for (int e = threadIdx.x; e < c * c; e += blockDim.x) {
        const int ii = e % c, kk = e / c;
        if (kk >= 1 && ii >= kk) tab[(c - 1 - kk) * (c - kk) / 2 + (ii - kk)] = make_short2((short)ii, (short)kk);
    }
}

// One CTA per supernode (split = 1), or `split` CTAs that each factorise the
// whole panel and take a share of the Schur update.
template <typename T, bool kReserve>
__global__ void __launch_bounds__(kFusedThreads)
factor_fused_kernel(Plan P, const int* __restrict__ lvl_sn, int split, T* __restrict__ Lx,
                    FailSink fail, T* __restrict__ dinv) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T rr[kFusedMaxC];           // 1 / d_j
    __shared__ T lh[2][kFusedMaxC];        // Lhat[.][j] of the diagonal block
    __shared__ short2 tab[kFusedMaxC * (kFusedMaxC - 1) / 2];
    const int s = lvl_sn[blockIdx.x / split];
    if (!kkt_in(P.berr, s >= 0 && s < P.ns, kBcSupernode)) return;
    if (!sn_on(P, s)) return;
    const int rank = (int)(blockIdx.x % split);
    const int f = P.sn_f[s], c = P.sn_c[s], r = P.sn_r[s], rb = r - c;
    T* U = reinterpret_cast<T*>(smem_raw);   // r x c, ld = r
    T* L21 = U + r * c;                      // rb x c, ld = rb (normalised rows below)
    T* g = Lx + P.sn_lptr[s];
    const int tid = threadIdx.x;
    for (int e = tid; e < r * c; e += kFusedThreads) U[e] = g[e];
    fused_tab<T>(tab, c);
    fused_panel<T, kReserve>(U, r, c, rb, f, fail, rr, lh, tab);
    // reciprocal square roots of the pivots for the solves; normalised panel
    if (rank == 0 && tid < c) {
        T d = U[tid + tid * r];
        if (!pivot_ok(d)) d = T(1.0);
        dinv[f + tid] = pivot_rsqrt(d);
    }
    for (int e = tid; e < r * c; e += kFusedThreads) {
        const int col = e / r, row = e - col * r;
        const T v = U[e] * rr[col];
        if (rank == 0) g[e] = v;
        if (row >= c) L21[(row - c) + col * rb] = v;
    }
    __syncthreads();
    if (rb > 0) {
        const int np = rb * (rb + 1) / 2;
        const int p0 = (int)((long long)np * rank / split);
        const int p1 = (int)((long long)np * (rank + 1) / split);
        syrk_pairs_ldl(P, s, c, (const T*)L21, rb, (const T*)(U + c), r, p0, p1, Lx);
    }
}

// Thread-block cluster of K CTAs per supernode (levels of a few supernodes):
// every CTA runs the pivot chain on the diagonal block, but only its own
// share of the rows below (rows [c + rb k / K, c + rb (k + 1) / K) for rank
// k), so the rows' updates are spread over K SMs.  Then: cluster barrier;
// each CTA copies the other CTAs' finished rows (unnormalised) from their
// shared memory (distributed shared memory) into its own; cluster barrier
// (no CTA leaves while its rows may still be read); each CTA takes 1/K of
// the Schur pairs.  Cluster barriers are hardware barriers of the cluster's
// co-scheduled CTAs: no spin-wait.  Shared memory layout: U = diagonal block
// + all rb rows (ld = r), L21 = normalised rows below (ld = rb).
template <typename T>
__global__ void __launch_bounds__(kFusedThreads)
factor_fused_cluster_kernel(Plan P, const int* __restrict__ lvl_sn, T* __restrict__ Lx, FailSink fail,
                            T* __restrict__ dinv) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T rr[kFusedMaxC];
    __shared__ T lh[2][kFusedMaxC];
    __shared__ short2 tab[kFusedMaxC * (kFusedMaxC - 1) / 2];
    const int K = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int s = lvl_sn[blockIdx.x / K];
    if (!kkt_in(P.berr, s >= 0 && s < P.ns, kBcSupernode)) {   // the whole cluster returns together
        return;
    }
    if (!sn_on(P, s)) return;   // switched-off instance: the whole cluster returns together
    const int f = P.sn_f[s], c = P.sn_c[s], r = P.sn_r[s], rb = r - c;
    const int i0 = (int)((long long)rb * rank / K), i1 = (int)((long long)rb * (rank + 1) / K);
    const int nr = i1 - i0;
    // own panel part: diagonal block + own rows, ld = c + nr (rows 0..c-1,
    // then rows c + i0 .. c + i1 - 1); afterwards the full panel at Uf
    T* Uo = reinterpret_cast<T*>(smem_raw);
    const int ro = c + nr;
    T* Uf = Uo + ro * c;                       // r x c, ld = r
    T* L21 = Uf + r * c;                       // rb x c, ld = rb
    T* g = Lx + P.sn_lptr[s];
    const int tid = threadIdx.x;
    for (int e = tid; e < ro * c; e += kFusedThreads) {
        const int col = e / ro, row = e - col * ro;
        Uo[e] = g[(row < c ? row : row + i0) + col * r];
    }
    fused_tab<T>(tab, c);
    fused_panel<T, true>(Uo, ro, c, nr, f, fail, rr, lh, tab);
    if (rank == 0 && tid < c) {
        T d = Uo[tid + tid * ro];
        if (!pivot_ok(d)) d = T(1.0);
        dinv[f + tid] = pivot_rsqrt(d);
    }
    // normalised panel part to global (rank 0 also the diagonal block)
    for (int e = tid; e < ro * c; e += kFusedThreads) {
        const int col = e / ro, row = e - col * ro;
        if (row >= c || rank == 0) g[(row < c ? row : row + i0) + col * r] = Uo[e] * rr[col];
    }
    cluster.sync();
    // gather every CTA's unnormalised rows below from its shared memory, one
    // peer at a time (its rows i0k .. i0k + nk - 1, ld c + nk there)
    for (int k = 0; k < K; ++k) {
        const int i0k = (int)((long long)rb * k / K), nk = (int)((long long)rb * (k + 1) / K) - i0k;
        if (nk == 0) continue;
        const T* remote = cluster.map_shared_rank(Uo, k);
        const int rk = c + nk;
        for (int e = tid; e < nk * c; e += kFusedThreads) {
            const int col = e / nk, i = e - col * nk;
            const T v = remote[c + i + col * rk];
            Uf[c + i0k + i + col * r] = v;
            L21[i0k + i + col * rb] = v * rr[col];
        }
    }
    cluster.sync();
    if (rb > 0) {
        const int np = rb * (rb + 1) / 2;
        const int p0 = (int)((long long)np * rank / K);
        const int p1 = (int)((long long)np * (rank + 1) / K);
        syrk_pairs_ldl(P, s, c, (const T*)L21, rb, (const T*)(Uf + c), r, p0, p1, Lx);
    }
}

}  // namespace kktgb
