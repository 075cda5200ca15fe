// Device kernels of the KKT library (sm_103a, FP64).
//
// On GB300 the FP64 pipe delivers about 1.2 TFLOP/s for the whole GPU, so
// the supernodal factorisation and the triangular solves are bound by DFMA
// issue, not by HBM.  The kernels therefore (i) never spend FP64 work on
// padding beyond the supernode panels, (ii) keep a panel in shared memory
// while it is factorised, and (iii) leave all index arithmetic to the
// integer pipes.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace kktgb {

constexpr int kThreads = 256;
constexpr int kRedBlocks = 296;   // 2 x 148..152 SMs: partial-sum slots

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
};

// ------------------------------------------------------------- assembly
// One thread per stored entry of the lower triangle of P K P^T: sums its
// sources (W entry, diagonal Sigma_x + delta_x, products D_r J_ra J_rb) and
// writes the panel slot.  Source encoding: b == -1 -> W[a];
// b == -2 -> sigma[a] + delta_x; b >= 0 -> D[jrow[a]] * J[a] * J[b].
__global__ void assemble_kernel(long long nk, const long long* __restrict__ slot,
                                const long long* __restrict__ sptr,
                                const int2* __restrict__ src, const int* __restrict__ jrow,
                                const double* __restrict__ W, const double* __restrict__ J,
                                const double* __restrict__ sigma, const double* __restrict__ D,
                                double Dconst, double delta_x, double* __restrict__ Lx) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nk;
         e += (long long)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (long long q = sptr[e]; q < sptr[e + 1]; ++q) {
            int2 s = src[q];
            if (s.y == -1) {
                v += W[s.x];
            } else if (s.y == -2) {
                v += sigma[s.x] + delta_x;
            } else {
                double d = D ? D[jrow[s.x]] : Dconst;
                v += d * J[s.x] * J[s.y];
            }
        }
        Lx[slot[e]] = v;
    }
}

// ------------------------------------------------------------- factor
// One CTA per supernode of a level: right-looking column Cholesky of the
// panel (POTRF of the diagonal block and TRSM of the rows below in one
// sweep), then the SYRK update L21 L21^T scattered into the ancestors'
// panels through the precomputed relative maps (FP64 atomics: ancestors
// are never in the same level, so a panel is only read after every update
// into it has landed).
__global__ void __launch_bounds__(kThreads)
factor_level_kernel(Plan P, const int* __restrict__ lvl_sn, double* __restrict__ Lx,
                    int* __restrict__ fail, long long smem_elems) {
    extern __shared__ double sm[];
    __shared__ double s_inv;
    const int s = lvl_sn[blockIdx.x];
    const int f = P.sn_f[s], c = P.sn_c[s], r = P.sn_r[s];
    const long long lp = P.sn_lptr[s];
    const int tid = threadIdx.x, nt = blockDim.x;
    const bool in_smem = (long long)r * c <= smem_elems;
    double* A = in_smem ? sm : Lx + lp;
    if (in_smem) {
        const double* g = Lx + lp;
        for (long long e = tid; e < (long long)r * c; e += nt) A[e] = g[e];
        __syncthreads();
    }
    for (int j = 0; j < c; ++j) {
        if (tid == 0) {
            double d = A[j + (long long)j * r];
            if (!(d > 0.0) || !isfinite(d)) {
                atomicMin(fail, f + j);
                d = 1.0;
            }
            double l = sqrt(d);
            A[j + (long long)j * r] = l;
            s_inv = 1.0 / l;
        }
        __syncthreads();
        const double inv = s_inv;
        double* colj = A + (long long)j * r;
        for (int i = j + 1 + tid; i < r; i += nt) colj[i] *= inv;
        __syncthreads();
        const int nk = c - 1 - j, len = r - 1 - j;
        for (int idx = tid; idx < nk * len; idx += nt) {
            const int kk = j + 1 + idx / len;
            const int ii = j + 1 + idx % len;
            if (ii >= kk) A[ii + (long long)kk * r] -= colj[ii] * colj[kk];
        }
        __syncthreads();
    }
    if (in_smem) {
        double* g = Lx + lp;
        for (long long e = tid; e < (long long)r * c; e += nt) g[e] = A[e];
    }
    const int rb = r - c;
    if (rb <= 0) return;
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    const int sp0 = P.seg_ptr[s], sp1 = P.seg_ptr[s + 1];
    const int* rows = P.rows + P.sn_rptr[s];
    for (int jj = warp; jj < rb; jj += nw) {
        int k = sp0;
        while (k < sp1 - 1 && jj >= P.seg_b[k]) ++k;
        const int t = P.seg_t[k], a = P.seg_a[k];
        const long long base =
            P.sn_lptr[t] + (long long)(rows[c + jj] - P.sn_f[t]) * P.sn_r[t];
        const int* rm = P.relmap + P.seg_map[k];
        for (int ii = jj + lane; ii < rb; ii += 32) {
            double sum = 0.0;
            for (int q = 0; q < c; ++q)
                sum += A[c + ii + (long long)q * r] * A[c + jj + (long long)q * r];
            atomicAdd(Lx + base + rm[ii - a], -sum);
        }
    }
}

// ------------------------------------------------------------- solves
// Forward substitution L z = b, one CTA per supernode of a level.
__global__ void __launch_bounds__(kThreads)
forward_level_kernel(Plan P, const int* __restrict__ lvl_sn, const double* __restrict__ Lx,
                     double* __restrict__ x) {
    extern __shared__ double z[];
    const int s = lvl_sn[blockIdx.x];
    const int f = P.sn_f[s], c = P.sn_c[s], r = P.sn_r[s];
    const double* A = Lx + P.sn_lptr[s];
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int k = tid; k < c; k += nt) z[k] = x[f + k];
    __syncthreads();
    for (int j = 0; j < c; ++j) {
        if (tid == 0) z[j] /= A[j + (long long)j * r];
        __syncthreads();
        const double zj = z[j];
        for (int i = j + 1 + tid; i < c; i += nt) z[i] -= A[i + (long long)j * r] * zj;
        __syncthreads();
    }
    for (int k = tid; k < c; k += nt) x[f + k] = z[k];
    const int* rows = P.rows + P.sn_rptr[s];
    for (int i = tid; i < r - c; i += nt) {
        double sum = 0.0;
        for (int k = 0; k < c; ++k) sum += A[c + i + (long long)k * r] * z[k];
        atomicAdd(x + rows[c + i], -sum);
    }
}

// Backward substitution L^T w = z, one CTA per supernode of a level
// (levels visited top-down).
__global__ void __launch_bounds__(kThreads)
backward_level_kernel(Plan P, const int* __restrict__ lvl_sn, const double* __restrict__ Lx,
                      double* __restrict__ x) {
    extern __shared__ double t[];
    const int s = lvl_sn[blockIdx.x];
    const int f = P.sn_f[s], c = P.sn_c[s], r = P.sn_r[s];
    const double* A = Lx + P.sn_lptr[s];
    const int* rows = P.rows + P.sn_rptr[s];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    const int rb = r - c;
    for (int k = warp; k < c; k += nw) {
        double sum = 0.0;
        for (int i = lane; i < rb; i += 32) sum += A[c + i + (long long)k * r] * x[rows[c + i]];
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
        if (lane == 0) t[k] = x[f + k] - sum;
    }
    __syncthreads();
    for (int j = c - 1; j >= 0; --j) {
        if (tid == 0) t[j] /= A[j + (long long)j * r];
        __syncthreads();
        const double tj = t[j];
        for (int k = tid; k < j; k += nt) t[k] -= A[j + (long long)k * r] * tj;
        __syncthreads();
    }
    for (int k = tid; k < c; k += nt) x[f + k] = t[k];
}

__global__ void gather_kernel(int n, const int* __restrict__ idx, const double* __restrict__ in,
                              double* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = in[idx[i]];
}

__global__ void scatter_kernel(int n, const int* __restrict__ idx, const double* __restrict__ in,
                               double* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[idx[i]] = in[i];
}

// ------------------------------------------------------------- sparse BLAS
// out_x = a_x + alpha * J^T (Dscale o a_y)    (Dscale NULL -> Dconst)
__global__ void jt_axpy_kernel(int n, const int* __restrict__ jt_ptr, const int* __restrict__ jt_row,
                               const int* __restrict__ jt_idx, const double* __restrict__ J,
                               const double* __restrict__ ax, const double* __restrict__ ay,
                               const double* __restrict__ Dscale, double Dconst, double alpha,
                               double* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int q = jt_ptr[i]; q < jt_ptr[i + 1]; ++q) {
            int r = jt_row[q];
            double d = Dscale ? Dscale[r] : Dconst;
            s += J[jt_idx[q]] * d * ay[r];
        }
        out[i] = (ax ? ax[i] : 0.0) + alpha * s;
    }
}

// out_y = Dscale o (J x - b_y)   (Dscale NULL -> Dconst; b_y NULL -> 0)
__global__ void j_apply_kernel(int m, const int* __restrict__ j_ptr, const int* __restrict__ j_col,
                               const double* __restrict__ J, const double* __restrict__ x,
                               const double* __restrict__ by, const double* __restrict__ Dscale,
                               double Dconst, double* __restrict__ out) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int q = j_ptr[r]; q < j_ptr[r + 1]; ++q) s += J[q] * x[j_col[q]];
        if (by) s -= by[r];
        out[r] = (Dscale ? Dscale[r] : Dconst) * s;
    }
}

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long*>(addr), __double_as_longlong(v));
}

__device__ __forceinline__ double block_max(double v) {
    __shared__ double red[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    }
    return v;
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

// Residual of the original system: r = b - K_orig v, with
//   K_orig = [[W + diag(sigma + delta_x), J^T], [J, -diag(C)]]
// and the max-norms of r, v, b accumulated into out[0..2].
__global__ void __launch_bounds__(kThreads)
residual_kernel(int n, int m, const int* __restrict__ wf_ptr, const int* __restrict__ wf_col,
                const int* __restrict__ wf_idx, const double* __restrict__ W,
                const int* __restrict__ j_ptr, const int* __restrict__ j_col,
                const int* __restrict__ jt_ptr, const int* __restrict__ jt_row,
                const int* __restrict__ jt_idx, const double* __restrict__ J,
                const double* __restrict__ sigma, double delta_x, const double* __restrict__ C,
                const double* __restrict__ bx, const double* __restrict__ by,
                const double* __restrict__ vx, const double* __restrict__ vy,
                double* __restrict__ rx, double* __restrict__ ry, double* __restrict__ out) {
    double mr = 0.0, mv = 0.0, mb = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
        if (i < n) {
            double s = (sigma[i] + delta_x) * vx[i];
            for (int q = wf_ptr[i]; q < wf_ptr[i + 1]; ++q) s += W[wf_idx[q]] * vx[wf_col[q]];
            for (int q = jt_ptr[i]; q < jt_ptr[i + 1]; ++q) s += J[jt_idx[q]] * vy[jt_row[q]];
            double r = bx[i] - s;
            rx[i] = r;
            mr = fmax(mr, fabs(r));
            mv = fmax(mv, fabs(vx[i]));
            mb = fmax(mb, fabs(bx[i]));
        } else {
            int k = i - n;
            double s = C ? -C[k] * vy[k] : 0.0;
            for (int q = j_ptr[k]; q < j_ptr[k + 1]; ++q) s += J[q] * vx[j_col[q]];
            double r = by[k] - s;
            ry[k] = r;
            mr = fmax(mr, fabs(r));
            mv = fmax(mv, fabs(vy[k]));
            mb = fmax(mb, fabs(by[k]));
        }
    }
    mr = block_max(mr);
    mv = block_max(mv);
    mb = block_max(mb);
    if (threadIdx.x == 0) {
        atomic_max_nonneg(out + 0, mr);
        atomic_max_nonneg(out + 1, mv);
        atomic_max_nonneg(out + 2, mb);
    }
}

// ||K_orig||_inf (row sums of |K_orig|) into out[0] (atomic max).
__global__ void __launch_bounds__(kThreads)
knorm_kernel(int n, int m, const int* __restrict__ wf_ptr, const int* __restrict__ wf_col,
             const int* __restrict__ wf_idx, const double* __restrict__ W,
             const int* __restrict__ j_ptr, const int* __restrict__ jt_ptr,
             const int* __restrict__ jt_idx, const double* __restrict__ J,
             const double* __restrict__ sigma, double delta_x, const double* __restrict__ C,
             double* __restrict__ out) {
    double mx = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        if (i < n) {
            double d = sigma[i] + delta_x;
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
        mx = fmax(mx, s);
    }
    mx = block_max(mx);
    if (threadIdx.x == 0) atomic_max_nonneg(out, mx);
}

// y += a * x over two concatenated segments
__global__ void axpy_kernel(int n, double a, const double* __restrict__ x, double* __restrict__ y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        y[i] += a * x[i];
}

__global__ void recip_kernel(int n, const double* __restrict__ x, double* __restrict__ y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        y[i] = 1.0 / x[i];
}

__global__ void fill_kernel(int n, double v, double* __restrict__ y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = v;
}

// Deterministic dot product: fixed grid of kRedBlocks CTAs writes partial
// sums, a single CTA adds them in a fixed order.
__global__ void __launch_bounds__(kThreads)
dot_partial_kernel(int n, const double* __restrict__ a, const double* __restrict__ b,
                   double* __restrict__ part) {
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        s += a[i] * b[i];
    s = block_sum(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads)
dot_final_kernel(int nparts, const double* __restrict__ part, double* __restrict__ out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += part[i];
    s = block_sum(s);
    if (threadIdx.x == 0) *out = s;
}

// CG updates with scalars kept on the device.
// x += alpha p; r -= alpha q   with alpha = sc[rr] / sc[pq]
__global__ void cg_update_xr_kernel(int m, const double* __restrict__ sc, int i_rr, int i_pq,
                                    const double* __restrict__ p, const double* __restrict__ q,
                                    double* __restrict__ x, double* __restrict__ r) {
    const double alpha = sc[i_rr] / sc[i_pq];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        x[i] += alpha * p[i];
        r[i] -= alpha * q[i];
    }
}

// p = r + beta p   with beta = sc[rr_new] / sc[rr_old]
__global__ void cg_update_p_kernel(int m, const double* __restrict__ sc, int i_new, int i_old,
                                   const double* __restrict__ r, double* __restrict__ p) {
    const double beta = sc[i_new] / sc[i_old];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        p[i] = r[i] + beta * p[i];
}

}  // namespace kktgb
