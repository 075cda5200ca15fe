// Block cyclic reduction of a block-tridiagonal SPD matrix (the condensed
// KKT matrix of a stage-structured problem with stage-major variables: W
// couples variables of one stage, the dynamics rows of J couple stage t with
// stage t-1, so K = W + Sigma + delta_x I + J^T D J has nonzero blocks only on
// and next to the block diagonal).  This is the structure-exploiting
// parallel-in-time alternative to the general supernodal factorisation.
//
// Storage (FP64, column-major b x b blocks, N = n / b blocks):
//   A[t]   diagonal block K[t, t] (full, both triangles), overwritten by L_t
//          inside the factor panel
//   C[t]   coupling K[t, prev(t)] with the previous still-active block
//   PN[t]  3b x b factor panel of block t: [L_t; L(prev, t); L(next, t)]
// Level l eliminates every other active block (one CTA each, "elim"
// entries {j, prev, next}); the survivors ("surv" entries {i, left elim,
// right elim}) then take the Schur updates of their eliminated neighbours.
#pragma once
#include "kernels.cuh"

namespace kktgb {

constexpr int kBcrMaxBlock = 80;   // 3 b^2 doubles of panel in shared memory

// Factor panel of elimination entry e = {j, jl, jr}: load [A_j; C_j^T; C_jr],
// factorise it (Cholesky of the b x b top, TRSM of the rest), store it in PN_j
// and write the fill coupling K'[jr, jl] = -L(jr, j) L(jl, j)^T into C_jr
// (zero when j has no left neighbour).
__global__ void __launch_bounds__(kThreads)
bcr_elim_kernel(int b, const int4* __restrict__ ent, double* __restrict__ A, double* __restrict__ C,
                double* __restrict__ PN, double* __restrict__ dinv, FailSink fail) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* P = reinterpret_cast<double*>(smem_raw);   // 3b x b, column-major
    const int4 e = ent[blockIdx.x];
    const int j = e.x, jl = e.y, jr = e.z;
    const int r = 3 * b;
    const long long bb = (long long)b * b;
    const double* Aj = A + j * bb;
    const double* Cj = C + j * bb;
    double* Cr = jr >= 0 ? C + jr * bb : nullptr;
    for (int q = threadIdx.x; q < r * b; q += blockDim.x) {
        const int row = q % r, col = q / r;
        double v = 0.0;
        if (row < b) {
            v = Aj[row + (long long)col * b];
        } else if (row < 2 * b) {
            if (jl >= 0) v = Cj[col + (long long)(row - b) * b];   // K[jl, j] = C_j^T
        } else {
            if (jr >= 0) v = Cr[(row - 2 * b) + (long long)col * b];   // K[jr, j]
        }
        P[q] = v;
    }
    __syncthreads();
    panel_factor<double>(P, j * b, b, r, r, fail, dinv);
    __syncthreads();
    double* out = PN + (long long)j * 3 * bb;
    for (int q = threadIdx.x; q < r * b; q += blockDim.x) out[q] = P[q];
    if (jr >= 0) {
        // K'[jr, jl](x, y) = -sum_c L(jr, j)(x, c) L(jl, j)(y, c)
        for (int q = threadIdx.x; q < b * b; q += blockDim.x) {
            const int x = q % b, y = q / b;
            double s = 0.0;
            if (jl >= 0)
                for (int c = 0; c < b; ++c) s = fma(P[2 * b + x + c * r], P[b + y + c * r], s);
            Cr[q] = -s;
        }
    }
}

// Survivor entry {i, el, er}: A_i -= L(i, el) L(i, el)^T + L(i, er) L(i, er)^T
// with L(i, el) the bottom block of el's panel (i follows el) and L(i, er)
// the middle block of er's panel (i precedes er).
__global__ void __launch_bounds__(kThreads)
bcr_update_kernel(int b, const int4* __restrict__ ent, double* __restrict__ A,
                  const double* __restrict__ PN) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* Ul = reinterpret_cast<double*>(smem_raw);   // b x b each
    double* Ur = Ul + b * b;
    const int4 e = ent[blockIdx.x];
    const int i = e.x, el = e.y, er = e.z;
    const long long bb = (long long)b * b;
    const int r = 3 * b;
    for (int q = threadIdx.x; q < b * b; q += blockDim.x) {
        const int x = q % b, c = q / b;
        Ul[q] = el >= 0 ? PN[el * 3 * bb + 2 * b + x + (long long)c * r] : 0.0;
        Ur[q] = er >= 0 ? PN[er * 3 * bb + b + x + (long long)c * r] : 0.0;
    }
    __syncthreads();
    double* Ai = A + i * bb;
    for (int q = threadIdx.x; q < b * b; q += blockDim.x) {
        const int x = q % b, y = q / b;
        double s = 0.0;
        for (int c = 0; c < b; ++c) {
            s = fma(Ul[x + c * b], Ul[y + c * b], s);
            s = fma(Ur[x + c * b], Ur[y + c * b], s);
        }
        Ai[q] -= s;
    }
}

// Forward solve, eliminated entry {j, ...}: z_j = L_j^{-1} v_j in place
// (reciprocal pivots in dinv; right-looking over the b x b block).
__global__ void __launch_bounds__(kThreads)
bcr_fwd_elim_kernel(int b, const int4* __restrict__ ent, const double* __restrict__ PN,
                    const double* __restrict__ dinv, double* __restrict__ v,
                    const int* __restrict__ active) {
    KKT_RETURN_IF_INACTIVE(active);
    __shared__ double z[kBcrMaxBlock];
    const int j = ent[blockIdx.x].x;
    const long long bb = (long long)b * b;
    const int r = 3 * b;
    const double* L = PN + j * 3 * bb;
    double* vj = v + (long long)j * b;
    for (int q = threadIdx.x; q < b; q += blockDim.x) z[q] = vj[q];
    __syncthreads();
    for (int c = 0; c < b; ++c) {
        const double zc = z[c] * dinv[j * b + c];
        __syncthreads();
        if (threadIdx.x == 0) z[c] = zc;
        for (int x = c + 1 + threadIdx.x; x < b; x += blockDim.x) z[x] -= L[x + (long long)c * r] * zc;
        __syncthreads();
    }
    for (int q = threadIdx.x; q < b; q += blockDim.x) vj[q] = z[q];
}

// Forward solve, survivor entry {i, el, er}: v_i -= L(i, el) z_el + L(i, er) z_er
__global__ void __launch_bounds__(kThreads)
bcr_fwd_update_kernel(int b, const int4* __restrict__ ent, const double* __restrict__ PN,
                      double* __restrict__ v, const int* __restrict__ active) {
    KKT_RETURN_IF_INACTIVE(active);
    const int4 e = ent[blockIdx.x];
    const int i = e.x, el = e.y, er = e.z;
    const long long bb = (long long)b * b;
    const int r = 3 * b;
    for (int x = threadIdx.x; x < b; x += blockDim.x) {
        double s = 0.0;
        if (el >= 0) {
            const double* Lb = PN + el * 3 * bb + 2 * b;
            const double* z = v + (long long)el * b;
            for (int c = 0; c < b; ++c) s = fma(Lb[x + (long long)c * r], z[c], s);
        }
        if (er >= 0) {
            const double* Lm = PN + er * 3 * bb + b;
            const double* z = v + (long long)er * b;
            for (int c = 0; c < b; ++c) s = fma(Lm[x + (long long)c * r], z[c], s);
        }
        v[(long long)i * b + x] -= s;
    }
}

// Backward solve, eliminated entry {j, jl, jr} (neighbours already final):
// w_j = L_j^{-T} (z_j - L(jl, j)^T w_jl - L(jr, j)^T w_jr), in place.
__global__ void __launch_bounds__(kThreads)
bcr_bwd_kernel(int b, const int4* __restrict__ ent, const double* __restrict__ PN,
               const double* __restrict__ dinv, double* __restrict__ v, const int* __restrict__ active) {
    KKT_RETURN_IF_INACTIVE(active);
    __shared__ double w[kBcrMaxBlock];
    const int4 e = ent[blockIdx.x];
    const int j = e.x, jl = e.y, jr = e.z;
    const long long bb = (long long)b * b;
    const int r = 3 * b;
    const double* L = PN + j * 3 * bb;
    double* vj = v + (long long)j * b;
    for (int c = threadIdx.x; c < b; c += blockDim.x) {
        double s = vj[c];
        if (jl >= 0) {
            const double* wl = v + (long long)jl * b;
            for (int y = 0; y < b; ++y) s -= L[b + y + (long long)c * r] * wl[y];
        }
        if (jr >= 0) {
            const double* wr = v + (long long)jr * b;
            for (int y = 0; y < b; ++y) s -= L[2 * b + y + (long long)c * r] * wr[y];
        }
        w[c] = s;
    }
    __syncthreads();
    for (int c = b - 1; c >= 0; --c) {
        const double wc = w[c] * dinv[j * b + c];
        __syncthreads();
        if (threadIdx.x == 0) w[c] = wc;
        for (int x = threadIdx.x; x < c; x += blockDim.x) w[x] -= L[c + (long long)x * r] * wc;
        __syncthreads();
    }
    for (int q = threadIdx.x; q < b; q += blockDim.x) vj[q] = w[q];
}

}  // namespace kktgb
