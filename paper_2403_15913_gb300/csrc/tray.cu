// Per-stage evaluation kernels of the distillation-column model
// (Sec. VI-A of Pacaud & Shin): objective, gradient, constraints, Jacobian
// and Lagrangian-Hessian values, one thread per (stage, tray).
//
// Model (k trays, stages t = 0..T, zero-based tray index i, feed tray kf):
//   L = u D, V = L + D, S = F + L
//   equilibrium   y_i - alpha x_i / (1 + (alpha - 1) x_i) = 0
//   balances g_i = M xdot_i:
//     i = 0         V (y_1 - x_0)
//     1 <= i < kf   L (x_{i-1} - x_i) - V (y_i - y_{i+1})
//     i = kf        F x_f + L x_{i-1} - S x_i - V (y_i - y_{i+1})
//     kf < i < k-1  S (x_{i-1} - x_i) - V (y_i - y_{i+1})
//     i = k-1       S x_{k-2} - (F - D) x_{k-1} - V y_{k-1}
//   dynamics (t >= 1)   x_{i,t} - x_{i,t-1} - (h / M) g_i(x_t, y_t, u_t) = 0
//   initial (t = 0)     x_{i,0} - xbar_0 = 0
//   objective  sum_t sum_i (x_{i,t} - xbar)^2 + rho (u_t - ubar)^2
#include <cmath>
#include <string>

#include "fp64_lean.cuh"
#include "kkt.h"
#include "tray_internal.h"

namespace {

struct TrayP {
    int k, T;
    double h, alpha, D, F, xf, M, xbar, ubar, rho, x0bar;
    double hm;   // h / M, formed once on the host
    __host__ __device__ int feed() const { return k / 2; }
    __host__ __device__ int nst() const { return 2 * k + 1; }
};

bool unpack(const double* p, TrayP& q) {
    if (!p) return false;
    if (!(p[0] >= 3 && p[0] <= 4096 && p[1] >= 0 && p[1] <= 1e7)) return false;
    q.k = (int)p[0];
    q.T = (int)p[1];
    q.h = p[2];
    q.alpha = p[3];
    q.D = p[4];
    q.F = p[5];
    q.xf = p[6];
    q.M = p[7];
    q.xbar = p[8];
    q.ubar = p[9];
    q.rho = p[10];
    q.x0bar = p[11];
    q.hm = q.h / q.M;
    if ((double)q.k != p[0] || (double)q.T != p[1]) return false;
    double n = (2.0 * q.k + 1) * (q.T + 1);
    return n < 2e9;
}

// CSR offsets of stage t's rows in J
__host__ __device__ inline long long j_stage_off(const TrayP& P, int t) {
    return t == 0 ? 0 : 3LL * P.k + (long long)(t - 1) * (8 * P.k - 3);
}
__host__ __device__ inline int j_dyn_row_off(int i) { return i == 0 ? 0 : 4 + 6 * (i - 1); }

__global__ void tray_eval_kernel(TrayP P, const double* __restrict__ x0v, const double* __restrict__ w,
                                 const double* __restrict__ lam, double objw, double* __restrict__ grad,
                                 double* __restrict__ c, double* __restrict__ Jv, double* __restrict__ Wv) {
    const int k = P.k;
    const long long total = (long long)(P.T + 1) * k;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int t = (int)(e / k), i = (int)(e % k);
        const long long base = (long long)t * P.nst();
        const double* xt = w + base;
        const double* yt = w + base + k;
        const double u = w[base + 2 * k];
        const double x = xt[i];
        const double den = 1.0 + (P.alpha - 1.0) * x;
        const double rden = kktgb::rcp_pos(den);   // one reciprocal for phi and its derivatives
        const double phi = P.alpha * x * rden;
        const double dphi = P.alpha * rden * rden;
        const double d2phi = -2.0 * P.alpha * (P.alpha - 1.0) * (rden * rden * rden);
        const long long crow_dyn = (long long)t * 2 * k + i;
        const long long crow_eq = crow_dyn + k;
        if (grad) {
            grad[base + i] = 2.0 * (x - P.xbar);
            grad[base + k + i] = 0.0;
            if (i == 0) grad[base + 2 * k] = 2.0 * P.rho * (u - P.ubar);
        }
        const double Lf = u * P.D, Vf = Lf + P.D, Sf = P.F + Lf;
        const double hm = P.hm;
        const int kf = P.feed();
        // partials of g_i (same stage): dxm = d/dx_{i-1}, dx = d/dx_i,
        // dy = d/dy_i, dyp = d/dy_{i+1}, du = d/du
        double g = 0, dxm = 0, dx = 0, dy = 0, dyp = 0, du = 0;
        if (t >= 1) {
            if (i == 0) {
                g = Vf * (yt[1] - xt[0]);
                dx = -Vf; dyp = Vf; du = P.D * (yt[1] - xt[0]);
            } else if (i == k - 1) {
                g = Sf * xt[i - 1] - (P.F - P.D) * x - Vf * yt[i];
                dxm = Sf; dx = -(P.F - P.D); dy = -Vf;
                du = P.D * xt[i - 1] - P.D * yt[i];
            } else {
                const double lin = i <= kf ? Lf : Sf;    // coefficient of x_{i-1}
                const double lout = i < kf ? Lf : Sf;    // coefficient of -x_i
                g = lin * xt[i - 1] - lout * x - Vf * (yt[i] - yt[i + 1]);
                if (i == kf) g += P.F * P.xf;
                dxm = lin; dx = -lout; dy = -Vf; dyp = Vf;
                du = P.D * (xt[i - 1] - x) - P.D * (yt[i] - yt[i + 1]);
            }
        }
        if (c) {
            c[crow_dyn] = t == 0 ? x - (x0v ? x0v[i] : P.x0bar) : x - w[base - P.nst() + i] - hm * g;
            c[crow_eq] = yt[i] - phi;
        }
        if (Jv) {
            const long long so = j_stage_off(P, t);
            if (t == 0) {
                Jv[so + i] = 1.0;
                Jv[so + k + 2 * i] = -dphi;
                Jv[so + k + 2 * i + 1] = 1.0;
            } else {
                long long q = so + j_dyn_row_off(i);
                Jv[q++] = -1.0;                        // x_{i,t-1}
                if (i >= 1) Jv[q++] = -hm * dxm;       // x_{i-1,t}
                Jv[q++] = 1.0 - hm * dx;               // x_{i,t}
                if (i >= 1) Jv[q++] = -hm * dy;        // y_{i,t}
                if (i <= k - 2) Jv[q++] = -hm * dyp;   // y_{i+1,t}
                Jv[q++] = -hm * du;                    // u_t
                const long long qe = so + (6LL * k - 3) + 2 * i;
                Jv[qe] = -dphi;
                Jv[qe + 1] = 1.0;
            }
        }
        if (Wv) {
            const long long wo = (long long)t * (4 * k + 1);
            const double* lt = lam + (long long)t * 2 * k;
            double ux = 0.0, uy = 0.0;
            if (t >= 1) {
                if (i <= k - 2) ux = hm * P.D * (lt[i] - lt[i + 1]);
                if (i >= 1) uy = hm * P.D * (lt[i] - lt[i - 1]);
            }
            Wv[wo + 2 * i] = objw * 2.0 - lt[k + i] * d2phi;
            Wv[wo + 2 * i + 1] = ux;
            Wv[wo + 2 * k + 2 * i] = 0.0;
            Wv[wo + 2 * k + 2 * i + 1] = uy;
            if (i == 0) Wv[wo + 4 * k] = objw * 2.0 * P.rho;
        }
    }
}

// Deterministic objective: one CTA, fixed order.
__global__ void tray_objective_kernel(TrayP P, const double* __restrict__ w, double* __restrict__ f) {
    __shared__ double red[256];
    const int k = P.k;
    const long long total = (long long)(P.T + 1) * (k + 1);
    double s = 0.0;
    for (long long e = threadIdx.x; e < total; e += blockDim.x) {
        const int t = (int)(e / (k + 1)), i = (int)(e % (k + 1));
        const long long base = (long long)t * P.nst();
        if (i < k) {
            const double d = w[base + i] - P.xbar;
            s += d * d;
        } else {
            const double d = w[base + 2 * k] - P.ubar;
            s += P.rho * d * d;
        }
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *f = red[0];
}

// Objective partials over a fixed grid: CTA b sums its grid-stride share of
// the (stage, tray) terms and writes part[b * stride].
__global__ void __launch_bounds__(256)
tray_objective_partials_kernel(TrayP P, const double* __restrict__ w, double* __restrict__ part,
                               int stride) {
    __shared__ double red[256 / 32];
    const int k = P.k;
    const long long total = (long long)(P.T + 1) * (k + 1);
    double s = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int t = (int)(e / (k + 1)), i = (int)(e % (k + 1));
        const long long base = (long long)t * P.nst();
        if (i < k) {
            const double d = w[base + i] - P.xbar;
            s = fma(d, d, s);
        } else {
            const double d = w[base + 2 * k] - P.ubar;
            s = fma(P.rho * d, d, s);
        }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double acc = 0.0;
        for (int q = 0; q < 256 / 32; ++q) acc += red[q];
        part[(long long)blockIdx.x * stride] = acc;
    }
}

}  // namespace

namespace kktgb {
bool tray_objective_partials(const double* params, const double* d_w, double* d_part, int stride,
                             int nblocks, cudaStream_t stream) {
    TrayP P;
    if (!unpack(params, P) || !d_w || !d_part || nblocks <= 0) return false;
    tray_objective_partials_kernel<<<nblocks, 256, 0, stream>>>(P, d_w, d_part, stride);
    return cudaGetLastError() == cudaSuccess;
}
}  // namespace kktgb

namespace kktgb {

kkt_status tray_eval(const double* params, const double* d_x0, const double* d_w, const double* d_lam,
                     double obj_weight, double* d_f, double* d_grad, double* d_c, double* d_Jval,
                     double* d_Wval, cudaStream_t stream) {
    TrayP P;
    if (!unpack(params, P) || !d_w) return KKT_ERR_ARG;
    if (d_Wval && !d_lam) return KKT_ERR_ARG;
    if (d_grad || d_c || d_Jval || d_Wval) {
        const long long total = (long long)(P.T + 1) * P.k;
        long long g = (total + 255) / 256;
        if (g > 152 * 32) g = 152 * 32;
        tray_eval_kernel<<<(int)g, 256, 0, stream>>>(P, d_x0, d_w, d_lam, obj_weight, d_grad, d_c, d_Jval,
                                                     d_Wval);
    }
    if (d_f) tray_objective_kernel<<<1, 256, 0, stream>>>(P, d_w, d_f);
    return cudaGetLastError() == cudaSuccess ? KKT_OK : KKT_ERR_CUDA;
}

}  // namespace kktgb

extern "C" {

kkt_status kkt_tray_sizes(const double* params, int* n, int* m, int* nnzW, int* nnzJ) {
    TrayP P;
    if (!unpack(params, P)) return KKT_ERR_ARG;
    const long long nn = (long long)(P.T + 1) * P.nst();
    const long long mm = (long long)(P.T + 1) * 2 * P.k;
    const long long nw = (long long)(P.T + 1) * (4 * P.k + 1);
    const long long nj = 3LL * P.k + (long long)P.T * (8 * P.k - 3);
    if (nj > 2000000000LL || nw > 2000000000LL) return KKT_ERR_ARG;
    if (n) *n = (int)nn;
    if (m) *m = (int)mm;
    if (nnzW) *nnzW = (int)nw;
    if (nnzJ) *nnzJ = (int)nj;
    return KKT_OK;
}

kkt_status kkt_tray_pattern(const double* params, int* W_colptr, int* W_rowind, int* J_rowptr,
                            int* J_colind) {
    TrayP P;
    if (!unpack(params, P)) return KKT_ERR_ARG;
    const int k = P.k, nst = P.nst();
    if (W_colptr && W_rowind) {
        int q = 0, col = 0;
        W_colptr[0] = 0;
        for (int t = 0; t <= P.T; ++t) {
            const int base = t * nst, ucol = base + 2 * k;
            for (int j = 0; j < 2 * k; ++j) {
                W_rowind[q++] = base + j;
                W_rowind[q++] = ucol;
                W_colptr[++col] = q;
            }
            W_rowind[q++] = ucol;
            W_colptr[++col] = q;
        }
    }
    if (J_rowptr && J_colind) {
        int q = 0, row = 0;
        J_rowptr[0] = 0;
        for (int t = 0; t <= P.T; ++t) {
            const int base = t * nst;
            for (int i = 0; i < k; ++i) {
                if (t == 0) {
                    J_colind[q++] = base + i;
                } else {
                    J_colind[q++] = base - nst + i;
                    if (i >= 1) J_colind[q++] = base + i - 1;
                    J_colind[q++] = base + i;
                    if (i >= 1) J_colind[q++] = base + k + i;
                    if (i <= k - 2) J_colind[q++] = base + k + i + 1;
                    J_colind[q++] = base + 2 * k;
                }
                J_rowptr[++row] = q;
            }
            for (int i = 0; i < k; ++i) {
                J_colind[q++] = base + i;
                J_colind[q++] = base + k + i;
                J_rowptr[++row] = q;
            }
        }
    }
    return KKT_OK;
}

kkt_status kkt_tray_eval(const double* params, const double* d_w, const double* d_lam, double obj_weight,
                         double* d_f, double* d_grad, double* d_c, double* d_Jval, double* d_Wval,
                         cudaStream_t stream) {
    return kktgb::tray_eval(params, nullptr, d_w, d_lam, obj_weight, d_f, d_grad, d_c, d_Jval, d_Wval,
                            stream);
}

}  // extern "C"
