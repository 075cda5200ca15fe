// Minimal filter line-search interior-point driver on the device (Sec. III of
// Pacaud & Shin: Newton steps on F_mu(w) = 0 with a fraction-to-boundary rule;
// the filter line search of Wachter & Biegler (2006), basic form).
//
// Per iteration (host logic in C++, every vector operation in a kernel):
//   1. derivatives of the column model at (x, y)          kkt_tray_eval
//   2. optimality error E_0; monotone barrier update      errors_kernel
//   3. Sigma_x, r_x = -(grad phi + J^T y), r_y            prepare_kernel
//   4. KKT factor (inertia-correction ladder) and solve   kkt_factor / kkt_solve
//   5. bound-multiplier steps, fraction to boundary,
//      directional derivative of the barrier function    recover_kernel
//   6. backtracking filter line search on (theta, phi)    trial/measure kernels
//   7. update with the bound-multiplier safeguard         accept_kernel
// Only scalars (norms, step lengths, filter measures) come back to the host.
// Constants are the published defaults of the reference algorithm.
#include <algorithm>
#include <cmath>
#include <string>
#include <utility>
#include <vector>

#include "fp64_lean.cuh"
#include "sparse_dot.cuh"
#include "kkt.h"
#include "tray_internal.h"

namespace {

using kktgb::is_pos;
using kktgb::lt_nonneg;
using kktgb::max_abs;
using kktgb::max_nonneg;
using kktgb::min_nonneg;
using kktgb::rcp_pos;

constexpr int kT = 256;
constexpr int kRB = 296;            // CTAs of the reduction kernels (fixed: deterministic sums)
constexpr int kQ = 8;               // quantities per reduction

// Wachter-Biegler defaults
constexpr double kKappaEps = 10.0, kKappaMu = 0.2, kThetaMu = 1.5, kTauMin = 0.99;
constexpr double kSMax = 100.0, kBoundPush = 1e-2, kBoundFrac = 1e-2, kKappaSigma = 1e10;
constexpr double kGammaTheta = 1e-5, kGammaPhi = 1e-8, kDelta = 1.0, kSTheta = 1.1, kSPhi = 2.3;
constexpr double kEtaPhi = 1e-8;
constexpr int kMaxLs = 40;
constexpr double kDeltaW0 = 1e-4, kDeltaMin = 1e-20, kDeltaMax = 1e40;
constexpr double kKappaWMinus = 1.0 / 3.0, kKappaWPlus = 8.0, kKappaWPlusBar = 100.0;

enum Op { SUM = 0, MAX = 1, MIN = 2 };

// every MAX / MIN quantity of the reductions is >= 0 (or a +-inf identity),
// so those are compared on the integer units
__device__ __forceinline__ double combine(double a, double b, int op) {
    return op == SUM ? a + b : (op == MAX ? max_nonneg(a, b) : min_nonneg(a, b));
}

__device__ __forceinline__ double block_reduce(double v, int op, double* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v = combine(v, __shfl_down_sync(0xffffffffu, v, o), op);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        const double id = op == SUM ? 0.0 : (op == MAX ? -INFINITY : INFINITY);
        v = lane < (int)(blockDim.x >> 5) ? red[lane] : id;
        for (int o = 16; o > 0; o >>= 1) v = combine(v, __shfl_down_sync(0xffffffffu, v, o), op);
    }
    return v;
}

// Writes the block's K partial results to part[blockIdx.x * kQ + q]; the
// CTA that finishes last (a device-wide counter taken after a fence) then
// reduces the gridDim.x partials of each quantity into out[q]: warp q takes
// quantity q, lane l combines blocks l, l + 32, ... in order, then a fixed
// shuffle tree -- the same order every time (deterministic), without a
// separate final launch.  The last CTA resets the counter.
template <int K>
__device__ __forceinline__ void store_partials(const double (&v)[K], const int (&ops)[K], double* part,
                                               unsigned* count, double* out) {
    static_assert(K <= kT / 32, "one warp per quantity");
    __shared__ double red[kT / 32];
    __shared__ bool last;
    for (int q = 0; q < K; ++q) {
        const double r = block_reduce(v[q], ops[q], red);
        if (threadIdx.x == 0) part[blockIdx.x * kQ + q] = r;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (q < K) {
        int op = SUM;
        for (int j = 0; j < K; ++j)
            if (j == q) op = ops[j];
        double acc = __ldcg(part + lane * kQ + q);
        for (int b = lane + 32; b < (int)gridDim.x; b += 32) acc = combine(acc, __ldcg(part + b * kQ + q), op);
        for (int o = 16; o > 0; o >>= 1) acc = combine(acc, __shfl_down_sync(0xffffffffu, acc, o), op);
        if (lane == 0) out[q] = acc;
    }
    if (threadIdx.x == 0) *count = 0u;
}

// Sum of kRB partials part[b * kQ] (the objective), in the order above.
__global__ void final_sum_kernel(const double* __restrict__ part, double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    double acc = part[lane * kQ];
    for (int b = lane + 32; b < kRB; b += 32) acc += part[b * kQ];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) out[0] = acc;
}

// sum of log(g) over a thread's elements as log(prod of mantissas) plus the
// exponents times ln 2: one logarithm per thread instead of one per element.
// The splits g = m 2^e are taken on the bit patterns (one FP64 multiply per
// element); zero, subnormal, infinite or negative g go through frexp.
struct LogSum {
    double mant = 1.0;
    long long expo = 0;
    __device__ __forceinline__ void add(double g) {
        double m;
        int e;
        if (!kktgb::split_pos(g, m, e)) m = frexp(g, &e);   // g = m 2^e, m in [0.5, 1)
        mant *= m;
        expo += e;
        int e2;
        double mm;
        if (!kktgb::split_pos(mant, mm, e2)) mm = frexp(mant, &e2);   // keep the product normalised
        mant = mm;
        expo += e2;
    }
    __device__ __forceinline__ double value() const {
        return log(mant) + (double)expo * 0.69314718055994530942;
    }
};

// Running minimum of ratios a / b (a >= 0, b > 0) compared by cross products
// (a b' < a' b), divided once at the end: a division costs several FP64
// instructions, a comparison by products two multiplies.  The minimum is the
// same rounded quotient a / b of the selected pair.
struct MinRatio {
    double a = 1.0, b = 1.0;
    __device__ __forceinline__ void add(double na, double nb) {
        if (lt_nonneg(na * b, a * nb)) { a = na; b = nb; }   // products >= 0: integer compare
    }
    __device__ __forceinline__ double value() const { return a / b; }
};

struct Bounds {
    const double *xlo, *xhi;
    double tau;   // slack bounds [-tau, tau]
};

// J^T v through the CSC of J (deterministic gather).
__global__ void jt_kernel(int n, const int* __restrict__ cp, const int* __restrict__ ri,
                          const int* __restrict__ idx, const double* __restrict__ J,
                          const double* __restrict__ v, double* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        out[i] = kktgb::gather_dot(cp[i], cp[i + 1], idx, ri, J, v, 0.0);
    }
}

__global__ void push_kernel(int n, const double* __restrict__ lo, const double* __restrict__ hi,
                            double clo, double chi, double* __restrict__ x) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double l = lo ? lo[i] : clo, h = hi ? hi[i] : chi;
        const double pl = fmin(kBoundPush * fmax(1.0, fabs(l)), kBoundFrac * (h - l));
        const double pu = fmin(kBoundPush * fmax(1.0, fabs(h)), kBoundFrac * (h - l));
        x[i] = fmin(fmax(x[i], l + pl), h - pu);
    }
}

__global__ void fill_kernel(int n, double v, double* __restrict__ y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = v;
}

__global__ void copy_kernel(int n, const double* __restrict__ a, double* __restrict__ b) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = a[i];
}

// Optimality measures: [max|du|, max|pr|, max z*gap, min z*gap, sum|y|, sum z, 0, 0]
__global__ void __launch_bounds__(kT)
errors_kernel(int n, int m, int relaxed, Bounds B, const double* __restrict__ x,
              const double* __restrict__ s, const double* __restrict__ y,
              const double* __restrict__ zl, const double* __restrict__ zu,
              const double* __restrict__ vl, const double* __restrict__ vu,
              const double* __restrict__ grad, const double* __restrict__ jty,
              const double* __restrict__ c, double* __restrict__ part, unsigned* count,
              double* __restrict__ out) {
    double v[6] = {0.0, 0.0, -INFINITY, INFINITY, 0.0, 0.0};
    const int ops[6] = {MAX, MAX, MAX, MIN, SUM, SUM};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
        if (i < n) {
            const double gl = x[i] - B.xlo[i], gu = B.xhi[i] - x[i];
            v[0] = max_abs(v[0], grad[i] + jty[i] - zl[i] + zu[i]);
            const double a = zl[i] * gl, b = zu[i] * gu;
            v[2] = max_nonneg(max_nonneg(v[2], a), b);
            v[3] = min_nonneg(min_nonneg(v[3], a), b);
            v[5] += zl[i] + zu[i];
        } else {
            const int k = i - n;
            v[1] = max_abs(v[1], relaxed ? c[k] - s[k] : c[k]);
            v[4] += fabs(y[k]);
            if (relaxed) {
                v[0] = max_abs(v[0], -y[k] - vl[k] + vu[k]);
                const double a = vl[k] * (s[k] + B.tau), b = vu[k] * (B.tau - s[k]);
                v[2] = max_nonneg(max_nonneg(v[2], a), b);
                v[3] = min_nonneg(min_nonneg(v[3], a), b);
                v[5] += vl[k] + vu[k];
            }
        }
    }
    store_partials<6>(v, ops, part, count, out);
}

__global__ void prepare_kernel(int n, int m, int relaxed, Bounds B, double mu,
                               const double* __restrict__ x, const double* __restrict__ s,
                               const double* __restrict__ y, const double* __restrict__ zl,
                               const double* __restrict__ zu, const double* __restrict__ vl,
                               const double* __restrict__ vu, const double* __restrict__ grad,
                               const double* __restrict__ jty, const double* __restrict__ c,
                               double* __restrict__ sigma, double* __restrict__ rx,
                               double* __restrict__ ry, double* __restrict__ D) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
        if (i < n) {
            const double igl = rcp_pos(x[i] - B.xlo[i]), igu = rcp_pos(B.xhi[i] - x[i]);
            sigma[i] = zl[i] * igl + zu[i] * igu;
            rx[i] = -(grad[i] - mu * igl + mu * igu + jty[i]);
        } else {
            const int k = i - n;
            if (relaxed) {
                const double ihl = rcp_pos(s[k] + B.tau), ihu = rcp_pos(B.tau - s[k]);
                const double sig = vl[k] * ihl + vu[k] * ihu;
                const double gphi = -mu * ihl + mu * ihu;
                D[k] = sig;
                ry[k] = -(c[k] - s[k]) - (gphi - y[k]) * rcp_pos(sig);
            } else {
                ry[k] = -c[k];
            }
        }
    }
}

// Step recovery, fraction to boundary and directional derivative:
// partials [alpha_pr (min), alpha_du (min), dphi (sum)].
__global__ void __launch_bounds__(kT)
recover_kernel(int n, int m, int relaxed, Bounds B, double mu, double tau,
               const double* __restrict__ x, const double* __restrict__ s,
               const double* __restrict__ y, const double* __restrict__ zl,
               const double* __restrict__ zu, const double* __restrict__ vl,
               const double* __restrict__ vu, const double* __restrict__ grad,
               const double* __restrict__ dx, const double* __restrict__ dy,
               double* __restrict__ ds, double* __restrict__ dzl, double* __restrict__ dzu,
               double* __restrict__ dvl, double* __restrict__ dvu, double* __restrict__ part,
               unsigned* count, double* __restrict__ out) {
    double v[3] = {1.0, 1.0, 0.0};
    const int ops[3] = {MIN, MIN, SUM};
    MinRatio apr, adu;   // tau gap / |step| over the blocking steps
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
        if (i < n) {
            const double gl = x[i] - B.xlo[i], gu = B.xhi[i] - x[i];
            const double igl = rcp_pos(gl), igu = rcp_pos(gu);
            const double d = dx[i];
            const double a = mu * igl - zl[i] - (zl[i] * igl) * d;
            const double b = mu * igu - zu[i] + (zu[i] * igu) * d;
            dzl[i] = a;
            dzu[i] = b;
            if (is_pos(-d)) apr.add(tau * gl, -d);   // sign tests on the bit patterns
            if (is_pos(d)) apr.add(tau * gu, d);
            if (is_pos(-a)) adu.add(tau * zl[i], -a);
            if (is_pos(-b)) adu.add(tau * zu[i], -b);
            v[2] += (grad[i] - mu * igl + mu * igu) * d;
        } else if (relaxed) {
            const int k = i - n;
            const double hl = s[k] + B.tau, hu = B.tau - s[k];
            const double ihl = rcp_pos(hl), ihu = rcp_pos(hu);
            const double sig = vl[k] * ihl + vu[k] * ihu;
            const double gphi = -mu * ihl + mu * ihu;
            const double d = (dy[k] - gphi + y[k]) * rcp_pos(sig);
            ds[k] = d;
            const double a = mu * ihl - vl[k] - (vl[k] * ihl) * d;
            const double b = mu * ihu - vu[k] + (vu[k] * ihu) * d;
            dvl[k] = a;
            dvu[k] = b;
            if (is_pos(-d)) apr.add(tau * hl, -d);
            if (is_pos(d)) apr.add(tau * hu, d);
            if (is_pos(-a)) adu.add(tau * vl[k], -a);
            if (is_pos(-b)) adu.add(tau * vu[k], -b);
            v[2] += gphi * d;
        }
    }
    v[0] = apr.value();
    v[1] = adu.value();
    store_partials<3>(v, ops, part, count, out);
}

// Trial point at step alpha, or at *alpha_dev when it is given (the first
// trial: the fraction-to-the-boundary step the recovery left on the device).
__global__ void trial_kernel(int n, int m, int relaxed, double alpha, const double* __restrict__ alpha_dev,
                             const double* __restrict__ x, const double* __restrict__ dx,
                             const double* __restrict__ s, const double* __restrict__ ds,
                             double* __restrict__ xt, double* __restrict__ st) {
    if (alpha_dev) alpha = *alpha_dev;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
        if (i < n) xt[i] = x[i] + alpha * dx[i];
        else if (relaxed) st[i - n] = s[i - n] + alpha * ds[i - n];
    }
}

// Filter measures at a point: partials [theta = sum |c - s|, sum log(gaps)].
__global__ void __launch_bounds__(kT)
measure_kernel(int n, int m, int relaxed, Bounds B, const double* __restrict__ x,
               const double* __restrict__ s, const double* __restrict__ c, double* __restrict__ part,
               unsigned* count, double* __restrict__ out) {
    double v[2] = {0.0, 0.0};
    const int ops[2] = {SUM, SUM};
    LogSum ls;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
        if (i < n) {
            ls.add(x[i] - B.xlo[i]);
            ls.add(B.xhi[i] - x[i]);
        } else {
            const int k = i - n;
            v[0] += fabs(relaxed ? c[k] - s[k] : c[k]);
            if (relaxed) {
                ls.add(s[k] + B.tau);
                ls.add(B.tau - s[k]);
            }
        }
    }
    v[1] = ls.value();
    store_partials<2>(v, ops, part, count, out);
}

__global__ void accept_kernel(int n, int m, int relaxed, Bounds B, double mu, double alpha,
                              double alpha_du, double* __restrict__ x, double* __restrict__ s,
                              double* __restrict__ y, double* __restrict__ zl,
                              double* __restrict__ zu, double* __restrict__ vl,
                              double* __restrict__ vu, const double* __restrict__ dx,
                              const double* __restrict__ ds, const double* __restrict__ dy,
                              const double* __restrict__ dzl, const double* __restrict__ dzu,
                              const double* __restrict__ dvl, const double* __restrict__ dvu) {
    const double k = kKappaSigma;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
        if (i < n) {
            const double xn = x[i] + alpha * dx[i];
            x[i] = xn;
            const double igl = rcp_pos(xn - B.xlo[i]), igu = rcp_pos(B.xhi[i] - xn);
            const double a = zl[i] + alpha_du * dzl[i], b = zu[i] + alpha_du * dzu[i];
            zl[i] = max_nonneg(min_nonneg(a, k * mu * igl), (mu / k) * igl);
            zu[i] = max_nonneg(min_nonneg(b, k * mu * igu), (mu / k) * igu);
        } else {
            const int q = i - n;
            y[q] += alpha * dy[q];
            if (relaxed) {
                const double sn = s[q] + alpha * ds[q];
                s[q] = sn;
                const double ihl = rcp_pos(sn + B.tau), ihu = rcp_pos(B.tau - sn);
                const double a = vl[q] + alpha_du * dvl[q], b = vu[q] + alpha_du * dvu[q];
                vl[q] = max_nonneg(min_nonneg(a, k * mu * ihl), (mu / k) * ihl);
                vu[q] = max_nonneg(min_nonneg(b, k * mu * ihu), (mu / k) * ihu);
            }
        }
    }
}

int grid(long long w) {
    long long g = (w + kT - 1) / kT;
    return (int)std::max<long long>(1, std::min<long long>(g, 152LL * 8));
}

}  // namespace

struct kkt_ipm {
    kkt_ipm_options opt{};
    double params[16];
    int n = 0, m = 0, nnzW = 0, nnzJ = 0;
    kkt_ctx* kkt = nullptr;
    std::string err;
    std::vector<void*> allocs;
    // device state
    double *x, *s, *y, *zl, *zu, *vl, *vu, *xlo, *xhi;
    double *grad, *c, *Jv, *Wv, *jty, *sigma, *rx, *ry, *D;
    double *dx, *dy, *ds, *dzl, *dzu, *dvl, *dvu, *xt, *st, *ct;
    double *part, *red, *f;
    unsigned* count;   // last-CTA counter of the reduction kernels (zero between launches)
    int *jt_cp, *jt_ri, *jt_idx;
    double* h_red = nullptr;   // pinned
    double* x0v = nullptr;     // per-tray initial state (device, k), NULL: x0bar
    double* x0buf = nullptr;
    long long dev_bytes = 0;   // device memory of this driver (the KKT context's excluded)
    // host state
    double mu = 0.1, theta_max = 0, theta_min = 0, delta_last = 0;
    std::vector<std::pair<double, double>> filter;
    int it = 0;
    int launches = 0;   // kernels launched by the driver in the current step
    bool started = false;
    bool graph_step = false;   // FP64 supernodal context: step 4 is one kkt_factor_solve graph launch
    cudaEvent_t ev[4] = {};
    // the iteration in progress: its report, the objective at its start,
    // and whether the report is complete (a result to hand back)
    kkt_ipm_info cur{};
    double fval = 0.0;
    bool report = false;
    // the filter line search in progress: step lengths, directional
    // derivative, theta and barrier function at the current point, the
    // trial step and the trials made
    double a_pr = 0, a_du = 0, dphi = 0, th = 0, ph = 0, alpha = 0;
    int ls = 0;
    int trial_slot = 0;   // red[] slot of the trial being judged
};

namespace {

kkt_status ierr(kkt_ipm* p, kkt_status st, const std::string& msg) {
    if (p) p->err = msg;
    return st;
}

#define ICUDA(p, call)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return ierr(p, e_ == cudaErrorMemoryAllocation ? KKT_ERR_OOM : KKT_ERR_CUDA,   \
                        std::string(#call) + ": " + cudaGetErrorString(e_));              \
    } while (0)

template <class T>
kkt_status dalloc(kkt_ipm* p, T** out, size_t count) {
    ICUDA(p, cudaMalloc((void**)out, std::max<size_t>(1, count) * sizeof(T)));
    p->allocs.push_back(*out);
    p->dev_bytes += (long long)(std::max<size_t>(1, count) * sizeof(T));
    return KKT_OK;
}

#define ITRY(x)                       \
    do {                              \
        kkt_status s_ = (x);          \
        if (s_ != KKT_OK) return s_;  \
    } while (0)

Bounds bounds_of(const kkt_ipm* p) { return Bounds{p->xlo, p->xhi, p->opt.tau_relax}; }

// Each phase of an iteration enqueues its kernels, whose reductions leave
// their results in slots of red, then one copy of the first nq slots to the
// pinned h_red; the host reads them after one synchronisation of the stream
// (shared by all members of a batch).
kkt_status fetch_red(kkt_ipm* p, int nq, cudaStream_t st) {
    ICUDA(p, cudaMemcpyAsync(p->h_red, p->red, nq * sizeof(double), cudaMemcpyDeviceToHost, st));
    return KKT_OK;
}

// objective at w via partials in part[b * kQ + kQ - 1] and the final reduce
// into red[slot]
kkt_status objective(kkt_ipm* p, const double* w, cudaStream_t st, int slot) {
    if (!kktgb::tray_objective_partials(p->params, w, p->part + (kQ - 1), kQ, kRB, st))
        return ierr(p, KKT_ERR_CUDA, "objective kernel launch failed");
    final_sum_kernel<<<1, 32, 0, st>>>(p->part + (kQ - 1), p->red + slot);
    p->launches += 2;
    return KKT_OK;
}

struct Errors {
    double du, pr, zg_max, zg_min, sum_y, sum_z;
};

double err_mu(const kkt_ipm* p, const Errors& e, double mu) {
    const int n = p->n, m = p->m;
    const bool rel = p->opt.relaxed;
    const double cnt_mult = m + 2.0 * n + (rel ? 2.0 * m : 0.0);
    const double cnt_z = 2.0 * n + (rel ? 2.0 * m : 0.0);
    const double s_d = std::max(kSMax, (e.sum_y + e.sum_z) / cnt_mult) / kSMax;
    const double s_c = std::max(kSMax, e.sum_z / cnt_z) / kSMax;
    const double compl_mu = std::max(e.zg_max - mu, mu - e.zg_min);
    return std::max(std::max(e.du / s_d, e.pr), compl_mu / s_c);
}

// constraint violation theta and the barrier log-sum at (x, s) into
// red[slot], red[slot + 1]
void measures(kkt_ipm* p, const double* x, const double* s, const double* c, cudaStream_t st, int slot) {
    measure_kernel<<<kRB, kT, 0, st>>>(p->n, p->m, p->opt.relaxed, bounds_of(p), x, s, c, p->part, p->count,
                                       p->red + slot);
    p->launches += 1;
}

// theta at the current point, on the host (one synchronisation)
kkt_status theta_now(kkt_ipm* p, cudaStream_t st, double* th) {
    measures(p, p->x, p->s, p->c, st, 0);
    ITRY(fetch_red(p, 2, st));
    ICUDA(p, cudaStreamSynchronize(st));
    *th = p->h_red[0];
    return KKT_OK;
}

}  // namespace

extern "C" {

void kkt_ipm_default_options(kkt_ipm_options* o) {
    if (!o) return;
    o->tol = 1e-8;
    o->max_iter = 200;
    o->mu_init = 0.1;
    o->relaxed = -1;   // decided from the scheme
    o->tau_relax = 1e-8;
}

namespace {
// own_kkt = false: a member of a kkt_ipm_batch -- no KKT context, and the
// KKT inputs and outputs (Wv, Jv, sigma, rx, ry, D, dx, dy) are slices of
// the batch's concatenated arrays, set by the batch.
kkt_status create_impl(const double* params, const kkt_options* kopt, const kkt_ipm_options* iopt,
                       bool own_kkt, kkt_ipm** out) {
    if (!params || !out) return KKT_ERR_ARG;
    *out = nullptr;
    kkt_ipm* p = new (std::nothrow) kkt_ipm();
    if (!p) return KKT_ERR_OOM;
    std::copy(params, params + 16, p->params);
    if (iopt) p->opt = *iopt; else kkt_ipm_default_options(&p->opt);
    kkt_options ko;
    if (kopt) ko = *kopt; else kkt_default_options(&ko);
    if (p->opt.relaxed < 0) p->opt.relaxed = ko.scheme == KKT_LIFTED ? 1 : 0;
    if (p->opt.relaxed && ko.scheme != KKT_LIFTED) {
        delete p;
        return KKT_ERR_ARG;
    }
    ko.target_relaxed = p->opt.relaxed ? 1 : 0;
    if (!(p->opt.tol > 0 && p->opt.mu_init > 0 && p->opt.tau_relax > 0)) {
        delete p;
        return KKT_ERR_ARG;
    }
    kkt_status stt = kkt_tray_sizes(params, &p->n, &p->m, &p->nnzW, &p->nnzJ);
    if (stt != KKT_OK) {
        delete p;
        return stt;
    }
    const int n = p->n, m = p->m;
    std::vector<int> Wc(n + 1), Wr(p->nnzW), Jr(m + 1), Jc(p->nnzJ);
    kkt_tray_pattern(params, Wc.data(), Wr.data(), Jr.data(), Jc.data());
    if (own_kkt) {
        stt = kkt_analyse(n, m, Wc.data(), Wr.data(), Jr.data(), Jc.data(), &ko, &p->kkt);
        if (stt != KKT_OK) {
            delete p;
            return stt;
        }
        p->graph_step = ko.precision == 0 && ko.solver == 0;
    }
    // CSC of J for J^T y
    std::vector<int> cp(n + 1, 0), ri(p->nnzJ), idx(p->nnzJ);
    for (int q = 0; q < p->nnzJ; ++q) cp[Jc[q] + 1]++;
    for (int i = 0; i < n; ++i) cp[i + 1] += cp[i];
    {
        std::vector<int> fillp(cp.begin(), cp.end() - 1);
        for (int r = 0; r < m; ++r)
            for (int q = Jr[r]; q < Jr[r + 1]; ++q) {
                ri[fillp[Jc[q]]] = r;
                idx[fillp[Jc[q]]++] = q;
            }
    }
    // bounds: 0 <= x, y <= 1 (x_lo, x_hi), 1 <= u <= 5 (u_lo, u_hi), stage-major
    const int k = (int)params[0];
    std::vector<double> lo(n), hi(n);
    for (int i = 0; i < n; ++i) {
        const bool is_u = (i % (2 * k + 1)) == 2 * k;
        lo[i] = is_u ? params[14] : params[12];
        hi[i] = is_u ? params[15] : params[13];
    }
    auto fail = [&](kkt_status s) {
        kkt_ipm_destroy(p);
        return s;
    };
    double** vecs_n[] = {&p->x, &p->zl, &p->zu, &p->xlo, &p->xhi, &p->grad, &p->jty, &p->dzl, &p->dzu, &p->xt};
    for (double** v : vecs_n)
        if (dalloc(p, v, n) != KKT_OK) return fail(KKT_ERR_OOM);
    double** vecs_m[] = {&p->s, &p->y, &p->vl, &p->vu, &p->c, &p->ds, &p->dvl, &p->dvu, &p->st, &p->ct};
    for (double** v : vecs_m)
        if (dalloc(p, v, m) != KKT_OK) return fail(KKT_ERR_OOM);
    if (own_kkt) {
        double** kn[] = {&p->sigma, &p->rx, &p->dx};
        for (double** v : kn)
            if (dalloc(p, v, n) != KKT_OK) return fail(KKT_ERR_OOM);
        double** km[] = {&p->ry, &p->D, &p->dy};
        for (double** v : km)
            if (dalloc(p, v, m) != KKT_OK) return fail(KKT_ERR_OOM);
        if (dalloc(p, &p->Jv, p->nnzJ) != KKT_OK || dalloc(p, &p->Wv, p->nnzW) != KKT_OK)
            return fail(KKT_ERR_OOM);
    }
    if (dalloc(p, &p->part, (size_t)kRB * kQ) != KKT_OK || dalloc(p, &p->red, kQ) != KKT_OK ||
        dalloc(p, &p->f, 1) != KKT_OK || dalloc(p, &p->count, 1) != KKT_OK ||
        dalloc(p, &p->jt_cp, n + 1) != KKT_OK || dalloc(p, &p->jt_ri, p->nnzJ) != KKT_OK ||
        dalloc(p, &p->jt_idx, p->nnzJ) != KKT_OK)
        return fail(KKT_ERR_OOM);
    if (cudaMemcpy(p->jt_cp, cp.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->jt_ri, ri.data(), p->nnzJ * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->jt_idx, idx.data(), p->nnzJ * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->xlo, lo.data(), n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->xhi, hi.data(), n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(p->count, 0, sizeof(unsigned)) != cudaSuccess)
        return fail(KKT_ERR_CUDA);
    if (cudaMallocHost((void**)&p->h_red, kQ * sizeof(double)) != cudaSuccess) return fail(KKT_ERR_OOM);
    for (auto& e : p->ev)
        if (cudaEventCreate(&e) != cudaSuccess) return fail(KKT_ERR_CUDA);
    *out = p;
    return KKT_OK;
}
}  // namespace

kkt_status kkt_ipm_create(const double* params, const kkt_options* kopt, const kkt_ipm_options* iopt,
                          kkt_ipm** out) {
    return create_impl(params, kopt, iopt, true, out);
}

kkt_status kkt_ipm_init(kkt_ipm* p, const double* d_x0, cudaStream_t st) {
    if (!p) return KKT_ERR_ARG;
    const int n = p->n, m = p->m;
    if (d_x0) {
        ICUDA(p, cudaMemcpyAsync(p->x, d_x0, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
        const int k = (int)p->params[0];
        std::vector<double> x0(n);
        for (int i = 0; i < n; ++i) x0[i] = (i % (2 * k + 1)) == 2 * k ? p->params[9] : p->params[11];
        ICUDA(p, cudaMemcpyAsync(p->x, x0.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
        ICUDA(p, cudaStreamSynchronize(st));
    }
    push_kernel<<<grid(n), kT, 0, st>>>(n, p->xlo, p->xhi, 0, 0, p->x);
    fill_kernel<<<grid(m), kT, 0, st>>>(m, 0.0, p->y);
    fill_kernel<<<grid(n), kT, 0, st>>>(n, 1.0, p->zl);
    fill_kernel<<<grid(n), kT, 0, st>>>(n, 1.0, p->zu);
    if (p->opt.relaxed) {
        ITRY(kktgb::tray_eval(p->params, p->x0v, p->x, nullptr, 1.0, nullptr, nullptr, p->s, nullptr, nullptr, st));
        push_kernel<<<grid(m), kT, 0, st>>>(m, nullptr, nullptr, -p->opt.tau_relax, p->opt.tau_relax, p->s);
        fill_kernel<<<grid(m), kT, 0, st>>>(m, 1.0, p->vl);
        fill_kernel<<<grid(m), kT, 0, st>>>(m, 1.0, p->vu);
    }
    ITRY(kktgb::tray_eval(p->params, p->x0v, p->x, nullptr, 1.0, nullptr, nullptr, p->c, nullptr, nullptr, st));
    double th = 0;
    ITRY(theta_now(p, st, &th));
    p->theta_max = 1e4 * std::max(1.0, th);
    p->theta_min = 1e-4 * std::max(1.0, th);
    p->mu = p->opt.mu_init;
    p->filter.clear();
    p->delta_last = 0.0;
    p->it = 0;
    p->started = true;
    ICUDA(p, cudaGetLastError());
    return KKT_OK;
}

namespace {

// Steps 1-3 of an iteration, split where the host needs reduction results:
// begin_issue enqueues the derivatives, the optimality-error reduction
// (red[0..5]) and the objective (red[6]) with their copy to the host;
// begin_finish, after the stream is synchronised, updates the barrier
// parameter and enqueues the right-hand side and diagonals.  KKT_CONVERGED
// when the optimality error is <= tol; the iteration's report accumulates
// in p->cur.
kkt_status begin_issue(kkt_ipm* p, cudaStream_t st) {
    const int n = p->n, m = p->m;
    const int rel = p->opt.relaxed;
    const Bounds B = bounds_of(p);
    kkt_ipm_info& inf = p->cur;
    inf = kkt_ipm_info{};
    inf.iter = p->it;
    p->launches = 0;
    cudaEventRecord(p->ev[0], st);
    // 1. derivatives
    ITRY(kktgb::tray_eval(p->params, p->x0v, p->x, p->y, 1.0, nullptr, p->grad, p->c, p->Jv, p->Wv, st));
    jt_kernel<<<grid(n), kT, 0, st>>>(n, p->jt_cp, p->jt_ri, p->jt_idx, p->Jv, p->y, p->jty);
    p->launches += 2;
    cudaEventRecord(p->ev[1], st);
    // 2. optimality error and objective
    errors_kernel<<<kRB, kT, 0, st>>>(n, m, rel, B, p->x, p->s, p->y, p->zl, p->zu, p->vl, p->vu,
                                      p->grad, p->jty, p->c, p->part, p->count, p->red);
    p->launches += 1;
    ITRY(objective(p, p->x, st, 6));
    return fetch_red(p, 7, st);
}

kkt_status begin_finish(kkt_ipm* p, cudaStream_t st) {
    const int n = p->n, m = p->m;
    const int rel = p->opt.relaxed;
    const Bounds B = bounds_of(p);
    kkt_ipm_info& inf = p->cur;
    const double* h = p->h_red;
    Errors E{h[0], h[1], h[2], h[3], h[4], h[5]};
    const double fval = h[6];
    const double e0 = err_mu(p, E, 0.0);
    inf.objective = fval;
    inf.inf_du = E.du;
    inf.inf_pr = E.pr;
    inf.inf_compl = std::max(std::fabs(E.zg_max), std::fabs(E.zg_min));
    inf.err0 = e0;
    inf.mu = p->mu;
    if (e0 <= p->opt.tol) {
        inf.launches = p->launches;
        p->report = true;
        return KKT_CONVERGED;
    }
    while (p->mu > p->opt.tol / 10) {
        if (err_mu(p, E, p->mu) > kKappaEps * p->mu) break;
        p->mu = std::max(p->opt.tol / 10, std::min(kKappaMu * p->mu, std::pow(p->mu, kThetaMu)));
        p->filter.clear();
    }
    const double mu = p->mu;
    inf.mu = mu;
    p->fval = fval;
    // 3. right-hand side and diagonals
    prepare_kernel<<<grid((long long)n + m), kT, 0, st>>>(n, m, rel, B, mu, p->x, p->s, p->y, p->zl,
                                                        p->zu, p->vl, p->vu, p->grad, p->jty, p->c,
                                                        p->sigma, p->rx, p->ry, p->D);
    p->launches += 1;
    return KKT_OK;
}

// Step 4 with the context's own KKT system: factor with the inertia-
// correction ladder, then the refined solve -- with the FP64 supernodal
// factor both as one graph launch (kkt_factor_solve: the refinement sweeps
// run as a conditional loop on the device, one host wait), otherwise as
// kkt_factor then kkt_solve.
kkt_status step_kkt(kkt_ipm* p, cudaStream_t st) {
    kkt_ipm_info& inf = p->cur;
    const int rel = p->opt.relaxed;
    // 4. factor with inertia correction, solve
    kkt_info ki{};
    double delta = 0.0;
    kkt_status fs;
    while (true) {
        if (p->graph_step)
            fs = kkt_factor_solve(p->kkt, p->Wv, p->Jv, p->sigma, rel ? p->D : nullptr, &delta, p->rx, p->ry,
                                  p->dx, p->dy, st, &ki);
        else
            fs = kkt_factor(p->kkt, p->Wv, p->Jv, p->sigma, rel ? p->D : nullptr, delta, st, &ki);
        if (fs == KKT_OK || (p->graph_step && (fs == KKT_ERR_MAXIT || fs == KKT_ERR_STALL))) break;
        if (fs != KKT_ERR_NOT_SPD) return ierr(p, fs, std::string("kkt_factor: ") + kkt_last_error(p->kkt));
        if (delta == 0.0)
            delta = p->delta_last == 0.0 ? kDeltaW0 : std::max(kDeltaMin, kKappaWMinus * p->delta_last);
        else
            delta *= p->delta_last == 0.0 ? kKappaWPlusBar : kKappaWPlus;
        if (delta > kDeltaMax) return ierr(p, KKT_ERR_NOT_SPD, "inertia correction gave up");
    }
    if (delta > 0) p->delta_last = delta;
    inf.delta_x = delta;
    if (!p->graph_step) {
        kkt_status ss = kkt_solve(p->kkt, p->rx, p->ry, p->dx, p->dy, nullptr, st, &ki);
        if (ss != KKT_OK && ss != KKT_ERR_MAXIT && ss != KKT_ERR_STALL)
            return ierr(p, ss, std::string("kkt_solve: ") + kkt_last_error(p->kkt));
    }
    inf.refine_iters = ki.refine_iters;
    inf.cg_iters = ki.cg_iters;
    inf.bwd_err = ki.bwd_err;
    return KKT_OK;
}

// Steps 5-7, split the same way: end_issue enqueues the recovery with the
// fraction-to-the-boundary steps and the directional derivative (red[0..2]),
// the measures at the current point (red[3..4]) and the first trial of the
// line search, whose step alpha_pr the recovery leaves in red[0] (its
// measures in red[5..6], its objective in red[7]); end_search_begin reads
// them and starts the filter line search.  Each further trial enqueues its
// point, model values, measures (red[0..1]) and objective (red[2])
// (trial_issue); a trial is judged after the synchronisation (trial_judge:
// 1 accepted, 0 try the halved step, -1 no trial left); accept_issue
// enqueues the update, and step_done closes the iteration once the stream
// has completed it.
constexpr int kFirstTrial = 5;   // red[] slot of the first trial's measures

// point, model values, measures into red[slot], red[slot + 1] and objective
// into red[slot + 2] of the trial at step alpha (or *alpha_dev)
kkt_status trial_enqueue(kkt_ipm* p, cudaStream_t st, const double* alpha_dev, int slot) {
    const int n = p->n, m = p->m;
    const int rel = p->opt.relaxed;
    trial_kernel<<<grid((long long)n + m), kT, 0, st>>>(n, m, rel, p->alpha, alpha_dev, p->x, p->dx, p->s, p->ds,
                                                      p->xt, p->st);
    p->launches += 1;
    ITRY(kktgb::tray_eval(p->params, p->x0v, p->xt, nullptr, 1.0, nullptr, nullptr, p->ct, nullptr, nullptr, st));
    p->launches += 1;
    measures(p, p->xt, p->st, p->ct, st, slot);
    return objective(p, p->xt, st, slot + 2);
}

kkt_status end_issue(kkt_ipm* p, cudaStream_t st) {
    const int n = p->n, m = p->m;
    const int rel = p->opt.relaxed;
    const Bounds B = bounds_of(p);
    const double mu = p->mu;
    cudaEventRecord(p->ev[2], st);
    // 5. recovery, fraction to boundary, directional derivative
    const double tau = std::max(kTauMin, 1.0 - mu);
    recover_kernel<<<kRB, kT, 0, st>>>(n, m, rel, B, mu, tau, p->x, p->s, p->y, p->zl, p->zu, p->vl,
                                       p->vu, p->grad, p->dx, p->dy, p->ds, p->dzl, p->dzu, p->dvl,
                                       p->dvu, p->part, p->count, p->red);
    p->launches += 1;
    measures(p, p->x, p->s, p->c, st, 3);
    ITRY(trial_enqueue(p, st, p->red, kFirstTrial));
    return fetch_red(p, kFirstTrial + 3, st);
}

void end_search_begin(kkt_ipm* p) {
    const double* h = p->h_red;
    p->a_pr = h[0];
    p->a_du = h[1];
    p->dphi = h[2];
    p->th = h[3];
    p->ph = p->fval - p->mu * h[4];
    p->alpha = p->a_pr;
    p->ls = 1;   // the first trial is in flight with the recovery
    p->trial_slot = kFirstTrial;
}

// 6. filter line search: the next trial step (after the first)
kkt_status trial_issue(kkt_ipm* p, cudaStream_t st) {
    ++p->ls;
    p->trial_slot = 0;
    ITRY(trial_enqueue(p, st, nullptr, 0));
    return fetch_red(p, 3, st);
}

int trial_judge(kkt_ipm* p) {
    const double* h = p->h_red + p->trial_slot;
    const double tht = h[0], pht = h[2] - p->mu * h[1];
    const double th = p->th, ph = p->ph, alpha = p->alpha, dphi = p->dphi;
    bool ok = tht <= p->theta_max;
    for (const auto& fe : p->filter)
        if (!(tht < fe.first || pht < fe.second)) { ok = false; break; }
    bool f_type = false;
    if (ok) {
        const bool switching = dphi < 0 && alpha * std::pow(-dphi, kSPhi) > kDelta * std::pow(th, kSTheta);
        if (th <= p->theta_min && switching) {
            ok = pht <= ph + kEtaPhi * alpha * dphi;
            f_type = true;
        } else {
            ok = tht <= (1 - kGammaTheta) * th || pht <= ph - kGammaPhi * th;
        }
    }
    if (ok) {
        if (!f_type) p->filter.emplace_back((1 - kGammaTheta) * th, ph - kGammaPhi * th);
        return 1;
    }
    p->alpha *= 0.5;
    return p->ls >= kMaxLs ? -1 : 0;
}

kkt_status search_failed(kkt_ipm* p) {
    p->cur.ls_trials = p->ls + 1;
    p->cur.launches = p->launches;
    p->report = true;
    return ierr(p, KKT_ERR_STALL, "line search failed (no restoration phase)");
}

// 7. update
void accept_issue(kkt_ipm* p, cudaStream_t st) {
    const int n = p->n, m = p->m;
    const int rel = p->opt.relaxed;
    const Bounds B = bounds_of(p);
    p->cur.ls_trials = p->ls;
    accept_kernel<<<grid((long long)n + m), kT, 0, st>>>(n, m, rel, B, p->mu, p->alpha, p->a_du, p->x, p->s,
                                                       p->y, p->zl, p->zu, p->vl, p->vu, p->dx,
                                                       p->ds, p->dy, p->dzl, p->dzu, p->dvl, p->dvu);
    p->launches += 1;
    cudaEventRecord(p->ev[3], st);
}

kkt_status step_done(kkt_ipm* p) {
    kkt_ipm_info& inf = p->cur;
    ICUDA(p, cudaEventSynchronize(p->ev[3]));
    float t01 = 0, t12 = 0, t03 = 0;
    cudaEventElapsedTime(&t01, p->ev[0], p->ev[1]);
    cudaEventElapsedTime(&t12, p->ev[1], p->ev[2]);
    cudaEventElapsedTime(&t03, p->ev[0], p->ev[3]);
    inf.t_eval_ms = t01;
    inf.t_kkt_ms = t12;
    inf.t_step_ms = t03;
    inf.alpha_pr = p->alpha;
    inf.alpha_du = p->a_du;
    p->it++;
    inf.iter = p->it;
    ICUDA(p, cudaGetLastError());
    inf.launches = p->launches;
    p->report = true;
    return KKT_OK;
}

// Steps 1-3 and 5-7 of one problem, each phase followed by its own
// synchronisation.
kkt_status step_begin(kkt_ipm* p, cudaStream_t st) {
    ITRY(begin_issue(p, st));
    ICUDA(p, cudaStreamSynchronize(st));
    return begin_finish(p, st);
}

kkt_status step_end(kkt_ipm* p, cudaStream_t st) {
    ITRY(end_issue(p, st));
    ICUDA(p, cudaStreamSynchronize(st));
    end_search_begin(p);
    while (true) {
        const int v = trial_judge(p);
        if (v > 0) break;
        if (v < 0) return search_failed(p);
        ITRY(trial_issue(p, st));
        ICUDA(p, cudaStreamSynchronize(st));
    }
    accept_issue(p, st);
    return step_done(p);
}

}  // namespace

kkt_status kkt_ipm_step(kkt_ipm* p, cudaStream_t st, kkt_ipm_info* info) {
    if (!p) return KKT_ERR_ARG;
    if (!p->started) return ierr(p, KKT_ERR_STATE, "kkt_ipm_step before kkt_ipm_init");
    if (!p->kkt) return ierr(p, KKT_ERR_STATE, "a member of a kkt_ipm_batch steps with the batch");
    p->report = false;
    kkt_status r = step_begin(p, st);
    if (r == KKT_OK) r = step_kkt(p, st);
    if (r == KKT_OK) r = step_end(p, st);
    if (info && p->report) *info = p->cur;
    return r;
}

kkt_status kkt_ipm_solve(kkt_ipm* p, cudaStream_t st, kkt_ipm_info* info) {
    if (!p) return KKT_ERR_ARG;
    kkt_ipm_info last{};
    for (int k = 0; k <= p->opt.max_iter; ++k) {
        const kkt_status s = kkt_ipm_step(p, st, &last);
        if (s != KKT_OK) {
            if (info) *info = last;
            return s;
        }
    }
    if (info) *info = last;
    return ierr(p, KKT_ERR_MAXIT, "kkt_ipm_solve: max_iter reached");
}

// stage t of the new start takes stage t + 1 of the previous solution; the
// last stage keeps its own values
__global__ void shift_stages_kernel(int n, int nst, const double* __restrict__ prev, double* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = i + nst < n ? prev[i + nst] : prev[i];
}

kkt_status kkt_ipm_set_initial_state(kkt_ipm* p, const double* x0, cudaStream_t st) {
    if (!p) return KKT_ERR_ARG;
    const int k = (int)p->params[0];
    if (!x0) {
        p->x0v = nullptr;
        return KKT_OK;
    }
    for (int i = 0; i < k; ++i)
        if (!std::isfinite(x0[i])) return ierr(p, KKT_ERR_ARG, "initial state is not finite");
    if (!p->x0buf) ITRY(dalloc(p, &p->x0buf, k));
    ICUDA(p, cudaMemcpyAsync(p->x0buf, x0, k * sizeof(double), cudaMemcpyHostToDevice, st));
    ICUDA(p, cudaStreamSynchronize(st));
    p->x0v = p->x0buf;
    return KKT_OK;
}

kkt_status kkt_ipm_init_shifted(kkt_ipm* p, const double* d_prev, cudaStream_t st) {
    if (!p || !d_prev) return KKT_ERR_ARG;
    const int nst = 2 * (int)p->params[0] + 1;
    shift_stages_kernel<<<grid(p->n), kT, 0, st>>>(p->n, nst, d_prev, p->xt);
    ICUDA(p, cudaGetLastError());
    return kkt_ipm_init(p, p->xt, st);
}

// shift a stage-major vector by one stage in place (through scratch)
static kkt_status shift_in_place(kkt_ipm* p, int len, int stride, double* v, double* scratch, cudaStream_t st) {
    shift_stages_kernel<<<grid(len), kT, 0, st>>>(len, stride, v, scratch);
    copy_kernel<<<grid(len), kT, 0, st>>>(len, scratch, v);
    ICUDA(p, cudaGetLastError());
    return KKT_OK;
}

// bound multipliers centred on the barrier parameter: z_L = mu / (x - lo),
// z_U = mu / (hi - x) (infinite bounds: 0) -- the slack-multiplier
// products start on the central path
__global__ void center_kernel(int n, const double* __restrict__ x, const double* __restrict__ lo,
                              const double* __restrict__ hi, double clo, double chi, double mu,
                              double* __restrict__ zl, double* __restrict__ zu) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double l = lo ? lo[i] : clo, h = hi ? hi[i] : chi;
        zl[i] = mu / fmax(x[i] - l, 1e-300);
        zu[i] = mu / fmax(h - x[i], 1e-300);
    }
}

kkt_status kkt_ipm_init_warm(kkt_ipm* p, double mu, int recenter, cudaStream_t st) {
    if (!p) return KKT_ERR_ARG;
    if (!p->started) return ierr(p, KKT_ERR_STATE, "kkt_ipm_init_warm needs a previous solve");
    if (!(mu > 0 && std::isfinite(mu))) return ierr(p, KKT_ERR_ARG, "bad mu");
    const int n = p->n, m = p->m, k = (int)p->params[0];
    const int nst = 2 * k + 1, mst = 2 * k;
    ITRY(shift_in_place(p, n, nst, p->x, p->xt, st));
    ITRY(shift_in_place(p, n, nst, p->zl, p->xt, st));
    ITRY(shift_in_place(p, n, nst, p->zu, p->xt, st));
    ITRY(shift_in_place(p, m, mst, p->y, p->ct, st));
    push_kernel<<<grid(n), kT, 0, st>>>(n, p->xlo, p->xhi, 0, 0, p->x);
    if (p->opt.relaxed) {
        ITRY(shift_in_place(p, m, mst, p->s, p->ct, st));
        ITRY(shift_in_place(p, m, mst, p->vl, p->ct, st));
        ITRY(shift_in_place(p, m, mst, p->vu, p->ct, st));
        push_kernel<<<grid(m), kT, 0, st>>>(m, nullptr, nullptr, -p->opt.tau_relax, p->opt.tau_relax, p->s);
    }
    if (recenter) {
        center_kernel<<<grid(n), kT, 0, st>>>(n, p->x, p->xlo, p->xhi, 0, 0, mu, p->zl, p->zu);
        if (p->opt.relaxed)
            center_kernel<<<grid(m), kT, 0, st>>>(m, p->s, nullptr, nullptr, -p->opt.tau_relax,
                                                  p->opt.tau_relax, mu, p->vl, p->vu);
    }
    ITRY(kktgb::tray_eval(p->params, p->x0v, p->x, nullptr, 1.0, nullptr, nullptr, p->c, nullptr, nullptr, st));
    double th = 0;
    ITRY(theta_now(p, st, &th));
    p->theta_max = 1e4 * std::max(1.0, th);
    p->theta_min = 1e-4 * std::max(1.0, th);
    p->mu = mu;
    p->filter.clear();
    p->delta_last = 0.0;
    p->it = 0;
    ICUDA(p, cudaGetLastError());
    return KKT_OK;
}

kkt_status kkt_ipm_device_bytes(const kkt_ipm* p, int64_t* bytes) {
    if (!p || !bytes) return KKT_ERR_ARG;
    int64_t kb = 0;
    if (p->kkt) {   // a batch member's KKT system belongs to the batch
        kkt_status s = kkt_device_bytes(p->kkt, &kb);
        if (s != KKT_OK) return s;
    }
    *bytes = kb + p->dev_bytes;
    return KKT_OK;
}

kkt_status kkt_ipm_get(const kkt_ipm* p, double* d_x, double* d_y, double* d_zl, double* d_zu,
                       double* d_s, cudaStream_t st) {
    if (!p) return KKT_ERR_ARG;
    const int n = p->n, m = p->m;
    if (d_x) copy_kernel<<<grid(n), kT, 0, st>>>(n, p->x, d_x);
    if (d_y) copy_kernel<<<grid(m), kT, 0, st>>>(m, p->y, d_y);
    if (d_zl) copy_kernel<<<grid(n), kT, 0, st>>>(n, p->zl, d_zl);
    if (d_zu) copy_kernel<<<grid(n), kT, 0, st>>>(n, p->zu, d_zu);
    if (d_s && p->opt.relaxed) copy_kernel<<<grid(m), kT, 0, st>>>(m, p->s, d_s);
    if (cudaStreamSynchronize(st) != cudaSuccess) return KKT_ERR_CUDA;
    return KKT_OK;
}

kkt_ctx* kkt_ipm_kkt(kkt_ipm* p) { return p ? p->kkt : nullptr; }

void kkt_ipm_destroy(kkt_ipm* p) {
    if (!p) return;
    for (auto& e : p->ev)
        if (e) cudaEventDestroy(e);
    for (void* a : p->allocs) cudaFree(a);
    if (p->h_red) cudaFreeHost(p->h_red);
    if (p->kkt) kkt_destroy(p->kkt);
    delete p;
}


// ---------------------------------------------------------------- batches
// Lock-step IPMs over many column problems with one KKT system: every
// member keeps its own iterate, barrier parameter, filter and line search
// (steps 1-3 and 5-7 above, unchanged), while step 4 factorises and solves
// the block-diagonal union of the members' KKT systems in one call (the
// batch context of kkt_analyse_batch; one graph launch in FP64, or the FP32
// factor with FP64 refinement).  The members' KKT inputs and outputs are
// slices of the batch's concatenated arrays, so nothing is copied.  Each
// phase enqueues the kernels of every member on the one stream and then
// synchronises once, so a tick costs the same few host round trips however
// many members step.  Members start and stop independently (continuous
// batching): one that does not step is switched off in the factorisation
// (kkt_batch_set_active) and has a zero right-hand side, so it costs no
// factorisation work and its refinement stops at once.
}  // extern "C"

struct kkt_ipm_batch {
    int count = 0;
    std::vector<kkt_ipm*> mem;
    kkt_ctx* kkt = nullptr;
    std::vector<void*> allocs;
    double *Wv = nullptr, *Jv = nullptr, *sigma = nullptr, *rx = nullptr, *ry = nullptr, *D = nullptr,
           *dx = nullptr, *dy = nullptr;
    std::vector<int> state;      // KKT_OK while a member iterates, else its final status
    std::vector<char> stepping;  // members in the current iteration's KKT step
    std::vector<double> delta;   // delta_x of every member's block in the last factor
    std::vector<int> fcol;       // scratch: failing columns of the last factor
    std::vector<char> searching; // scratch: members whose line search goes on
    // reduced precision (kopt precision 1 or 2): members whose solve saw the
    // union fall back to FP64; while one of them steps, the union is
    // factorised in FP64 directly (later iterations only widen Sigma)
    std::vector<char> fell_back;
    int precision = 0;
    bool relaxed = false, graph = false;
    long long dev_bytes = 0;     // the union's value and vector arrays
    long long kkt_steps = 0, factor_calls = 0;
    std::string err;
};

namespace {
kkt_status berr(kkt_ipm_batch* b, kkt_status st, const std::string& msg) {
    if (b) b->err = msg;
    return st;
}
#define TRY_B(b, x)                   \
    do {                              \
        kkt_status s_ = (x);          \
        if (s_ != KKT_OK) return s_;  \
    } while (0)
}  // namespace

extern "C" {

kkt_status kkt_ipm_batch_create(int count, const double* params, const kkt_options* kopt,
                                const kkt_ipm_options* iopt, kkt_ipm_batch** out) {
    if (count < 1 || !params || !out) return KKT_ERR_ARG;
    *out = nullptr;
    kkt_ipm_batch* b = new (std::nothrow) kkt_ipm_batch();
    if (!b) return KKT_ERR_OOM;
    auto fail = [&](kkt_status st) {
        kkt_ipm_batch_destroy(b);
        return st;
    };
    b->count = count;
    b->mem.assign(count, nullptr);
    for (int i = 0; i < count; ++i) {
        kkt_status st = create_impl(params + 16 * (size_t)i, kopt, iopt, false, &b->mem[i]);
        if (st != KKT_OK) return fail(st);
    }
    kkt_options ko;
    if (kopt) ko = *kopt; else kkt_default_options(&ko);
    b->relaxed = b->mem[0]->opt.relaxed != 0;
    ko.target_relaxed = b->relaxed ? 1 : 0;
    b->graph = ko.precision == 0 && ko.solver == 0;
    b->precision = ko.solver == 0 ? ko.precision : 0;
    std::vector<int> n(count), m(count);
    std::vector<std::vector<int>> Wc(count), Wr(count), Jr(count), Jc(count);
    std::vector<const int*> pWc(count), pWr(count), pJr(count), pJc(count);
    long long N = 0, M = 0, NW = 0, NJ = 0;
    for (int i = 0; i < count; ++i) {
        kkt_ipm* p = b->mem[i];
        n[i] = p->n;
        m[i] = p->m;
        Wc[i].resize(p->n + 1);
        Wr[i].resize(std::max(1, p->nnzW));
        Jr[i].resize(p->m + 1);
        Jc[i].resize(std::max(1, p->nnzJ));
        kkt_tray_pattern(p->params, Wc[i].data(), Wr[i].data(), Jr[i].data(), Jc[i].data());
        pWc[i] = Wc[i].data();
        pWr[i] = Wr[i].data();
        pJr[i] = Jr[i].data();
        pJc[i] = Jc[i].data();
        N += p->n;
        M += p->m;
        NW += p->nnzW;
        NJ += p->nnzJ;
    }
    kkt_status st = kkt_analyse_batch(count, n.data(), m.data(), pWc.data(), pWr.data(), pJr.data(), pJc.data(),
                                      &ko, &b->kkt);
    if (st != KKT_OK) return fail(st);
    // zero values, unit diagonals: a member that never stepped has the
    // identity block and a zero right-hand side
    auto dal = [&](double** v, long long cnt, double fillv) {
        const long long c1 = std::max<long long>(1, cnt);
        if (cudaMalloc((void**)v, c1 * sizeof(double)) != cudaSuccess) return false;
        b->allocs.push_back(*v);
        b->dev_bytes += c1 * (long long)sizeof(double);
        std::vector<double> h((size_t)c1, fillv);
        return cudaMemcpy(*v, h.data(), c1 * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
    };
    if (!dal(&b->Wv, NW, 0.0) || !dal(&b->Jv, NJ, 0.0) || !dal(&b->sigma, N, 1.0) || !dal(&b->rx, N, 0.0) ||
        !dal(&b->dx, N, 0.0) || !dal(&b->ry, M, 0.0) || !dal(&b->D, M, 1.0) || !dal(&b->dy, M, 0.0))
        return fail(KKT_ERR_OOM);
    // the union concatenates the members in order: variables, constraints,
    // W and J values
    long long xo = 0, yo = 0, wo = 0, jo = 0;
    for (int i = 0; i < count; ++i) {
        kkt_ipm* p = b->mem[i];
        p->Wv = b->Wv + wo;
        p->Jv = b->Jv + jo;
        p->sigma = b->sigma + xo;
        p->rx = b->rx + xo;
        p->dx = b->dx + xo;
        p->ry = b->ry + yo;
        p->D = b->D + yo;
        p->dy = b->dy + yo;
        xo += p->n;
        yo += p->m;
        wo += p->nnzW;
        jo += p->nnzJ;
    }
    std::vector<int> lx(count + 1), ly(count + 1);
    st = kkt_batch_layout(b->kkt, nullptr, lx.data(), ly.data());
    if (st != KKT_OK) return fail(st);
    long long cx = 0, cy = 0;
    for (int i = 0; i < count; ++i) {
        if (lx[i] != cx || ly[i] != cy) return fail(berr(b, KKT_ERR_INTERNAL, "batch layout mismatch"));
        cx += n[i];
        cy += m[i];
    }
    b->state.assign(count, (int)KKT_ERR_STATE);
    b->stepping.assign(count, 0);
    b->searching.assign(count, 0);
    b->fell_back.assign(count, 0);
    b->delta.assign(count, 0.0);
    b->fcol.assign(count, -1);
    *out = b;
    return KKT_OK;
}

kkt_status kkt_ipm_batch_start(kkt_ipm_batch* b) {
    if (!b) return KKT_ERR_ARG;
    for (int i = 0; i < b->count; ++i) {
        if (!b->mem[i]->started) return berr(b, KKT_ERR_STATE, "member " + std::to_string(i) + " not initialised");
        b->state[i] = KKT_OK;
    }
    return KKT_OK;
}

kkt_status kkt_ipm_batch_start_member(kkt_ipm_batch* b, int i) {
    if (!b || i < 0 || i >= b->count) return KKT_ERR_ARG;
    if (!b->mem[i]->started) return berr(b, KKT_ERR_STATE, "member " + std::to_string(i) + " not initialised");
    if (b->state[i] == KKT_OK) return berr(b, KKT_ERR_STATE, "member " + std::to_string(i) + " is iterating");
    b->state[i] = KKT_OK;
    return KKT_OK;
}

kkt_status kkt_ipm_batch_member_status(const kkt_ipm_batch* b, int i, int* status, int* iters) {
    if (!b || i < 0 || i >= b->count) return KKT_ERR_ARG;
    if (status) *status = b->state[i];
    if (iters) *iters = b->mem[i]->it;
    return KKT_OK;
}

kkt_status kkt_ipm_batch_device_bytes(const kkt_ipm_batch* b, int64_t* bytes) {
    if (!b || !bytes) return KKT_ERR_ARG;
    int64_t total = b->dev_bytes, x = 0;
    for (const kkt_ipm* p : b->mem) {
        kkt_ipm_device_bytes(p, &x);
        total += x;
    }
    if (kkt_device_bytes(b->kkt, &x) == KKT_OK) total += x;
    *bytes = total;
    return KKT_OK;
}

kkt_status kkt_ipm_batch_step(kkt_ipm_batch* b, cudaStream_t st, kkt_ipm_info* info) {
    if (!b) return KKT_ERR_ARG;
    const int cnt = b->count;
    auto sync = [&]() -> kkt_status {
        const cudaError_t e = cudaStreamSynchronize(st);
        return e == cudaSuccess ? KKT_OK : berr(b, KKT_ERR_CUDA, std::string("batch step: ") + cudaGetErrorString(e));
    };
    auto stop = [&](int i, kkt_status r) {
        b->stepping[i] = 0;
        b->searching[i] = 0;
        b->fell_back[i] = 0;
        b->state[i] = r;
        if (info && b->mem[i]->report) info[i] = b->mem[i]->cur;
    };
    // steps 1-3 of every member still iterating
    for (int i = 0; i < cnt; ++i) {
        b->stepping[i] = 0;
        if (b->state[i] != KKT_OK) continue;
        kkt_ipm* p = b->mem[i];
        p->report = false;
        const kkt_status r = begin_issue(p, st);
        if (r == KKT_OK)
            b->stepping[i] = 1;
        else
            stop(i, r);
    }
    TRY_B(b, sync());
    int running = 0;
    for (int i = 0; i < cnt; ++i) {
        if (!b->stepping[i]) continue;
        const kkt_status r = begin_finish(b->mem[i], st);
        if (r == KKT_OK)
            ++running;
        else
            stop(i, r);
    }
    if (running == 0) return KKT_CONVERGED;
    // members that do not step keep their last block; a zero right-hand side
    // ends their refinement at once
    for (int i = 0; i < cnt; ++i) {
        if (b->stepping[i]) continue;
        const kkt_ipm* p = b->mem[i];
        if (cudaMemsetAsync(p->rx, 0, (size_t)p->n * sizeof(double), st) != cudaSuccess ||
            cudaMemsetAsync(p->ry, 0, (size_t)p->m * sizeof(double), st) != cudaSuccess)
            return berr(b, KKT_ERR_CUDA, "batch step: clearing an idle member's right-hand side");
    }
    // step 4 for all of them at once: the inertia-correction ladder per
    // member (a member whose block fails raises its own delta_x); members
    // that do not step are switched off (no factorisation work; their zero
    // right-hand side solves to zero)
    std::vector<double> d(cnt);
    for (int i = 0; i < cnt; ++i) d[i] = b->stepping[i] ? 0.0 : b->delta[i];
    if (cnt > 1) {
        std::vector<int> on(b->stepping.begin(), b->stepping.end());
        const kkt_status as = kkt_batch_set_active(b->kkt, on.data());
        if (as != KKT_OK) return berr(b, as, std::string("batch step: ") + kkt_last_error(b->kkt));
    }
    if (b->precision != 0) {
        bool fp64 = false;
        for (int i = 0; i < cnt; ++i) fp64 = fp64 || (b->stepping[i] && b->fell_back[i]);
        const kkt_status ps = kkt_set_precision(b->kkt, fp64 ? 0 : b->precision);
        if (ps != KKT_OK) return berr(b, ps, std::string("batch step: ") + kkt_last_error(b->kkt));
    }
    kkt_info ki{};
    while (true) {
        kkt_status fs;
        if (b->graph) {
            fs = kkt_factor_solve(b->kkt, b->Wv, b->Jv, b->sigma, b->relaxed ? b->D : nullptr, d.data(), b->rx, b->ry,
                                  b->dx, b->dy, st, &ki);
        } else {
            fs = kkt_factor_batch(b->kkt, b->Wv, b->Jv, b->sigma, b->relaxed ? b->D : nullptr, d.data(), st, &ki);
        }
        ++b->factor_calls;
        if (fs != KKT_OK && fs != KKT_ERR_NOT_SPD && fs != KKT_ERR_MAXIT && fs != KKT_ERR_STALL)
            return berr(b, fs, std::string("batch KKT step: ") + kkt_last_error(b->kkt));
        kkt_status rs = kkt_batch_results(b->kkt, nullptr, nullptr, nullptr, nullptr, b->fcol.data());
        if (rs != KKT_OK) return berr(b, rs, "kkt_batch_results");
        bool again = false;
        for (int i = 0; i < cnt; ++i) {
            if (b->fcol[i] < 0 || !b->stepping[i]) continue;
            kkt_ipm* p = b->mem[i];
            if (d[i] == 0.0)
                d[i] = p->delta_last == 0.0 ? kDeltaW0 : std::max(kDeltaMin, kKappaWMinus * p->delta_last);
            else
                d[i] *= p->delta_last == 0.0 ? kKappaWPlusBar : kKappaWPlus;
            if (d[i] > kDeltaMax) {   // this member gives up; the others go on
                stop(i, ierr(p, KKT_ERR_NOT_SPD, "inertia correction gave up"));
                --running;
            } else {
                again = true;
            }
        }
        if (!again) break;
    }
    bool fell = ki.status_detail == 2;   // a reduced-precision pivot failed: refactorised in FP64
    if (!b->graph && running > 0) {
        const kkt_status ss = kkt_solve(b->kkt, b->rx, b->ry, b->dx, b->dy, nullptr, st, &ki);
        fell = fell || ki.status_detail == 2;   // the refinement did not reach its tolerance
        if (ss != KKT_OK && ss != KKT_ERR_MAXIT && ss != KKT_ERR_STALL && ss != KKT_ERR_NOT_SPD)
            return berr(b, ss, std::string("batch kkt_solve: ") + kkt_last_error(b->kkt));
    }
    ++b->kkt_steps;
    if (b->precision != 0 && fell)   // this iteration fell back to FP64
        for (int i = 0; i < cnt; ++i)
            if (b->stepping[i]) b->fell_back[i] = 1;
    std::vector<int> ref(cnt), cg(cnt);
    std::vector<double> eta(cnt);
    kkt_status rs = kkt_batch_results(b->kkt, nullptr, ref.data(), cg.data(), eta.data(), nullptr);
    if (rs != KKT_OK) return berr(b, rs, "kkt_batch_results");
    // steps 5-7 per member: recovery, then line-search rounds in which every
    // member still searching tries its next step, then the updates
    for (int i = 0; i < cnt; ++i) {
        if (!b->stepping[i]) continue;
        kkt_ipm* p = b->mem[i];
        b->delta[i] = d[i];
        if (d[i] > 0) p->delta_last = d[i];
        p->cur.delta_x = d[i];
        p->cur.refine_iters = ref[i];
        p->cur.cg_iters = cg[i];
        p->cur.bwd_err = eta[i];
        const kkt_status r = end_issue(p, st);
        if (r != KKT_OK) stop(i, r);
    }
    TRY_B(b, sync());
    int searching = 0;
    for (int i = 0; i < cnt; ++i) {
        b->searching[i] = b->stepping[i];
        if (!b->stepping[i]) continue;
        end_search_begin(b->mem[i]);
        ++searching;
    }
    while (searching > 0) {
        // judge the trials in flight (the first came with the recovery)
        for (int i = 0; i < cnt; ++i) {
            if (!b->searching[i]) continue;
            const int v = trial_judge(b->mem[i]);
            if (v > 0) {
                b->searching[i] = 0;
                --searching;
            } else if (v < 0) {
                stop(i, search_failed(b->mem[i]));
                --searching;
            }
        }
        if (searching == 0) break;
        for (int i = 0; i < cnt; ++i) {
            if (!b->searching[i]) continue;
            const kkt_status r = trial_issue(b->mem[i], st);
            if (r != KKT_OK) {
                stop(i, r);
                --searching;
            }
        }
        TRY_B(b, sync());
    }
    for (int i = 0; i < cnt; ++i)
        if (b->stepping[i]) accept_issue(b->mem[i], st);
    for (int i = 0; i < cnt; ++i) {
        if (!b->stepping[i]) continue;
        kkt_ipm* p = b->mem[i];
        const kkt_status r = step_done(p);
        if (r != KKT_OK) {
            stop(i, r);
            continue;
        }
        if (info) info[i] = p->cur;
        if (p->it > p->opt.max_iter) b->state[i] = KKT_ERR_MAXIT;
    }
    return KKT_OK;
}

kkt_status kkt_ipm_batch_solve(kkt_ipm_batch* b, cudaStream_t st, int* status, int* iters,
                               kkt_ipm_info* info) {
    if (!b) return KKT_ERR_ARG;
    TRY_B(b, kkt_ipm_batch_start(b));
    int max_iter = 0;
    for (kkt_ipm* p : b->mem) max_iter = std::max(max_iter, p->opt.max_iter);
    kkt_status r = KKT_OK;
    for (int k = 0; k <= max_iter + 1; ++k) {
        r = kkt_ipm_batch_step(b, st, info);
        if (r != KKT_OK) break;
    }
    if (r != KKT_OK && r != KKT_CONVERGED) return r;
    kkt_status out = KKT_CONVERGED;
    for (int i = 0; i < b->count; ++i) {
        if (b->state[i] == KKT_OK) b->state[i] = KKT_ERR_MAXIT;
        if (status) status[i] = b->state[i];
        if (iters) iters[i] = b->mem[i]->it;
        if (b->state[i] != KKT_CONVERGED && out == KKT_CONVERGED) out = (kkt_status)b->state[i];
    }
    return out;
}

kkt_ipm* kkt_ipm_batch_member(kkt_ipm_batch* b, int i) {
    return b && i >= 0 && i < b->count ? b->mem[i] : nullptr;
}

kkt_ctx* kkt_ipm_batch_kkt(kkt_ipm_batch* b) { return b ? b->kkt : nullptr; }

const char* kkt_ipm_batch_last_error(const kkt_ipm_batch* b) { return b ? b->err.c_str() : ""; }

void kkt_ipm_batch_destroy(kkt_ipm_batch* b) {
    if (!b) return;
    for (kkt_ipm* p : b->mem)
        if (p) kkt_ipm_destroy(p);
    for (void* a : b->allocs) cudaFree(a);
    if (b->kkt) kkt_destroy(b->kkt);
    delete b;
}

}  // extern "C"
