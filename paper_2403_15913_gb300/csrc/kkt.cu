// C ABI of the GB300 KKT library: symbolic analysis, numeric factorisation
// and the two hybrid solves of Pacaud & Shin (arXiv 2403.15913, Sec. IV-V).
#include "kkt.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "bcr_kernels.cuh"
#include "df64.cuh"
#include "kernels.cuh"
#include "symbolic.h"

using namespace kktgb;

// ---------------------------------------------------------------------------
// Allocation-free backsolve.  The permuted work vector lives in a file-scope
// device array; host code must not use the symbol's name as a pointer (it is
// a host-side stand-in), so its device address is looked up once per device,
// with that device current, when a context is set up on it (kkt_analyse):
// that lookup is also what places the array on the device, so the
// allocation-free call itself takes no device memory and touches no module
// loading.
static __device__ __align__(256) double g_noalloc_scratch[KKT_STATIC_SCRATCH_DOUBLES];


namespace {

constexpr long long kSmemCapElems = (200 * 1024) / 8;   // panel kept in smem up to 200 KB
constexpr int kBackwardSmemBytes = 192 * 1024;   // backward level solve: diagonal block + staged x
constexpr size_t kStagedSmemBytes = 96 * 1024;   // staged level solves: panel (+ x and indices below)
constexpr size_t kFlowSmemBytes = 100 * 1024;    // dataflow solves: widest staged panel (+ x and indices below)
constexpr int kSyrkStageBytes = 96 * 1024;       // split-level SYRK: L21 staged in shared memory
constexpr int kClusterLevelMax = 32;             // split levels this small run as one cluster launch
constexpr int kClusterSmemBytes = 96 * 1024;     // its diagonal block / staged L21
constexpr int kNumSMs = 152;   // GB300
constexpr int kSplitLevel = 2 * kNumSMs;   // levels with fewer supernodes use split launches

template <class T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
};

}  // namespace

struct kkt_ctx {
    kkt_options opt{};
    std::string err;
    int n = 0, m = 0, nnzW = 0, nnzJ = 0;
    Symbolic sym;
    // host copies of the plan (for exports and launches)
    std::vector<int> h_sn_f, h_sn_c, h_sn_r, h_sn_rptr;
    std::vector<long long> h_sn_lptr;
    std::vector<int> h_lvl_ptr, h_lvl_sn;
    std::vector<int> lvl_max_c;
    std::vector<int> lvl_max_rb;
    std::vector<long long> lvl_max_rc;
    // levels with few supernodes are factorised by split POTRF/TRSM/SYRK
    // launches over these task lists (per level offsets into the arrays)
    std::vector<char> lvl_split;
    std::vector<int> lvl_trsm_ptr, lvl_syrk_ptr;
    int2* d_trsm_tasks = nullptr;
    int4* d_syrk_tasks = nullptr;

    double* d_dinv = nullptr;
    long long panel = 0;
    long long nk = 0;
    int nlev = 0;          // levels of the supernodes outside small-subtree tasks
    int tree_levels = 0;   // levels of the whole supernodal tree
    // small-subtree tasks: supernodes of task b are task_sn[task_ptr[b] ..]
    int ntasks = 0;
    int* d_task_ptr = nullptr;
    int* d_task_sn = nullptr;
    int n_norm = 0;               // supernodes normalised after the factorisation
    int* d_norm_list = nullptr;
    // levels factorised by the fused kernels (FP64 and FP32 panels; every
    // level of supernodes with <= kFusedMaxC columns and <= kFusedMaxRb rows
    // below, wide or split), and the normalisation list that leaves their
    // supernodes out
    std::vector<char> lvl_fused;
    // co-resident clusters of factor_fused_cluster_kernel for K = 2, 4, 8
    // CTAs (index log2 K; 0 = not queried): a level takes K only if all its
    // clusters run in one wave
    int fused_clusters[4] = {0, 0, 0, 0};
    int n_norm_fused = 0;
    int* d_norm_list_fused = nullptr;
    long long task_max_rc = 0, task_max_cc = 0, task_max_ccrb = 0;
    long long task_max_cols = 0;   // widest column range of a subtree task (its slice of x in the solves)
    // dataflow triangular solves (staged_solve = 2): work items in
    // topological order, the item each one feeds and its number of feeders,
    // arrival counters, epochs and tickets; the mapped host word a wait that
    // gave up sets; shared memory bounds and launch grids per precision
    // (0 double, 1 float, 2 double-float) and direction (0 forward)
    bool flow = false;
    int flow_items = 0;
    int *d_flow_item = nullptr, *d_flow_up = nullptr, *d_flow_nchild = nullptr, *d_flow_cnt = nullptr;
    int* d_flow_nchild_lv = nullptr;   // feeders among the level supernodes only (staged_solve = 3)
    unsigned *d_flow_done = nullptr, *d_flow_ctrl = nullptr;
    int* h_flow_err = nullptr;   // pinned, mapped
    int* d_flow_err = nullptr;   // its device address
    long long flow_fwd_elems = 0, flow_bwd_elems = 0, flow_bwd_ints = 0;
    int flow_grid[3][2] = {};
    // device allocations (all freed in kkt_destroy) and their total size
    std::vector<void*> allocs;
    long long dev_bytes = 0;
    Plan plan{};
    int* d_lvl_sn = nullptr;
    int *d_perm = nullptr, *d_iperm = nullptr;
    long long *d_k_slot = nullptr, *d_k_sptr = nullptr;
    int2* d_k_src = nullptr;
    int *d_wf_ptr = nullptr, *d_wf_col = nullptr, *d_wf_idx = nullptr;
    int *d_j_ptr = nullptr, *d_j_col = nullptr;
    int *d_jt_ptr = nullptr, *d_jt_row = nullptr, *d_jt_idx = nullptr;
    double* d_Lx = nullptr;
    int* d_fail = nullptr;
    // work vectors
    double *w_xp = nullptr, *w_t = nullptr, *w_r = nullptr, *w_d = nullptr;
    double *w_q = nullptr, *w_p = nullptr, *w_sp = nullptr, *w_res = nullptr, *w_cgx = nullptr;
    double *w_rg = nullptr, *w_tn = nullptr;
    // private copies of the values of the last kkt_factor (residuals of the
    // following solves read them, so callers may free their buffers)
    double *v_W = nullptr, *v_J = nullptr, *v_sigma = nullptr, *v_D = nullptr;
    double* v_Js = nullptr;     // J scaled by sqrt(D) for the assembly
    // FP32 factor (precision = 1): panels, reciprocal pivots, permuted vector
    float *d_Lx32 = nullptr, *d_dinv32 = nullptr, *w_xp32 = nullptr;
    // precision of the current factor: 0 FP64, 1 FP32, 2 double-float (kept
    // in the FP64 buffers: a float pair is 8 bytes); the graphs of the
    // reduced precision (1 or 2) are tri_exec32 / cg_exec32
    int cur_prec = 0;
    // factor inputs of the last kkt_factor
    bool factored = false;
    const double *f_W = nullptr, *f_J = nullptr, *f_sigma = nullptr, *f_D = nullptr;
    double f_delta_x = 0.0, f_Dconst = 0.0;
    double knorm = 0.0;
    const double* f_C = nullptr;   // dual block of the target system (device) or NULL
    DevBuf<double> d_Cbuf;
    bool device_ready = false;   // false for host-only analyses
    int analysed_precision = 0;  // opt.precision at the analysis (its storage exists)
    // device address of the allocation-free backsolve's static scratch,
    // looked up when the context is set up (null with noalloc_err set if
    // the lookup failed)
    double* noalloc_ptr = nullptr;
    std::string noalloc_err;
    // bounds-check error word (device) and the test hook's map entry
    int* d_berr = nullptr;
    long long dbg_relmap_pos = -1;
    int dbg_relmap_bad = 0, dbg_relmap_old = 0;
    bool dbg_corrupted = false;
    bool dbg_flow_raised = false;
    // CUDA graphs captured once after the analysis: the triangular solves on
    // w_xp, and one HyKKT CG iteration on the internal CG vectors
    cudaGraph_t tri_graph = nullptr, cg_graph = nullptr, tri_graph32 = nullptr, cg_graph32 = nullptr;
    cudaGraphExec_t tri_exec = nullptr, cg_exec = nullptr, tri_exec32 = nullptr, cg_exec32 = nullptr;
    size_t tri_nodes = 0, cg_nodes = 0, tri_nodes32 = 0, cg_nodes32 = 0;
    int* d_cg = nullptr;        // [some instance's CG active, unused]
    int* h_cg = nullptr;        // pinned
    // Block-diagonal batch of nb independent systems (nb = 1 for a single
    // one): instance i owns primal rows [xoff[i], xoff[i+1]) and dual rows
    // [yoff[i], yoff[i+1]).  Reductions run over chunks of rows of one
    // instance: d_ch_xy covers the n + m rows (the nch_x primal chunks
    // first), d_ch_y the m dual rows, instance i owning dual chunks
    // [chy_ptr[i], chy_ptr[i+1]).
    int nb = 1;
    std::vector<int> h_xoff, h_yoff, h_chy_ptr;
    int4 *d_ch_xy = nullptr, *d_ch_y = nullptr;
    int nch_xy = 0, nch_x = 0, nch_y = 0;
    int* d_chy_ptr = nullptr;
    int* d_col_inst = nullptr;   // instance of every permuted column (nb > 1)
    int* d_sn_inst = nullptr;    // instance of every supernode (nb > 1)
    int* d_inst_on = nullptr;    // per-instance factorisation switch (nb > 1; all on by default)
    int* h_inst_on = nullptr;    // pinned: the switch kkt_batch_set_active gave
    bool inst_on_pending = false;   // h_inst_on not yet copied to d_inst_on
    double* d_knorm = nullptr;   // ||K_orig,i||_inf per instance
    double* d_red = nullptr;     // residual maxima, 3 per instance
    int* d_act = nullptr;        // instances whose refinement still runs
    double* d_cgs = nullptr;     // CG scalars, 4 per instance
    int* d_cgi = nullptr;        // CG active flag and iterations, 2 per instance
    double* d_part_y = nullptr;  // partial sums, one per dual chunk
    double* d_dvec = nullptr;    // per-variable delta_x of a batch factor
    double* d_dval = nullptr;    // per-instance delta_x
    const double* f_dvec = nullptr;   // d_dvec when the last factor used it
    double* h_red = nullptr;     // pinned: 3 nb residual maxima
    int* h_act = nullptr;        // pinned: nb
    int* h_int = nullptr;        // pinned: 2 nb
    std::vector<double> h_knorm, h_delta;
    // per-instance results of the last factor / solve
    std::vector<int> r_status, r_refine, r_cg, r_fail;
    std::vector<double> r_eta;
    // side stream: ||K_orig||_inf is computed while the factorisation runs
    cudaStream_t side = nullptr;
    cudaEvent_t ev_in = nullptr, ev_side = nullptr;
    // block cyclic reduction (opt.solver == 1): N blocks of b variables;
    // level l eliminates bcr_elim[elim_ptr[l] ..] then updates the survivors
    // bcr_surv[surv_ptr[l] ..]; the last level eliminates the root alone
    int bcr_b = 0, bcr_N = 0, bcr_nlev = 0;
    std::vector<int> bcr_elim_ptr, bcr_surv_ptr;
    int4 *d_bcr_elim = nullptr, *d_bcr_surv = nullptr;
    double* d_bcr = nullptr;     // A blocks then C blocks (2 N b^2)
    double* d_bcr_pn = nullptr;  // factor panels (3 N b^2)
    long long bcr_nk = 0;
    long long *d_bcr_slot = nullptr, *d_bcr_sptr = nullptr;
    int2* d_bcr_src = nullptr;
    double bcr_flops = 0.0;
    // tracing
    bool profiling = false;
    kkt_stats stats{};
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    struct Span {
        cudaEvent_t a, b;
        int kind;   // 0 assemble, 1 factor, 2 solve, 3 other
    };
    std::vector<Span> spans;
    // one-graph factor + refined solve (kkt_factor_solve): the graph, the
    // device pointers it was captured with, its capture streams (main,
    // refinement body, CG body) and external event nodes (factor start,
    // factor end, end); device refinement state; pinned results; kernel
    // launches per replay (before the loop, per sweep, per CG iteration)
    bool capturing = false;   // enqueue solves directly, no nested graph launch
    cudaGraph_t step_graph = nullptr;
    cudaGraphExec_t step_exec = nullptr;
    const void* step_key[9] = {};
    cudaStream_t cap[3] = {};
    cudaEvent_t step_ev[4] = {};   // start, factor end, end, assembly end (factor kernels start)
    int* d_rst = nullptr;       // 4 per instance (state, stalled, sweeps, CG iterations)
    double* d_reta = nullptr;   // 2 per instance (eta, previous eta)
    int* d_rctl = nullptr;      // next sweep, CG iterations run
    int* h_rst = nullptr;       // pinned: rst (4 nb), fail (nb), ctl (2)
    double* h_reta = nullptr;   // pinned: reta (2 nb), knorm (nb)
    double* hp_delta = nullptr; // pinned: delta_x per instance
    long long step_pre = 0, step_sweep = 0, step_cgit = 0, step_fl = 0;
};

namespace {

constexpr int kCgBatch = 8;   // CG iterations enqueued between convergence checks

thread_local std::string g_err;   // last error of calls that have no context

kkt_status set_err(kkt_ctx* c, kkt_status st, const std::string& msg) {
    if (c) c->err = msg;
    else g_err = msg;
    return st;
}

#define CUDA_TRY(ctx, call)                                                              \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return set_err(ctx, e_ == cudaErrorMemoryAllocation ? KKT_ERR_OOM : KKT_ERR_CUDA, \
                           std::string(#call) + ": " + cudaGetErrorString(e_));          \
    } while (0)

template <class T>
kkt_status upload(kkt_ctx* c, T** dst, const std::vector<T>& src) {
    size_t bytes = std::max<size_t>(1, src.size()) * sizeof(T);
    CUDA_TRY(c, cudaMalloc((void**)dst, bytes));
    c->allocs.push_back(*dst);
    c->dev_bytes += (long long)bytes;
    if (!src.empty()) CUDA_TRY(c, cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    return KKT_OK;
}

template <class T>
kkt_status alloc(kkt_ctx* c, T** dst, size_t count) {
    CUDA_TRY(c, cudaMalloc((void**)dst, std::max<size_t>(1, count) * sizeof(T)));
    c->allocs.push_back(*dst);
    c->dev_bytes += (long long)(std::max<size_t>(1, count) * sizeof(T));
    return KKT_OK;
}

#define TRY(x)                         \
    do {                               \
        kkt_status s_ = (x);           \
        if (s_ != KKT_OK) return s_;   \
    } while (0)

int grid_for(long long work) {
    long long g = (work + kThreads - 1) / kThreads;
    return (int)std::max<long long>(1, std::min<long long>(g, 152LL * 16));
}

// ------------------------------------------------------------- tracing
cudaEvent_t next_event(kkt_ctx* c) {
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        c->ev_pool.push_back(e);
    }
    return c->ev_pool[c->ev_used++];
}

// returns an open span index or -1
int span_begin(kkt_ctx* c, int kind, cudaStream_t st) {
    if (!c->profiling) return -1;
    cudaEvent_t a = next_event(c), b = next_event(c);
    if (!a || !b) return -1;
    cudaEventRecord(a, st);
    c->spans.push_back({a, b, kind});
    return (int)c->spans.size() - 1;
}

void span_end(kkt_ctx* c, int idx, cudaStream_t st) {
    if (idx >= 0) cudaEventRecord(c->spans[idx].b, st);
}

// after a stream synchronisation: accumulate and recycle the events
void spans_collect(kkt_ctx* c) {
    for (auto& sp : c->spans) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, sp.a, sp.b) != cudaSuccess) continue;
        double* dst = sp.kind == 0 ? &c->stats.assemble_ms
                      : sp.kind == 1 ? &c->stats.factor_ms
                      : sp.kind == 2 ? &c->stats.solve_ms : &c->stats.other_ms;
        *dst += ms;
    }
    c->spans.clear();
    c->ev_used = 0;
}

// Plan of the block cyclic reduction: dense-block assembly map (every entry
// of K lands in A[t] (both triangles) or in C[t] = K[t, t-1]), level
// schedule, flop count.  Rejects patterns that are not block tridiagonal.
kkt_status build_bcr(kkt_ctx* c, const int* W_colptr, const int* W_rowind, const int* J_rowptr,
                     const int* J_colind) {
    const int n = c->n, m = c->m, b = c->opt.block;
    if (c->nb != 1) return set_err(c, KKT_ERR_ARG, "block-tridiagonal solver: single instance only");
    if (c->opt.precision != 0) return set_err(c, KKT_ERR_ARG, "block-tridiagonal solver: FP64 only");
    if (b < 1 || b > kBcrMaxBlock || n % b != 0)
        return set_err(c, KKT_ERR_ARG, "block-tridiagonal solver: block must divide n and be <= " +
                                           std::to_string(kBcrMaxBlock));
    const int N = n / b;
    const long long bb = (long long)b * b;
    struct E {
        long long slot;
        int a, bsrc;
    };
    std::vector<E> ents;
    bool ok = true;
    auto put = [&](int i, int j, int a, int bs) {   // K[i, j] += source, i >= j in value
        const int ti = i / b, tj = j / b;
        if (ti == tj) {
            ents.push_back({(long long)ti * bb + (i % b) + (long long)(j % b) * b, a, bs});
            if (i != j) ents.push_back({(long long)ti * bb + (j % b) + (long long)(i % b) * b, a, bs});
        } else if (ti == tj + 1) {
            ents.push_back({(long long)(N + ti) * bb + (i % b) + (long long)(j % b) * b, a, bs});
        } else if (tj == ti + 1) {
            ents.push_back({(long long)(N + tj) * bb + (j % b) + (long long)(i % b) * b, a, bs});
        } else {
            ok = false;
        }
    };
    for (int col = 0; col < n; ++col)
        for (int p = W_colptr[col]; p < W_colptr[col + 1]; ++p) put(W_rowind[p], col, p, -1);
    for (int v = 0; v < n; ++v) put(v, v, v, -2);
    for (int r = 0; r < m && ok; ++r)
        for (int p = J_rowptr[r]; p < J_rowptr[r + 1]; ++p)
            for (int q = p; q < J_rowptr[r + 1]; ++q) put(J_colind[p], J_colind[q], p, q);
    if (!ok) return set_err(c, KKT_ERR_ARG, "block-tridiagonal solver: K is not block tridiagonal for block " +
                                                std::to_string(b));
    std::stable_sort(ents.begin(), ents.end(), [](const E& x, const E& y) { return x.slot < y.slot; });
    std::vector<long long> slot, sptr;
    std::vector<int2> src;
    src.reserve(ents.size());
    for (size_t q = 0; q < ents.size(); ++q) {
        if (q == 0 || ents[q].slot != ents[q - 1].slot) {
            slot.push_back(ents[q].slot);
            sptr.push_back((long long)q);
        }
        src.push_back(make_int2(ents[q].a, ents[q].bsrc));
    }
    sptr.push_back((long long)ents.size());
    // level schedule: eliminate the even positions of the active chain
    std::vector<int> active(N);
    for (int t = 0; t < N; ++t) active[t] = t;
    std::vector<int4> elim, surv;
    c->bcr_elim_ptr.assign(1, 0);
    c->bcr_surv_ptr.assign(1, 0);
    double fl = 0.0;
    const double b3 = (double)b * b * b;
    while (true) {
        const int A = (int)active.size();
        std::vector<int> next;
        for (int q = 0; q < A; ++q) {
            const int prev = q > 0 ? active[q - 1] : -1, nxt = q + 1 < A ? active[q + 1] : -1;
            if (A == 1 || q % 2 == 0) {
                elim.push_back(make_int4(active[q], prev, nxt, 0));
                const int nb2 = (prev >= 0) + (nxt >= 0);
                // POTRF, TRSM of the neighbour rows, fill GEMM, neighbour updates
                fl += b3 / 3.0 + b3 * nb2 + (prev >= 0 && nxt >= 0 ? 2.0 * b3 : 0.0) + 2.0 * b3 * nb2;
            } else {
                surv.push_back(make_int4(active[q], prev, nxt, 0));
                next.push_back(active[q]);
            }
        }
        c->bcr_elim_ptr.push_back((int)elim.size());
        c->bcr_surv_ptr.push_back((int)surv.size());
        if (A == 1) break;
        active.swap(next);
    }
    c->bcr_nlev = (int)c->bcr_elim_ptr.size() - 1;
    c->bcr_b = b;
    c->bcr_N = N;
    c->bcr_flops = fl;
    c->bcr_nk = (long long)slot.size();
    TRY(upload(c, &c->d_bcr_elim, elim));
    TRY(upload(c, &c->d_bcr_surv, surv));
    TRY(upload(c, &c->d_bcr_slot, slot));
    TRY(upload(c, &c->d_bcr_sptr, sptr));
    TRY(upload(c, &c->d_bcr_src, src));
    TRY(alloc(c, &c->d_bcr, (size_t)2 * N * bb));
    TRY(alloc(c, &c->d_bcr_pn, (size_t)3 * N * bb));
    return KKT_OK;
}

// Build the device plan from the symbolic analysis and the input patterns.
kkt_status build_plan(kkt_ctx* c, const int* W_colptr, const int* W_rowind, const int* J_rowptr,
                      const int* J_colind) {
    const Symbolic& S = c->sym;
    const int n = c->n, m = c->m, ns = S.ns();
    std::vector<int>& sn_f = c->h_sn_f;
    std::vector<int>& sn_c = c->h_sn_c;
    std::vector<int>& sn_r = c->h_sn_r;
    std::vector<long long>& sn_lptr = c->h_sn_lptr;
    sn_f.resize(ns);
    sn_c.resize(ns);
    sn_r.resize(ns);
    sn_lptr.resize(ns + 1);
    c->h_sn_rptr = S.sn_rowptr;
    std::vector<int> snode(n);
    long long off = 0;
    for (int s = 0; s < ns; ++s) {
        sn_f[s] = S.sn_ptr[s];
        sn_c[s] = S.sn_ptr[s + 1] - S.sn_ptr[s];
        sn_r[s] = S.sn_rowptr[s + 1] - S.sn_rowptr[s];
        sn_lptr[s] = off;
        off += (long long)sn_r[s] * sn_c[s];
        for (int j = sn_f[s]; j < S.sn_ptr[s + 1]; ++j) snode[j] = s;
    }
    sn_lptr[ns] = off;
    c->panel = off;

    // position of every row inside rows(s), computed on demand
    std::vector<int> pos(n, -1);
    auto fill_pos = [&](int s) {
        for (int q = S.sn_rowptr[s]; q < S.sn_rowptr[s + 1]; ++q) pos[S.sn_rows[q]] = q - S.sn_rowptr[s];
    };
    auto clear_pos = [&](int s) {
        for (int q = S.sn_rowptr[s]; q < S.sn_rowptr[s + 1]; ++q) pos[S.sn_rows[q]] = -1;
    };

    // ---- assembly sources, grouped by panel slot
    struct Src {
        long long slot;
        int a, b;
    };
    std::vector<Src> srcs;
    // collect (new row, new col) for every source, then resolve slots per supernode
    struct Raw {
        int i, j, a, b;
    };
    std::vector<Raw> raw;
    raw.reserve((size_t)W_colptr[n] + n + 16 * (size_t)J_rowptr[m]);
    for (int col = 0; col < n; ++col)
        for (int p = W_colptr[col]; p < W_colptr[col + 1]; ++p) {
            int a = S.iperm[W_rowind[p]], b = S.iperm[col];
            raw.push_back({std::max(a, b), std::min(a, b), p, -1});
        }
    for (int v = 0; v < n; ++v) raw.push_back({S.iperm[v], S.iperm[v], v, -2});
    for (int r = 0; r < m; ++r)
        for (int p = J_rowptr[r]; p < J_rowptr[r + 1]; ++p) {
            for (int q = p; q < J_rowptr[r + 1]; ++q) {
                int a = S.iperm[J_colind[p]], b = S.iperm[J_colind[q]];
                raw.push_back({std::max(a, b), std::min(a, b), p, q});
            }
        }
    // bucket by supernode of the column, then resolve the slot
    std::vector<long long> bucket_ptr(ns + 1, 0);
    for (const Raw& x : raw) bucket_ptr[snode[x.j] + 1]++;
    for (int s = 0; s < ns; ++s) bucket_ptr[s + 1] += bucket_ptr[s];
    std::vector<Raw> sorted(raw.size());
    {
        std::vector<long long> fillp(bucket_ptr.begin(), bucket_ptr.end() - 1);
        for (const Raw& x : raw) sorted[fillp[snode[x.j]]++] = x;
    }
    std::vector<Raw>().swap(raw);
    srcs.reserve(sorted.size());
    for (int s = 0; s < ns; ++s) {
        fill_pos(s);
        for (long long q = bucket_ptr[s]; q < bucket_ptr[s + 1]; ++q) {
            const Raw& x = sorted[q];
            int pi = pos[x.i];
            if (pi < 0) {
                clear_pos(s);
                return set_err(c, KKT_ERR_INTERNAL, "assembly entry outside the supernode structure");
            }
            long long slot = sn_lptr[s] + (long long)(x.j - sn_f[s]) * sn_r[s] + pi;
            srcs.push_back({slot, x.a, x.b});
        }
        clear_pos(s);
    }
    std::vector<Raw>().swap(sorted);
    std::stable_sort(srcs.begin(), srcs.end(), [](const Src& x, const Src& y) { return x.slot < y.slot; });
    std::vector<long long> k_slot, k_sptr;
    std::vector<int2> k_src;
    k_src.reserve(srcs.size());
    for (size_t q = 0; q < srcs.size(); ++q) {
        if (q == 0 || srcs[q].slot != srcs[q - 1].slot) {
            k_slot.push_back(srcs[q].slot);
            k_sptr.push_back((long long)q);
        }
        k_src.push_back(make_int2(srcs[q].a, srcs[q].b));
    }
    k_sptr.push_back((long long)srcs.size());
    c->nk = (long long)k_slot.size();
    std::vector<Src>().swap(srcs);

    // ---- update segments and relative maps
    std::vector<int> seg_ptr{0}, seg_t, seg_a, seg_b, relmap;
    std::vector<long long> seg_map;
    for (int s = 0; s < ns; ++s) {
        const int cc = sn_c[s], rr = sn_r[s], rb = rr - cc;
        const int* rows = S.sn_rows.data() + S.sn_rowptr[s];
        int i = 0;
        while (i < rb) {
            int t = snode[rows[cc + i]];
            int e = i;
            while (e < rb && snode[rows[cc + e]] == t) ++e;
            seg_t.push_back(t);
            seg_a.push_back(i);
            seg_b.push_back(e);
            seg_map.push_back((long long)relmap.size());
            fill_pos(t);
            if (c->dbg_relmap_pos < 0 && rb > 0) {
                c->dbg_relmap_pos = (long long)relmap.size();
                c->dbg_relmap_bad = sn_r[t];
            }
            for (int q = i; q < rb; ++q) {
                int pq = pos[rows[cc + q]];
                if (pq < 0) {
                    clear_pos(t);
                    return set_err(c, KKT_ERR_INTERNAL, "supernode row structure is not nested");
                }
                relmap.push_back(pq);
            }
            clear_pos(t);
            i = e;
        }
        seg_ptr.push_back((int)seg_t.size());
    }

    // ---- small-subtree tasks, then levels of the remaining supernodes
    std::vector<int> sub_cols(ns, 0);
    std::vector<char> small_ok(ns, 1);
    const long long kTaskPanelCap = 6144;   // panel entries kept in the task CTA's smem
    const int kTaskColsCap = 1024;          // columns of a task (its slice of x in the solves' smem)
    for (int s = 0; s < ns; ++s) {
        sub_cols[s] += sn_c[s];
        if ((long long)sn_r[s] * sn_c[s] > kTaskPanelCap) small_ok[s] = 0;
        const int p = S.sn_parent[s];
        if (p >= 0) {
            sub_cols[p] += sub_cols[s];
            if (!small_ok[s]) small_ok[p] = 0;
        }
    }
    std::vector<char> in_task(ns, 0);
    for (int s = 0; s < ns; ++s)
        in_task[s] = c->opt.subtree_cols > 0 && sub_cols[s] <= std::min(c->opt.subtree_cols, kTaskColsCap) &&
                     small_ok[s];
    std::vector<int> task_of(ns, -1), task_root;
    for (int s = ns - 1; s >= 0; --s) {
        if (!in_task[s]) continue;
        const int p = S.sn_parent[s];
        if (p >= 0 && in_task[p]) {
            task_of[s] = task_of[p];
        } else {
            task_of[s] = (int)task_root.size();
            task_root.push_back(s);
        }
    }
    c->ntasks = (int)task_root.size();
    std::vector<int> task_ptr(c->ntasks + 1, 0), task_sn;
    for (int s = 0; s < ns; ++s)
        if (task_of[s] >= 0) task_ptr[task_of[s] + 1]++;
    for (int b = 0; b < c->ntasks; ++b) task_ptr[b + 1] += task_ptr[b];
    task_sn.resize(task_ptr[c->ntasks]);
    {
        std::vector<int> fillp(task_ptr.begin(), task_ptr.end() - 1);
        for (int s = 0; s < ns; ++s)   // increasing s: postorder inside every task
            if (task_of[s] >= 0) {
                task_sn[fillp[task_of[s]]++] = s;
                c->task_max_rc = std::max(c->task_max_rc, (long long)sn_r[s] * sn_c[s]);
                c->task_max_cc = std::max(c->task_max_cc, (long long)sn_c[s] * sn_c[s]);
                c->task_max_ccrb = std::max(c->task_max_ccrb,
                                            (long long)sn_c[s] * sn_c[s] + sn_r[s] - sn_c[s]);
            }
    }
    // a task's columns are one range (a subtree in postorder): the solves
    // keep that slice of x in shared memory
    for (int b = 0; b < c->ntasks; ++b) {
        const int q0 = task_ptr[b], q1 = task_ptr[b + 1];
        long long cols = 0;
        for (int q = q0; q < q1; ++q) cols += sn_c[task_sn[q]];
        const long long w = (long long)sn_f[task_sn[q1 - 1]] + sn_c[task_sn[q1 - 1]] - sn_f[task_sn[q0]];
        if (q1 <= q0 || w != cols) return set_err(c, KKT_ERR_INTERNAL, "subtree task columns are not contiguous");
        c->task_max_cols = std::max(c->task_max_cols, w);
    }
    std::vector<int> level(ns, 0);
    for (int s = 0; s < ns; ++s) {
        const int p = S.sn_parent[s];
        if (in_task[s] || p < 0) continue;
        level[p] = std::max(level[p], level[s] + 1);
    }
    int nlev = 0;
    for (int s = 0; s < ns; ++s)
        if (!in_task[s]) nlev = std::max(nlev, level[s] + 1);
    c->nlev = nlev;
    c->h_lvl_ptr.assign(nlev + 1, 0);
    for (int s = 0; s < ns; ++s)
        if (!in_task[s]) c->h_lvl_ptr[level[s] + 1]++;
    for (int l = 0; l < nlev; ++l) c->h_lvl_ptr[l + 1] += c->h_lvl_ptr[l];
    c->h_lvl_sn.resize(c->h_lvl_ptr[nlev]);
    c->lvl_max_c.assign(nlev, 0);
    c->lvl_max_rb.assign(nlev, 0);
    c->lvl_max_rc.assign(nlev, 0);
    {
        std::vector<int> fillp(c->h_lvl_ptr.begin(), c->h_lvl_ptr.end() - 1);
        for (int s = 0; s < ns; ++s) {
            if (in_task[s]) continue;
            c->h_lvl_sn[fillp[level[s]]++] = s;
            c->lvl_max_c[level[s]] = std::max(c->lvl_max_c[level[s]], sn_c[s]);
            c->lvl_max_rb[level[s]] = std::max(c->lvl_max_rb[level[s]], sn_r[s] - sn_c[s]);
            c->lvl_max_rc[level[s]] =
                std::max(c->lvl_max_rc[level[s]], (long long)sn_c[s] * sn_r[s]);
        }
    }
    std::vector<int2> trsm_tasks;
    std::vector<int4> syrk_tasks;
    c->lvl_split.assign(nlev, 0);
    c->lvl_fused.assign(nlev, 0);
    c->lvl_trsm_ptr.assign(nlev + 1, 0);
    c->lvl_syrk_ptr.assign(nlev + 1, 0);
    for (int l = 0; l < nlev; ++l) {
        const int cnt = c->h_lvl_ptr[l + 1] - c->h_lvl_ptr[l];
        // Split launches spread a supernode over many CTAs.  They serve levels
        // with fewer supernodes than SMs can hold, and levels where one
        // supernode would straggle: with one CTA per supernode the largest
        // panel runs on one SM (two FP64 FMAs a clock), so when its panel
        // work exceeds twice the level's average work per SM it alone would
        // set the level's time (a few separators among many tiny supernodes).
        double fl_max = 0.0, fl_sum = 0.0;
        for (int q = c->h_lvl_ptr[l]; q < c->h_lvl_ptr[l + 1]; ++q) {
            const int s = c->h_lvl_sn[q];
            const double cc = sn_c[s], rr = sn_r[s];
            // sum over the columns j < c of (r - j)^2: the panel's FMA count x 2
            const double f = cc * rr * rr - rr * cc * (cc - 1.0) + (cc - 1.0) * cc * (2.0 * cc - 1.0) / 6.0;
            fl_max = std::max(fl_max, f);
            fl_sum += f;
        }
        c->lvl_split[l] = cnt < kSplitLevel || fl_max > 2.0 * fl_sum / kNumSMs;
        c->lvl_fused[l] = c->lvl_max_c[l] <= kFusedMaxC && c->lvl_max_rb[l] <= kFusedMaxRb;
        if (c->lvl_split[l]) {
            // SYRK tasks: chunks of the packed lower triangle of each
            // supernode, sized so the level gives about four CTAs per SM
            long long pairs = 0;
            for (int q = c->h_lvl_ptr[l]; q < c->h_lvl_ptr[l + 1]; ++q) {
                const long long rb = sn_r[c->h_lvl_sn[q]] - sn_c[c->h_lvl_sn[q]];
                pairs += rb * (rb + 1) / 2;
            }
            const long long want = (pairs + 4LL * kNumSMs - 1) / (4LL * kNumSMs);
            const int chunk = (int)std::min<long long>(1024, std::max<long long>(128, (want + 127) / 128 * 128));
            for (int q = c->h_lvl_ptr[l]; q < c->h_lvl_ptr[l + 1]; ++q) {
                const int sn = c->h_lvl_sn[q];
                const int rb = sn_r[sn] - sn_c[sn];
                for (int r0 = 0; r0 < rb; r0 += kTrsmWarps) trsm_tasks.push_back(make_int2(sn, r0));
                const int np = rb * (rb + 1) / 2;
                for (int p0 = 0; p0 < np; p0 += chunk)
                    syrk_tasks.push_back(make_int4(sn, p0, std::min(np, p0 + chunk), 0));
            }
        }
        c->lvl_trsm_ptr[l + 1] = (int)trsm_tasks.size();
        c->lvl_syrk_ptr[l + 1] = (int)syrk_tasks.size();
    }

    // ---- supernodes whose panels the factor kernels do not write back
    // normalised (split narrow levels, panels too large for shared memory):
    // the normalisation pass after the factorisation covers only these
    {
        std::vector<int> norm_list, norm_list_fused;
        for (int s = 0; s < ns; ++s) {
            if (in_task[s]) continue;
            const bool fused_smem = !c->lvl_split[level[s]] && (long long)sn_r[s] * sn_c[s] <= kSmemCapElems;
            if (!fused_smem) norm_list.push_back(s);
            if (!fused_smem && !c->lvl_fused[level[s]]) norm_list_fused.push_back(s);
        }
        c->n_norm = (int)norm_list.size();
        c->n_norm_fused = (int)norm_list_fused.size();
        TRY(upload(c, &c->d_norm_list, norm_list));
        TRY(upload(c, &c->d_norm_list_fused, norm_list_fused));
    }

    // ---- SpMV structures (original labels)
    std::vector<int> wf_ptr(n + 1, 0), wf_col, wf_idx;
    for (int col = 0; col < n; ++col)
        for (int p = W_colptr[col]; p < W_colptr[col + 1]; ++p) {
            wf_ptr[W_rowind[p] + 1]++;
            if (W_rowind[p] != col) wf_ptr[col + 1]++;
        }
    for (int i = 0; i < n; ++i) wf_ptr[i + 1] += wf_ptr[i];
    wf_col.resize(wf_ptr[n]);
    wf_idx.resize(wf_ptr[n]);
    {
        std::vector<int> fillp(wf_ptr.begin(), wf_ptr.end() - 1);
        for (int col = 0; col < n; ++col)
            for (int p = W_colptr[col]; p < W_colptr[col + 1]; ++p) {
                int r = W_rowind[p];
                wf_col[fillp[r]] = col;
                wf_idx[fillp[r]++] = p;
                if (r != col) {
                    wf_col[fillp[col]] = r;
                    wf_idx[fillp[col]++] = p;
                }
            }
    }
    std::vector<int> j_ptr(J_rowptr, J_rowptr + m + 1), j_col(J_colind, J_colind + J_rowptr[m]);
    std::vector<int> jt_ptr(n + 1, 0), jt_row(J_rowptr[m]), jt_idx(J_rowptr[m]);
    for (int p = 0; p < J_rowptr[m]; ++p) jt_ptr[J_colind[p] + 1]++;
    for (int i = 0; i < n; ++i) jt_ptr[i + 1] += jt_ptr[i];
    {
        std::vector<int> fillp(jt_ptr.begin(), jt_ptr.end() - 1);
        for (int r = 0; r < m; ++r)
            for (int p = J_rowptr[r]; p < J_rowptr[r + 1]; ++p) {
                int col = J_colind[p];
                jt_row[fillp[col]] = r;
                jt_idx[fillp[col]++] = p;
            }
    }

    // ---- validate every index the kernels will dereference
    for (size_t e = 0; e < k_slot.size(); ++e)
        if (k_slot[e] < 0 || k_slot[e] >= c->panel)
            return set_err(c, KKT_ERR_INTERNAL, "assembly slot out of range");
    for (const int2& q : k_src) {
        bool ok = q.y == -1 ? (q.x >= 0 && q.x < W_colptr[n])
                : q.y == -2 ? (q.x >= 0 && q.x < n)
                            : (q.x >= 0 && q.x < J_rowptr[m] && q.y < J_rowptr[m]);
        if (!ok) return set_err(c, KKT_ERR_INTERNAL, "assembly source out of range");
    }
    for (int s = 0; s < ns; ++s) {
        const int cc = sn_c[s], rb = sn_r[s] - cc;
        const int* rows = S.sn_rows.data() + S.sn_rowptr[s];
        for (int q = 0; q < sn_r[s]; ++q)
            if (rows[q] < 0 || rows[q] >= n) return set_err(c, KKT_ERR_INTERNAL, "row out of range");
        if (rb > 0 && seg_ptr[s + 1] <= seg_ptr[s])
            return set_err(c, KKT_ERR_INTERNAL, "missing update segment");
        for (int k = seg_ptr[s]; k < seg_ptr[s + 1]; ++k) {
            const int t = seg_t[k];
            if (t <= s || t >= ns) return set_err(c, KKT_ERR_INTERNAL, "bad segment target");
            for (int i = seg_a[k]; i < seg_b[k]; ++i) {
                int colo = rows[cc + i] - sn_f[t];
                if (colo < 0 || colo >= sn_c[t]) return set_err(c, KKT_ERR_INTERNAL, "bad column offset");
            }
            for (int i = seg_a[k]; i < rb; ++i) {
                int rp = relmap[seg_map[k] + (i - seg_a[k])];
                if (rp < 0 || rp >= sn_r[t]) return set_err(c, KKT_ERR_INTERNAL, "bad relative row");
            }
        }
    }

    if (S.sn_rowmask.size() != S.sn_rows.size())
        return set_err(c, KKT_ERR_INTERNAL, "structural masks missing (supernode wider than 64)");
    for (int s = 0; s < ns; ++s)
        if (sn_c[s] > 64) return set_err(c, KKT_ERR_INTERNAL, "supernode wider than 64 columns");

    // ---- reduction chunks (rows of one instance each) and column instances
    const int nb = c->nb;
    std::vector<int4> ch_xy, ch_y;
    c->h_chy_ptr.assign(nb + 1, 0);
    auto make_chunks = [](const std::vector<int>& off, int base, std::vector<int4>& out,
                          std::vector<int>* inst_ptr) {
        for (int i = 0; i + 1 < (int)off.size(); ++i) {
            if (inst_ptr) (*inst_ptr)[i] = (int)out.size();
            for (int lo = off[i]; lo < off[i + 1]; lo += kChunkRows)
                out.push_back(make_int4(base + lo, base + std::min(off[i + 1], lo + kChunkRows), i, 0));
        }
        if (inst_ptr) inst_ptr->back() = (int)out.size();
    };
    make_chunks(c->h_xoff, 0, ch_xy, nullptr);
    c->nch_x = (int)ch_xy.size();
    make_chunks(c->h_yoff, n, ch_xy, nullptr);
    c->nch_xy = (int)ch_xy.size();
    make_chunks(c->h_yoff, 0, ch_y, &c->h_chy_ptr);
    c->nch_y = (int)ch_y.size();
    if (c->h_xoff.size() != (size_t)nb + 1 || c->h_xoff.back() != n || c->h_yoff.back() != m)
        return set_err(c, KKT_ERR_INTERNAL, "batch offsets do not cover the system");
    TRY(upload(c, &c->d_ch_xy, ch_xy));
    TRY(upload(c, &c->d_ch_y, ch_y));
    TRY(upload(c, &c->d_chy_ptr, c->h_chy_ptr));
    if (nb > 1) {
        std::vector<int> col_inst(n);
        for (int j = 0; j < n; ++j) {
            const int v = S.perm[j];
            col_inst[j] = (int)(std::upper_bound(c->h_xoff.begin(), c->h_xoff.end(), v) - c->h_xoff.begin()) - 1;
        }
        TRY(upload(c, &c->d_col_inst, col_inst));
        std::vector<int> sn_inst(ns);
        for (int s = 0; s < ns; ++s) sn_inst[s] = col_inst[S.sn_ptr[s]];
        TRY(upload(c, &c->d_sn_inst, sn_inst));
        TRY(upload(c, &c->d_inst_on, std::vector<int>(nb, 1)));
        CUDA_TRY(c, cudaMallocHost((void**)&c->h_inst_on, (size_t)nb * sizeof(int)));
        for (int i = 0; i < nb; ++i) c->h_inst_on[i] = 1;
        TRY(alloc(c, &c->d_dvec, n));
        TRY(alloc(c, &c->d_dval, nb));
    }
    TRY(alloc(c, &c->d_knorm, nb));
    TRY(alloc(c, &c->d_red, 3 * (size_t)nb));
    TRY(alloc(c, &c->d_act, nb));
    TRY(alloc(c, &c->d_cgs, 4 * (size_t)nb));
    TRY(alloc(c, &c->d_cgi, 2 * (size_t)nb));
    TRY(alloc(c, &c->d_part_y, std::max(1, c->nch_y)));
    CUDA_TRY(c, cudaMallocHost((void**)&c->h_red, 3 * (size_t)nb * sizeof(double)));
    CUDA_TRY(c, cudaMallocHost((void**)&c->h_act, (size_t)nb * sizeof(int)));
    CUDA_TRY(c, cudaMallocHost((void**)&c->h_int, 2 * (size_t)nb * sizeof(int)));
    c->h_knorm.assign(nb, 0.0);
    c->h_delta.assign(nb, 0.0);
    c->r_status.assign(nb, 0);
    c->r_refine.assign(nb, 0);
    c->r_cg.assign(nb, 0);
    c->r_fail.assign(nb, -1);
    c->r_eta.assign(nb, 0.0);

    // ---- upload
    int *d_sn_f, *d_sn_c, *d_sn_r, *d_sn_rptr, *d_rows, *d_seg_ptr, *d_seg_t, *d_seg_a, *d_seg_b,
        *d_relmap;
    long long *d_sn_lptr, *d_seg_map;
    TRY(upload(c, &d_sn_f, sn_f));
    TRY(upload(c, &d_sn_c, sn_c));
    TRY(upload(c, &d_sn_r, sn_r));
    TRY(upload(c, &d_sn_lptr, sn_lptr));
    TRY(upload(c, &d_sn_rptr, S.sn_rowptr));
    TRY(upload(c, &d_rows, S.sn_rows));
    TRY(upload(c, &d_seg_ptr, seg_ptr));
    TRY(upload(c, &d_seg_t, seg_t));
    TRY(upload(c, &d_seg_a, seg_a));
    TRY(upload(c, &d_seg_b, seg_b));
    TRY(upload(c, &d_seg_map, seg_map));
    TRY(upload(c, &d_relmap, relmap));
    unsigned long long* d_rmask;
    {
        std::vector<unsigned long long> rm(S.sn_rowmask.begin(), S.sn_rowmask.end());
        TRY(upload(c, &d_rmask, rm));
    }
    TRY(alloc(c, &c->d_berr, 1));
    CUDA_TRY(c, cudaMemset(c->d_berr, 0, sizeof(int)));
    c->plan = Plan{d_sn_f, d_sn_c, d_sn_r, d_sn_lptr, d_sn_rptr, d_rows,
                   d_seg_ptr, d_seg_t, d_seg_a, d_seg_b, d_seg_map, d_relmap, d_rmask,
                   c->d_berr, ns, n, c->panel, c->d_sn_inst, c->d_inst_on};
    TRY(upload(c, &c->d_lvl_sn, c->h_lvl_sn));
    TRY(upload(c, &c->d_trsm_tasks, trsm_tasks));
    TRY(upload(c, &c->d_task_ptr, task_ptr));

    TRY(upload(c, &c->d_task_sn, task_sn));
    // ---- dataflow solves: the subtree tasks, then the supernodes of the
    // levels bottom-up (a topological order of the tree: every item comes
    // after the items that feed it); each item feeds the item holding the
    // parent of its (root) supernode
    {
        const int nitems = c->ntasks + (int)c->h_lvl_sn.size();
        std::vector<int> item(nitems), up(nitems, -1), nchild(nitems, 0), item_of(ns, -1);
        for (int b = 0; b < c->ntasks; ++b) item[b] = -(b + 1);
        for (size_t q = 0; q < c->h_lvl_sn.size(); ++q) {
            item[c->ntasks + q] = c->h_lvl_sn[q];
            item_of[c->h_lvl_sn[q]] = c->ntasks + (int)q;
        }
        std::vector<int> nchild_lv(nitems, 0);
        for (int i = 0; i < nitems; ++i) {
            const int s = item[i] >= 0 ? item[i] : task_root[-item[i] - 1];
            const int p = S.sn_parent[s];
            if (p < 0) continue;
            up[i] = item_of[p];
            if (up[i] <= i) return set_err(c, KKT_ERR_INTERNAL, "dataflow solve order is not topological");
            nchild[up[i]]++;
            if (item[i] >= 0) nchild_lv[up[i]]++;
        }
        c->flow_fwd_elems = c->task_max_cc + c->task_max_cols;
        c->flow_bwd_elems = c->task_max_ccrb + c->task_max_cols;
        c->flow_bwd_ints = 0;
        for (int s : c->h_lvl_sn) {
            const long long ldc = (long long)staged_ld(sn_r[s]) * sn_c[s], rb = sn_r[s] - sn_c[s];
            c->flow_fwd_elems = std::max(c->flow_fwd_elems, ldc);
            c->flow_bwd_elems = std::max(c->flow_bwd_elems, ldc + rb);
            c->flow_bwd_ints = std::max(c->flow_bwd_ints, rb);
        }
        c->flow_items = nitems;
        if (nitems > 0) {
            TRY(upload(c, &c->d_flow_item, item));
            TRY(upload(c, &c->d_flow_up, up));
            TRY(upload(c, &c->d_flow_nchild, nchild));
            TRY(upload(c, &c->d_flow_nchild_lv, nchild_lv));
            TRY(alloc(c, &c->d_flow_cnt, nitems));
            TRY(alloc(c, &c->d_flow_done, nitems));
            TRY(alloc(c, &c->d_flow_ctrl, 4));
            CUDA_TRY(c, cudaMemset(c->d_flow_cnt, 0, (size_t)nitems * sizeof(int)));
            CUDA_TRY(c, cudaMemset(c->d_flow_done, 0, (size_t)nitems * sizeof(unsigned)));
            CUDA_TRY(c, cudaMemset(c->d_flow_ctrl, 0, 4 * sizeof(unsigned)));
            CUDA_TRY(c, cudaHostAlloc((void**)&c->h_flow_err, sizeof(int), cudaHostAllocMapped));
            *c->h_flow_err = 0;
            CUDA_TRY(c, cudaHostGetDevicePointer((void**)&c->d_flow_err, c->h_flow_err, 0));
        }
    }
    TRY(upload(c, &c->d_syrk_tasks, syrk_tasks));
    TRY(alloc(c, &c->d_dinv, n));
    // zero: a batch instance switched off before its first factorisation
    // solves with these pivots (times a zero right-hand side)
    CUDA_TRY(c, cudaMemset(c->d_dinv, 0, (size_t)n * sizeof(double)));
    TRY(upload(c, &c->d_perm, S.perm));
    TRY(upload(c, &c->d_iperm, S.iperm));
    TRY(upload(c, &c->d_k_slot, k_slot));
    TRY(upload(c, &c->d_k_sptr, k_sptr));
    TRY(upload(c, &c->d_k_src, k_src));
    TRY(upload(c, &c->d_wf_ptr, wf_ptr));
    TRY(upload(c, &c->d_wf_col, wf_col));
    TRY(upload(c, &c->d_wf_idx, wf_idx));
    TRY(upload(c, &c->d_j_ptr, j_ptr));
    TRY(upload(c, &c->d_j_col, j_col));
    TRY(upload(c, &c->d_jt_ptr, jt_ptr));
    TRY(upload(c, &c->d_jt_row, jt_row));
    TRY(upload(c, &c->d_jt_idx, jt_idx));
    TRY(alloc(c, &c->d_Lx, (size_t)c->panel));
    TRY(alloc(c, &c->d_fail, nb));
    const size_t nm = (size_t)n + m;
    TRY(alloc(c, &c->w_xp, n));
    TRY(alloc(c, &c->w_t, n));
    TRY(alloc(c, &c->w_r, nm));
    TRY(alloc(c, &c->w_d, nm));
    TRY(alloc(c, &c->w_q, n));
    TRY(alloc(c, &c->w_p, std::max(n, m)));
    TRY(alloc(c, &c->w_sp, std::max(n, m)));
    TRY(alloc(c, &c->w_res, m));
    TRY(alloc(c, &c->w_cgx, m));
    TRY(alloc(c, &c->w_rg, n));
    TRY(alloc(c, &c->w_tn, n));
    TRY(alloc(c, &c->v_W, std::max(1, W_colptr[n])));
    TRY(alloc(c, &c->v_J, std::max(1, J_rowptr[m])));
    TRY(alloc(c, &c->v_Js, std::max(1, J_rowptr[m])));
    TRY(alloc(c, &c->v_sigma, n));
    TRY(alloc(c, &c->v_D, std::max(1, m)));
    TRY(alloc(c, &c->d_cg, 2));
    if (c->opt.precision == 1) {
        TRY(alloc(c, &c->d_Lx32, (size_t)c->panel));
        TRY(alloc(c, &c->d_dinv32, n));
        CUDA_TRY(c, cudaMemset(c->d_dinv32, 0, (size_t)n * sizeof(float)));
        TRY(alloc(c, &c->w_xp32, n));
    }
    CUDA_TRY(c, cudaMallocHost((void**)&c->h_cg, 2 * sizeof(int)));
    return KKT_OK;
}

df64* as_df(double* p) { return reinterpret_cast<df64*>(p); }

// Block cyclic reduction: K^{-1} v in place (natural order), levels forward
// then backward.
void enqueue_bcr_solve(kkt_ctx* c, double* v, cudaStream_t st, const int* active) {
    const int b = c->bcr_b;
    for (int l = 0; l < c->bcr_nlev; ++l) {
        const int ne = c->bcr_elim_ptr[l + 1] - c->bcr_elim_ptr[l];
        const int ns = c->bcr_surv_ptr[l + 1] - c->bcr_surv_ptr[l];
        if (ne > 0)
            bcr_fwd_elim_kernel<<<ne, kThreads, 0, st>>>(b, c->d_bcr_elim + c->bcr_elim_ptr[l], c->d_bcr_pn,
                                                         c->d_dinv, v, active);
        if (ns > 0)
            bcr_fwd_update_kernel<<<ns, kThreads, 0, st>>>(b, c->d_bcr_surv + c->bcr_surv_ptr[l], c->d_bcr_pn,
                                                           v, active);
    }
    for (int l = c->bcr_nlev - 1; l >= 0; --l) {
        const int ne = c->bcr_elim_ptr[l + 1] - c->bcr_elim_ptr[l];
        if (ne > 0)
            bcr_bwd_kernel<<<ne, kThreads, 0, st>>>(b, c->d_bcr_elim + c->bcr_elim_ptr[l], c->d_bcr_pn,
                                                    c->d_dinv, v, active);
    }
}

template <typename T>
void set_backward_smem_limit() {
    cudaFuncSetAttribute(backward_level_kernel<T, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kBackwardSmemBytes);
    cudaFuncSetAttribute(backward_level_kernel<T, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kBackwardSmemBytes);
    cudaFuncSetAttribute(forward_level_staged_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kStagedSmemBytes);
    // subtree tasks: diagonal block (and rows below) of <= 6144 entries plus
    // the task's slice of x (<= 1024 columns)
    cudaFuncSetAttribute(forward_subtree_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    cudaFuncSetAttribute(backward_subtree_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    cudaFuncSetAttribute(backward_level_staged_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kStagedSmemBytes);
}

// Launch with programmatic stream serialisation: the kernel may start while
// the previous kernel of the stream runs; it waits for that kernel's
// completion itself (grid_dependency_wait).  Captured into a graph this is
// a programmatic dependency edge.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t st,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3((unsigned)block, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Shared memory of the staged level kernels for level l: the widest panel at
// the padded leading dimension, and for the backward pass x and the row
// indices of the rows below.
size_t staged_panel_elems(const kkt_ctx* c, int l) { return (size_t)c->lvl_max_rc[l] + c->lvl_max_c[l]; }
template <typename T>
size_t staged_backward_bytes(const kkt_ctx* c, int l) {
    return (staged_panel_elems(c, l) + c->lvl_max_rb[l]) * sizeof(T) + (size_t)c->lvl_max_rb[l] * sizeof(int);
}

template <typename T>
constexpr int flow_prec() {
    return std::is_same<T, double>::value ? 0 : std::is_same<T, float>::value ? 1 : 2;
}
template <typename T>
size_t flow_fwd_bytes(const kkt_ctx* c) {
    return (size_t)c->flow_fwd_elems * sizeof(T);
}
template <typename T>
size_t flow_bwd_bytes(const kkt_ctx* c) {
    return (size_t)c->flow_bwd_elems * sizeof(T) + (size_t)c->flow_bwd_ints * sizeof(int);
}
// staged_solve = 3: the subtree tasks keep their own launches, the dataflow
// kernels take the level supernodes only
bool flow_levels_only(const kkt_ctx* c) { return c->opt.staged_solve == 3 && c->ntasks > 0; }
Flow flow_of(const kkt_ctx* c) {
    const bool lv = flow_levels_only(c);
    return Flow{c->d_flow_item, c->d_flow_up, lv ? c->d_flow_nchild_lv : c->d_flow_nchild, c->d_flow_cnt,
                c->d_flow_done, c->d_flow_ctrl, c->d_flow_err, lv ? c->ntasks : 0, c->flow_items,
                (int)c->task_max_cc, (int)c->task_max_ccrb};
}

// Dataflow solves are used with staged_solve = 2 (3: levels only) when the
// widest staged panel fits kFlowSmemBytes; the launch grid is what stays
// resident on the device
// (a CTA waits only for items that running CTAs hold, so fewer resident
// CTAs make it slower, never stuck).
template <typename T>
bool flow_grids(kkt_ctx* c, int sms) {
    const int p = flow_prec<T>();
    const size_t fb = flow_fwd_bytes<T>(c), bb = flow_bwd_bytes<T>(c);
    // the attribute is per kernel, not per context: every context sets the
    // same bound, so contexts of other sizes (e.g. the clients of a server,
    // created on several threads) never lower it below what one needs
    if (cudaFuncSetAttribute(forward_flow_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kFlowSmemBytes) != cudaSuccess ||
        cudaFuncSetAttribute(backward_flow_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kFlowSmemBytes) != cudaSuccess)
        return false;
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, forward_flow_kernel<T>, kFlowThreads, fb) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, backward_flow_kernel<T>, kFlowThreads, bb) != cudaSuccess ||
        a < 1 || b < 1)
        return false;
    c->flow_grid[p][0] = std::max(1, std::min(c->flow_items, a * sms));
    c->flow_grid[p][1] = std::max(1, std::min(c->flow_items, b * sms));
    return true;
}

void setup_flow(kkt_ctx* c) {
    c->flow = false;
    if (c->opt.staged_solve < 2 || c->opt.solver != 0 || c->flow_items == 0 || !c->h_flow_err) return;
    if (flow_bwd_bytes<double>(c) > kFlowSmemBytes) return;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || sms < 1) {
        cudaGetLastError();
        return;
    }
    c->flow = flow_grids<double>(c, sms) && flow_grids<float>(c, sms) && flow_grids<df64>(c, sms);
    cudaGetLastError();
}

// L z = xp, L^T w = z in place on the permuted vector xp: subtree tasks and
// levels bottom-up, then levels top-down and subtree tasks (panels Lx and
// reciprocal pivots dinv of the precision T).
template <typename T>
void enqueue_triangular_solves(kkt_ctx* c, const T* Lx, const T* dinv, T* xp, cudaStream_t st,
                               const int* active) {
    if (c->flow) {   // one dependency-driven launch per direction
        const int p = flow_prec<T>();
        const Flow F = flow_of(c);
        const bool tasks = flow_levels_only(c);
        if (tasks)
            forward_subtree_kernel<T><<<c->ntasks, kSubtreeThreads,
                                        (size_t)(c->task_max_cc + c->task_max_cols) * sizeof(T), st>>>(
                c->plan, c->d_task_ptr, c->d_task_sn, Lx, dinv, xp, (int)c->task_max_cc, active);
        if (F.nitems > F.first) {
            forward_flow_kernel<T><<<c->flow_grid[p][0], kFlowThreads, flow_fwd_bytes<T>(c), st>>>(
                c->plan, F, c->d_task_ptr, c->d_task_sn, Lx, xp, active);
            backward_flow_kernel<T><<<c->flow_grid[p][1], kFlowThreads, flow_bwd_bytes<T>(c), st>>>(
                c->plan, F, c->d_task_ptr, c->d_task_sn, Lx, dinv, xp, active);
        }
        if (tasks)
            backward_subtree_kernel<T><<<c->ntasks, kSubtreeThreads,
                                         (size_t)(c->task_max_ccrb + c->task_max_cols) * sizeof(T), st>>>(
                c->plan, c->d_task_ptr, c->d_task_sn, Lx, dinv, xp, (int)c->task_max_ccrb, active);
        return;
    }
    if (c->ntasks > 0)
        forward_subtree_kernel<T><<<c->ntasks, kSubtreeThreads,
                                    (size_t)(c->task_max_cc + c->task_max_cols) * sizeof(T), st>>>(
            c->plan, c->d_task_ptr, c->d_task_sn, Lx, dinv, xp, (int)c->task_max_cc, active);
    // Levels with more supernodes than 256-thread CTAs keep resident at once
    // (six per SM by registers) run 128-thread CTAs with the diagonal block
    // sized for the level's widest supernode: one wave instead of two.
    // Narrower levels keep a fixed 64 x 64 block.
    // Levels whose panels fit kStagedSmemBytes run the staged kernels with
    // programmatic dependent launch.
    for (int l = 0; l < c->nlev; ++l) {
        const int cnt = c->h_lvl_ptr[l + 1] - c->h_lvl_ptr[l];
        const int* lsn = c->d_lvl_sn + c->h_lvl_ptr[l];
        const size_t fsm = staged_panel_elems(c, l) * sizeof(T);
        if (c->opt.staged_solve && fsm <= kStagedSmemBytes) {
            launch_pdl(forward_level_staged_kernel<T>, cnt, cnt > 6 * kNumSMs ? kThreads / 2 : kThreads, fsm, st,
                       c->plan, lsn, (const T*)Lx, xp, active);
        } else if (cnt > 6 * kNumSMs) {
            const size_t dsm = (size_t)c->lvl_max_c[l] * c->lvl_max_c[l] * sizeof(T);
            forward_level_kernel<T, true><<<cnt, kThreads / 2, dsm, st>>>(c->plan, lsn, Lx, dinv, xp, active);
        } else {
            forward_level_kernel<T, false><<<cnt, kThreads, 0, st>>>(c->plan, lsn, Lx, dinv, xp, active);
        }
    }
    for (int l = c->nlev - 1; l >= 0; --l) {
        const int cnt = c->h_lvl_ptr[l + 1] - c->h_lvl_ptr[l];
        const int* lsn = c->d_lvl_sn + c->h_lvl_ptr[l];
        const bool wide = cnt > 6 * kNumSMs;
        const size_t bsm = staged_backward_bytes<T>(c, l);
        if (c->opt.staged_solve && bsm <= kStagedSmemBytes) {
            launch_pdl(backward_level_staged_kernel<T>, cnt, wide ? kThreads / 2 : kThreads, bsm, st, c->plan, lsn,
                       (const T*)Lx, (const T*)dinv, xp, (int)staged_panel_elems(c, l), c->lvl_max_rb[l], active);
            continue;
        }
        const int dsz = wide ? c->lvl_max_c[l] * c->lvl_max_c[l] : 0;
        const size_t xsm = (size_t)c->lvl_max_rb[l] * sizeof(T);
        const size_t dbytes = wide ? (size_t)dsz * sizeof(T) : 64 * 64 * sizeof(T);   // dynamic or static
        const bool stage = dbytes + xsm <= kBackwardSmemBytes;
        const size_t sm = (size_t)dsz * sizeof(T) + (stage ? xsm : 0);
        const int nt = wide ? kThreads / 2 : kThreads;
        if (wide && stage)
            backward_level_kernel<T, true, true><<<cnt, nt, sm, st>>>(c->plan, lsn, Lx, dinv, xp, dsz, active);
        else if (wide)
            backward_level_kernel<T, false, true><<<cnt, nt, sm, st>>>(c->plan, lsn, Lx, dinv, xp, dsz, active);
        else if (stage)
            backward_level_kernel<T, true, false><<<cnt, nt, sm, st>>>(c->plan, lsn, Lx, dinv, xp, dsz, active);
        else
            backward_level_kernel<T, false, false><<<cnt, nt, sm, st>>>(c->plan, lsn, Lx, dinv, xp, dsz, active);
    }
    if (c->ntasks > 0)
        backward_subtree_kernel<T><<<c->ntasks, kSubtreeThreads,
                                     (size_t)(c->task_max_ccrb + c->task_max_cols) * sizeof(T), st>>>(
            c->plan, c->d_task_ptr, c->d_task_sn, Lx, dinv, xp, (int)c->task_max_ccrb, active);
}

void enqueue_triangular_solves(kkt_ctx* c, double* xp, cudaStream_t st, const int* active) {
    enqueue_triangular_solves<double>(c, c->d_Lx, c->d_dinv, xp, st, active);
}

// x <- K^{-1} x  (in and out may alias; uses w_xp)
kkt_status apply_kinv(kkt_ctx* c, const double* in, double* out, cudaStream_t st) {
    const int n = c->n;
    const int sp = span_begin(c, 2, st);
    c->stats.kinv_calls++;
    c->stats.launches += 2 + (c->flow ? 2LL + (flow_levels_only(c) ? 2 : 0) : 2LL * c->nlev + (c->ntasks > 0 ? 2 : 0));
    if (c->opt.solver == 1) {
        CUDA_TRY(c, cudaMemcpyAsync(c->w_xp, in, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        if (c->tri_exec) {
            CUDA_TRY(c, cudaGraphLaunch(c->tri_exec, st));
        } else {
            enqueue_bcr_solve(c, c->w_xp, st, nullptr);
        }
        CUDA_TRY(c, cudaMemcpyAsync(out, c->w_xp, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else if (c->cur_prec == 2) {
        gather_kernel<<<grid_for(n), kThreads, 0, st>>>(n, c->d_perm, in, as_df(c->w_xp), nullptr);
        if (c->tri_exec32) {
            CUDA_TRY(c, cudaGraphLaunch(c->tri_exec32, st));
        } else {
            enqueue_triangular_solves<df64>(c, as_df(c->d_Lx), as_df(c->d_dinv), as_df(c->w_xp), st, nullptr);
        }
        scatter_kernel<<<grid_for(n), kThreads, 0, st>>>(n, c->d_perm, as_df(c->w_xp), out, nullptr);
    } else if (c->cur_prec == 1) {
        gather_kernel<<<grid_for(n), kThreads, 0, st>>>(n, c->d_perm, in, c->w_xp32, nullptr);
        if (c->tri_exec32) {
            CUDA_TRY(c, cudaGraphLaunch(c->tri_exec32, st));
        } else {
            enqueue_triangular_solves<float>(c, c->d_Lx32, c->d_dinv32, c->w_xp32, st, nullptr);
        }
        scatter_kernel<<<grid_for(n), kThreads, 0, st>>>(n, c->d_perm, c->w_xp32, out, nullptr);
    } else {
        gather_kernel<<<grid_for(n), kThreads, 0, st>>>(n, c->d_perm, in, c->w_xp, nullptr);
        if (c->tri_exec && !c->capturing) {
            CUDA_TRY(c, cudaGraphLaunch(c->tri_exec, st));
        } else {
            enqueue_triangular_solves(c, c->w_xp, st, nullptr);
        }
        scatter_kernel<<<grid_for(n), kThreads, 0, st>>>(n, c->d_perm, c->w_xp, out, nullptr);
    }
    span_end(c, sp, st);
    CUDA_TRY(c, cudaGetLastError());
    return KKT_OK;
}

// Per-instance dot products of two dual-space vectors into cgs[4 i + slot].
void seg_dot(kkt_ctx* c, const double* a, const double* b, int slot, cudaStream_t st,
             const int* active = nullptr) {
    c->stats.launches += 2;
    if (c->nch_y > 0)
        seg_dot_partial_kernel<<<c->nch_y, kThreads, 0, st>>>(c->d_ch_y, a, b, c->d_part_y, active);
    constexpr int kWarps = kThreads / 32;
    seg_dot_final_kernel<<<(c->nb + kWarps - 1) / kWarps, kThreads, 0, st>>>(
        c->nb, c->d_chy_ptr, c->d_part_y, c->d_cgs, slot, active);
}

// r = b - K_orig v and the backward error of every instance (host sync):
// eta_i = ||r_i||_inf / (||K_i||_inf ||v_i||_inf + ||b_i||_inf).
kkt_status enqueue_residual(kkt_ctx* c, const double* bx, const double* by, const double* vx,
                            const double* vy, double* rx, double* ry, cudaStream_t st) {
    CUDA_TRY(c, cudaMemsetAsync(c->d_red, 0, 3 * (size_t)c->nb * sizeof(double), st));
    c->stats.launches += 1;
    residual_kernel<<<c->nch_xy, kThreads, 0, st>>>(
        c->d_ch_xy, c->n, c->d_wf_ptr, c->d_wf_col, c->d_wf_idx, c->f_W, c->d_j_ptr, c->d_j_col,
        c->d_jt_ptr, c->d_jt_row, c->d_jt_idx, c->f_J, c->f_sigma, c->f_delta_x, c->f_dvec, c->f_C,
        bx, by, vx, vy, rx, ry, c->d_red);
    return KKT_OK;
}

kkt_status residual(kkt_ctx* c, const double* bx, const double* by, const double* vx,
                    const double* vy, double* rx, double* ry, cudaStream_t st, std::vector<double>& eta) {
    const int nb = c->nb;
    TRY(enqueue_residual(c, bx, by, vx, vy, rx, ry, st));
    CUDA_TRY(c, cudaMemcpyAsync(c->h_red, c->d_red, 3 * (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c, cudaStreamSynchronize(st));
    eta.resize(nb);
    for (int i = 0; i < nb; ++i) {
        const double rmax = c->h_red[3 * i], vmax = c->h_red[3 * i + 1], bmax = c->h_red[3 * i + 2];
        const double den = c->h_knorm[i] * vmax + bmax;
        eta[i] = den > 0 ? rmax / den : (rmax > 0 ? INFINITY : 0.0);
    }
    return KKT_OK;
}

// Lifted-KKT preconditioner: d = M^{-1} r with M = [[H, J^T], [J, -D^{-1}]]
kkt_status lifted_precond(kkt_ctx* c, const double* rx, const double* ry, double* dx, double* dy,
                          cudaStream_t st) {
    const int n = c->n, m = c->m;
    c->stats.launches += 2;
    jt_axpy_kernel<<<grid_for(n), kThreads, 0, st>>>(n, c->d_jt_ptr, c->d_jt_row, c->d_jt_idx,
                                                     c->f_J, rx, ry, c->f_D, c->f_Dconst, 1.0,
                                                     c->w_t, nullptr);
    TRY(apply_kinv(c, c->w_t, dx, st));
    j_apply_kernel<<<grid_for(m), kThreads, 0, st>>>(m, c->d_j_ptr, c->d_j_col, c->f_J, dx, ry,
                                                     c->f_D, c->f_Dconst, dy, nullptr);
    return KKT_OK;
}

// One CG iteration on S_gamma = J K_gamma^{-1} J^T with the internal vectors
// (p = w_p, S p = w_sp, x = w_cgx, r = w_res), every kernel guarded by the
// device flag d_cg[0].
template <typename T>
void enqueue_cg_iteration(kkt_ctx* c, const T* Lx, const T* dinv, T* xp, cudaStream_t st) {
    const int n = c->n, m = c->m;
    const int* act = c->d_cg;
    if (c->opt.solver == 1) {
        jt_axpy_kernel<<<grid_for(n), kThreads, 0, st>>>(n, c->d_jt_ptr, c->d_jt_row, c->d_jt_idx, c->v_J,
                                                         nullptr, c->w_p, nullptr, 1.0, 1.0, c->w_tn, act);
        enqueue_bcr_solve(c, c->w_tn, st, act);
        j_apply_kernel<<<grid_for(m), kThreads, 0, st>>>(m, c->d_j_ptr, c->d_j_col, c->v_J, c->w_tn,
                                                         nullptr, nullptr, 1.0, c->w_sp, act);
    } else {
        // J^T p into the permuted vector, the solves, J x from it: the
        // permutations folded into the products
        jt_gather_kernel<T><<<grid_for(n), kThreads, 0, st>>>(n, c->d_perm, c->d_jt_ptr, c->d_jt_row, c->d_jt_idx,
                                                              c->v_J, c->w_p, xp, act);
        enqueue_triangular_solves<T>(c, Lx, dinv, xp, st, act);
        j_apply_perm_kernel<T><<<grid_for(m), kThreads, 0, st>>>(m, c->d_j_ptr, c->d_j_col, c->v_J, c->d_iperm,
                                                                 xp, c->w_sp, act);
    }
    seg_dot(c, c->w_p, c->w_sp, 2, st, act);
    if (c->nch_y > 0)
        cg_update_xr_kernel<<<c->nch_y, kThreads, 0, st>>>(c->d_ch_y, c->d_cgs, c->d_cgi, c->w_p, c->w_sp,
                                                           c->w_cgx, c->w_res, act);
    seg_dot(c, c->w_res, c->w_res, 1, st, act);
    if (c->nch_y > 0)
        cg_update_p_kernel<<<c->nch_y, kThreads, 0, st>>>(c->d_ch_y, c->d_cgs, c->d_cgi, c->w_res, c->w_p, act);
    cg_check_kernel<<<1, kThreads, 0, st>>>(c->nb, c->d_cgs, c->d_cgi, c->opt.max_cg, c->d_cg);
}

// Capture the triangular-solve sequence and (HyKKT) one CG iteration as
// CUDA graphs; they only touch buffers owned by the context.
kkt_status capture_graphs(kkt_ctx* c) {
    cudaStream_t cs;
    CUDA_TRY(c, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    auto capture = [&](auto&& body, cudaGraph_t* g, cudaGraphExec_t* e, size_t* nodes) -> cudaError_t {
        cudaError_t err = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (err != cudaSuccess) return err;
        body();
        err = cudaStreamEndCapture(cs, g);
        if (err != cudaSuccess) return err;
        err = cudaGraphInstantiate(e, *g, 0);
        if (err != cudaSuccess) return err;
        return cudaGraphGetNodes(*g, nullptr, nodes);
    };
    cudaError_t err = capture([&] {
        if (c->opt.solver == 1) enqueue_bcr_solve(c, c->w_xp, cs, nullptr);
        else enqueue_triangular_solves(c, c->w_xp, cs, nullptr);
    }, &c->tri_graph, &c->tri_exec, &c->tri_nodes);
    if (err == cudaSuccess && c->opt.scheme == KKT_HYKKT)
        err = capture([&] { enqueue_cg_iteration<double>(c, c->d_Lx, c->d_dinv, c->w_xp, cs); },
                      &c->cg_graph, &c->cg_exec, &c->cg_nodes);
    if (err == cudaSuccess && c->opt.precision == 2) {
        err = capture([&] { enqueue_triangular_solves<df64>(c, as_df(c->d_Lx), as_df(c->d_dinv), as_df(c->w_xp), cs,
                                                            nullptr); },
                      &c->tri_graph32, &c->tri_exec32, &c->tri_nodes32);
        if (err == cudaSuccess && c->opt.scheme == KKT_HYKKT)
            err = capture([&] { enqueue_cg_iteration<df64>(c, as_df(c->d_Lx), as_df(c->d_dinv), as_df(c->w_xp), cs); },
                          &c->cg_graph32, &c->cg_exec32, &c->cg_nodes32);
    }
    if (err == cudaSuccess && c->opt.precision == 1) {
        err = capture([&] { enqueue_triangular_solves<float>(c, c->d_Lx32, c->d_dinv32, c->w_xp32, cs, nullptr); },
                      &c->tri_graph32, &c->tri_exec32, &c->tri_nodes32);
        if (err == cudaSuccess && c->opt.scheme == KKT_HYKKT)
            err = capture([&] { enqueue_cg_iteration<float>(c, c->d_Lx32, c->d_dinv32, c->w_xp32, cs); },
                          &c->cg_graph32, &c->cg_exec32, &c->cg_nodes32);
    }
    cudaStreamDestroy(cs);
    if (err != cudaSuccess) return set_err(c, KKT_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(err));
    return KKT_OK;
}

// HyKKT inner solve (Eq. hykkt / Eq. schurcomp): d = K_orig^{-1} r up to the
// CG tolerance, one CG per instance (instances with d_act = 0 keep dy = 0).
// Adds every instance's CG iterations to its[i].  The CG iterations run as
// graph launches in batches of kCgBatch between convergence checks; the
// device flags make the iterations after convergence no-ops, so the counts
// equal those of a check after every iteration.
kkt_status hykkt_inner(kkt_ctx* c, const double* rx, const double* ry, double* dx, double* dy,
                       cudaStream_t st, std::vector<int>& its) {
    const int n = c->n, m = c->m, nb = c->nb;
    const double gamma = c->f_Dconst;
    c->stats.launches += 4;
    // r_gamma = r_x + gamma J^T r_y ; q = K_gamma^{-1} r_gamma
    jt_axpy_kernel<<<grid_for(n), kThreads, 0, st>>>(n, c->d_jt_ptr, c->d_jt_row, c->d_jt_idx,
                                                     c->f_J, rx, ry, nullptr, 1.0, gamma, c->w_rg, nullptr);
    TRY(apply_kinv(c, c->w_rg, c->w_q, st));
    // rhs = J q - r_y (the CG residual starts at rhs, x at 0)
    j_apply_kernel<<<grid_for(m), kThreads, 0, st>>>(m, c->d_j_ptr, c->d_j_col, c->f_J, c->w_q, ry,
                                                     nullptr, 1.0, c->w_res, nullptr);
    CUDA_TRY(c, cudaMemsetAsync(c->w_cgx, 0, m * sizeof(double), st));
    CUDA_TRY(c, cudaMemcpyAsync(c->w_p, c->w_res, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
    seg_dot(c, c->w_res, c->w_res, 0, st);
    cg_init_kernel<<<1, kThreads, 0, st>>>(nb, c->d_cgs, c->d_cgi, c->d_act, c->opt.tol_cg, c->opt.max_cg,
                                           c->d_cg);
    const int sp = span_begin(c, 3, st);
    while (true) {
        const bool f32 = c->cur_prec != 0;
        for (int b = 0; b < kCgBatch; ++b) {
            cudaGraphExec_t ex = f32 ? c->cg_exec32 : c->cg_exec;
            if (ex) {
                CUDA_TRY(c, cudaGraphLaunch(ex, st));
            } else if (c->cur_prec == 2) {
                enqueue_cg_iteration<df64>(c, as_df(c->d_Lx), as_df(c->d_dinv), as_df(c->w_xp), st);
            } else if (f32) {
                enqueue_cg_iteration<float>(c, c->d_Lx32, c->d_dinv32, c->w_xp32, st);
            } else {
                enqueue_cg_iteration<double>(c, c->d_Lx, c->d_dinv, c->w_xp, st);
            }
        }
        c->stats.launches += (long long)kCgBatch * (long long)(f32 ? c->cg_nodes32 : c->cg_nodes);
        CUDA_TRY(c, cudaMemcpyAsync(c->h_cg, c->d_cg, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(c, cudaStreamSynchronize(st));
        if (c->h_cg[0] == 0) break;
    }
    span_end(c, sp, st);
    CUDA_TRY(c, cudaMemcpyAsync(c->h_int, c->d_cgi, 2 * (size_t)nb * sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c, cudaStreamSynchronize(st));
    int it_max = 0;
    for (int i = 0; i < nb; ++i) {
        its[i] += c->h_int[2 * i + 1];
        it_max = std::max(it_max, c->h_int[2 * i + 1]);
    }
    c->stats.kinv_calls += it_max;
    // dx = K_gamma^{-1} (r_gamma - J^T dy)
    jt_axpy_kernel<<<grid_for(n), kThreads, 0, st>>>(n, c->d_jt_ptr, c->d_jt_row, c->d_jt_idx,
                                                     c->f_J, c->w_rg, c->w_cgx, nullptr, 1.0, -1.0,
                                                     c->w_tn, nullptr);
    TRY(apply_kinv(c, c->w_tn, dx, st));
    CUDA_TRY(c, cudaMemcpyAsync(dy, c->w_cgx, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
    return KKT_OK;
}

// Zero the panels, assemble, factorise (subtree tasks, levels), normalise to
// unit diagonal: everything the numeric factorisation enqueues for the panel
// precision T.  The fail words (one per instance) are reset first to
// kNoFail, above every column index.
constexpr int kNoFail = 0x7f7f7f7f;

// Block cyclic reduction: assemble the dense blocks, then per level the
// eliminations (factor panels, fill couplings) and the survivor updates.
kkt_status enqueue_bcr_factor(kkt_ctx* c, double delta_x, cudaStream_t st) {
    const int b = c->bcr_b, N = c->bcr_N;
    const long long bb = (long long)b * b;
    const int sp_a = span_begin(c, 0, st);
    CUDA_TRY(c, cudaMemsetAsync(c->d_bcr, 0, (size_t)2 * N * bb * sizeof(double), st));
    assemble_kernel<double><<<grid_for(c->bcr_nk), kThreads, 0, st>>>(
        c->bcr_nk, c->d_bcr_slot, c->d_bcr_sptr, c->d_bcr_src, c->f_W, c->v_Js, c->f_sigma, delta_x,
        c->f_dvec, c->d_bcr, (long long)2 * N * bb, c->d_berr);
    span_end(c, sp_a, st);
    CUDA_TRY(c, cudaMemsetAsync(c->d_fail, 0x7f, sizeof(int), st));
    const FailSink fs{c->d_fail, nullptr};
    const int sp_f = span_begin(c, 1, st);
    c->stats.factor_calls++;
    double* A = c->d_bcr;
    double* C = c->d_bcr + (size_t)N * bb;
    for (int l = 0; l < c->bcr_nlev; ++l) {
        const int ne = c->bcr_elim_ptr[l + 1] - c->bcr_elim_ptr[l];
        const int ns = c->bcr_surv_ptr[l + 1] - c->bcr_surv_ptr[l];
        if (ne > 0)
            bcr_elim_kernel<<<ne, kThreads, (size_t)3 * bb * sizeof(double), st>>>(
                b, c->d_bcr_elim + c->bcr_elim_ptr[l], A, C, c->d_bcr_pn, c->d_dinv, fs);
        if (ns > 0)
            bcr_update_kernel<<<ns, kThreads, (size_t)2 * bb * sizeof(double), st>>>(
                b, c->d_bcr_surv + c->bcr_surv_ptr[l], A, c->d_bcr_pn);
        c->stats.launches += 2;
        c->stats.factor_launches += 2;
    }
    span_end(c, sp_f, st);
    CUDA_TRY(c, cudaGetLastError());
    return KKT_OK;
}

// Shared memory requested by the fused launches that must run one CTA per
// SM (more than half of an SM's 228 KB): two CTAs on one SM would put both
// pivot chains on sub-partition 0 and its single FP64 unit.
constexpr size_t kOneCtaPerSmBytes = 120 * 1024;

// panel types the fused narrow-level kernels are instantiated for
template <typename T>
constexpr bool kFusedType = std::is_same<T, double>::value || std::is_same<T, float>::value;

// One split level of supernodes with <= 32 columns and <= 128 rows below:
// one CTA per supernode when the level fills the SMs, otherwise a cluster of
// K = 2, 4 or 8 CTAs per supernode sharing its rows and Schur pairs, K the
// largest for which the level's clusters are resident at once (clusters of
// 8 one-per-SM CTAs: 15 at a time on GB300, so a level of 16 supernodes
// takes K = 4 in one wave rather than K = 8 in two).
template <typename T>
kkt_status launch_fused_level(kkt_ctx* c, int l, int cnt, const int* lsn, T* Lx, FailSink fs, T* dinv,
                              cudaStream_t st) {
    const size_t mc = (size_t)c->lvl_max_c[l], mrb = (size_t)c->lvl_max_rb[l];
    int K = 1;
    while (K < kFusedClusterMax && (long long)cnt * K * 2 <= kNumSMs) {
        const int q = c->fused_clusters[K == 1 ? 1 : K == 2 ? 2 : 3];
        if (q > 0 && cnt > q) break;   // clusters of 2K CTAs would not all be resident at once
        K *= 2;
    }
    if (K == 1) {
        const size_t fsm = ((size_t)c->lvl_max_rc[l] + mrb * mc) * sizeof(T);
        if (cnt <= kNumSMs)   // one CTA per SM: the chain keeps its sub-partition's FP64 unit to itself
            factor_fused_kernel<T, true><<<cnt, kFusedThreads, std::max(fsm, kOneCtaPerSmBytes), st>>>(
                c->plan, lsn, 1, Lx, fs, dinv);
        else
            factor_fused_kernel<T, false><<<cnt, kFusedThreads, fsm, st>>>(c->plan, lsn, 1, Lx, fs, dinv);
        CUDA_TRY(c, cudaGetLastError());
        return KKT_OK;
    }
    const size_t own = (mc + (mrb + K - 1) / K) * mc;
    const size_t fsm = (own + (size_t)c->lvl_max_rc[l] + mrb * mc) * sizeof(T);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(cnt * K), 1, 1);
    cfg.blockDim = dim3(kFusedThreads, 1, 1);
    cfg.dynamicSmemBytes = std::max(fsm, kOneCtaPerSmBytes);   // one CTA of the cluster per SM
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)K;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CUDA_TRY(c, cudaLaunchKernelEx(&cfg, factor_fused_cluster_kernel<T>, c->plan, lsn, Lx, fs, dinv));
    return KKT_OK;
}

// after_assembly (captured graphs only): an external event recorded between
// the assembly and the factor kernels, for the graph's phase times
template <typename T>
kkt_status enqueue_numeric_factor(kkt_ctx* c, T* Lx, T* dinv, double delta_x, cudaStream_t st,
                                  cudaEvent_t after_assembly = nullptr) {
    if (c->inst_on_pending) {
        CUDA_TRY(c, cudaMemcpyAsync(c->d_inst_on, c->h_inst_on, (size_t)c->nb * sizeof(int), cudaMemcpyHostToDevice,
                                    st));
        c->inst_on_pending = false;
    }
    const int sp_a = span_begin(c, 0, st);
    CUDA_TRY(c, cudaMemsetAsync(Lx, 0, (size_t)c->panel * sizeof(T), st));
    assemble_kernel<T><<<grid_for(c->nk), kThreads, 0, st>>>(c->nk, c->d_k_slot, c->d_k_sptr, c->d_k_src,
                                                             c->f_W, c->v_Js, c->f_sigma, delta_x,
                                                             c->f_dvec, Lx, c->panel, c->d_berr);
    span_end(c, sp_a, st);
    if (after_assembly) CUDA_TRY(c, cudaEventRecordWithFlags(after_assembly, st, cudaEventRecordExternal));
    CUDA_TRY(c, cudaMemsetAsync(c->d_fail, 0x7f, (size_t)c->nb * sizeof(int), st));
    const FailSink fs{c->d_fail, c->nb > 1 ? c->d_col_inst : nullptr};
    const int sp_f = span_begin(c, 1, st);
    c->stats.factor_calls++;
    c->stats.launches += 2 + c->nlev;
    c->stats.factor_launches += c->nlev;
    if (c->ntasks > 0) {
        factor_subtree_kernel<T><<<c->ntasks, kSubtreeThreads, (size_t)c->task_max_rc * sizeof(T), st>>>(
            c->plan, c->d_task_ptr, c->d_task_sn, Lx, fs, dinv);
        c->stats.launches += 1;
        c->stats.factor_launches += 1;
    }
    for (int l = 0; l < c->nlev; ++l) {
        const int cnt = c->h_lvl_ptr[l + 1] - c->h_lvl_ptr[l];
        const int* lsn = c->d_lvl_sn + c->h_lvl_ptr[l];
        if constexpr (kFusedType<T>) {
            if (c->lvl_fused[l]) {
                TRY(launch_fused_level<T>(c, l, cnt, lsn, Lx, fs, dinv, st));
                continue;
            }
        }
        if (!c->lvl_split[l]) {
            // (Levels the fused kernel does not take: double-float panels,
            // or supernodes wider than 32 columns / 128 rows below.)
            // At 60 registers a thread, 256-thread CTAs fit four to an SM: a
            // level of 600-1200 narrow supernodes (c <= 32) takes two waves,
            // where 128-thread CTAs (same warps per SM, twice the supernodes
            // in flight) take one.  Wider supernodes or other counts keep 256.
            const bool half = cnt > 4 * kNumSMs && cnt <= 8 * kNumSMs && c->lvl_max_c[l] <= 32;
            long long need = std::min<long long>(c->lvl_max_rc[l], kSmemCapElems);
            factor_level_kernel<T><<<cnt, half ? kThreads / 2 : kThreads, (size_t)need * sizeof(T), st>>>(
                c->plan, lsn, Lx, fs, need, dinv);
            continue;
        }
        const size_t dsm = (size_t)c->lvl_max_c[l] * c->lvl_max_c[l] * sizeof(T);
        // the small top levels: one cluster launch instead of three launches
        const size_t csm = std::max(dsm, (size_t)c->lvl_max_rb[l] * c->lvl_max_c[l] * sizeof(T));
        if (cnt <= kClusterLevelMax && csm <= kClusterSmemBytes) {
            narrow_level_cluster_kernel<T><<<cnt * kClusterCtas, kThreads, csm, st>>>(c->plan, lsn, Lx, fs, dinv);
            continue;
        }
        potrf_diag_kernel<T><<<cnt, kThreads, dsm, st>>>(c->plan, lsn, Lx, fs, dinv);
        const int nt = c->lvl_trsm_ptr[l + 1] - c->lvl_trsm_ptr[l];
        if (nt > 0)
            trsm_rows_kernel<T><<<nt, 32 * kTrsmWarps, 0, st>>>(
                c->plan, c->d_trsm_tasks + c->lvl_trsm_ptr[l], Lx, dinv);
        const int ny = c->lvl_syrk_ptr[l + 1] - c->lvl_syrk_ptr[l];
        if (ny > 0) {
            const size_t l21 = (size_t)c->lvl_max_rb[l] * c->lvl_max_c[l] * sizeof(T);
            const int stage = l21 <= kSyrkStageBytes;
            syrk_stage_kernel<T><<<ny, kThreads, stage ? l21 : 0, st>>>(
                c->plan, c->d_syrk_tasks + c->lvl_syrk_ptr[l], Lx, stage);
        }
        c->stats.launches += 2;
    }
    const int n_norm = kFusedType<T> ? c->n_norm_fused : c->n_norm;
    if (n_norm > 0) {
        normalize_panels_kernel<T><<<std::min(n_norm, 152 * 16), kThreads, 0, st>>>(
            c->plan, kFusedType<T> ? c->d_norm_list_fused : c->d_norm_list, n_norm, Lx, dinv);
        c->stats.launches += 1;
    }
    span_end(c, sp_f, st);
    CUDA_TRY(c, cudaGetLastError());
    return KKT_OK;
}

}  // namespace

extern "C" {

void kkt_default_options(kkt_options* o) {
    if (!o) return;
    o->scheme = KKT_LIFTED;
    o->leaf_size = 8;
    o->relax_cols = 32;
    o->relax_zeros = 128;
    o->max_width = 32;
    o->delta = 1e-8;
    o->gamma = 1e4;
    o->tol_refine = 1e-10;
    o->tol_cg = 1e-10;
    o->max_refine = 20;
    o->max_cg = 200;
    o->target_relaxed = 0;
    o->subtree_cols = 32;
    o->precision = 0;
    o->solver = 0;
    o->block = 0;
    o->staged_solve = 1;
}

namespace {
kkt_status new_ctx(const kkt_options* opt, kkt_ctx** out) {
    if (!out) return set_err(nullptr, KKT_ERR_ARG, "out is NULL");
    *out = nullptr;
    kkt_ctx* c = new (std::nothrow) kkt_ctx();
    if (!c) return set_err(nullptr, KKT_ERR_OOM, "host allocation failed");
    if (opt) c->opt = *opt; else kkt_default_options(&c->opt);
    if (c->opt.scheme != KKT_LIFTED && c->opt.scheme != KKT_HYKKT) {
        delete c;
        return set_err(nullptr, KKT_ERR_ARG, "unknown scheme");
    }
    if (c->opt.precision < 0 || c->opt.precision > 2) {
        delete c;
        return set_err(nullptr, KKT_ERR_ARG, "precision must be 0 (FP64), 1 (FP32) or 2 (double-float factor)");
    }
    if (c->opt.solver != 0 && c->opt.solver != 1) {
        delete c;
        return set_err(nullptr, KKT_ERR_ARG, "solver must be 0 (supernodal) or 1 (block tridiagonal)");
    }
    if (c->opt.max_width <= 0 || c->opt.max_width > 64) c->opt.max_width = 64;
    *out = c;
    return KKT_OK;
}

// Allocation-free backsolve: device address of its static scratch (below).
constexpr int kMaxDevices = 64;
double* g_noalloc_ptr[kMaxDevices] = {};
std::mutex g_noalloc_mu;

// Address of the static scratch on the current device (cached per device).
cudaError_t noalloc_lookup(double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        if (!p) return cudaErrorInvalidSymbol;
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

SymbolicOptions symbolic_options(const kkt_options& o) {
    SymbolicOptions so;
    so.leaf_size = o.leaf_size;
    so.relax_cols = o.relax_cols;
    so.relax_zeros = o.relax_zeros;
    so.max_width = o.max_width;
    return so;
}

// After c->sym, sizes and batch offsets are set: tree height, device plan,
// kernel attributes and graphs.  Destroys c on failure.
kkt_status finish_ctx(kkt_ctx* c, const int* W_colptr, const int* W_rowind, const int* J_rowptr,
                      const int* J_colind, bool device, kkt_ctx** out) {
    const int ns = c->sym.ns();
    c->h_sn_c.resize(ns);
    c->h_sn_r.resize(ns);
    for (int s = 0; s < ns; ++s) {
        c->h_sn_c[s] = c->sym.sn_ptr[s + 1] - c->sym.sn_ptr[s];
        c->h_sn_r[s] = c->sym.sn_rowptr[s + 1] - c->sym.sn_rowptr[s];
    }
    {
        std::vector<int> level(ns, 0);
        int nlev = 0;
        for (int s = 0; s < ns; ++s) {
            if (c->sym.sn_parent[s] >= 0)
                level[c->sym.sn_parent[s]] = std::max(level[c->sym.sn_parent[s]], level[s] + 1);
            nlev = std::max(nlev, level[s] + 1);
        }
        c->tree_levels = nlev;
    }
    if (device) {
        kkt_status st = build_plan(c, W_colptr, W_rowind, J_rowptr, J_colind);
        if (st == KKT_OK && c->opt.solver == 1) st = build_bcr(c, W_colptr, W_rowind, J_rowptr, J_colind);
        if (st == KKT_OK && (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
                             cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess ||
                             cudaEventCreateWithFlags(&c->ev_side, cudaEventDisableTiming) != cudaSuccess))
            st = set_err(c, KKT_ERR_CUDA, "side stream or events could not be created");
        if (st != KKT_OK) {
            set_err(nullptr, st, c->err);
            kkt_destroy(c);
            return st;
        }
        cudaFuncSetAttribute(bcr_elim_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(3 * kBcrMaxBlock * kBcrMaxBlock * sizeof(double)));
        cudaFuncSetAttribute(bcr_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(2 * kBcrMaxBlock * kBcrMaxBlock * sizeof(double)));
        cudaFuncSetAttribute(factor_level_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kSmemCapElems * sizeof(double)));
        cudaFuncSetAttribute(factor_level_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kSmemCapElems * sizeof(float)));
        cudaFuncSetAttribute(factor_level_kernel<df64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kSmemCapElems * sizeof(df64)));
        cudaFuncSetAttribute(narrow_level_cluster_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kClusterSmemBytes);
        cudaFuncSetAttribute(narrow_level_cluster_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kClusterSmemBytes);
        cudaFuncSetAttribute(narrow_level_cluster_kernel<df64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kClusterSmemBytes);
        {
            const int fb = std::max((int)kOneCtaPerSmBytes,
                                    (int)(((kFusedMaxC + kFusedMaxRb) * kFusedMaxC + kFusedMaxRb * kFusedMaxC) * sizeof(double)));
            const int fcb = std::max((int)kOneCtaPerSmBytes,
                                     fb + (int)((kFusedMaxC + kFusedMaxRb / 2) * kFusedMaxC * sizeof(double)));
            cudaFuncSetAttribute(factor_fused_kernel<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, fb);
            cudaFuncSetAttribute(factor_fused_kernel<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, fb);
            cudaFuncSetAttribute(factor_fused_kernel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, fb);
            cudaFuncSetAttribute(factor_fused_kernel<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, fb);
            cudaFuncSetAttribute(factor_fused_cluster_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, fcb);
            cudaFuncSetAttribute(factor_fused_cluster_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, fcb);
            for (int q = 1; q <= 3; ++q) {   // launches of 1 CTA per SM (kOneCtaPerSmBytes), K = 2^q
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3((unsigned)(kNumSMs << q), 1, 1);
                cfg.blockDim = dim3(kFusedThreads, 1, 1);
                cfg.dynamicSmemBytes = kOneCtaPerSmBytes;
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeClusterDimension;
                attr[0].val.clusterDim.x = 1u << q;
                attr[0].val.clusterDim.y = 1;
                attr[0].val.clusterDim.z = 1;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                int nc = 0;
                if (cudaOccupancyMaxActiveClusters(&nc, factor_fused_cluster_kernel<double>, &cfg) == cudaSuccess)
                    c->fused_clusters[q] = nc;
                else
                    cudaGetLastError();   // unknown: the SM-count rule alone
            }
        }
        cudaFuncSetAttribute(syrk_stage_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSyrkStageBytes);
        cudaFuncSetAttribute(syrk_stage_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSyrkStageBytes);
        cudaFuncSetAttribute(syrk_stage_kernel<df64>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSyrkStageBytes);
        set_backward_smem_limit<df64>();
        set_backward_smem_limit<double>();
        set_backward_smem_limit<float>();
        setup_flow(c);
        st = capture_graphs(c);
        if (st != KKT_OK) {
            set_err(nullptr, st, c->err);
            kkt_destroy(c);
            return st;
        }
        // a failed lookup only disables kkt_backsolve_noalloc
        const cudaError_t e = noalloc_lookup(&c->noalloc_ptr);
        if (e != cudaSuccess) {
            c->noalloc_ptr = nullptr;
            c->noalloc_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            cudaGetLastError();
        }
    }
    c->device_ready = device;
    c->analysed_precision = c->opt.precision;
    *out = c;
    return KKT_OK;
}

kkt_status analyse_common(int n, int m, const int* W_colptr, const int* W_rowind,
                          const int* J_rowptr, const int* J_colind, const kkt_options* opt,
                          bool device, kkt_ctx** out) {
    if (!out) return set_err(nullptr, KKT_ERR_ARG, "out is NULL");
    *out = nullptr;
    kkt_ctx* c = nullptr;
    TRY(new_ctx(opt, &c));
    c->n = n;
    c->m = m;
    std::string e;
    try {
        Graph g;
        e = build_graph(n, m, W_colptr, W_rowind, J_rowptr, J_colind, g);
        if (e.empty()) {
            c->nnzW = W_colptr[n];
            c->nnzJ = J_rowptr[m];
            e = analyse(g, symbolic_options(c->opt), c->sym);
        }
    } catch (const std::bad_alloc&) {
        delete c;
        return set_err(nullptr, KKT_ERR_OOM, "kkt_analyse: host allocation failed");
    } catch (const std::exception& ex) {
        delete c;
        return set_err(nullptr, KKT_ERR_INTERNAL, std::string("kkt_analyse: ") + ex.what());
    }
    if (!e.empty()) {
        delete c;
        return set_err(nullptr, KKT_ERR_ARG, "kkt_analyse: " + e);
    }
    c->nb = 1;
    c->h_xoff = {0, n};
    c->h_yoff = {0, m};
    return finish_ctx(c, W_colptr, W_rowind, J_rowptr, J_colind, device, out);
}

// Batch: every instance analysed on its own (worker threads), the analyses
// concatenated, the union's patterns built for the plan.
kkt_status analyse_batch(int count, const int* n, const int* m, const int* const* W_colptr,
                         const int* const* W_rowind, const int* const* J_rowptr,
                         const int* const* J_colind, const kkt_options* opt, bool device,
                         kkt_ctx** out) {
    if (!out) return set_err(nullptr, KKT_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (count < 1 || !n || !m || !W_colptr || !W_rowind || !J_rowptr || !J_colind)
        return set_err(nullptr, KKT_ERR_ARG, "kkt_analyse_batch: count < 1 or NULL array");
    long long nt = 0, mt = 0, wt = 0, jt = 0;
    for (int i = 0; i < count; ++i) {
        if (n[i] < 1 || m[i] < 0 || !W_colptr[i] || !W_rowind[i] || !J_rowptr[i] || !J_colind[i])
            return set_err(nullptr, KKT_ERR_ARG, "kkt_analyse_batch: bad instance " + std::to_string(i));
        nt += n[i];
        mt += m[i];
        wt += W_colptr[i][n[i]];
        jt += J_rowptr[i][m[i]];
    }
    if (nt + mt > 0x7fffffffLL || wt > 0x7fffffffLL || jt > 0x7fffffffLL)
        return set_err(nullptr, KKT_ERR_ARG, "kkt_analyse_batch: the union exceeds 32-bit indices");
    kkt_ctx* c = nullptr;
    TRY(new_ctx(opt, &c));
    std::vector<Symbolic> parts(count);
    std::vector<std::string> errs(count);
    SymbolicOptions so = symbolic_options(c->opt);
    so.parallel = false;   // the instances themselves run on the worker threads
    std::atomic<int> next(0);
    auto work = [&]() {
        for (int i = next++; i < count; i = next++) {
            try {
                Graph g;
                errs[i] = build_graph(n[i], m[i], W_colptr[i], W_rowind[i], J_rowptr[i], J_colind[i], g);
                if (errs[i].empty()) errs[i] = analyse(g, so, parts[i]);
            } catch (const std::exception& ex) {
                errs[i] = std::string("analysis failed: ") + ex.what();
            }
        }
    };
    const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
    const int nw = std::min(count, std::min(hw, 32));
    std::vector<std::thread> pool;
    for (int w = 1; w < nw; ++w) pool.emplace_back(work);
    work();
    for (auto& t : pool) t.join();
    for (int i = 0; i < count; ++i)
        if (!errs[i].empty()) {
            delete c;
            return set_err(nullptr, KKT_ERR_ARG, "kkt_analyse_batch: instance " + std::to_string(i) + ": " + errs[i]);
        }
    concat(parts, c->sym);
    std::vector<Symbolic>().swap(parts);
    c->n = (int)nt;
    c->m = (int)mt;
    c->nb = count;
    c->h_xoff.assign(count + 1, 0);
    c->h_yoff.assign(count + 1, 0);
    std::vector<int> Wc(nt + 1, 0), Wr, Jr(mt + 1, 0), Jc;
    Wr.reserve(wt);
    Jc.reserve(jt);
    for (int i = 0; i < count; ++i) {
        const int x0 = c->h_xoff[i], y0 = c->h_yoff[i];
        const int w0 = (int)Wr.size(), j0 = (int)Jc.size();
        for (int k = 0; k < n[i]; ++k) Wc[x0 + k + 1] = w0 + W_colptr[i][k + 1];
        for (int q = 0; q < W_colptr[i][n[i]]; ++q) Wr.push_back(W_rowind[i][q] + x0);
        for (int r = 0; r < m[i]; ++r) Jr[y0 + r + 1] = j0 + J_rowptr[i][r + 1];
        for (int q = 0; q < J_rowptr[i][m[i]]; ++q) Jc.push_back(J_colind[i][q] + x0);
        c->h_xoff[i + 1] = x0 + n[i];
        c->h_yoff[i + 1] = y0 + m[i];
    }
    c->nnzW = (int)wt;
    c->nnzJ = (int)jt;
    return finish_ctx(c, Wc.data(), Wr.data(), Jr.data(), Jc.data(), device, out);
}
}  // namespace

kkt_status kkt_analyse(int n, int m, const int* W_colptr, const int* W_rowind, const int* J_rowptr,
                       const int* J_colind, const kkt_options* opt, kkt_ctx** out) {
    return analyse_common(n, m, W_colptr, W_rowind, J_rowptr, J_colind, opt, true, out);
}

kkt_status kkt_analyse_host(int n, int m, const int* W_colptr, const int* W_rowind,
                            const int* J_rowptr, const int* J_colind, const kkt_options* opt,
                            kkt_ctx** out) {
    return analyse_common(n, m, W_colptr, W_rowind, J_rowptr, J_colind, opt, false, out);
}

kkt_status kkt_analyse_batch(int count, const int* n, const int* m, const int* const* W_colptr,
                             const int* const* W_rowind, const int* const* J_rowptr,
                             const int* const* J_colind, const kkt_options* opt, kkt_ctx** out) {
    return analyse_batch(count, n, m, W_colptr, W_rowind, J_rowptr, J_colind, opt, true, out);
}

kkt_status kkt_analyse_batch_host(int count, const int* n, const int* m, const int* const* W_colptr,
                                  const int* const* W_rowind, const int* const* J_rowptr,
                                  const int* const* J_colind, const kkt_options* opt, kkt_ctx** out) {
    return analyse_batch(count, n, m, W_colptr, W_rowind, J_rowptr, J_colind, opt, false, out);
}

kkt_status kkt_batch_layout(const kkt_ctx* c, int* count, int* x_off, int* y_off) {
    if (!c) return KKT_ERR_ARG;
    if (count) *count = c->nb;
    if (x_off) std::copy(c->h_xoff.begin(), c->h_xoff.end(), x_off);
    if (y_off) std::copy(c->h_yoff.begin(), c->h_yoff.end(), y_off);
    return KKT_OK;
}

// Autotuner of the supernode partition for a batch: the candidates differ in
// the relaxed amalgamation (width and explicit-zero budget), the width cut
// and the small-subtree threshold, which together fix the panel (tile)
// shapes every factor kernel works on.  Each candidate is analysed on an
// evenly spaced sample of the instances and its numeric factorisation timed
// on the device with synthetic SPD values (W = 0, Sigma = 1, J = 1, D = 1:
// K = I + J^T J); the fastest wins.
kkt_status kkt_autotune_batch(int count, const int* n, const int* m, const int* const* W_colptr,
                              const int* const* W_rowind, const int* const* J_rowptr,
                              const int* const* J_colind, const kkt_options* base, int sample,
                              cudaStream_t stream, kkt_options* best, double* best_ms) {
    if (count < 1 || !n || !m || !W_colptr || !W_rowind || !J_rowptr || !J_colind || !best)
        return set_err(nullptr, KKT_ERR_ARG, "kkt_autotune_batch: bad arguments");
    kkt_options b0;
    if (base) b0 = *base; else kkt_default_options(&b0);
    const int ns = std::max(1, std::min(count, sample > 0 ? sample : 32));
    std::vector<int> pick(ns);
    for (int i = 0; i < ns; ++i) pick[i] = (int)((long long)i * count / ns);
    std::vector<int> sn(ns), sm(ns);
    std::vector<const int*> wc(ns), wr(ns), jr(ns), jc(ns);
    for (int i = 0; i < ns; ++i) {
        const int q = pick[i];
        sn[i] = n[q];
        sm[i] = m[q];
        wc[i] = W_colptr[q];
        wr[i] = W_rowind[q];
        jr[i] = J_rowptr[q];
        jc[i] = J_colind[q];
    }
    struct Cand { int relax_cols, relax_zeros, max_width, subtree_cols; };
    const Cand cands[] = {{32, 128, 64, 48}, {16, 64, 64, 48}, {48, 1024, 64, 48}, {64, 4096, 64, 48},
                          {32, 128, 32, 48}, {32, 128, 64, 0},  {32, 128, 64, 24},  {0, 0, 64, 48}};
    double best_t = INFINITY;
    kkt_options won = b0;
    for (const Cand& cd : cands) {
        kkt_options o = b0;
        o.scheme = KKT_LIFTED;
        o.delta = 1.0;
        o.precision = b0.precision;
        o.relax_cols = cd.relax_cols;
        o.relax_zeros = cd.relax_zeros;
        o.max_width = cd.max_width;
        o.subtree_cols = cd.subtree_cols;
        kkt_ctx* c = nullptr;
        TRY(analyse_batch(ns, sn.data(), sm.data(), wc.data(), wr.data(), jr.data(), jc.data(), &o, true, &c));
        double* buf = nullptr;
        const size_t nw = std::max(1, c->nnzW), nj = std::max(1, c->nnzJ);
        cudaError_t e = cudaMalloc((void**)&buf, (nw + nj + c->n) * sizeof(double));
        if (e != cudaSuccess) {
            kkt_destroy(c);
            return set_err(nullptr, KKT_ERR_OOM, "kkt_autotune_batch: device allocation failed");
        }
        double *dW = buf, *dJ = buf + nw, *dS = buf + nw + nj;
        fill_kernel<<<grid_for((long long)nw), kThreads, 0, stream>>>((int)nw, 0.0, dW);
        fill_kernel<<<grid_for((long long)nj), kThreads, 0, stream>>>((int)nj, 1.0, dJ);
        fill_kernel<<<grid_for(c->n), kThreads, 0, stream>>>(c->n, 1.0, dS);
        kkt_status st = kkt_factor(c, dW, dJ, dS, nullptr, 0.0, stream, nullptr);
        std::vector<float> t;
        cudaEvent_t a = nullptr, z = nullptr;
        if (st == KKT_OK && cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&z) == cudaSuccess) {
            for (int r = 0; r < 3 && st == KKT_OK; ++r) {
                cudaEventRecord(a, stream);
                st = kkt_factor(c, dW, dJ, dS, nullptr, 0.0, stream, nullptr);
                cudaEventRecord(z, stream);
                cudaEventSynchronize(z);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, a, z);
                t.push_back(ms);
            }
        }
        if (a) cudaEventDestroy(a);
        if (z) cudaEventDestroy(z);
        cudaFree(buf);
        kkt_destroy(c);
        if (st != KKT_OK) return set_err(nullptr, st, "kkt_autotune_batch: factorisation failed");
        std::sort(t.begin(), t.end());
        const double med = t.empty() ? INFINITY : t[t.size() / 2];
        if (med < best_t) {
            best_t = med;
            won = b0;
            won.relax_cols = cd.relax_cols;
            won.relax_zeros = cd.relax_zeros;
            won.max_width = cd.max_width;
            won.subtree_cols = cd.subtree_cols;
        }
    }
    *best = won;
    if (best_ms) *best_ms = best_t;
    return KKT_OK;
}

kkt_status kkt_set_precision(kkt_ctx* c, int precision) {
    if (!c) return KKT_ERR_ARG;
    if (!c->device_ready) return set_err(c, KKT_ERR_STATE, "no device context");
    if (precision != 0 && precision != c->analysed_precision)
        return set_err(c, KKT_ERR_ARG, "precision must be 0 or the one the context was analysed with");
    c->opt.precision = precision;
    return KKT_OK;
}

kkt_status kkt_batch_set_active(kkt_ctx* c, const int* active) {
    if (!c) return KKT_ERR_ARG;
    if (!c->device_ready) return set_err(c, KKT_ERR_STATE, "no device context");
    if (c->nb < 2) return active ? set_err(c, KKT_ERR_ARG, "not a batch context") : KKT_OK;
    for (int i = 0; i < c->nb; ++i) c->h_inst_on[i] = active ? (active[i] != 0) : 1;
    c->inst_on_pending = true;
    return KKT_OK;
}

kkt_status kkt_batch_results(const kkt_ctx* c, int* status, int* refine_iters, int* cg_iters,
                             double* bwd_err, int* failed_col) {
    if (!c) return KKT_ERR_ARG;
    if (!c->device_ready) return KKT_ERR_STATE;
    if (status) std::copy(c->r_status.begin(), c->r_status.end(), status);
    if (refine_iters) std::copy(c->r_refine.begin(), c->r_refine.end(), refine_iters);
    if (cg_iters) std::copy(c->r_cg.begin(), c->r_cg.end(), cg_iters);
    if (bwd_err) std::copy(c->r_eta.begin(), c->r_eta.end(), bwd_err);
    if (failed_col) std::copy(c->r_fail.begin(), c->r_fail.end(), failed_col);
    return KKT_OK;
}

kkt_status kkt_symbolic_sizes(const kkt_ctx* c, int* ns, int64_t* nnz_L, int64_t* panel,
                              int64_t* row_entries, int* levels, double* flops) {
    if (!c) return KKT_ERR_ARG;
    if (ns) *ns = c->sym.ns();
    if (nnz_L) *nnz_L = c->sym.nnz_L;
    if (panel) {
        int64_t p = 0;
        for (int s = 0; s < c->sym.ns(); ++s) {
            int64_t cc = c->h_sn_c[s], rr = c->h_sn_r[s];
            p += cc * rr - cc * (cc - 1) / 2;
        }
        *panel = p;
    }
    if (row_entries) *row_entries = (int64_t)c->sym.sn_rows.size();
    if (levels) *levels = c->opt.solver == 1 ? c->bcr_nlev : c->tree_levels;
    if (flops) *flops = c->opt.solver == 1 ? c->bcr_flops : c->sym.flops;
    return KKT_OK;
}

kkt_status kkt_symbolic_export(const kkt_ctx* c, int* perm, int* parent, int* colcount, int* sn_ptr,
                               int* sn_rowptr, int* sn_rows) {
    if (!c) return KKT_ERR_ARG;
    const Symbolic& S = c->sym;
    if (perm) std::copy(S.perm.begin(), S.perm.end(), perm);
    if (parent) std::copy(S.parent.begin(), S.parent.end(), parent);
    if (colcount) std::copy(S.colcount.begin(), S.colcount.end(), colcount);
    if (sn_ptr) std::copy(S.sn_ptr.begin(), S.sn_ptr.end(), sn_ptr);
    if (sn_rowptr) std::copy(S.sn_rowptr.begin(), S.sn_rowptr.end(), sn_rowptr);
    if (sn_rows) std::copy(S.sn_rows.begin(), S.sn_rows.end(), sn_rows);
    return KKT_OK;
}

// Numeric factorisation shared by kkt_factor (one delta_x) and
// kkt_factor_batch (h_delta: one delta_x per instance, host).
static kkt_status factor_impl(kkt_ctx* c, const double* d_Wval, const double* d_Jval,
                              const double* d_sigma, const double* d_D, double delta_x,
                              const double* h_delta, cudaStream_t st, kkt_info* info) {
    if (!c) return KKT_ERR_ARG;
    if (!c->device_ready) return set_err(c, KKT_ERR_STATE, "context was analysed on the host only");
    if (!d_Wval && c->nnzW > 0) return set_err(c, KKT_ERR_ARG, "d_Wval is NULL");
    if (!d_Jval && c->nnzJ > 0) return set_err(c, KKT_ERR_ARG, "d_Jval is NULL");
    if (!d_sigma) return set_err(c, KKT_ERR_ARG, "d_sigma is NULL");
    if (c->opt.scheme == KKT_HYKKT && d_D) return set_err(c, KKT_ERR_ARG, "HyKKT takes D = gamma");
    const int nb = c->nb;
    if (h_delta) {
        for (int i = 0; i < nb; ++i)
            if (!(std::isfinite(h_delta[i]) && h_delta[i] >= 0))
                return set_err(c, KKT_ERR_ARG, "bad delta_x of instance " + std::to_string(i));
        delta_x = 0.0;
    } else if (!(std::isfinite(delta_x) && delta_x >= 0)) {
        return set_err(c, KKT_ERR_ARG, "bad delta_x");
    }
    c->factored = false;
    if (c->nnzW > 0)
        CUDA_TRY(c, cudaMemcpyAsync(c->v_W, d_Wval, (size_t)c->nnzW * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (c->nnzJ > 0)
        CUDA_TRY(c, cudaMemcpyAsync(c->v_J, d_Jval, (size_t)c->nnzJ * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(c, cudaMemcpyAsync(c->v_sigma, d_sigma, (size_t)c->n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    const bool hasD = c->opt.scheme == KKT_LIFTED && d_D;
    if (hasD && c->m > 0)
        CUDA_TRY(c, cudaMemcpyAsync(c->v_D, d_D, (size_t)c->m * sizeof(double), cudaMemcpyDeviceToDevice, st));
    c->f_W = c->v_W;
    c->f_J = c->v_J;
    c->f_sigma = c->v_sigma;
    c->f_D = hasD ? c->v_D : nullptr;
    c->f_Dconst = c->opt.scheme == KKT_LIFTED ? 1.0 / c->opt.delta : c->opt.gamma;
    c->f_delta_x = delta_x;
    c->f_dvec = nullptr;
    if (h_delta) {
        if (nb == 1) {
            c->f_delta_x = delta_x = h_delta[0];
        } else {
            for (int i = 0; i < nb; ++i) c->h_delta[i] = h_delta[i];
            CUDA_TRY(c, cudaMemcpyAsync(c->d_dval, c->h_delta.data(), (size_t)nb * sizeof(double),
                                        cudaMemcpyHostToDevice, st));
            expand_kernel<<<c->nch_x, kThreads, 0, st>>>(c->d_ch_xy, c->d_dval, c->d_dvec);
            c->f_dvec = c->d_dvec;
        }
    }
    if (!c->f_dvec) std::fill(c->h_delta.begin(), c->h_delta.end(), c->f_delta_x);
    // dual block of the target system: C = 1/D (relaxed problem) or none
    c->f_C = nullptr;
    if (c->opt.scheme == KKT_LIFTED && c->opt.target_relaxed) {
        if (!c->d_Cbuf.p) {
            TRY(alloc(c, &c->d_Cbuf.p, c->m));
            c->d_Cbuf.n = c->m;
        }
        c->f_C = c->d_Cbuf.p;
    }
    const int m = c->m;
    const int sp_a = span_begin(c, 0, st);
    if (c->nnzJ > 0)
        scale_rows_sqrt_kernel<<<grid_for(m), kThreads, 0, st>>>(m, c->d_j_ptr, c->f_J, c->f_D,
                                                                 c->f_Dconst, c->v_Js);
    span_end(c, sp_a, st);
    auto fetch_fail = [&]() -> kkt_status {
        CUDA_TRY(c, cudaMemcpyAsync(c->h_int, c->d_fail, (size_t)nb * sizeof(int), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(c, cudaStreamSynchronize(st));
        return KKT_OK;
    };
    auto any_fail = [&]() {
        for (int i = 0; i < nb; ++i)
            if (c->h_int[i] != kNoFail) return true;
        return false;
    };
    // ||K_orig,i||_inf (and the dual block C of the relaxed target) on the side
    // stream, overlapping the factorisation, which does not read them
    CUDA_TRY(c, cudaEventRecord(c->ev_in, st));
    CUDA_TRY(c, cudaStreamWaitEvent(c->side, c->ev_in, 0));
    CUDA_TRY(c, cudaMemsetAsync(c->d_knorm, 0, (size_t)nb * sizeof(double), c->side));
    if (c->f_C) {
        if (c->f_D) recip_kernel<<<grid_for(m), kThreads, 0, c->side>>>(m, c->f_D, c->d_Cbuf.p);
        else fill_kernel<<<grid_for(m), kThreads, 0, c->side>>>(m, c->opt.delta, c->d_Cbuf.p);
    }
    knorm_kernel<<<c->nch_xy, kThreads, 0, c->side>>>(c->d_ch_xy, c->n, c->d_wf_ptr, c->d_wf_col, c->d_wf_idx,
                                                      c->f_W, c->d_j_ptr, c->d_jt_ptr, c->d_jt_idx, c->f_J,
                                                      c->f_sigma, c->f_delta_x, c->f_dvec, c->f_C, c->d_knorm);
    CUDA_TRY(c, cudaEventRecord(c->ev_side, c->side));
    // detail: 0 FP64, 1 FP32, 2 FP64 after a failed reduced-precision
    // factor, 3 double-float
    int detail = 0;
    bool need64 = true;
    if (c->opt.solver == 1) {
        TRY(enqueue_bcr_factor(c, delta_x, st));
        c->cur_prec = 0;
        need64 = false;
    } else if (c->opt.precision == 1 || c->opt.precision == 2) {
        if (c->opt.precision == 1) {
            TRY(enqueue_numeric_factor<float>(c, c->d_Lx32, c->d_dinv32, delta_x, st));
        } else {
            TRY(enqueue_numeric_factor<df64>(c, as_df(c->d_Lx), as_df(c->d_dinv), delta_x, st));
        }
        TRY(fetch_fail());
        c->stats.fp32_factors++;
        c->cur_prec = c->opt.precision;
        detail = c->opt.precision == 1 ? 1 : 3;
        need64 = false;
        if (any_fail()) {            // a reduced-precision pivot failed: factorise in FP64
            c->stats.fp64_fallbacks++;
            detail = 2;
            need64 = true;
        }
    }
    if (need64) {
        TRY(enqueue_numeric_factor<double>(c, c->d_Lx, c->d_dinv, delta_x, st));
        c->cur_prec = 0;
    }
    const bool reduced_ok = detail == 1 || detail == 3;
    CUDA_TRY(c, cudaStreamWaitEvent(st, c->ev_side, 0));   // ||K_orig,i||_inf done on the side stream
    CUDA_TRY(c, cudaMemcpyAsync(c->h_red, c->d_knorm, (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (reduced_ok) {
        CUDA_TRY(c, cudaStreamSynchronize(st));
    } else {
        TRY(fetch_fail());   // synchronises
    }
    spans_collect(c);
    int first_fail = -1, nfail = 0;
    for (int i = 0; i < nb; ++i) {
        c->h_knorm[i] = c->h_red[i];
        const int w = reduced_ok ? kNoFail : c->h_int[i];
        c->r_fail[i] = w == kNoFail ? -1 : w;
        c->r_status[i] = w == kNoFail ? KKT_OK : KKT_ERR_NOT_SPD;
        if (w != kNoFail) {
            ++nfail;
            if (first_fail < 0) first_fail = w;
        }
    }
    c->knorm = c->h_knorm[0];
    if (info) {
        info->failed_col = first_fail;
        info->delta_x = c->f_delta_x;
        info->status_detail = detail;
    }
    if (nfail > 0) {
        // a batch keeps the factors of its other instances usable
        c->factored = nb > 1 && nfail < nb;
        return set_err(c, KKT_ERR_NOT_SPD, "factorization: non-positive pivot in column " +
                                               std::to_string(first_fail) +
                                               (nb > 1 ? " (" + std::to_string(nfail) + " of " +
                                                             std::to_string(nb) + " instances failed)"
                                                       : std::string()));
    }
    c->factored = true;
    return KKT_OK;
}

}  // extern "C"

namespace {
// Bounds-check builds: after a factor or solve call, the device error word;
// a recorded failure becomes KKT_ERR_INTERNAL (the word is cleared for the
// next call).  Ordinary builds return the call's own status.
kkt_status bounds_verdict(kkt_ctx* c, cudaStream_t st, kkt_status s0) {
#if KKT_BOUNDS_CHECK
    if (!c || !c->d_berr) return s0;
    int h = 0;
    if (cudaMemcpyAsync(&h, c->d_berr, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return set_err(c, KKT_ERR_CUDA, "bounds check: the error word could not be read");
    if (h == 0) return s0;
    cudaMemsetAsync(c->d_berr, 0, sizeof(int), st);
    cudaStreamSynchronize(st);
    static const char* what[] = {"", "assembly slot outside the panel storage",
                                 "level or task entry outside the supernodes",
                                 "update segment target is not an ancestor",
                                 "Schur update column outside its target supernode",
                                 "relative row outside its target supernode",
                                 "solve row index outside 0..n-1"};
    return set_err(c, KKT_ERR_INTERNAL,
                   std::string("device bounds check failed: ") + (h >= 1 && h <= 6 ? what[h] : "unknown code"));
#else
    (void)c;
    (void)st;
    return s0;
#endif
}
// After a call that synchronised its stream: a dataflow solve whose wait
// gave up has left x invalid and its counters unknown; they are cleared so
// the next solve starts clean, and the call reports KKT_ERR_TIMEOUT.
kkt_status flow_verdict(kkt_ctx* c, kkt_status s0) {
    if (!c || !c->h_flow_err || *(volatile int*)c->h_flow_err == 0) return s0;
    *(volatile int*)c->h_flow_err = 0;
    cudaMemset(c->d_flow_cnt, 0, (size_t)c->flow_items * sizeof(int));
    cudaMemset(c->d_flow_done, 0, (size_t)c->flow_items * sizeof(unsigned));
    cudaMemset(c->d_flow_ctrl, 0, 4 * sizeof(unsigned));
    cudaDeviceSynchronize();
    return set_err(c, KKT_ERR_TIMEOUT, "a dependency wait of the dataflow triangular solve gave up");
}
}  // namespace

extern "C" {

kkt_status kkt_factor(kkt_ctx* c, const double* d_Wval, const double* d_Jval, const double* d_sigma,
                      const double* d_D, double delta_x, cudaStream_t st, kkt_info* info) {
    return bounds_verdict(c, st, factor_impl(c, d_Wval, d_Jval, d_sigma, d_D, delta_x, nullptr, st, info));
}

kkt_status kkt_factor_batch(kkt_ctx* c, const double* d_Wval, const double* d_Jval,
                            const double* d_sigma, const double* d_D, const double* delta_x,
                            cudaStream_t st, kkt_info* info) {
    if (!delta_x) return set_err(c, KKT_ERR_ARG, "delta_x is NULL");
    return bounds_verdict(c, st, factor_impl(c, d_Wval, d_Jval, d_sigma, d_D, 0.0, delta_x, st, info));
}

static kkt_status solve_impl(kkt_ctx* c, const double* d_rx, const double* d_ry, double* d_dx, double* d_dy,
                             double* d_ds, cudaStream_t st, kkt_info* info);

kkt_status kkt_solve(kkt_ctx* c, const double* d_rx, const double* d_ry, double* d_dx, double* d_dy,
                     double* d_ds, cudaStream_t st, kkt_info* info) {
    return flow_verdict(c, bounds_verdict(c, st, solve_impl(c, d_rx, d_ry, d_dx, d_dy, d_ds, st, info)));
}

static kkt_status solve_impl(kkt_ctx* c, const double* d_rx, const double* d_ry, double* d_dx, double* d_dy,
                             double* d_ds, cudaStream_t st, kkt_info* info) {
    if (!c) return KKT_ERR_ARG;
    if (!c->factored) return set_err(c, KKT_ERR_STATE, "kkt_solve called without a successful kkt_factor");
    if (!d_rx || !d_ry || !d_dx || !d_dy) return set_err(c, KKT_ERR_ARG, "NULL vector");
    const int n = c->n, m = c->m, nb = c->nb;
    double* rx = c->w_r;
    double* ry = c->w_r + n;
    double* dx = c->w_d;
    double* dy = c->w_d + n;
    // Richardson on every instance: an instance stops at eta <= tol_refine
    // (KKT_OK), at two successive sweeps with eta > 0.9 eta_prev (STALL), or
    // after max_refine sweeps (MAXIT); instances whose factor failed take no
    // part (NOT_SPD).  Stopped instances keep their solution: the correction
    // is added only where d_act is set.
    constexpr int kRunning = 1;
    std::vector<char> failed(nb);
    for (int i = 0; i < nb; ++i) failed[i] = c->r_fail[i] >= 0;
    std::vector<double> eta(nb, INFINITY), prev(nb, INFINITY);
    std::vector<int> slow(nb, 0), state(nb, 0);
    std::fill(c->r_cg.begin(), c->r_cg.end(), 0);
    int detail = c->cur_prec == 2 ? 3 : c->cur_prec;
    for (int attempt = 0; attempt < 2; ++attempt) {
        CUDA_TRY(c, cudaMemsetAsync(d_dx, 0, n * sizeof(double), st));
        CUDA_TRY(c, cudaMemsetAsync(d_dy, 0, m * sizeof(double), st));
        CUDA_TRY(c, cudaMemcpyAsync(rx, d_rx, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        CUDA_TRY(c, cudaMemcpyAsync(ry, d_ry, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
        int running = 0;
        for (int i = 0; i < nb; ++i) {
            state[i] = failed[i] ? (int)KKT_ERR_NOT_SPD : kRunning;
            slow[i] = 0;
            prev[i] = INFINITY;
            eta[i] = INFINITY;
            c->r_refine[i] = 0;
            c->h_act[i] = state[i] == kRunning;
            running += c->h_act[i];
        }
        CUDA_TRY(c, cudaMemcpyAsync(c->d_act, c->h_act, (size_t)nb * sizeof(int), cudaMemcpyHostToDevice, st));
        for (int it = 0; it <= c->opt.max_refine && running > 0; ++it) {
            if (c->opt.scheme == KKT_LIFTED) {
                TRY(lifted_precond(c, rx, ry, dx, dy, st));
            } else {
                TRY(hykkt_inner(c, rx, ry, dx, dy, st, c->r_cg));
            }
            c->stats.launches += 2;
            seg_axpy_kernel<<<c->nch_xy, kThreads, 0, st>>>(c->d_ch_xy, n, c->d_act, dx, dy, d_dx, d_dy);
            TRY(residual(c, d_rx, d_ry, d_dx, d_dy, rx, ry, st, eta));
            running = 0;
            for (int i = 0; i < nb; ++i) {
                if (state[i] != kRunning) continue;
                c->r_refine[i] = it;
                if (eta[i] <= c->opt.tol_refine) {
                    state[i] = KKT_OK;
                } else if (it > 0 && eta[i] > 0.9 * prev[i]) {   // stagnation
                    if (++slow[i] >= 2) state[i] = KKT_ERR_STALL;
                } else {
                    slow[i] = 0;
                }
                prev[i] = eta[i];
                c->r_eta[i] = eta[i];
                c->h_act[i] = state[i] == kRunning;
                running += c->h_act[i];
            }
            if (running > 0)
                CUDA_TRY(c, cudaMemcpyAsync(c->d_act, c->h_act, (size_t)nb * sizeof(int), cudaMemcpyHostToDevice, st));
        }
        bool all_ok = true;
        for (int i = 0; i < nb; ++i) {
            if (state[i] == kRunning) state[i] = KKT_ERR_MAXIT;
            if (state[i] != KKT_OK && !failed[i]) all_ok = false;
        }
        if (all_ok || c->cur_prec == 0) break;
        // the FP32 factor did not carry the refinement to the tolerance:
        // factorise the same system in FP64 and solve again
        TRY(enqueue_numeric_factor<double>(c, c->d_Lx, c->d_dinv, c->f_delta_x, st));
        CUDA_TRY(c, cudaMemcpyAsync(c->h_int, c->d_fail, (size_t)nb * sizeof(int), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(c, cudaStreamSynchronize(st));
        c->cur_prec = 0;
        c->stats.fp64_fallbacks++;
        detail = 2;
        int nfail = 0, first = -1;
        for (int i = 0; i < nb; ++i) {
            if (c->h_int[i] != kNoFail) {
                failed[i] = 1;
                c->r_fail[i] = c->h_int[i];
                if (first < 0) first = c->h_int[i];
            }
            nfail += failed[i];
        }
        if (nfail == nb) {
            c->factored = false;
            for (int i = 0; i < nb; ++i) c->r_status[i] = KKT_ERR_NOT_SPD;
            if (info) { info->failed_col = first; info->status_detail = detail; }
            return set_err(c, KKT_ERR_NOT_SPD, "FP64 refactorization after FP32 fallback: non-positive pivot in column " +
                                                   std::to_string(first));
        }
    }
    if (d_ds && c->opt.scheme == KKT_LIFTED && c->opt.target_relaxed) {
        j_apply_kernel<<<grid_for(m), kThreads, 0, st>>>(m, c->d_j_ptr, c->d_j_col, c->f_J, d_dx, d_ry,
                                                         nullptr, 1.0, d_ds, nullptr);
    }
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaStreamSynchronize(st));
    spans_collect(c);
    kkt_status result = KKT_OK;
    int refine_max = 0, cg_total = 0;
    double eta_max = 0.0;
    for (int i = 0; i < nb; ++i) {
        c->r_status[i] = state[i];
        cg_total += c->r_cg[i];
        if (failed[i]) {
            c->r_eta[i] = INFINITY;
            result = KKT_ERR_NOT_SPD;
            continue;
        }
        refine_max = std::max(refine_max, c->r_refine[i]);
        eta_max = std::max(eta_max, c->r_eta[i]);
        if (state[i] != KKT_OK && result == KKT_OK) result = (kkt_status)state[i];
    }
    if (info) {
        info->refine_iters = refine_max;
        info->cg_iters = cg_total;
        info->bwd_err = eta_max;
        info->status_detail = detail;
    }
    if (result != KKT_OK)
        set_err(c, result, result == KKT_ERR_STALL ? "refinement stalled"
                           : result == KKT_ERR_MAXIT ? "refinement hit max_refine"
                                                     : "some instances have no factor (non-positive pivot)");
    return result;
}

}  // extern "C"

namespace {
// ------------------------------------------------------------- one-graph step
// A WHILE node on the conditional handle h after the work captured so far on
// st; the capture continues after the node.  Returns the (empty) body graph.
kkt_status add_while_node(kkt_ctx* c, cudaStream_t st, cudaGraphConditionalHandle h, cudaGraph_t* body) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    CUDA_TRY(c, cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd));
    if (cs != cudaStreamCaptureStatusActive) return set_err(c, KKT_ERR_INTERNAL, "WHILE node outside a capture");
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CUDA_TRY(c, cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
    *body = np.conditional.phGraph_out[0];
    CUDA_TRY(c, cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return KKT_OK;
}

// Kernel nodes of a graph (not counting the bodies of its conditional nodes).
long long kernel_nodes(cudaGraph_t g) {
    size_t nn = 0;
    if (cudaGraphGetNodes(g, nullptr, &nn) != cudaSuccess || nn == 0) return 0;
    std::vector<cudaGraphNode_t> nodes(nn);
    if (cudaGraphGetNodes(g, nodes.data(), &nn) != cudaSuccess) return 0;
    long long k = 0;
    for (size_t i = 0; i < nn; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

kkt_status new_handle(kkt_ctx* c, cudaStream_t st, cudaGraphConditionalHandle* h) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    CUDA_TRY(c, cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, nullptr, nullptr, nullptr));
    if (cs != cudaStreamCaptureStatusActive) return set_err(c, KKT_ERR_INTERNAL, "handle outside a capture");
    CUDA_TRY(c, cudaGraphConditionalHandleCreate(h, g, 0, 0));
    return KKT_OK;
}

// HyKKT inner solve inside the captured step: the steps of hykkt_inner,
// with the CG loop as a WHILE node (condition: some instance's CG runs,
// checked after every iteration) and the CG counts added on the device.
kkt_status hykkt_inner_graph(kkt_ctx* c, const double* rx, const double* ry, double* dx, double* dy,
                             cudaStream_t st) {
    const int n = c->n, m = c->m, nb = c->nb;
    const double gamma = c->f_Dconst;
    jt_axpy_kernel<<<grid_for(n), kThreads, 0, st>>>(n, c->d_jt_ptr, c->d_jt_row, c->d_jt_idx,
                                                     c->f_J, rx, ry, nullptr, 1.0, gamma, c->w_rg, nullptr);
    TRY(apply_kinv(c, c->w_rg, c->w_q, st));
    j_apply_kernel<<<grid_for(m), kThreads, 0, st>>>(m, c->d_j_ptr, c->d_j_col, c->f_J, c->w_q, ry,
                                                     nullptr, 1.0, c->w_res, nullptr);
    CUDA_TRY(c, cudaMemsetAsync(c->w_cgx, 0, m * sizeof(double), st));
    CUDA_TRY(c, cudaMemcpyAsync(c->w_p, c->w_res, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
    seg_dot(c, c->w_res, c->w_res, 0, st);
    cg_init_kernel<<<1, kThreads, 0, st>>>(nb, c->d_cgs, c->d_cgi, c->d_act, c->opt.tol_cg, c->opt.max_cg,
                                           c->d_cg);
    cudaGraphConditionalHandle h;
    TRY(new_handle(c, st, &h));
    cg_cond_kernel<<<1, 32, 0, st>>>(c->d_cg, h, c->d_rctl + 1, 0);
    cudaGraph_t body = nullptr;
    TRY(add_while_node(c, st, h, &body));
    cudaStream_t bs = c->cap[2];
    CUDA_TRY(c, cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    enqueue_cg_iteration<double>(c, c->d_Lx, c->d_dinv, c->w_xp, bs);
    cg_cond_kernel<<<1, 32, 0, bs>>>(c->d_cg, h, c->d_rctl + 1, 1);
    cudaGraph_t done = nullptr;
    CUDA_TRY(c, cudaStreamEndCapture(bs, &done));
    c->step_cgit = kernel_nodes(body);
    cg_count_kernel<<<grid_for(nb), kThreads, 0, st>>>(nb, c->d_cgi, c->d_rst);
    jt_axpy_kernel<<<grid_for(n), kThreads, 0, st>>>(n, c->d_jt_ptr, c->d_jt_row, c->d_jt_idx,
                                                     c->f_J, c->w_rg, c->w_cgx, nullptr, 1.0, -1.0,
                                                     c->w_tn, nullptr);
    TRY(apply_kinv(c, c->w_tn, dx, st));
    CUDA_TRY(c, cudaMemcpyAsync(dy, c->w_cgx, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
    return KKT_OK;
}

// The whole step on the capture stream: input copies, per-instance
// delta_x, assembly and factorisation (||K||_inf on the side stream),
// then the refinement loop as a WHILE node and the copies of the results
// to pinned host memory.  The f_* inputs are set by the caller.
kkt_status capture_step_body(kkt_ctx* c, const double* W, const double* J, const double* sigma,
                             const double* D, const double* d_rx, const double* d_ry, double* d_dx,
                             double* d_dy) {
    cudaStream_t st = c->cap[0];
    const int n = c->n, m = c->m, nb = c->nb;
    CUDA_TRY(c, cudaEventRecordWithFlags(c->step_ev[0], st, cudaEventRecordExternal));
    if (c->nnzW > 0)
        CUDA_TRY(c, cudaMemcpyAsync(c->v_W, W, (size_t)c->nnzW * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (c->nnzJ > 0)
        CUDA_TRY(c, cudaMemcpyAsync(c->v_J, J, (size_t)c->nnzJ * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(c, cudaMemcpyAsync(c->v_sigma, sigma, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (c->f_D && m > 0)
        CUDA_TRY(c, cudaMemcpyAsync(c->v_D, D, (size_t)m * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(c, cudaMemcpyAsync(c->d_dval, c->hp_delta, (size_t)nb * sizeof(double), cudaMemcpyHostToDevice, st));
    expand_kernel<<<c->nch_x, kThreads, 0, st>>>(c->d_ch_xy, c->d_dval, c->d_dvec);
    if (c->nnzJ > 0)
        scale_rows_sqrt_kernel<<<grid_for(m), kThreads, 0, st>>>(m, c->d_j_ptr, c->f_J, c->f_D, c->f_Dconst,
                                                                 c->v_Js);
    CUDA_TRY(c, cudaEventRecord(c->ev_in, st));
    CUDA_TRY(c, cudaStreamWaitEvent(c->side, c->ev_in, 0));
    CUDA_TRY(c, cudaMemsetAsync(c->d_knorm, 0, (size_t)nb * sizeof(double), c->side));
    if (c->f_C) {
        if (c->f_D) recip_kernel<<<grid_for(m), kThreads, 0, c->side>>>(m, c->f_D, c->d_Cbuf.p);
        else fill_kernel<<<grid_for(m), kThreads, 0, c->side>>>(m, c->opt.delta, c->d_Cbuf.p);
    }
    knorm_kernel<<<c->nch_xy, kThreads, 0, c->side>>>(c->d_ch_xy, n, c->d_wf_ptr, c->d_wf_col, c->d_wf_idx,
                                                      c->f_W, c->d_j_ptr, c->d_jt_ptr, c->d_jt_idx, c->f_J,
                                                      c->f_sigma, 0.0, c->f_dvec, c->f_C, c->d_knorm);
    CUDA_TRY(c, cudaEventRecord(c->ev_side, c->side));
    const long long f0 = c->stats.factor_launches;
    // the instance switch is read from pinned memory at every replay
    if (nb > 1)
        CUDA_TRY(c, cudaMemcpyAsync(c->d_inst_on, c->h_inst_on, (size_t)nb * sizeof(int), cudaMemcpyHostToDevice,
                                    st));
    c->inst_on_pending = false;
    TRY(enqueue_numeric_factor<double>(c, c->d_Lx, c->d_dinv, 0.0, st, c->step_ev[3]));
    c->step_fl = c->stats.factor_launches - f0;
    CUDA_TRY(c, cudaStreamWaitEvent(st, c->ev_side, 0));
    CUDA_TRY(c, cudaEventRecordWithFlags(c->step_ev[1], st, cudaEventRecordExternal));
    // refinement (the rules of kkt_solve, on the device)
    double* rx = c->w_r;
    double* ry = c->w_r + n;
    double* dx = c->w_d;
    double* dy = c->w_d + n;
    CUDA_TRY(c, cudaMemsetAsync(d_dx, 0, n * sizeof(double), st));
    CUDA_TRY(c, cudaMemsetAsync(d_dy, 0, m * sizeof(double), st));
    CUDA_TRY(c, cudaMemcpyAsync(rx, d_rx, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(c, cudaMemcpyAsync(ry, d_ry, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(c, cudaMemsetAsync(c->d_rctl, 0, 2 * sizeof(int), st));
    cudaGraphConditionalHandle h;
    TRY(new_handle(c, st, &h));
    refine_init_kernel<<<1, kThreads, 0, st>>>(nb, c->d_fail, kNoFail, (int)KKT_ERR_NOT_SPD, c->d_act, c->d_rst,
                                               c->d_reta, c->d_rctl, h);
    cudaGraph_t body = nullptr;
    TRY(add_while_node(c, st, h, &body));
    cudaStream_t bs = c->cap[1];
    CUDA_TRY(c, cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    if (c->opt.scheme == KKT_LIFTED) {
        TRY(lifted_precond(c, rx, ry, dx, dy, bs));
    } else {
        TRY(hykkt_inner_graph(c, rx, ry, dx, dy, bs));
    }
    seg_axpy_kernel<<<c->nch_xy, kThreads, 0, bs>>>(c->d_ch_xy, n, c->d_act, dx, dy, d_dx, d_dy);
    TRY(enqueue_residual(c, d_rx, d_ry, d_dx, d_dy, rx, ry, bs));
    refine_update_kernel<<<1, kThreads, 0, bs>>>(nb, c->d_red, c->d_knorm, c->opt.tol_refine, c->opt.max_refine,
                                                 (int)KKT_OK, (int)KKT_ERR_STALL, c->d_act, c->d_rst, c->d_reta,
                                                 c->d_rctl, h);
    cudaGraph_t done = nullptr;
    CUDA_TRY(c, cudaStreamEndCapture(bs, &done));
    c->step_sweep = kernel_nodes(body);
    CUDA_TRY(c, cudaEventRecordWithFlags(c->step_ev[2], st, cudaEventRecordExternal));
    CUDA_TRY(c, cudaMemcpyAsync(c->h_rst, c->d_rst, 4 * (size_t)nb * sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c, cudaMemcpyAsync(c->h_rst + 4 * nb, c->d_fail, (size_t)nb * sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c, cudaMemcpyAsync(c->h_rst + 5 * nb, c->d_rctl, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c, cudaMemcpyAsync(c->h_reta, c->d_reta, 2 * (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c, cudaMemcpyAsync(c->h_reta + 2 * nb, c->d_knorm, (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost,
                                st));
    return KKT_OK;
}

kkt_status build_step_graph(kkt_ctx* c, const double* W, const double* J, const double* sigma, const double* D,
                            const double* d_rx, const double* d_ry, double* d_dx, double* d_dy) {
    const int nb = c->nb;
    for (auto& s : c->cap)
        if (!s) CUDA_TRY(c, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    for (auto& e : c->step_ev)
        if (!e) CUDA_TRY(c, cudaEventCreate(&e));
    if (!c->d_rst) {
        TRY(alloc(c, &c->d_rst, 4 * (size_t)nb));
        TRY(alloc(c, &c->d_reta, 2 * (size_t)nb));
        TRY(alloc(c, &c->d_rctl, 2));
        CUDA_TRY(c, cudaMallocHost((void**)&c->h_rst, (5 * (size_t)nb + 2) * sizeof(int)));
        CUDA_TRY(c, cudaMallocHost((void**)&c->h_reta, 3 * (size_t)nb * sizeof(double)));
    }
    if (!c->d_dvec) TRY(alloc(c, &c->d_dvec, c->n));
    if (!c->d_dval) TRY(alloc(c, &c->d_dval, nb));
    if (c->step_exec) cudaGraphExecDestroy(c->step_exec);
    if (c->step_graph) cudaGraphDestroy(c->step_graph);
    c->step_exec = nullptr;
    c->step_graph = nullptr;
    const kkt_stats saved = c->stats;
    const bool prof = c->profiling;
    c->profiling = false;
    c->capturing = true;
    c->step_cgit = 0;
    kkt_status r = KKT_OK;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->cap[0], cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        r = capture_step_body(c, W, J, sigma, D, d_rx, d_ry, d_dx, d_dy);
        e = cudaStreamEndCapture(c->cap[0], &g);
    }
    c->capturing = false;
    c->profiling = prof;
    c->stats = saved;
    if (r == KKT_OK && e != cudaSuccess) r = set_err(c, KKT_ERR_CUDA, std::string("step graph capture: ") +
                                                                       cudaGetErrorString(e));
    if (r == KKT_OK) {
        e = cudaGraphInstantiate(&c->step_exec, g, 0);
        if (e != cudaSuccess) r = set_err(c, KKT_ERR_CUDA, std::string("step graph instantiate: ") +
                                                             cudaGetErrorString(e));
    }
    if (r != KKT_OK) {
        if (g) cudaGraphDestroy(g);
        c->step_exec = nullptr;
        cudaGetLastError();
        return r;
    }
    c->step_graph = g;
    c->step_pre = kernel_nodes(g);
    c->step_key[0] = W;
    c->step_key[1] = J;
    c->step_key[2] = sigma;
    c->step_key[3] = D;
    c->step_key[4] = d_rx;
    c->step_key[5] = d_ry;
    c->step_key[6] = d_dx;
    c->step_key[7] = d_dy;
    c->step_key[8] = reinterpret_cast<const void*>((intptr_t)(c->opt.target_relaxed + 2));
    return KKT_OK;
}

kkt_status factor_solve_impl(kkt_ctx* c, const double* d_Wval, const double* d_Jval, const double* d_sigma,
                             const double* d_D, const double* delta_x, const double* d_rx, const double* d_ry,
                             double* d_dx, double* d_dy, cudaStream_t st, kkt_info* info) {
    if (!c) return KKT_ERR_ARG;
    if (!c->device_ready) return set_err(c, KKT_ERR_STATE, "context was analysed on the host only");
    if (c->opt.solver != 0 || c->opt.precision != 0)
        return set_err(c, KKT_ERR_ARG, "kkt_factor_solve: supernodal FP64 factor only (solver 0, precision 0)");
    if (!d_Wval && c->nnzW > 0) return set_err(c, KKT_ERR_ARG, "d_Wval is NULL");
    if (!d_Jval && c->nnzJ > 0) return set_err(c, KKT_ERR_ARG, "d_Jval is NULL");
    if (!d_sigma) return set_err(c, KKT_ERR_ARG, "d_sigma is NULL");
    if (!d_rx || !d_ry || !d_dx || !d_dy) return set_err(c, KKT_ERR_ARG, "NULL vector");
    if (!delta_x) return set_err(c, KKT_ERR_ARG, "delta_x is NULL");
    if (c->opt.scheme == KKT_HYKKT && d_D) return set_err(c, KKT_ERR_ARG, "HyKKT takes D = gamma");
    const int nb = c->nb, m = c->m;
    for (int i = 0; i < nb; ++i)
        if (!(std::isfinite(delta_x[i]) && delta_x[i] >= 0))
            return set_err(c, KKT_ERR_ARG, "bad delta_x of instance " + std::to_string(i));
    if (!c->hp_delta) CUDA_TRY(c, cudaMallocHost((void**)&c->hp_delta, (size_t)nb * sizeof(double)));
    // the launch below reads hp_delta; no earlier replay is in flight, since
    // every call waits for its own replay before it returns
    for (int i = 0; i < nb; ++i) c->hp_delta[i] = delta_x[i];
    c->factored = false;
    const bool hasD = c->opt.scheme == KKT_LIFTED && d_D;
    c->f_W = c->v_W;
    c->f_J = c->v_J;
    c->f_sigma = c->v_sigma;
    c->f_D = hasD ? c->v_D : nullptr;
    c->f_Dconst = c->opt.scheme == KKT_LIFTED ? 1.0 / c->opt.delta : c->opt.gamma;
    c->f_delta_x = 0.0;
    c->f_C = nullptr;
    if (c->opt.scheme == KKT_LIFTED && c->opt.target_relaxed) {
        if (!c->d_Cbuf.p) {
            TRY(alloc(c, &c->d_Cbuf.p, m));
            c->d_Cbuf.n = m;
        }
        c->f_C = c->d_Cbuf.p;
    }
    if (!c->d_dvec) TRY(alloc(c, &c->d_dvec, c->n));
    c->f_dvec = c->d_dvec;
    const void* key[9] = {d_Wval, d_Jval, d_sigma, hasD ? d_D : nullptr, d_rx, d_ry, d_dx, d_dy,
                          reinterpret_cast<const void*>((intptr_t)(c->opt.target_relaxed + 2))};
    if (!c->step_exec || !std::equal(key, key + 9, c->step_key))
        TRY(build_step_graph(c, d_Wval, d_Jval, d_sigma, hasD ? d_D : nullptr, d_rx, d_ry, d_dx, d_dy));
    CUDA_TRY(c, cudaGraphLaunch(c->step_exec, st));
    CUDA_TRY(c, cudaStreamSynchronize(st));
    // results and counters
    const int* rs = c->h_rst;
    const int* fail = c->h_rst + 4 * nb;
    const int sweeps = c->h_rst[5 * nb], cgits = c->h_rst[5 * nb + 1];
    c->stats.graph_steps++;
    c->stats.factor_calls++;
    c->stats.factor_launches += c->step_fl;
    c->stats.launches += c->step_pre + (long long)sweeps * c->step_sweep + (long long)cgits * c->step_cgit;
    c->stats.kinv_calls += c->opt.scheme == KKT_LIFTED ? sweeps : 2LL * sweeps + cgits;
    if (c->profiling) {
        float a = 0.f, b = 0.f;
        float a0 = 0;
        if (cudaEventElapsedTime(&a0, c->step_ev[0], c->step_ev[3]) == cudaSuccess) c->stats.assemble_ms += a0;
        if (cudaEventElapsedTime(&a, c->step_ev[3], c->step_ev[1]) == cudaSuccess) c->stats.factor_ms += a;
        if (cudaEventElapsedTime(&b, c->step_ev[1], c->step_ev[2]) == cudaSuccess) c->stats.solve_ms += b;
    }
    int nfail = 0, first_fail = -1, refine_max = 0, cg_total = 0;
    double eta_max = 0.0;
    kkt_status result = KKT_OK;
    for (int i = 0; i < nb; ++i) {
        const bool failed = fail[i] != kNoFail;
        int state = rs[4 * i];
        if (state == kRefineRunning) state = KKT_ERR_MAXIT;
        c->r_fail[i] = failed ? fail[i] : -1;
        c->r_status[i] = state;
        c->r_refine[i] = rs[4 * i + 2];
        c->r_cg[i] = rs[4 * i + 3];
        c->r_eta[i] = failed ? INFINITY : c->h_reta[2 * i];
        c->h_knorm[i] = c->h_reta[2 * nb + i];
        cg_total += c->r_cg[i];
        if (failed) {
            ++nfail;
            if (first_fail < 0) first_fail = fail[i];
            continue;
        }
        refine_max = std::max(refine_max, c->r_refine[i]);
        eta_max = std::max(eta_max, c->r_eta[i]);
        if (state != KKT_OK && result == KKT_OK) result = (kkt_status)state;
    }
    c->knorm = c->h_knorm[0];
    c->cur_prec = 0;
    c->factored = nfail == 0 || (nb > 1 && nfail < nb);
    if (info) {
        info->failed_col = first_fail;
        info->delta_x = c->hp_delta[0];
        info->status_detail = 0;
        info->refine_iters = refine_max;
        info->cg_iters = cg_total;
        info->bwd_err = eta_max;
    }
    if (nfail > 0)
        return set_err(c, KKT_ERR_NOT_SPD, "factorization: non-positive pivot in column " +
                                               std::to_string(first_fail) + " (" + std::to_string(nfail) +
                                               " of " + std::to_string(nb) + " instances failed)");
    if (result != KKT_OK)
        set_err(c, result, result == KKT_ERR_STALL ? "refinement stalled" : "refinement hit max_refine");
    return result;
}
}  // namespace

extern "C" {

kkt_status kkt_factor_solve(kkt_ctx* c, const double* d_Wval, const double* d_Jval, const double* d_sigma,
                            const double* d_D, const double* delta_x, const double* d_rx, const double* d_ry,
                            double* d_dx, double* d_dy, cudaStream_t st, kkt_info* info) {
    return flow_verdict(c, bounds_verdict(c, st, factor_solve_impl(c, d_Wval, d_Jval, d_sigma, d_D, delta_x, d_rx,
                                                                   d_ry, d_dx, d_dy, st, info)));
}

kkt_status kkt_backsolve(kkt_ctx* c, const double* d_b, double* d_x, cudaStream_t st) {
    if (!c || !d_b || !d_x) return set_err(c, KKT_ERR_ARG, "NULL argument");
    if (!c->factored) return set_err(c, KKT_ERR_STATE, "kkt_backsolve called without a factor");
    TRY(apply_kinv(c, d_b, d_x, st));
    CUDA_TRY(c, cudaStreamSynchronize(st));
    TRY(flow_verdict(c, bounds_verdict(c, st, KKT_OK)));
    spans_collect(c);
    return KKT_OK;
}

kkt_status kkt_backsolve_noalloc(kkt_ctx* c, const double* d_b, double* d_x, cudaStream_t st) {
    if (!c || !d_b || !d_x) return set_err(c, KKT_ERR_ARG, "NULL argument");
    if (!c->factored) return set_err(c, KKT_ERR_STATE, "kkt_backsolve_noalloc called without a factor");
    if ((long long)c->n > (long long)KKT_STATIC_SCRATCH_DOUBLES)
        return set_err(c, KKT_ERR_ARG, "n = " + std::to_string(c->n) +
                                           " exceeds the static scratch of kkt_backsolve_noalloc (" +
                                           std::to_string(KKT_STATIC_SCRATCH_DOUBLES) + " doubles)");
    double* xp = c->noalloc_ptr;
    if (!xp) return set_err(c, KKT_ERR_CUDA, c->noalloc_err.empty() ? "no device scratch" : c->noalloc_err);
    const int n = c->n;
    if (c->opt.solver == 1) {
        CUDA_TRY(c, cudaMemcpyAsync(xp, d_b, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        enqueue_bcr_solve(c, xp, st, nullptr);
        CUDA_TRY(c, cudaMemcpyAsync(d_x, xp, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else if (c->cur_prec == 2) {   // double-float factor: n pairs
        df64* xd = as_df(xp);
        gather_kernel<<<grid_for(n), kThreads, 0, st>>>(n, c->d_perm, d_b, xd, nullptr);
        enqueue_triangular_solves<df64>(c, as_df(c->d_Lx), as_df(c->d_dinv), xd, st, nullptr);
        scatter_kernel<<<grid_for(n), kThreads, 0, st>>>(n, c->d_perm, xd, d_x, nullptr);
    } else if (c->cur_prec == 1) {   // FP32 factor: the scratch holds n floats
        float* xp32 = reinterpret_cast<float*>(xp);
        gather_kernel<<<grid_for(n), kThreads, 0, st>>>(n, c->d_perm, d_b, xp32, nullptr);
        enqueue_triangular_solves<float>(c, c->d_Lx32, c->d_dinv32, xp32, st, nullptr);
        scatter_kernel<<<grid_for(n), kThreads, 0, st>>>(n, c->d_perm, xp32, d_x, nullptr);
    } else {
        gather_kernel<<<grid_for(n), kThreads, 0, st>>>(n, c->d_perm, d_b, xp, nullptr);
        enqueue_triangular_solves(c, xp, st, nullptr);
        scatter_kernel<<<grid_for(n), kThreads, 0, st>>>(n, c->d_perm, xp, d_x, nullptr);
    }
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaStreamSynchronize(st));
    return flow_verdict(c, KKT_OK);
}

kkt_status kkt_debug_corrupt_map(kkt_ctx* c, int what) {
#if KKT_BOUNDS_CHECK
    if (!c || !c->device_ready || c->opt.solver != 0) return set_err(c, KKT_ERR_STATE, "no supernodal device context");
    if (what < 0 || what > 2)
        return set_err(c, KKT_ERR_ARG, "what must be 0 (restore), 1 (corrupt the row map) or 2 (raise a wait)");
    // the arrival count the last dataflow item waits for, raised by one
    // (what = 2, no solve can meet it, so the wait runs out) or restored
    auto flow_target = [&](int delta) -> kkt_status {
        int* q = c->d_flow_nchild + (c->flow_items - 1);
        int v = 0;
        CUDA_TRY(c, cudaMemcpy(&v, q, sizeof(int), cudaMemcpyDeviceToHost));
        v += delta;
        CUDA_TRY(c, cudaMemcpy(q, &v, sizeof(int), cudaMemcpyHostToDevice));
        return KKT_OK;
    };
    if (what == 2) {
        if (!c->flow) return set_err(c, KKT_ERR_STATE, "the dataflow solves are not in use");
        if (!c->dbg_flow_raised) TRY(flow_target(1));
        c->dbg_flow_raised = true;
        return KKT_OK;
    }
    if (what == 0 && c->dbg_flow_raised) {
        TRY(flow_target(-1));
        c->dbg_flow_raised = false;
    }
    if (what == 0 && !c->dbg_corrupted) return KKT_OK;
    if (c->dbg_relmap_pos < 0) return set_err(c, KKT_ERR_STATE, "no Schur update in this tree");
    int* p = const_cast<int*>(c->plan.relmap) + c->dbg_relmap_pos;
    if (what == 1 && !c->dbg_corrupted) {
        CUDA_TRY(c, cudaMemcpy(&c->dbg_relmap_old, p, sizeof(int), cudaMemcpyDeviceToHost));
        CUDA_TRY(c, cudaMemcpy(p, &c->dbg_relmap_bad, sizeof(int), cudaMemcpyHostToDevice));
        c->dbg_corrupted = true;
    } else if (what == 0) {
        CUDA_TRY(c, cudaMemcpy(p, &c->dbg_relmap_old, sizeof(int), cudaMemcpyHostToDevice));
        c->dbg_corrupted = false;
    }
    return KKT_OK;
#else
    (void)what;
    return set_err(c, KKT_ERR_STATE, "kkt_debug_corrupt_map needs a bounds-check build");
#endif
}

kkt_status kkt_factor_export(kkt_ctx* c, int64_t* colptr, int* rowind, double* val) {
    if (!c) return KKT_ERR_ARG;
    if (!c->factored) return set_err(c, KKT_ERR_STATE, "no factor");
    if (c->opt.solver == 1) return set_err(c, KKT_ERR_STATE, "the block-tridiagonal factor has no supernodal form");
    const int ns = c->sym.ns();
    std::vector<double> Lh((size_t)c->panel), dv(c->n);
    if (val && c->cur_prec == 2) {
        std::vector<df64> Lf((size_t)c->panel), df(c->n);
        CUDA_TRY(c, cudaMemcpy(Lf.data(), c->d_Lx, (size_t)c->panel * sizeof(df64), cudaMemcpyDeviceToHost));
        CUDA_TRY(c, cudaMemcpy(df.data(), c->d_dinv, (size_t)c->n * sizeof(df64), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < Lf.size(); ++i) Lh[i] = (double)Lf[i];
        for (int i = 0; i < c->n; ++i) dv[i] = (double)df[i];
    } else if (val && c->cur_prec == 1) {
        std::vector<float> Lf((size_t)c->panel), df(c->n);
        CUDA_TRY(c, cudaMemcpy(Lf.data(), c->d_Lx32, (size_t)c->panel * sizeof(float), cudaMemcpyDeviceToHost));
        CUDA_TRY(c, cudaMemcpy(df.data(), c->d_dinv32, (size_t)c->n * sizeof(float), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < Lf.size(); ++i) Lh[i] = Lf[i];
        for (int i = 0; i < c->n; ++i) dv[i] = df[i];
    } else if (val) {
        CUDA_TRY(c, cudaMemcpy(Lh.data(), c->d_Lx, (size_t)c->panel * sizeof(double), cudaMemcpyDeviceToHost));
        CUDA_TRY(c, cudaMemcpy(dv.data(), c->d_dinv, (size_t)c->n * sizeof(double), cudaMemcpyDeviceToHost));
    }
    int64_t q = 0;
    if (colptr) colptr[0] = 0;
    for (int s = 0; s < ns; ++s) {
        const int f = c->h_sn_f[s], cc = c->h_sn_c[s], rr = c->h_sn_r[s];
        const int* rows = c->sym.sn_rows.data() + c->sym.sn_rowptr[s];
        for (int j = 0; j < cc; ++j) {
            for (int i = j; i < rr; ++i) {
                if (rowind) rowind[q] = rows[i];
                // the device keeps Lhat = L diag(1/l) below the diagonal and
                // the reciprocals 1/l; export L
                if (val) val[q] = i == j ? 1.0 / dv[f + j] : Lh[c->h_sn_lptr[s] + (long long)j * rr + i] / dv[f + j];
                ++q;
            }
            if (colptr) colptr[f + j + 1] = q;
        }
    }
    return KKT_OK;
}

kkt_status kkt_set_profiling(kkt_ctx* c, int enable) {
    if (!c) return KKT_ERR_ARG;
    c->profiling = enable != 0;
    return KKT_OK;
}

kkt_status kkt_get_stats(const kkt_ctx* c, kkt_stats* out) {
    if (!c || !out) return KKT_ERR_ARG;
    *out = c->stats;
    return KKT_OK;
}

kkt_status kkt_reset_stats(kkt_ctx* c) {
    if (!c) return KKT_ERR_ARG;
    c->stats = kkt_stats{};
    return KKT_OK;
}

kkt_status kkt_device_bytes(const kkt_ctx* c, int64_t* bytes) {
    if (!c || !bytes) return KKT_ERR_ARG;
    *bytes = c->dev_bytes;
    return KKT_OK;
}

const char* kkt_last_error(const kkt_ctx* c) { return c ? c->err.c_str() : g_err.c_str(); }

void kkt_destroy(kkt_ctx* c) {
    if (!c) return;
    if (c->tri_exec32) cudaGraphExecDestroy(c->tri_exec32);
    if (c->tri_graph32) cudaGraphDestroy(c->tri_graph32);
    if (c->cg_exec32) cudaGraphExecDestroy(c->cg_exec32);
    if (c->cg_graph32) cudaGraphDestroy(c->cg_graph32);
    if (c->tri_exec) cudaGraphExecDestroy(c->tri_exec);
    if (c->tri_graph) cudaGraphDestroy(c->tri_graph);
    if (c->cg_exec) cudaGraphExecDestroy(c->cg_exec);
    if (c->cg_graph) cudaGraphDestroy(c->cg_graph);
    if (c->step_exec) cudaGraphExecDestroy(c->step_exec);
    if (c->step_graph) cudaGraphDestroy(c->step_graph);
    for (cudaStream_t q : c->cap)
        if (q) cudaStreamDestroy(q);
    for (cudaEvent_t e : c->step_ev)
        if (e) cudaEventDestroy(e);
    if (c->h_rst) cudaFreeHost(c->h_rst);
    if (c->h_reta) cudaFreeHost(c->h_reta);
    if (c->hp_delta) cudaFreeHost(c->hp_delta);
    if (c->h_cg) cudaFreeHost(c->h_cg);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_side) cudaEventDestroy(c->ev_side);
    if (c->side) cudaStreamDestroy(c->side);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    for (void* p : c->allocs) cudaFree(p);
    if (c->h_red) cudaFreeHost(c->h_red);
    if (c->h_act) cudaFreeHost(c->h_act);
    if (c->h_int) cudaFreeHost(c->h_int);
    if (c->h_flow_err) cudaFreeHost(c->h_flow_err);
    if (c->h_inst_on) cudaFreeHost(c->h_inst_on);
    delete c;
}

}  // extern "C"

// ------------------------------------------------------------------ helpers
namespace {

__global__ void eval_fn_kernel(int fn, int n, const double* __restrict__ x, double* __restrict__ y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double a = x[i];
        double r = 0.0;
        switch (fn) {
            case KKT_FN_RSQRT: r = kktgb::rsqrt_householder(a); break;
            case KKT_FN_RCP: r = kktgb::rcp_pos(a); break;
            case KKT_FN_SPLIT_M:
            case KKT_FN_SPLIT_E: {
                double m;
                int e;
                if (kktgb::split_pos(a, m, e)) r = fn == KKT_FN_SPLIT_M ? m : (double)e;
                else r = __longlong_as_double(0x7ff8000000000000LL);
                break;
            }
            case KKT_FN_MAX_ABS: r = kktgb::max_abs(a, x[n + i]); break;
            case KKT_FN_MAX_NN: r = kktgb::max_nonneg(a, x[n + i]); break;
            case KKT_FN_MIN_NN: r = kktgb::min_nonneg(a, x[n + i]); break;
            default: r = kktgb::f64_of(kktgb::f32_of(a)); break;
        }
        y[i] = r;
    }
}

}  // namespace

extern "C" kkt_status kkt_eval_fn(int fn, int n, const double* x, double* y, void* stream) {
    if (fn < KKT_FN_RSQRT || fn > KKT_FN_F32_ROUNDTRIP || n < 0 || (n > 0 && (!x || !y))) return KKT_ERR_ARG;
    if (n == 0) return KKT_OK;
    eval_fn_kernel<<<std::min((n + 255) / 256, 152 * 8), 256, 0, (cudaStream_t)stream>>>(fn, n, x, y);
    return cudaGetLastError() == cudaSuccess ? KKT_OK : KKT_ERR_CUDA;
}
