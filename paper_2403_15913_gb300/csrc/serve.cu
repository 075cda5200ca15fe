// Receding-horizon (NMPC) serving of the column model: many controllers
// ("clients"), each re-solving its own horizon-T problem whenever a new state
// arrives, served concurrently on one GPU.
//
// The paper's motivation for keeping the symbolic factorisation (Sec. V-B) is
// exactly this reuse: a client's context -- symbolic analysis, supernodal
// storage, CUDA graphs, IPM buffers and its previous solution -- stays
// resident on the device between requests, and every new request starts
// from the previous solution shifted by one stage (warm start), with the
// stage-0 state pinned to the new measurement.
//
// Scheduling: requests wait in one queue in submission order; a worker slot
// (host thread + its own non-blocking CUDA stream) takes the first request
// whose client is idle and can be made resident, so requests of different
// clients overlap on the device while each client's requests run in order.
// Admission: resident contexts may hold at most hbm_budget bytes; a client
// that is not resident is admitted when its estimated footprint fits after
// evicting idle contexts (least recently used first); otherwise its requests
// wait while resident clients proceed.  A context larger than the whole
// budget is admitted only when nothing else is resident.
//
// Batched mode (batch > 0): clients are grouped, in the order they are
// added, into cohorts of up to `batch` clients (a cohort closes when full
// or at the first request for one of its clients).  A cohort's context is
// one kkt_ipm_batch whose members are its clients: each IPM iteration of
// all its running requests is ONE factorisation and refined solve of the
// union of their KKT systems (optionally the FP32 factor with FP64
// refinement).  A worker owns a cohort while it has work; between two
// iterations it retires the requests that finished and starts the requests
// that arrived for its idle clients (continuous batching at iteration
// granularity).  Cohorts are admitted and evicted as a unit.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kkt.h"

namespace {

struct Client {
    double params[16];
    int k = 0, n = 0, m = 0;
    int cohort = -1, member = -1;   // batched mode: its cohort and member index
    kkt_ipm* ipm = nullptr;       // resident context, or NULL
    double* d_prev = nullptr;     // previous solution (device, n)
    bool has_prev = false;
    bool busy = false;
    bool loading = false;         // a worker is creating its context
    long long bytes = 0;          // device bytes while resident
    unsigned long long last_used = 0;
};

struct Request {
    long long id = 0;
    int client = 0;
    bool has_x0 = false;
    std::vector<double> x0;
    bool keep = false;
    double t_submit = 0;
};

struct Cohort {
    std::vector<int> clients;       // member i is client clients[i]
    kkt_ipm_batch* b = nullptr;     // resident batch, or NULL
    bool sealed = false;            // no more clients join
    bool owned = false;             // a worker runs it
    bool loading = false;
    long long bytes = 0;
    unsigned long long last_used = 0;
};

}  // namespace

struct kkt_server {
    kkt_server_options opt{};
    int device = 0;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::deque<Client> clients;            // stable references while clients are added
    std::deque<Cohort> cohorts;            // batched mode
    double cohort_bytes_per_row = 4096.0;  // device bytes per (n + m) row of a cohort (learned)
    bool cohort_learned = false;
    std::deque<Request> queue;
    std::unordered_map<long long, kkt_request_result> done;
    std::unordered_map<long long, std::vector<double>> solutions;
    long long next_id = 1;
    unsigned long long tick = 0;
    long long resident = 0;   // bytes of resident contexts plus reservations of loads in flight
    long long peak = 0;       // largest resident total seen after a load completed
    long long created = 0, evicted = 0, completed = 0, failed = 0;
    std::map<int, double> bytes_per_var;   // learned footprint per tray count
    std::vector<std::thread> workers;
    // evicted contexts and their solution buffers, freed outside the lock
    std::vector<std::pair<kkt_ipm*, double*>> graveyard;
    std::vector<kkt_ipm_batch*> batch_graveyard;

    double now_ms() const {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

long long estimate(kkt_server* S, const Client& c) {
    auto it = S->bytes_per_var.find(c.k);
    const double per = it != S->bytes_per_var.end() ? it->second : 4096.0;
    return (long long)(per * (double)(c.n + c.m) * 1.05) + (1 << 20);
}

// Under the lock: make room for `need` bytes by evicting idle resident
// clients, least recently used first.  Returns whether it fits.
bool make_room(kkt_server* S, long long need) {
    const long long budget = (long long)(S->opt.hbm_budget_gb * 1e9);
    while (S->resident + need > budget) {
        int victim = -1;
        for (int i = 0; i < (int)S->clients.size(); ++i) {
            const Client& c = S->clients[i];
            if (c.ipm && !c.busy && !c.loading &&
                (victim < 0 || c.last_used < S->clients[victim].last_used))
                victim = i;
        }
        if (victim < 0) return S->resident == 0;   // alone it may exceed the budget
        Client& v = S->clients[victim];
        S->graveyard.push_back({v.ipm, v.d_prev});
        v.ipm = nullptr;
        v.d_prev = nullptr;
        v.has_prev = false;
        S->resident -= v.bytes;
        v.bytes = 0;
        S->evicted++;
    }
    return true;
}

void flush_graveyard(kkt_server* S, std::unique_lock<std::mutex>& lk) {
    if (S->graveyard.empty() && S->batch_graveyard.empty()) return;
    std::vector<std::pair<kkt_ipm*, double*>> g;
    std::vector<kkt_ipm_batch*> gb;
    g.swap(S->graveyard);
    gb.swap(S->batch_graveyard);
    lk.unlock();
    for (auto& e : g) {
        kkt_ipm_destroy(e.first);
        cudaFree(e.second);
    }
    for (kkt_ipm_batch* b : gb) kkt_ipm_batch_destroy(b);
    lk.lock();
}

// Under the lock: index into the queue of the first request that can run now,
// reserving room for a client that is not resident.  -1 if none.
int pick(kkt_server* S, long long* reserved) {
    for (int q = 0; q < (int)S->queue.size(); ++q) {
        Client& c = S->clients[S->queue[q].client];
        if (c.busy || c.loading) continue;
        // keep each client's requests in order: skip if an earlier one waits
        bool earlier = false;
        for (int e = 0; e < q; ++e)
            if (S->queue[e].client == S->queue[q].client) { earlier = true; break; }
        if (earlier) continue;
        if (c.ipm) {
            *reserved = 0;
            return q;
        }
        const long long est = estimate(S, c);
        if (make_room(S, est)) {
            S->resident += est;   // reservation; the measured size replaces it after the load
            *reserved = est;
            return q;
        }
    }
    return -1;
}

void solver_options(const kkt_server* S, kkt_options* ko, kkt_ipm_options* io) {
    kkt_default_options(ko);
    ko->scheme = S->opt.scheme;
    ko->precision = S->opt.precision;
    ko->gamma = S->opt.gamma;
    ko->max_cg = 500;
    kkt_ipm_default_options(io);
    io->tol = S->opt.tol;
    io->max_iter = S->opt.max_iter;
    io->mu_init = S->opt.mu_init;
}

// Create a client's context and solution buffer (no lock held; c is a copy).
kkt_status load(kkt_server* S, const Client& c, kkt_ipm** ipm, double** prev_out, long long* bytes) {
    kkt_options ko;
    kkt_ipm_options io;
    solver_options(S, &ko, &io);
    kkt_ipm* p = nullptr;
    kkt_status s = kkt_ipm_create(c.params, &ko, &io, &p);
    if (s != KKT_OK) return s;
    double* prev = nullptr;
    if (cudaMalloc((void**)&prev, (size_t)c.n * sizeof(double)) != cudaSuccess) {
        kkt_ipm_destroy(p);
        return KKT_ERR_OOM;
    }
    int64_t b = 0;
    kkt_ipm_device_bytes(p, &b);
    *ipm = p;
    *prev_out = prev;
    *bytes = b + (long long)c.n * (long long)sizeof(double);
    return KKT_OK;
}

// Start a request's solve on IPM p (the client's own context or its member
// of a cohort): the stage-0 state is the request's, else stage 1 of the
// client's previous solution (the column advanced one step as predicted),
// else xbar_0; warm start from the previous solution when there is one.
kkt_status begin_request(const kkt_server* S, const Client& c, const Request& r, kkt_ipm* p, cudaStream_t st,
                         std::vector<double>& x1, kkt_request_result& res) {
    kkt_status s;
    if (r.has_x0) {
        s = kkt_ipm_set_initial_state(p, r.x0.data(), st);
    } else if (c.has_prev) {
        x1.resize(c.k);
        const int nst = 2 * c.k + 1;
        const int off = c.n > nst ? nst : 0;
        if (cudaMemcpyAsync(x1.data(), c.d_prev + off, c.k * sizeof(double), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            s = KKT_ERR_CUDA;
        else
            s = kkt_ipm_set_initial_state(p, x1.data(), st);
    } else {
        s = kkt_ipm_set_initial_state(p, nullptr, st);
    }
    if (s != KKT_OK) return s;
    if (c.has_prev && S->opt.warm_start) {
        res.warm = 1;
        return kkt_ipm_init_warm(p, S->opt.warm_mu, S->opt.warm_recenter, st);
    }
    return kkt_ipm_init(p, nullptr, st);
}

bool solved(int status) { return status == KKT_CONVERGED || status == KKT_OK || status == KKT_ERR_MAXIT; }

// After a solve that produced an iterate: keep it as the client's previous
// solution (device) and, if asked, copy it to the host.
void keep_solution(const Client& c, const kkt_ipm* p, bool keep, cudaStream_t st, std::vector<double>& sol) {
    kkt_ipm_get(p, c.d_prev, nullptr, nullptr, nullptr, nullptr, st);
    if (keep) {
        sol.resize(c.n);
        cudaMemcpyAsync(sol.data(), c.d_prev, c.n * sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
    }
}

// Under the lock: a finished request's result and the client's state.
void complete(kkt_server* S, const Request& r, const kkt_request_result& res, std::vector<double>& sol) {
    Client& c = S->clients[r.client];
    c.busy = false;
    c.last_used = ++S->tick;
    if (solved(res.status)) {
        c.has_prev = true;
    } else {
        c.has_prev = false;   // its iterate may be unusable: the next request starts cold
        S->failed++;
    }
    S->completed++;
    S->done[r.id] = res;
    if (r.keep) S->solutions[r.id] = std::move(sol);
}

void worker_batched(kkt_server* S, int slot);

void worker(kkt_server* S, int slot) {
    if (S->opt.batch > 0) {
        worker_batched(S, slot);
        return;
    }
    cudaSetDevice(S->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    std::vector<double> x1;
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        flush_graveyard(S, lk);
        if (S->stop) break;
        long long reserved = 0;
        const int q = pick(S, &reserved);
        if (q < 0) {
            S->cv_work.wait(lk);
            continue;
        }
        Request r = std::move(S->queue[q]);
        S->queue.erase(S->queue.begin() + q);
        Client& c = S->clients[r.client];   // deque: stable while clients are added
        c.busy = true;
        kkt_request_result res{};
        res.id = r.id;
        res.client = r.client;
        res.slot = slot;
        res.t_submit_ms = r.t_submit;
        res.cold = 0;
        kkt_status s = KKT_OK;
        if (!c.ipm) {
            c.loading = true;
            res.cold = 1;
            const Client copy = c;
            flush_graveyard(S, lk);
            lk.unlock();
            long long bytes = 0;
            kkt_ipm* ipm = nullptr;
            double* prev = nullptr;
            s = load(S, copy, &ipm, &prev, &bytes);
            lk.lock();
            c.loading = false;
            if (s == KKT_OK) {
                c.ipm = ipm;
                c.d_prev = prev;
                c.has_prev = false;
                S->resident += bytes - reserved;
                S->peak = std::max(S->peak, S->resident);
                c.bytes = bytes;
                const double per = (double)bytes / (double)(c.n + c.m);
                double& learned = S->bytes_per_var[c.k];
                learned = std::max(learned, per);
                S->created++;
            } else {
                S->resident -= reserved;
            }
        }
        Client snapshot = c;
        lk.unlock();
        res.t_start_ms = S->now_ms();
        std::vector<double> sol;
        if (s == KKT_OK) {
            kkt_ipm* p = snapshot.ipm;
            s = begin_request(S, snapshot, r, p, st, x1, res);
            kkt_ipm_info info{};
            if (s == KKT_OK) s = kkt_ipm_solve(p, st, &info);
            res.status = s;
            res.iters = info.iter;
            res.objective = info.objective;
            res.inf_pr = info.inf_pr;
            res.inf_du = info.inf_du;
            if (solved(s)) keep_solution(snapshot, p, r.keep, st, sol);
        } else {
            res.status = s;
        }
        res.t_done_ms = S->now_ms();
        lk.lock();
        complete(S, r, res, sol);
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
    lk.unlock();
    cudaStreamDestroy(st);
}

// ---- batched mode
long long estimate_cohort(const kkt_server* S, const Cohort& h) {
    long long rows = 0;
    for (int ci : h.clients) rows += (long long)S->clients[ci].n + S->clients[ci].m;
    return (long long)(S->cohort_bytes_per_row * (double)rows * 1.05) + (8LL << 20);
}

// Under the lock: make room for `need` bytes by evicting idle resident
// cohorts, least recently used first (their clients' previous solutions go
// with them).  Returns whether it fits.
bool make_room_cohorts(kkt_server* S, long long need) {
    const long long budget = (long long)(S->opt.hbm_budget_gb * 1e9);
    while (S->resident + need > budget) {
        int victim = -1;
        for (int i = 0; i < (int)S->cohorts.size(); ++i) {
            const Cohort& h = S->cohorts[i];
            if (h.b && !h.owned && !h.loading && (victim < 0 || h.last_used < S->cohorts[victim].last_used))
                victim = i;
        }
        if (victim < 0) return S->resident == 0;   // alone it may exceed the budget
        Cohort& v = S->cohorts[victim];
        S->batch_graveyard.push_back(v.b);
        for (int ci : v.clients) {
            Client& c = S->clients[ci];
            if (c.d_prev) S->graveyard.push_back({nullptr, c.d_prev});
            c.d_prev = nullptr;
            c.has_prev = false;
        }
        v.b = nullptr;
        S->resident -= v.bytes;
        v.bytes = 0;
        S->evicted++;
    }
    return true;
}

// Under the lock: a cohort with a queued request for an idle client that
// no worker runs, reserving room for it if it is not resident.  -1 if none.
int pick_cohort(kkt_server* S, long long* reserved) {
    for (const Request& r : S->queue) {
        const Client& c = S->clients[r.client];
        Cohort& h = S->cohorts[c.cohort];
        if (h.owned || h.loading || c.busy) continue;
        if (h.b) {
            *reserved = 0;
            return c.cohort;
        }
        const long long est = estimate_cohort(S, h);
        if (make_room_cohorts(S, est)) {
            S->resident += est;   // reservation; the measured size replaces it after the load
            *reserved = est;
            return c.cohort;
        }
    }
    return -1;
}

// Create a cohort's batch and its clients' solution buffers (no lock held;
// cl are copies of its clients in member order).
kkt_status load_cohort(kkt_server* S, const std::vector<Client>& cl, kkt_ipm_batch** out,
                       std::vector<double*>& prev, long long* bytes) {
    kkt_options ko;
    kkt_ipm_options io;
    solver_options(S, &ko, &io);
    const int count = (int)cl.size();
    std::vector<double> params(16 * (size_t)count);
    for (int i = 0; i < count; ++i) std::copy(cl[i].params, cl[i].params + 16, params.begin() + 16 * (size_t)i);
    kkt_ipm_batch* b = nullptr;
    kkt_status s = kkt_ipm_batch_create(count, params.data(), &ko, &io, &b);
    if (s != KKT_OK) return s;
    prev.assign(count, nullptr);
    long long extra = 0;
    for (int i = 0; i < count; ++i) {
        if (cudaMalloc((void**)&prev[i], (size_t)cl[i].n * sizeof(double)) != cudaSuccess) {
            for (double* q : prev) cudaFree(q);
            prev.clear();
            kkt_ipm_batch_destroy(b);
            return KKT_ERR_OOM;
        }
        extra += (long long)cl[i].n * (long long)sizeof(double);
    }
    int64_t bb = 0;
    kkt_ipm_batch_device_bytes(b, &bb);
    *bytes = bb + extra;
    *out = b;
    return KKT_OK;
}

// The worker owns cohort h (lock held on entry and exit): between two
// iterations of its batch it starts the queued requests of its idle clients
// (a client's requests in submission order) and retires the finished ones,
// until none runs and none waits.
void run_cohort(kkt_server* S, int hi, int slot, cudaStream_t st, std::unique_lock<std::mutex>& lk) {
    Cohort& h = S->cohorts[hi];   // deque: stable while cohorts are added
    const int count = (int)h.clients.size();
    kkt_ipm_batch* b = h.b;
    std::vector<Request> req(count);
    std::vector<kkt_request_result> res(count);
    std::vector<char> live(count, 0);
    std::vector<kkt_ipm_info> infos(count);
    std::vector<double> x1;
    bool cold = h.last_used == 0;
    bool failed_batch = false;
    while (true) {
        // admit: queued requests of this cohort's idle clients, oldest first
        std::vector<int> admitted;
        for (size_t q = 0; q < S->queue.size();) {
            Client& c = S->clients[S->queue[q].client];
            if (c.cohort != hi || c.busy) {
                ++q;
                continue;
            }
            const int i = c.member;
            req[i] = std::move(S->queue[q]);
            S->queue.erase(S->queue.begin() + (long)q);
            c.busy = true;
            admitted.push_back(i);
        }
        bool any = !admitted.empty();
        for (int i = 0; i < count && !any; ++i) any = live[i] != 0;
        if (!any) break;
        std::vector<Client> snap(admitted.size());
        for (size_t a = 0; a < admitted.size(); ++a) snap[a] = S->clients[h.clients[admitted[a]]];
        lk.unlock();
        std::vector<int> finished;
        for (size_t a = 0; a < admitted.size(); ++a) {
            const int i = admitted[a];
            kkt_request_result& rr = res[i];
            rr = kkt_request_result{};
            rr.id = req[i].id;
            rr.client = req[i].client;
            rr.slot = slot;
            rr.t_submit_ms = req[i].t_submit;
            rr.t_start_ms = S->now_ms();
            rr.cold = cold ? 1 : 0;
            kkt_ipm* p = kkt_ipm_batch_member(b, i);
            kkt_status s = begin_request(S, snap[a], req[i], p, st, x1, rr);
            if (s == KKT_OK) s = kkt_ipm_batch_start_member(b, i);
            if (s == KKT_OK) {
                live[i] = 1;
            } else {
                rr.status = s;
                finished.push_back(i);
            }
        }
        cold = false;
        kkt_status bs = KKT_OK;
        bool stepping = false;
        for (int i = 0; i < count && !stepping; ++i) stepping = live[i] != 0;
        if (stepping) bs = kkt_ipm_batch_step(b, st, infos.data());
        for (int i = 0; i < count; ++i) {
            if (!live[i]) continue;
            int status = KKT_OK, iters = 0;
            kkt_ipm_batch_member_status(b, i, &status, &iters);
            if (bs != KKT_OK && bs != KKT_CONVERGED) status = bs;   // batch-wide failure
            if (status == KKT_OK) continue;
            kkt_request_result& rr = res[i];
            rr.status = status;
            rr.iters = iters;
            rr.objective = infos[i].objective;
            rr.inf_pr = infos[i].inf_pr;
            rr.inf_du = infos[i].inf_du;
            live[i] = 0;
            finished.push_back(i);
        }
        std::vector<std::vector<double>> sols(finished.size());
        for (size_t f = 0; f < finished.size(); ++f) {
            const int i = finished[f];
            if (solved(res[i].status)) {
                lk.lock();
                const Client c = S->clients[h.clients[i]];
                lk.unlock();
                keep_solution(c, kkt_ipm_batch_member(b, i), req[i].keep, st, sols[f]);
            }
            res[i].t_done_ms = S->now_ms();
        }
        lk.lock();
        for (size_t f = 0; f < finished.size(); ++f) complete(S, req[finished[f]], res[finished[f]], sols[f]);
        if (!finished.empty()) S->cv_done.notify_all();
        if (bs != KKT_OK && bs != KKT_CONVERGED) {   // every live request was retired above
            failed_batch = true;
            break;
        }
    }
    h.owned = false;
    h.last_used = ++S->tick;
    if (failed_batch) {   // its context is not reused: the next request rebuilds it
        S->batch_graveyard.push_back(h.b);
        for (int ci : h.clients) {
            Client& c = S->clients[ci];
            if (c.d_prev) S->graveyard.push_back({nullptr, c.d_prev});
            c.d_prev = nullptr;
            c.has_prev = false;
        }
        h.b = nullptr;
        S->resident -= h.bytes;
        h.bytes = 0;
    }
    S->cv_work.notify_all();
}

void worker_batched(kkt_server* S, int slot) {
    cudaSetDevice(S->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        flush_graveyard(S, lk);
        if (S->stop) break;
        long long reserved = 0;
        const int hi = pick_cohort(S, &reserved);
        if (hi < 0) {
            S->cv_work.wait(lk);
            continue;
        }
        Cohort& h = S->cohorts[hi];
        h.sealed = true;
        h.owned = true;
        if (!h.b) {
            h.loading = true;
            std::vector<Client> cl;
            for (int ci : h.clients) cl.push_back(S->clients[ci]);
            flush_graveyard(S, lk);
            lk.unlock();
            long long bytes = 0;
            kkt_ipm_batch* b = nullptr;
            std::vector<double*> prev;
            const kkt_status s = load_cohort(S, cl, &b, prev, &bytes);
            lk.lock();
            h.loading = false;
            if (s != KKT_OK) {
                // every queued request of its clients fails with the load's status
                S->resident -= reserved;
                for (size_t q = 0; q < S->queue.size();) {
                    const Request& r = S->queue[q];
                    if (S->clients[r.client].cohort != hi) {
                        ++q;
                        continue;
                    }
                    kkt_request_result rr{};
                    rr.id = r.id;
                    rr.client = r.client;
                    rr.slot = slot;
                    rr.status = s;
                    rr.t_submit_ms = r.t_submit;
                    rr.t_start_ms = rr.t_done_ms = S->now_ms();
                    std::vector<double> none;
                    const Request rc = r;
                    S->queue.erase(S->queue.begin() + (long)q);
                    S->clients[rc.client].busy = true;
                    complete(S, rc, rr, none);
                }
                h.owned = false;
                S->cv_done.notify_all();
                S->cv_work.notify_all();
                continue;
            }
            h.b = b;
            h.bytes = bytes;
            h.last_used = 0;   // the first round's requests are cold
            for (size_t i = 0; i < h.clients.size(); ++i) {
                Client& c = S->clients[h.clients[i]];
                c.d_prev = prev[i];
                c.has_prev = false;
            }
            S->resident += bytes - reserved;
            S->peak = std::max(S->peak, S->resident);
            long long rows = 0;
            for (int ci : h.clients) rows += (long long)S->clients[ci].n + S->clients[ci].m;
            const double per = (double)bytes / (double)std::max(1LL, rows);
            S->cohort_bytes_per_row = S->cohort_learned ? std::max(S->cohort_bytes_per_row, per) : per;
            S->cohort_learned = true;
            S->created++;
        }
        run_cohort(S, hi, slot, st, lk);
    }
    lk.unlock();
    cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

void kkt_server_default_options(kkt_server_options* o) {
    if (!o) return;
    o->slots = 8;
    o->hbm_budget_gb = 40.0;
    o->scheme = KKT_LIFTED;
    o->precision = 0;
    o->gamma = 1e7;
    o->tol = 1e-8;
    o->max_iter = 200;
    o->mu_init = 0.1;
    o->warm_start = 1;
    o->warm_mu = 1e-4;
    o->warm_recenter = 1;
    o->batch = 0;
}

kkt_status kkt_server_create(const kkt_server_options* opt, int device, kkt_server** out) {
    if (!out) return KKT_ERR_ARG;
    *out = nullptr;
    kkt_server* S = new (std::nothrow) kkt_server();
    if (!S) return KKT_ERR_OOM;
    if (opt) S->opt = *opt; else kkt_server_default_options(&S->opt);
    if (S->opt.slots < 1 || S->opt.slots > 256 || !(S->opt.hbm_budget_gb > 0) || S->opt.batch < 0 ||
        S->opt.batch > 4096 ||
        (S->opt.scheme != KKT_LIFTED && S->opt.scheme != KKT_HYKKT) || !(S->opt.warm_mu > 0)) {
        delete S;
        return KKT_ERR_ARG;
    }
    S->device = device;
    S->t0 = std::chrono::steady_clock::now();
    for (int w = 0; w < S->opt.slots; ++w) S->workers.emplace_back(worker, S, w);
    *out = S;
    return KKT_OK;
}

kkt_status kkt_server_add_client(kkt_server* S, const double* params, int* client) {
    if (!S || !params || !client) return KKT_ERR_ARG;
    int n = 0, m = 0, nw = 0, nj = 0;
    kkt_status s = kkt_tray_sizes(params, &n, &m, &nw, &nj);
    if (s != KKT_OK) return s;
    std::lock_guard<std::mutex> g(S->mu);
    Client c;
    std::copy(params, params + 16, c.params);
    c.k = (int)params[0];
    c.n = n;
    c.m = m;
    const int id = (int)S->clients.size();
    if (S->opt.batch > 0) {   // joins the open cohort, or opens the next one
        if (S->cohorts.empty() || S->cohorts.back().sealed || (int)S->cohorts.back().clients.size() >= S->opt.batch)
            S->cohorts.emplace_back();
        Cohort& h = S->cohorts.back();
        c.cohort = (int)S->cohorts.size() - 1;
        c.member = (int)h.clients.size();
        h.clients.push_back(id);
        if ((int)h.clients.size() >= S->opt.batch) h.sealed = true;
    }
    S->clients.push_back(c);
    *client = id;
    return KKT_OK;
}

kkt_status kkt_server_submit(kkt_server* S, int client, const double* x0, int keep_solution,
                             int64_t* id) {
    if (!S || !id) return KKT_ERR_ARG;
    std::lock_guard<std::mutex> g(S->mu);
    if (client < 0 || client >= (int)S->clients.size()) return KKT_ERR_ARG;
    Request r;
    r.id = S->next_id++;
    r.client = client;
    r.keep = keep_solution != 0;
    if (x0) {
        r.has_x0 = true;
        r.x0.assign(x0, x0 + S->clients[client].k);
    }
    r.t_submit = S->now_ms();
    *id = r.id;
    if (S->opt.batch > 0) S->cohorts[S->clients[client].cohort].sealed = true;
    S->queue.push_back(std::move(r));
    S->cv_work.notify_one();
    return KKT_OK;
}

kkt_status kkt_server_wait(kkt_server* S, int64_t id, kkt_request_result* out, double* h_x) {
    if (!S) return KKT_ERR_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    if (id <= 0 || id >= S->next_id) return KKT_ERR_ARG;
    S->cv_done.wait(lk, [&] { return S->done.count(id) > 0; });
    const kkt_request_result& r = S->done[id];
    if (out) *out = r;
    auto it = S->solutions.find(id);
    if (it != S->solutions.end()) {
        if (h_x && !it->second.empty()) std::memcpy(h_x, it->second.data(), it->second.size() * sizeof(double));
        S->solutions.erase(it);
    }
    return KKT_OK;
}

kkt_status kkt_server_drain(kkt_server* S) {
    if (!S) return KKT_ERR_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv_done.wait(lk, [&] {
        if (!S->queue.empty()) return false;
        for (const Client& c : S->clients)
            if (c.busy || c.loading) return false;
        return true;
    });
    return KKT_OK;
}

kkt_status kkt_server_get_stats(kkt_server* S, kkt_server_stats* st) {
    if (!S || !st) return KKT_ERR_ARG;
    std::lock_guard<std::mutex> g(S->mu);
    st->completed = S->completed;
    st->failed = S->failed;
    st->contexts_created = S->created;
    st->evictions = S->evicted;
    st->resident_bytes = S->resident;
    st->peak_resident_bytes = S->peak;
    st->queued = (int64_t)S->queue.size();
    int res = 0;
    for (const Client& c : S->clients) res += c.ipm != nullptr;
    for (const Cohort& h : S->cohorts)
        if (h.b) res += (int)h.clients.size();
    st->resident_clients = res;
    return KKT_OK;
}

void kkt_server_destroy(kkt_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto& t : S->workers) t.join();
    for (auto& e : S->graveyard) {
        kkt_ipm_destroy(e.first);
        cudaFree(e.second);
    }
    for (kkt_ipm_batch* b : S->batch_graveyard) kkt_ipm_batch_destroy(b);
    for (Cohort& h : S->cohorts)
        if (h.b) kkt_ipm_batch_destroy(h.b);
    for (Client& c : S->clients) {
        if (c.ipm) kkt_ipm_destroy(c.ipm);
        if (c.d_prev) cudaFree(c.d_prev);
    }
    delete S;
}

}  // extern "C"
