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

}  // namespace

struct kkt_server {
    kkt_server_options opt{};
    int device = 0;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::deque<Client> clients;            // stable references while clients are added
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
    if (S->graveyard.empty()) return;
    std::vector<std::pair<kkt_ipm*, double*>> g;
    g.swap(S->graveyard);
    lk.unlock();
    for (auto& e : g) {
        kkt_ipm_destroy(e.first);
        cudaFree(e.second);
    }
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

// Create a client's context and solution buffer (no lock held; c is a copy).
kkt_status load(kkt_server* S, const Client& c, kkt_ipm** ipm, double** prev_out, long long* bytes) {
    kkt_options ko;
    kkt_default_options(&ko);
    ko.scheme = S->opt.scheme;
    ko.precision = S->opt.precision;
    ko.gamma = S->opt.gamma;
    ko.max_cg = 500;
    kkt_ipm_options io;
    kkt_ipm_default_options(&io);
    io.tol = S->opt.tol;
    io.max_iter = S->opt.max_iter;
    io.mu_init = S->opt.mu_init;
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

void worker(kkt_server* S, int slot) {
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
            // initial state: given, else the previous solution's stage 1
            // (the column advanced one step as predicted), else x0bar
            if (r.has_x0) {
                s = kkt_ipm_set_initial_state(p, r.x0.data(), st);
            } else if (snapshot.has_prev) {
                x1.resize(snapshot.k);
                const int nst = 2 * snapshot.k + 1;
                const int off = snapshot.n > nst ? nst : 0;
                if (cudaMemcpyAsync(x1.data(), snapshot.d_prev + off, snapshot.k * sizeof(double),
                                    cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                    cudaStreamSynchronize(st) != cudaSuccess)
                    s = KKT_ERR_CUDA;
                else
                    s = kkt_ipm_set_initial_state(p, x1.data(), st);
            } else {
                s = kkt_ipm_set_initial_state(p, nullptr, st);
            }
            if (s == KKT_OK) {
                if (snapshot.has_prev && S->opt.warm_start) {
                    s = kkt_ipm_init_warm(p, S->opt.warm_mu, S->opt.warm_recenter, st);
                    res.warm = 1;
                } else {
                    s = kkt_ipm_init(p, nullptr, st);
                }
            }
            kkt_ipm_info info{};
            if (s == KKT_OK) s = kkt_ipm_solve(p, st, &info);
            res.status = s;
            res.iters = info.iter;
            res.objective = info.objective;
            res.inf_pr = info.inf_pr;
            res.inf_du = info.inf_du;
            if (s == KKT_CONVERGED || s == KKT_OK || s == KKT_ERR_MAXIT) {
                kkt_ipm_get(p, snapshot.d_prev, nullptr, nullptr, nullptr, nullptr, st);
                if (r.keep) {
                    sol.resize(snapshot.n);
                    cudaMemcpyAsync(sol.data(), snapshot.d_prev, snapshot.n * sizeof(double),
                                    cudaMemcpyDeviceToHost, st);
                    cudaStreamSynchronize(st);
                }
            }
        } else {
            res.status = s;
        }
        res.t_done_ms = S->now_ms();
        lk.lock();
        Client& c2 = S->clients[r.client];
        c2.busy = false;
        c2.last_used = ++S->tick;
        if (res.status == KKT_CONVERGED || res.status == KKT_OK || res.status == KKT_ERR_MAXIT) {
            c2.has_prev = true;
        } else {
            c2.has_prev = false;   // its iterate may be unusable: the next request starts cold
            S->failed++;
        }
        S->completed++;
        S->done[r.id] = res;
        if (r.keep) S->solutions[r.id] = std::move(sol);
        S->cv_done.notify_all();
        S->cv_work.notify_all();
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
}

kkt_status kkt_server_create(const kkt_server_options* opt, int device, kkt_server** out) {
    if (!out) return KKT_ERR_ARG;
    *out = nullptr;
    kkt_server* S = new (std::nothrow) kkt_server();
    if (!S) return KKT_ERR_OOM;
    if (opt) S->opt = *opt; else kkt_server_default_options(&S->opt);
    if (S->opt.slots < 1 || S->opt.slots > 256 || !(S->opt.hbm_budget_gb > 0) ||
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
    S->clients.push_back(c);
    *client = (int)S->clients.size() - 1;
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
    for (Client& c : S->clients)
        if (c.ipm) {
            kkt_ipm_destroy(c.ipm);
            cudaFree(c.d_prev);
        }
    delete S;
}

}  // extern "C"
