// icm_server.cpp -- the request server of include/icmpt.h (continuous
// batching of whole runs to the thermalization test).
//
// Native runtime around the batch API: a queue of requests, shape classes
// (one slot-table batch and one CUDA stream each), admission by a
// device-memory budget, non-blocking collection of finished launches
// (icm_query), the doubling-window thermalization test (icm_therm_update)
// and result records.  It calls only the public entry points of icmpt.h.
#include "icmpt.h"

#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

namespace {

struct Request {
    uint64_t ticket = 0;
    int32_t lattice = 0, L = 0, disorder = 0;
    std::vector<double> T;
    double T_icm = 0.0;
    uint64_t seed = 0;
    uint32_t instance_id = 0;
    std::vector<unsigned char> couplings;   // [N_b] int8 or float32
    std::vector<int8_t> spins;              // [2 n_T][N] or empty
};

struct Slot {
    bool used = false;
    bool cancel = false;     // release at the next collection
    uint64_t ticket = 0;
    uint32_t t = 0;          // sweeps run
    uint32_t boundary = 0;   // end of the current window
    icm_therm_state state{};
};

struct ShapeKey {
    int32_t lattice, L, disorder;
    std::vector<double> T;
    double T_icm;
    uint64_t seed;
    bool operator<(const ShapeKey &o) const
    {
        if (lattice != o.lattice) return lattice < o.lattice;
        if (L != o.L) return L < o.L;
        if (disorder != o.disorder) return disorder < o.disorder;
        if (T != o.T) return T < o.T;
        if (T_icm != o.T_icm) return T_icm < o.T_icm;
        return seed < o.seed;
    }
};

struct ShapeClass {
    ShapeKey key;
    int32_t N = 0, Nb = 0;
    cudaStream_t stream = nullptr;
    icm_ctx *ctx = nullptr;
    icm_batch *batch = nullptr;
    uint64_t bytes = 0;
    std::vector<Slot> slots;
    std::vector<int> free;           // free slot indices (back = next)
    std::vector<int> in_flight;      // slots of the running launch
    int active = 0;
    // host buffers of the window test
    std::vector<double> accE;
    std::vector<int64_t> acc_d, n_meas;
    std::vector<int32_t> nb;
};

double now_seconds()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Device bytes of a class batch of n slots: the state, staging and
// observable arrays that icm_batch_create allocates (an estimate used for
// admission; the geometry tables and scratch are small next to it).
uint64_t class_bytes(int32_t lattice, int32_t N, int32_t Nb, int32_t n_T, bool gauss, int32_t n)
{
    const uint64_t Z = lattice == ICM_SQUARE2D ? 4 : lattice == ICM_HYPERCUBIC4D ? 8 : 6;
    const uint64_t R = 2 * (uint64_t)n_T, G = (R + 31) / 32;
    const uint64_t per = (gauss ? N * Z * 4 : N)                    // expanded couplings
                         + G * N * 4                                 // packed spins
                         + R * 4 * 2 + R * 8                         // energies (both kinds), staging
                         + (uint64_t)Nb * (gauss ? 4 : 1)            // bond couplings
                         + R * N                                     // spin staging
                         + N * Z * 2 + N + 4                         // dilution tables
                         + (uint64_t)n_T * (N + 1) * 8               // P(q) histograms
                         + (uint64_t)n_T * 8 * 5 + 8                 // accumulators
                         + (uint64_t)n_T * 4 * 6 + 2 * (uint64_t)n_T;  // trace
    return per * (uint64_t)n + 64 * 1024;
}

}  // namespace

struct icm_server {
    int32_t device = 0;
    icm_server_config cfg{};
    std::string err = "no error";
    uint64_t next_ticket = 1;
    uint64_t used = 0;
    std::deque<Request> queue;
    std::map<ShapeKey, std::unique_ptr<ShapeClass>> classes;
    std::vector<ShapeClass *> order;     // creation order
    std::map<uint64_t, icm_result> results;
};

namespace {

icm_status fail(icm_server *s, icm_status code, const std::string &msg)
{
    s->err = msg;
    return code;
}

icm_status from_ctx(icm_server *s, icm_ctx *ctx, icm_status code, const char *what)
{
    return fail(s, code, std::string(what) + ": " + icm_last_error(ctx));
}

void destroy_class(ShapeClass *c)
{
    if (c->ctx) {
        icm_sync(c->ctx);
        icm_ctx_destroy(c->ctx);      // frees the batch too
    }
    if (c->stream) cudaStreamDestroy(c->stream);
    c->ctx = nullptr;
    c->batch = nullptr;
    c->stream = nullptr;
}

icm_status create_class(icm_server *s, const Request &r, ShapeClass **out)
{
    std::unique_ptr<ShapeClass> c(new (std::nothrow) ShapeClass());
    if (!c) return fail(s, ICM_ERR_OOM, "host allocation failed");
    c->key = ShapeKey{r.lattice, r.L, r.disorder, r.T, r.T_icm, r.seed};
    if (icm_lattice_size(r.lattice, r.L, &c->N, &c->Nb)) return fail(s, ICM_ERR_ARG, "bad lattice");
    const int32_t n = s->cfg.slots_per_class, n_T = (int32_t)r.T.size();
    const bool gauss = r.disorder == ICM_GAUSS;
    c->bytes = class_bytes(r.lattice, c->N, c->Nb, n_T, gauss, n);
    if (cudaSetDevice(s->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(s, ICM_ERR_CUDA, "stream creation failed");
    }
    if (icm_ctx_create(&c->ctx, s->device, c->stream) != ICM_OK) {
        destroy_class(c.get());
        return fail(s, ICM_ERR_CUDA, "context creation failed");
    }
    // placeholder couplings of the free slots: every bond present (a zero
    // coupling is an absent bond and would select the diluted kernels)
    std::vector<unsigned char> J((size_t)n * c->Nb * (gauss ? 4 : 1));
    if (gauss) {
        const float one = 1.0f;
        for (size_t i = 0; i < (size_t)n * c->Nb; ++i) std::memcpy(&J[i * 4], &one, 4);
    } else {
        std::memset(J.data(), 1, J.size());
    }
    icm_status st = icm_batch_create(c->ctx, r.lattice, r.L, r.disorder, n, J.data(), nullptr, nullptr, r.T.data(),
                                     n_T, r.T_icm, r.seed, 0, &c->batch);
    if (st == ICM_OK) st = icm_batch_set_active(c->batch, -1, 0);
    if (st == ICM_OK) {
        // a class of large instances (one wide CTA each) runs each instance on
        // a thread-block cluster instead: lower latency per request.  8 CTAs
        // of 512 threads for 8192 sites and more, of 256 below (2D L=64 and
        // 3D L=16, 1 or 20 instances: 36-81 us per sweep, against 37-95
        // with 512 threads)
        int32_t th = 0, cps = 0, grid = 0, smem = 0;
        int64_t launches = 0;
        st = icm_batch_info(c->batch, &th, &cps, &grid, &smem, &launches);
        if (st == ICM_OK && th > 128 && icm_batch_set_cluster(c->batch, 8, c->N >= 8192 ? 512 : 256) != ICM_OK &&
            icm_batch_set_cluster(c->batch, 4, 512) != ICM_OK)
            st = icm_batch_set_cluster(c->batch, 0, th);          // keep the one-CTA layout
    }
    if (st != ICM_OK) {
        icm_status e = from_ctx(s, c->ctx, st, "class batch");
        destroy_class(c.get());
        return e;
    }
    c->slots.assign(n, Slot{});
    for (int i = n - 1; i >= 0; --i) c->free.push_back(i);
    c->accE.resize((size_t)n * n_T);
    c->acc_d.resize((size_t)n * n_T);
    c->n_meas.resize(n);
    c->nb.resize(n);
    *out = c.get();
    s->used += c->bytes;
    s->order.push_back(c.get());
    s->classes[c->key] = std::move(c);
    return ICM_OK;
}

}  // namespace

namespace {

// Admit queued requests, first come first served, into free slots of idle
// classes (a class's slot tables are written between its launches).
icm_status admit(icm_server *s)
{
    std::deque<Request> waiting;
    icm_status st = ICM_OK;
    while (!s->queue.empty()) {
        Request r = std::move(s->queue.front());
        s->queue.pop_front();
        const ShapeKey key{r.lattice, r.L, r.disorder, r.T, r.T_icm, r.seed};
        auto it = s->classes.find(key);
        ShapeClass *c = it == s->classes.end() ? nullptr : it->second.get();
        if (!c) {
            int32_t N, Nb;
            icm_lattice_size(r.lattice, r.L, &N, &Nb);
            const uint64_t need = class_bytes(r.lattice, N, Nb, (int32_t)r.T.size(), r.disorder == ICM_GAUSS,
                                              s->cfg.slots_per_class);
            if (s->used + need > s->cfg.hbm_budget || st != ICM_OK) {
                waiting.push_back(std::move(r));     // admission by memory budget: wait
                continue;
            }
            if ((st = create_class(s, r, &c)) != ICM_OK) {
                waiting.push_back(std::move(r));
                continue;
            }
        }
        if (c->free.empty() || !c->in_flight.empty()) {
            waiting.push_back(std::move(r));
            continue;
        }
        const int slot = c->free.back();
        icm_status e = icm_batch_set_slot(c->batch, slot, r.couplings.empty() ? nullptr : r.couplings.data(),
                                          r.spins.empty() ? nullptr : r.spins.data(), r.instance_id, 0);
        if (e == ICM_OK) e = icm_batch_start_window(c->batch, slot, s->cfg.quantum);   // first window [Q, 2Q)
        if (e != ICM_OK) {
            st = from_ctx(s, c->ctx, e, "slot admission");
            waiting.push_back(std::move(r));
            continue;
        }
        c->free.pop_back();
        Slot &sl = c->slots[slot];
        sl = Slot{};
        sl.used = true;
        sl.ticket = r.ticket;
        sl.boundary = 2u * (uint32_t)s->cfg.quantum;
        c->active += 1;
        icm_result &res = s->results[r.ticket];
        res.slot = slot;
        res.t_admit = now_seconds();
    }
    s->queue.swap(waiting);
    return st;
}

// Free a slot whose request was cancelled.
icm_status release_cancelled(icm_server *s, ShapeClass *c, int slot)
{
    Slot &sl = c->slots[slot];
    icm_result &res = s->results[sl.ticket];
    res.status = ICM_CANCELLED;
    res.sweeps = sl.t;
    res.t_done = now_seconds();
    const icm_status st = icm_batch_set_active(c->batch, slot, 0);
    if (st != ICM_OK) return from_ctx(s, c->ctx, st, "slot release");
    sl = Slot{};
    c->free.push_back(slot);
    c->active -= 1;
    return ICM_OK;
}

// The window of `slot` ended: thermalization test at T_min, then finish the
// request or start the next window [t, 2t).
icm_status close_window(icm_server *s, ShapeClass *c, int slot, int *finished)
{
    Slot &sl = c->slots[slot];
    const int32_t nT = (int32_t)c->key.T.size();
    const double m = (double)(c->n_meas[slot] > 0 ? c->n_meas[slot] : 1);
    const double nb = c->nb[slot] > 0 ? (double)c->nb[slot] : 1.0;
    const double e = c->accE[(size_t)slot * nT] / (2.0 * c->N * m);
    const double ql = 1.0 - 2.0 * (double)c->acc_d[(size_t)slot * nT] / (nb * m);
    int32_t done = 0;
    icm_status st = icm_therm_update(&sl.state, &s->cfg.crit, e, ql, c->key.T[0], nb / c->N, &done);
    if (st != ICM_OK) return fail(s, st, "thermalization test");
    if (done || sl.t >= s->cfg.max_sweeps) {
        icm_result &res = s->results[sl.ticket];
        res.status = ICM_OK;
        res.thermalized = done ? 1 : 0;
        res.sweeps = sl.t;
        res.e = e;
        res.q_l = ql;
        res.delta = sl.state.delta;
        res.accE = c->accE[(size_t)slot * nT];
        res.acc_d = c->acc_d[(size_t)slot * nT];
        res.n_meas = c->n_meas[slot];
        res.t_done = now_seconds();
        if ((st = icm_batch_set_active(c->batch, slot, 0)) != ICM_OK) return from_ctx(s, c->ctx, st, "slot release");
        sl = Slot{};
        c->free.push_back(slot);
        c->active -= 1;
        *finished += 1;
        return ICM_OK;
    }
    if ((st = icm_batch_start_window(c->batch, slot, sl.t)) != ICM_OK) return from_ctx(s, c->ctx, st, "window");
    sl.boundary = 2u * sl.t;
    return ICM_OK;
}

}  // namespace

extern "C" {

double icm_server_clock(void) { return now_seconds(); }

icm_status icm_server_create(int32_t device, const icm_server_config *cfg, icm_server **out)
{
    if (!out) return ICM_ERR_ARG;
    *out = nullptr;
    icm_server_config c{64, 64, 1u << 16, {0.005, 0.01, 2}, 8ull << 30};
    if (cfg) c = *cfg;
    if (c.slots_per_class < 1 || c.quantum < 1 || (c.quantum & (c.quantum - 1)) || c.max_sweeps < 1 ||
        c.crit.need < 1 || !(c.crit.eps_e >= 0) || !(c.crit.eps_ql >= 0))
        return ICM_ERR_ARG;
    icm_server *s = new (std::nothrow) icm_server();
    if (!s) return ICM_ERR_OOM;
    s->device = device;
    s->cfg = c;
    *out = s;
    return ICM_OK;
}

icm_status icm_server_destroy(icm_server *s)
{
    if (!s) return ICM_ERR_ARG;
    for (ShapeClass *c : s->order) destroy_class(c);
    delete s;
    return ICM_OK;
}

const char *icm_server_last_error(const icm_server *s) { return s ? s->err.c_str() : "null server"; }

icm_status icm_server_submit(icm_server *s, const icm_request *r, uint64_t *ticket)
{
    if (!s) return ICM_ERR_ARG;
    if (!r || !ticket) return fail(s, ICM_ERR_ARG, "request and ticket are required");
    int32_t N = 0, Nb = 0;
    if (icm_lattice_size(r->lattice, r->L, &N, &Nb) != ICM_OK) return fail(s, ICM_ERR_ARG, "bad lattice");
    if (r->disorder != ICM_PM_J && r->disorder != ICM_GAUSS) return fail(s, ICM_ERR_ARG, "unknown disorder kind");
    if (!r->T || r->n_T < 1 || r->n_T > 32) return fail(s, ICM_ERR_ARG, "need 1 <= n_T <= 32 temperatures");
    for (int k = 0; k < r->n_T; ++k)
        if (!(r->T[k] > 0.0) || !std::isfinite(r->T[k]) || (k && !(r->T[k] > r->T[k - 1])))
            return fail(s, ICM_ERR_ARG, "temperatures must be finite, > 0 and strictly ascending");
    if (r->instance_id >= (1u << 24)) return fail(s, ICM_ERR_ARG, "instance ids must be < 2^24");
    if (class_bytes(r->lattice, N, Nb, r->n_T, r->disorder == ICM_GAUSS, s->cfg.slots_per_class) >
        s->cfg.hbm_budget)
        return fail(s, ICM_ERR_BUDGET, "the request's class alone exceeds the server's memory budget");
    Request q;
    q.ticket = s->next_ticket++;
    q.lattice = r->lattice;
    q.L = r->L;
    q.disorder = r->disorder;
    q.T.assign(r->T, r->T + r->n_T);
    q.T_icm = r->T_icm;
    q.seed = r->seed;
    q.instance_id = r->instance_id;
    const size_t cb = (size_t)Nb * (r->disorder == ICM_GAUSS ? 4 : 1);
    if (r->couplings)   // else drawn from the request's seed and instance id when it is admitted
        q.couplings.assign((const unsigned char *)r->couplings, (const unsigned char *)r->couplings + cb);
    if (r->spins) q.spins.assign(r->spins, r->spins + (size_t)2 * r->n_T * N);
    icm_result res{};
    res.status = ICM_PENDING;
    res.slot = -1;
    res.t_submit = now_seconds();
    s->results[q.ticket] = res;
    *ticket = q.ticket;
    s->queue.push_back(std::move(q));
    return ICM_OK;
}

icm_status icm_server_step(icm_server *s, int32_t *finished, int32_t *launched)
{
    if (!s) return ICM_ERR_ARG;
    int fin = 0, lau = 0;
    icm_status st = admit(s);
    for (ShapeClass *c : s->order) {
        if (st != ICM_OK) break;
        if (!c->in_flight.empty()) {
            const icm_status q = icm_query(c->ctx);
            if (q == ICM_PENDING) continue;
            if (q != ICM_OK) {
                st = from_ctx(s, c->ctx, q, "class stream");
                break;
            }
            std::vector<int> due;
            for (int slot : c->in_flight) {
                Slot &sl = c->slots[slot];
                sl.t += (uint32_t)s->cfg.quantum;
                if (sl.cancel) {
                    if ((st = release_cancelled(s, c, slot)) != ICM_OK) break;
                    continue;
                }
                if (sl.t >= sl.boundary) due.push_back(slot);
            }
            c->in_flight.clear();
            if (st != ICM_OK) break;
            if (!due.empty()) {
                icm_status e = icm_read_observables(c->batch, c->accE.data(), nullptr, nullptr, nullptr,
                                                    c->acc_d.data(), nullptr, c->n_meas.data(), 0);
                if (e == ICM_OK) e = icm_read_bond_counts(c->batch, c->nb.data());
                if (e != ICM_OK) {
                    st = from_ctx(s, c->ctx, e, "window read");
                    break;
                }
                for (int slot : due)
                    if ((st = close_window(s, c, slot, &fin)) != ICM_OK) break;
                if (st != ICM_OK) break;
            }
        }
        if (c->active > 0) {
            icm_status e = icm_run_sweeps(c->batch, (uint32_t)s->cfg.quantum);
            if (e != ICM_OK) {
                st = from_ctx(s, c->ctx, e, "launch");
                break;
            }
            for (int i = 0; i < (int)c->slots.size(); ++i)
                if (c->slots[i].used) c->in_flight.push_back(i);
            lau += 1;
        }
    }
    if (finished) *finished = fin;
    if (launched) *launched = lau;
    return st;
}

icm_status icm_server_poll(const icm_server *s, uint64_t ticket, icm_result *out)
{
    if (!s || !out) return ICM_ERR_ARG;
    auto it = s->results.find(ticket);
    if (it == s->results.end()) return ICM_ERR_ARG;
    *out = it->second;
    return ICM_OK;
}

icm_status icm_server_cancel(icm_server *s, uint64_t ticket)
{
    if (!s) return ICM_ERR_ARG;
    auto it = s->results.find(ticket);
    if (it == s->results.end()) return fail(s, ICM_ERR_ARG, "unknown ticket");
    if (it->second.status != ICM_PENDING) return fail(s, ICM_ERR_STATE, "the request is no longer pending");
    for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
        if (q->ticket == ticket) {
            s->queue.erase(q);
            it->second.status = ICM_CANCELLED;
            it->second.t_done = now_seconds();
            return ICM_OK;
        }
    for (ShapeClass *c : s->order)
        for (int i = 0; i < (int)c->slots.size(); ++i) {
            Slot &sl = c->slots[i];
            if (!sl.used || sl.ticket != ticket) continue;
            if (c->in_flight.empty()) return release_cancelled(s, c, i);
            sl.cancel = true;               // released when the running launch is collected
            return ICM_OK;
        }
    return fail(s, ICM_ERR_STATE, "request not found in the queue or a slot");
}

icm_status icm_server_status(const icm_server *s, int32_t *queued, int32_t *active, int32_t *classes)
{
    if (!s) return ICM_ERR_ARG;
    int a = 0;
    for (const ShapeClass *c : s->order) a += c->active;
    if (queued) *queued = (int32_t)s->queue.size();
    if (active) *active = a;
    if (classes) *classes = (int32_t)s->order.size();
    return ICM_OK;
}

icm_status icm_server_class_info(const icm_server *s, int32_t i, int32_t *lattice, int32_t *L, int32_t *disorder,
                                 int32_t *n_T, int32_t *threads, int32_t *active)
{
    if (!s || i < 0 || i >= (int32_t)s->order.size()) return ICM_ERR_ARG;
    const ShapeClass *c = s->order[i];
    if (lattice) *lattice = c->key.lattice;
    if (L) *L = c->key.L;
    if (disorder) *disorder = c->key.disorder;
    if (n_T) *n_T = (int32_t)c->key.T.size();
    if (active) *active = c->active;
    if (threads) {
        int32_t th = 0, cps = 0, grid = 0, smem = 0;
        int64_t launches = 0;
        if (icm_batch_info(c->batch, &th, &cps, &grid, &smem, &launches) != ICM_OK) return ICM_ERR_STATE;
        *threads = th;
    }
    return ICM_OK;
}

}  // extern "C"
