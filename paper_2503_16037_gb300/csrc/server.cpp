// Serving: continuous batching of scene solves over a pool of resident
// scenes (slots).  See the tursca_server_* declarations for the contract.
//
// Scheduling.  Requests wait in FIFO order.  A free worker takes the first
// request it can start now: one whose shape has an idle slot, or one whose
// new slot fits the memory budget (after evicting idle slots of other shapes,
// least recently used first).  A request at the head that has waited longer
// than kAgingMs for memory stops later requests from building new slots, so
// large scenes cannot be starved by a stream of small ones.  Each slot owns a
// CUDA stream; the library's per-request host synchronisations block only
// the worker that issued them, so the device runs the kernels of concurrent
// requests side by side.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "batcher.h"
#include "tursca.h"

namespace {

constexpr double kAgingMs = 50.0;

using Clock = std::chrono::steady_clock;

// shape of a slot: everything of the grid descriptor
using ShapeKey = std::tuple<int, int, int, double, double, double, int, int, int, int>;

ShapeKey key_of(const tursca_grid_desc &d) {
    return ShapeKey(d.nx, d.ny, d.nz, d.hx, d.hy, d.hz, d.stencil_radius, d.n_species, d.fib_points, d.precision);
}

struct Slot {
    tursca_scene *sc = nullptr;
    cudaStream_t st = nullptr;
    ShapeKey key;
    size_t bytes = 0;
    bool busy = false;
    long long last_use = 0;
};

struct Request {
    long long ticket = 0;
    tursca_grid_desc desc;
    tursca_geometry geom;
    const void *mu_abs = nullptr, *mu_sca = nullptr;
    std::vector<double> g;
    double albedo = 0.0, rtol = 1e-10;
    void *radiance = nullptr;
    tursca_request_info info;
    bool done = false;
};

}  // namespace

struct tursca_server {
    size_t budget = 0, used = 0, peak = 0;
    int workers_n = 0, device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> pending;
    std::unordered_map<long long, std::unique_ptr<Request>> reqs;
    std::vector<std::unique_ptr<Slot>> slots;
    std::map<ShapeKey, size_t> slot_bytes;  // measured device bytes of a slot per shape
    std::map<ShapeKey, tursca_graph_stats> shape_stats;  // graph counts per shape (validated descriptors)
    std::vector<std::thread> workers;
    long long next_ticket = 1, use_clock = 0;
    int evictions = 0, built = 0, reserving = 0;
    bool stop = false;
    bool batch_solves = false;          // TURSCA_SERVER_BATCH_SOLVES
    tk::ChebBatcher *batcher = nullptr;  // created with the first FP32 slot
    Clock::time_point t0 = Clock::now();

    double now_ms() const { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }
};

namespace {

// device bytes of a new slot for this shape: measured once built; before
// that, the scene's allocations itemised from the graph counts (with room for
// the GMRES basis the solver may need) plus a tenth
size_t slot_estimate(tursca_server *srv, const tursca_grid_desc &d) {
    auto it = srv->slot_bytes.find(key_of(d));
    if (it != srv->slot_bytes.end()) return it->second;
    auto is = srv->shape_stats.find(key_of(d));
    if (is == srv->shape_stats.end()) return srv->budget;  // not reached: submit records every shape
    const tursca_graph_stats &st = is->second;
    const double es = d.precision == TURSCA_FP64 ? 8.0 : 4.0;
    const double R = d.stencil_radius, S = d.n_species;
    const double lp = (d.nx + 2 * R) * (d.ny + 2 * R), npad = (d.nz + 1) * lp;
    const double na = st.n_atm, nn = st.n_nodes;
    const double nc = st.n_dirs / 2.0;
    const double gm = d.precision == TURSCA_FP64 ? 41.0 : 31.0;  // GMRES basis vectors
    double b = es * ((double)st.nnz                      // values of K
                     + (nc + 5 + S + 4 + gm) * npad       // segment table, haloed copies, solver vectors, basis
                     + (double)st.n_up_dirs * na          // tau_inf
                     + (double)st.n_gdirs * lp            // ground TOA planes
                     + (3 + S + 3) * na + 3 * nn)         // fields, e1, s, emission
               + 24.0 * npad                              // FP64 x and r, FP32 pair of x
               + 96.0 * 8.0 * st.max_row * (d.nz + 1)     // template descriptors (upper bound)
               + (2 << 20);                               // partial sums, view taps, small tables
    return (size_t)(1.1 * b);
}

// take one admissible request (caller holds the lock); returns null if none
Request *pick(tursca_server *srv, Slot **slot_out, bool *build_out, size_t *reserve_out) {
    const double now = srv->now_ms();
    bool head_blocked = false;
    for (auto it = srv->pending.begin(); it != srv->pending.end(); ++it) {
        Request *r = *it;
        const ShapeKey k = key_of(r->desc);
        // an idle resident slot of the same shape
        Slot *best = nullptr;
        for (auto &s : srv->slots)
            if (!s->busy && s->key == k) {
                best = s.get();
                break;
            }
        if (best) {
            best->busy = true;
            best->last_use = ++srv->use_clock;
            *slot_out = best;
            *build_out = false;
            *reserve_out = 0;
            srv->pending.erase(it);
            return r;
        }
        if (head_blocked) continue;  // an aged head keeps new slots for itself
        const size_t need = slot_estimate(srv, r->desc);
        // evict idle slots, least recently used first, until the new one fits
        size_t freeable = 0;
        for (auto &s : srv->slots)
            if (!s->busy) freeable += s->bytes;
        if (srv->used + need <= srv->budget || (srv->used - freeable + need <= srv->budget)) {
            while (srv->used + need > srv->budget) {
                Slot *lru = nullptr;
                for (auto &s : srv->slots)
                    if (!s->busy && (!lru || s->last_use < lru->last_use)) lru = s.get();
                if (!lru) break;
                tursca_scene_destroy(lru->sc);
                cudaStreamDestroy(lru->st);
                srv->used -= lru->bytes;
                srv->evictions++;
                srv->slots.erase(std::find_if(srv->slots.begin(), srv->slots.end(),
                                              [&](const std::unique_ptr<Slot> &p) { return p.get() == lru; }));
            }
            if (srv->used + need <= srv->budget) {
                srv->used += need;  // reserved until the slot's real size is known
                srv->peak = std::max(srv->peak, srv->used);
                *slot_out = nullptr;
                *build_out = true;
                *reserve_out = need;
                srv->pending.erase(it);
                return r;
            }
        }
        if (it == srv->pending.begin() && now - r->info.submit_ms > kAgingMs) head_blocked = true;
    }
    return nullptr;
}

// a request whose slot can never fit the budget fails instead of waiting
Request *pick_impossible(tursca_server *srv) {
    for (auto it = srv->pending.begin(); it != srv->pending.end(); ++it) {
        Request *r = *it;
        if (slot_estimate(srv, r->desc) > srv->budget) {
            bool resident = false;
            for (auto &s : srv->slots) resident = resident || s->key == key_of(r->desc);
            if (!resident) {
                srv->pending.erase(it);
                return r;
            }
        }
    }
    return nullptr;
}

void run_request(tursca_server *srv, Request *r, Slot *slot) {
    tursca_scene *sc = slot->sc;
    tursca_status e = tursca_set_medium(sc, r->mu_abs, r->mu_sca, r->g.data(), r->albedo);
    if (!e) e = tursca_assemble_flux(sc, &r->geom);
    tursca_solve_info si;
    std::memset(&si, 0, sizeof(si));
    if (!e) e = tursca_solve(sc, r->rtol, 5000, &si);
    if (!e) e = tursca_render_radiance(sc, r->radiance, nullptr);
    r->info.iters = si.iters;
    r->info.rel_resid64 = si.rel_resid64;
    r->info.status = e;
}

void worker(tursca_server *srv) {
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    for (;;) {
        Request *r = nullptr;
        Slot *slot = nullptr;
        bool build = false;
        size_t reserve = 0;
        srv->cv_work.wait(lk, [&] {
            if (srv->stop && srv->pending.empty()) return true;
            r = pick_impossible(srv);
            if (r) return true;
            r = pick(srv, &slot, &build, &reserve);
            return r != nullptr;
        });
        if (!r) return;  // stopping
        r->info.start_ms = srv->now_ms();
        if (!slot && !build) {  // cannot ever fit
            r->info.status = TURSCA_E_NOMEM;
            r->info.end_ms = r->info.start_ms;
            r->done = true;
            srv->cv_done.notify_all();
            continue;
        }
        if (build) {
            // a new slot, built outside the lock
            lk.unlock();
            auto s = std::unique_ptr<Slot>(new Slot());
            s->key = key_of(r->desc);
            tursca_status e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) == cudaSuccess
                                  ? TURSCA_OK
                                  : TURSCA_E_CUDA;
            if (!e) e = tursca_scene_create(&r->desc, s->st, &s->sc);
            if (!e) e = tursca_build_graph(s->sc);
            lk.lock();
            if (!e && srv->batch_solves && r->desc.precision == TURSCA_FP32_REFINE) {
                if (!srv->batcher) srv->batcher = tk::batcher_create();
                tk::scene_attach_batcher(s->sc, srv->batcher);  // a null batcher leaves the scene's own passes
            }
            if (e) {
                if (s->sc) tursca_scene_destroy(s->sc);
                if (s->st) cudaStreamDestroy(s->st);
                srv->used -= reserve;
                r->info.status = e;
                r->info.end_ms = srv->now_ms();
                r->done = true;
                srv->cv_done.notify_all();
                srv->cv_work.notify_all();
                continue;
            }
            s->busy = true;
            s->last_use = ++srv->use_clock;
            s->bytes = reserve;  // corrected after the first request (fields are allocated then)
            slot = s.get();
            srv->slots.push_back(std::move(s));
            srv->built++;
        }
        r->info.slot_reused = build ? 0 : 1;
        lk.unlock();
        run_request(srv, r, slot);
        const size_t real = tursca_scene_device_bytes(slot->sc);
        lk.lock();
        // the slot's measured size replaces the estimate
        srv->used = srv->used - slot->bytes + real;
        slot->bytes = real;
        srv->slot_bytes[slot->key] = std::max(srv->slot_bytes[slot->key], real);
        srv->peak = std::max(srv->peak, srv->used);
        slot->busy = false;
        r->info.end_ms = srv->now_ms();
        r->done = true;
        srv->cv_done.notify_all();
        srv->cv_work.notify_all();
    }
}

}  // namespace

extern "C" {

tursca_status tursca_server_create(size_t hbm_budget_bytes, int max_concurrent, tursca_server **out) {
    if (!out) return TURSCA_E_INVALID;
    *out = nullptr;
    if (max_concurrent < 1 || max_concurrent > 64 || hbm_budget_bytes == 0) return TURSCA_E_INVALID;
    tursca_server *srv = new (std::nothrow) tursca_server();
    if (!srv) return TURSCA_E_NOMEM;
    srv->budget = hbm_budget_bytes;
    srv->workers_n = max_concurrent;
    if (cudaGetDevice(&srv->device) != cudaSuccess) {
        delete srv;
        return TURSCA_E_CUDA;
    }
    for (int i = 0; i < max_concurrent; ++i) srv->workers.emplace_back(worker, srv);
    *out = srv;
    return TURSCA_OK;
}

tursca_status tursca_server_submit(tursca_server *srv, const tursca_grid_desc *desc, const tursca_geometry *geom,
                                   const void *mu_abs, const void *mu_sca, const double *g, double albedo,
                                   double rtol, void *radiance, long long *ticket) {
    if (!srv || !desc || !geom || !mu_abs || !mu_sca || !g || !radiance || !ticket) return TURSCA_E_INVALID;
    if (!(rtol > 0.0)) return TURSCA_E_INVALID;
    if (desc->n_species < 1) return TURSCA_E_INVALID;
    // the graph counts of a shape (and the check of its descriptor) are
    // computed once per shape, outside the lock
    const ShapeKey key = key_of(*desc);
    bool known;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        known = srv->shape_stats.count(key) != 0;
    }
    if (!known) {
        tursca_graph_stats st;
        std::memset(&st, 0, sizeof(st));
        if (tursca_graph_info(desc, &st) != TURSCA_OK) return TURSCA_E_INVALID;
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->shape_stats[key] = st;
    }
    auto r = std::unique_ptr<Request>(new Request());
    r->desc = *desc;
    r->geom = *geom;
    r->mu_abs = mu_abs;
    r->mu_sca = mu_sca;
    r->g.assign(g, g + desc->n_species);
    r->albedo = albedo;
    r->rtol = rtol;
    r->radiance = radiance;
    std::memset(&r->info, 0, sizeof(r->info));
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stop) return TURSCA_E_STATE;
    r->ticket = srv->next_ticket++;
    r->info.submit_ms = srv->now_ms();
    *ticket = r->ticket;
    srv->pending.push_back(r.get());
    srv->reqs[r->ticket] = std::move(r);
    srv->cv_work.notify_one();
    return TURSCA_OK;
}

tursca_status tursca_server_wait(tursca_server *srv, long long ticket, tursca_request_info *info) {
    if (!srv) return TURSCA_E_INVALID;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return TURSCA_E_INVALID;
    Request *r = it->second.get();
    srv->cv_done.wait(lk, [&] { return r->done; });
    if (info) *info = r->info;
    const tursca_status e = r->info.status;
    srv->reqs.erase(it);
    return e;
}

tursca_status tursca_server_stats_get(tursca_server *srv, tursca_server_stats *out) {
    if (!srv || !out) return TURSCA_E_INVALID;
    std::lock_guard<std::mutex> lk(srv->mu);
    out->budget_bytes = srv->budget;
    out->used_bytes = srv->used;
    out->peak_bytes = srv->peak;
    out->slots = (int)srv->slots.size();
    out->busy_slots = 0;
    for (auto &s : srv->slots) out->busy_slots += s->busy ? 1 : 0;
    out->pending = (int)srv->pending.size();
    out->evictions = srv->evictions;
    out->slots_built = srv->built;
    out->batches = out->batched_refinements = 0;
    out->max_batch = 0;
    if (srv->batcher) tk::batcher_stats(srv->batcher, &out->batches, &out->batched_refinements, &out->max_batch);
    return TURSCA_OK;
}

tursca_status tursca_server_configure(tursca_server *srv, int option, double value) {
    if (!srv) return TURSCA_E_INVALID;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (option != TURSCA_SERVER_BATCH_SOLVES || (value != 0.0 && value != 1.0)) return TURSCA_E_INVALID;
    if (srv->built > 0 || srv->next_ticket > 1) return TURSCA_E_STATE;  // before the first request
    srv->batch_solves = value != 0.0;
    return TURSCA_OK;
}

tursca_status tursca_server_destroy(tursca_server *srv) {
    if (!srv) return TURSCA_E_INVALID;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        srv->cv_work.notify_all();
    }
    for (auto &t : srv->workers) t.join();
    tk::batcher_destroy(srv->batcher);  // idle: every request has finished
    for (auto &s : srv->slots) {
        tursca_scene_destroy(s->sc);
        cudaStreamDestroy(s->st);
    }
    delete srv;
    return TURSCA_OK;
}

}  // extern "C"
