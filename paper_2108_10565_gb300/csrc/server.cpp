// Continuous-batching server for ensembles of independent poroelastic
// simulations (poro_server_*, poro_submit, ...).
//
// A scheduler thread admits queued requests in arrival order while a slot
// is free and the sum of the admitted requests' device-memory footprints
// stays within the budget.  Each admitted request is set up (context, mesh,
// flux solvers, clusters, sources, receivers) on a worker thread of its own.
//
// Batched mode (the default): set-up requests join one executor thread.  It
// groups the running requests by degree, precision, refinement, CTA variant
// and cluster count, and advances every group a chunk of cycles at a time
// with poro::group_enqueue: each tick's predictors of all of a group's runs
// are a single launch, followed by each run's LTS buffers, correctors,
// sources and receivers, the cycle captured once as a CUDA graph.  Groups of
// different degrees run concurrently on their own streams.  Requests that
// arrive while others run join their group at the next chunk.
//
// Stream mode (poro_server_set_batching(s, 0)): each request runs on its
// worker thread with its own context and CUDA stream, advancing one chunk of
// cycles at a time, so requests overlap on the device through streams.
//
// In both modes a cancel takes effect between chunks, and a request that
// fails (invalid input, footprint above the whole budget, a CUDA error of its
// own calls) ends in PORO_REQ_FAILED alone; in batched mode a failure of a
// group's shared predictor launch fails that group's requests.
// The paper has no counterpart: it runs one simulation per MPI job.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "poro_internal.h"

namespace {
using clk = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    int32_t state = PORO_REQ_QUEUED;
    std::string err;
    // copied scenario
    int32_t N = 0, prec = 0, C = 1, refine = 1;
    double cfl = 0.5, t_end = 0.0;
    std::vector<double> xyz;
    std::vector<int64_t> tet, nb;
    std::vector<int32_t> tag;
    std::vector<poro_material> mat;
    std::vector<double> src_xyz, src_w, src_f0, src_t0, src_amp;
    std::vector<double> rec_xyz;
    std::vector<double> q0;
    size_t footprint = 0;
    bool cancel = false;
    double sim_t = 0.0;
    clk::time_point t_submit, t_start, t_done;
    std::vector<std::vector<double>> seis_t, seis_q;
    // batched mode: the set-up context and the cycles to run
    poro_ctx* ctx = nullptr;
    int64_t total = 0, done = 0;
    double dt_cycle = 0.0;
};
}  // namespace

struct poro_server {
    int device = 0;
    size_t budget = 0, used = 0;
    int max_slots = 1;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    bool stop = false;
    uint64_t next = 1;
    std::map<uint64_t, std::unique_ptr<Request>> reqs;
    std::deque<uint64_t> queue;
    int running = 0;
    std::thread scheduler;
    std::vector<std::thread> workers;
    std::string err;
    // batched mode
    bool batched = true;
    std::deque<uint64_t> ready;      // set up, waiting to join the executor
    bool exec_stop = false;
    std::condition_variable exec_cv;
    std::thread executor;
};

namespace {
thread_local std::string g_srv_err;

poro_status sfail(poro_server* s, poro_status st, const std::string& m) {
    if (s) {
        std::lock_guard<std::mutex> l(s->mu);
        s->err = m;
    } else {
        g_srv_err = m;
    }
    return st;
}

// device bytes one request needs (element data, faces, predictors, buffers,
// reference and face matrices, receivers), with 25 % headroom
size_t footprint_bytes(int N, int64_t ne, int C, int nrec) {
    const size_t B = (size_t)poro::n_modes(N), T = (size_t)N + 1, QB = poro::NQ * B;
    size_t per = (size_t)poro::elem_const_stride(N) * 8 + 2 * QB * 8 + QB * T * 8 + 4 * (4 + 4 + 8) +
                 4 * 2 * poro::NQ * poro::NQ * 8;
    if (C > 1) per += (size_t)(C - 1) * QB * 8 / 2 + 8 * C;
    size_t fixed = 96 * B * B * 8 + 4 * B * B * 8 + (size_t)3 * B * B * 8 * 2 + (size_t)nrec * 1024 * poro::NQ * 8;
    return (size_t)((double)(per * (size_t)ne + fixed) * 1.25) + (64u << 20);
}

// Context, mesh, materials, clusters, sources and receivers of a request;
// on success r.ctx, r.total (cycles) and r.dt_cycle are set.
poro_status setup_request(poro_server* s, Request& r) {
    poro_ctx* ctx = nullptr;
    poro_status st = poro_create(s->device, r.N, (poro_precision)r.prec, &ctx);
    if (st != PORO_OK) {
        r.err = poro_last_error(nullptr);
        return st;
    }
    auto bail = [&](poro_status e) {
        r.err = poro_last_error(ctx);
        poro_destroy(ctx);
        return e;
    };
    const int64_t ne = (int64_t)r.tet.size() / 4;
    if (r.prec != PORO_FP64 && (st = poro_set_refinement(ctx, r.refine)) != PORO_OK) return bail(st);
    if ((st = poro_set_mesh(ctx, (int64_t)r.xyz.size() / 3, r.xyz.data(), ne, r.tet.data(), r.nb.data(),
                            r.tag.data())) != PORO_OK)
        return bail(st);
    if ((st = poro_set_materials(ctx, r.mat.data())) != PORO_OK) return bail(st);
    double dtmin = 0.0;
    if ((st = poro_set_clusters(ctx, r.cfl, r.C, &dtmin, nullptr)) != PORO_OK) return bail(st);
    if (!r.q0.empty() && (st = poro_set_dofs(ctx, r.q0.data())) != PORO_OK) return bail(st);
    for (size_t i = 0; i < r.src_f0.size(); ++i)
        if ((st = poro_add_point_source(ctx, &r.src_xyz[3 * i], &r.src_w[13 * i], r.src_f0[i], r.src_t0[i],
                                        r.src_amp[i])) != PORO_OK)
            return bail(st);
    const int nrec = (int)(r.rec_xyz.size() / 3);
    for (int i = 0; i < nrec; ++i)
        if ((st = poro_add_receiver(ctx, &r.rec_xyz[3 * i], nullptr)) != PORO_OK) return bail(st);
    r.ctx = ctx;
    r.dt_cycle = std::ldexp(dtmin, r.C - 1);
    r.total = (int64_t)std::floor(r.t_end / r.dt_cycle + 1e-9);
    r.done = 0;
    return PORO_OK;
}

// Receiver samples into the request, context released.
void collect_request(Request& r) {
    poro_ctx* ctx = r.ctx;
    const int nrec = (int)(r.rec_xyz.size() / 3);
    r.seis_t.assign(nrec, {});
    r.seis_q.assign(nrec, {});
    for (int i = 0; i < nrec; ++i) {
        int64_t n = 0;
        poro_get_seismogram(ctx, i, 0, nullptr, nullptr, &n);
        r.seis_t[i].resize(n);
        r.seis_q[i].resize((size_t)n * poro::NQ);
        poro_get_seismogram(ctx, i, n, r.seis_t[i].data(), r.seis_q[i].data(), &n);
    }
    poro_destroy(ctx);
    r.ctx = nullptr;
}

// Stream mode: the request's own context and stream, one chunk of cycles at a
// time.
poro_status run_request(poro_server* s, Request& r) {
    poro_status st = setup_request(s, r);
    if (st != PORO_OK) return st;
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(64, r.total / 8 + 1));
    while (r.done < r.total) {
        {
            std::lock_guard<std::mutex> l(s->mu);
            if (r.cancel) {
                poro_destroy(r.ctx);
                r.ctx = nullptr;
                return PORO_ETIMEOUT;  // marker: cancelled
            }
        }
        const int64_t n = std::min(chunk, r.total - r.done);
        if ((st = poro_advance(r.ctx, (double)(r.done + n) * r.dt_cycle * (1.0 + 1e-12))) != PORO_OK) {
            r.err = poro_last_error(r.ctx);
            poro_destroy(r.ctx);
            r.ctx = nullptr;
            return st;
        }
        r.done += n;
        double t = 0.0;
        poro_get_time(r.ctx, &t, nullptr);
        std::lock_guard<std::mutex> l(s->mu);
        r.sim_t = t;
    }
    collect_request(r);
    return PORO_OK;
}

// End state of a request; releases its slot and budget.
void finalize(poro_server* s, Request* r, poro_status st) {
    std::lock_guard<std::mutex> l(s->mu);
    r->t_done = clk::now();
    if (st == PORO_OK) r->state = PORO_REQ_DONE;
    else if (st == PORO_ETIMEOUT && r->cancel) r->state = PORO_REQ_CANCELLED;
    else r->state = PORO_REQ_FAILED;
    s->used -= r->footprint;
    s->running -= 1;
    s->cv.notify_all();
    s->done_cv.notify_all();
}

void worker_main(poro_server* s, uint64_t ticket) {
    Request* r;
    {
        std::lock_guard<std::mutex> l(s->mu);
        r = s->reqs[ticket].get();
    }
    finalize(s, r, run_request(s, *r));
}

// Batched mode, set-up half: build the context, then hand the request to the
// executor.
void setup_main(poro_server* s, uint64_t ticket) {
    Request* r;
    {
        std::lock_guard<std::mutex> l(s->mu);
        r = s->reqs[ticket].get();
    }
    poro_status st = setup_request(s, *r);
    if (st != PORO_OK) {
        finalize(s, r, st);
        return;
    }
    std::lock_guard<std::mutex> l(s->mu);
    s->ready.push_back(ticket);
    s->exec_cv.notify_all();
}

// requests that can share predictor launches (the server's contexts all keep
// the default CTA variant)
struct GroupKey {
    int N, prec, refine, C;
    bool operator<(const GroupKey& o) const {
        return std::tie(N, prec, refine, C) < std::tie(o.N, o.prec, o.refine, o.C);
    }
};

// cycles of one chunk: about 32 ticks, at least one cycle
int64_t chunk_cycles(int C) { return std::max<int64_t>(1, 32 >> (C - 1)); }

void executor_main(poro_server* s) {
    std::vector<Request*> active;
    std::map<std::vector<uint64_t>, poro::RunGroup*> groups;  // by the sorted tickets of their runs
    for (;;) {
        {
            std::unique_lock<std::mutex> l(s->mu);
            s->exec_cv.wait(l, [&] { return s->exec_stop || !s->ready.empty() || !active.empty(); });
            if (s->exec_stop && s->ready.empty() && active.empty()) break;
            while (!s->ready.empty()) {
                active.push_back(s->reqs[s->ready.front()].get());
                s->ready.pop_front();
            }
        }
        // cancellations (between chunks)
        std::vector<Request*> keep;
        for (Request* r : active) {
            bool cancel;
            {
                std::lock_guard<std::mutex> l(s->mu);
                cancel = r->cancel;
            }
            if (!cancel) {
                keep.push_back(r);
                continue;
            }
            for (auto& kv : groups) poro::group_destroy(kv.second);
            groups.clear();
            poro_destroy(r->ctx);
            r->ctx = nullptr;
            finalize(s, r, PORO_ETIMEOUT);
        }
        active.swap(keep);
        if (active.empty()) continue;
        // groups of the running requests; a changed composition is rebuilt
        std::map<GroupKey, std::vector<Request*>> by;
        for (Request* r : active) by[GroupKey{r->N, r->prec, r->prec == PORO_FP64 ? 0 : r->refine, r->C}].push_back(r);
        std::map<std::vector<uint64_t>, poro::RunGroup*> next;
        std::vector<std::pair<poro::RunGroup*, std::vector<Request*>>> work;
        std::vector<Request*> failed;
        for (auto& kv : by) {
            std::vector<Request*>& rs = kv.second;
            std::sort(rs.begin(), rs.end(), [](const Request* a, const Request* b) { return a->ticket < b->ticket; });
            std::vector<uint64_t> key;
            std::vector<poro_ctx*> ctxs;
            for (Request* r : rs) {
                key.push_back(r->ticket);
                ctxs.push_back(r->ctx);
            }
            poro::RunGroup* g = nullptr;
            auto it = groups.find(key);
            if (it != groups.end()) {
                g = it->second;
                groups.erase(it);
            } else {
                std::string err;
                g = poro::group_create(ctxs.data(), (int)ctxs.size(), err);
                if (!g) {
                    for (Request* r : rs) {
                        r->err = err;
                        failed.push_back(r);
                    }
                    continue;
                }
            }
            next[key] = g;
            work.emplace_back(g, rs);
        }
        for (auto& kv : groups) poro::group_destroy(kv.second);
        groups.swap(next);
        // one chunk per group: all groups are enqueued before any is awaited
        std::vector<int64_t> chunk(work.size(), 0);
        std::vector<std::string> errs(work.size());
        std::vector<bool> ok(work.size(), true);
        for (size_t i = 0; i < work.size(); ++i) {
            int64_t n = chunk_cycles(work[i].second[0]->C);
            for (Request* r : work[i].second) n = std::min(n, r->total - r->done);
            chunk[i] = n;
            if (n > 0 && poro::group_enqueue(work[i].first, n, errs[i]) != 0) ok[i] = false;
        }
        for (size_t i = 0; i < work.size(); ++i) {
            if (ok[i] && chunk[i] > 0 && poro::group_finish(work[i].first, errs[i]) != PORO_OK) ok[i] = false;
            if (!ok[i]) {
                for (Request* r : work[i].second) {
                    r->err = errs[i];
                    failed.push_back(r);
                }
                continue;
            }
            for (Request* r : work[i].second) {
                r->done += chunk[i];
                double t = 0.0;
                poro_get_time(r->ctx, &t, nullptr);
                std::lock_guard<std::mutex> l(s->mu);
                r->sim_t = t;
            }
        }
        // finished and failed requests leave (their groups first)
        std::vector<Request*> still;
        std::vector<Request*> finished;
        for (Request* r : active) {
            if (std::find(failed.begin(), failed.end(), r) != failed.end()) continue;
            (r->done >= r->total ? finished : still).push_back(r);
        }
        // groups that hold a leaving run go (the others keep their tables
        // and captured cycle)
        if (!finished.empty() || !failed.empty()) {
            std::vector<uint64_t> gone;
            for (Request* r : finished) gone.push_back(r->ticket);
            for (Request* r : failed) gone.push_back(r->ticket);
            for (auto it = groups.begin(); it != groups.end();) {
                bool hit = false;
                for (uint64_t t : it->first) hit = hit || std::find(gone.begin(), gone.end(), t) != gone.end();
                if (hit) {
                    poro::group_destroy(it->second);
                    it = groups.erase(it);
                } else {
                    ++it;
                }
            }
        }
        for (Request* r : finished) {
            collect_request(*r);
            finalize(s, r, PORO_OK);
        }
        for (Request* r : failed) {
            poro_destroy(r->ctx);
            r->ctx = nullptr;
            finalize(s, r, PORO_ECUDA);
        }
        active.swap(still);
    }
    for (auto& kv : groups) poro::group_destroy(kv.second);
}

void scheduler_main(poro_server* s) {
    std::unique_lock<std::mutex> l(s->mu);
    while (!s->stop) {
        bool admitted = false;
        while (!s->queue.empty() && s->running < s->max_slots) {
            Request* r = s->reqs[s->queue.front()].get();
            if (r->cancel) {
                r->state = PORO_REQ_CANCELLED;
                r->t_done = clk::now();
                s->queue.pop_front();
                s->done_cv.notify_all();
                continue;
            }
            if (r->footprint > s->budget) {
                r->state = PORO_REQ_FAILED;
                r->err = "request needs more device memory than the server budget";
                r->t_done = clk::now();
                s->queue.pop_front();
                s->done_cv.notify_all();
                continue;
            }
            if (s->used + r->footprint > s->budget) break;  // wait for memory (arrival order)
            s->queue.pop_front();
            s->used += r->footprint;
            s->running += 1;
            r->state = PORO_REQ_RUNNING;
            r->t_start = clk::now();
            if (s->batched)
                s->workers.emplace_back(setup_main, s, r->ticket);
            else
                s->workers.emplace_back(worker_main, s, r->ticket);
            admitted = true;
        }
        if (!admitted) s->cv.wait(l);
    }
}
}  // namespace

extern "C" {

poro_status poro_server_create(int device, size_t hbm_budget, int32_t max_slots, poro_server** out) {
    if (!out || max_slots < 1 || hbm_budget == 0) return sfail(nullptr, PORO_EINVAL, "poro_server_create: bad argument");
    poro_server* s = new poro_server();
    s->device = device;
    s->budget = hbm_budget;
    s->max_slots = max_slots;
    s->scheduler = std::thread(scheduler_main, s);
    s->executor = std::thread(executor_main, s);
    *out = s;
    return PORO_OK;
}

poro_status poro_server_set_batching(poro_server* s, int32_t on) {
    if (!s) return sfail(nullptr, PORO_EINVAL, "poro_server_set_batching: NULL server");
    std::lock_guard<std::mutex> l(s->mu);
    s->batched = on != 0;
    return PORO_OK;
}

poro_status poro_server_destroy(poro_server* s) {
    if (!s) return PORO_OK;
    {
        std::lock_guard<std::mutex> l(s->mu);
        for (auto& kv : s->reqs)
            if (kv.second->state == PORO_REQ_QUEUED || kv.second->state == PORO_REQ_RUNNING) kv.second->cancel = true;
        s->stop = true;
        s->cv.notify_all();
    }
    s->scheduler.join();
    for (auto& w : s->workers)
        if (w.joinable()) w.join();
    {
        std::lock_guard<std::mutex> l(s->mu);
        for (uint64_t t : s->ready) s->reqs[t]->cancel = true;
        s->exec_stop = true;
        s->exec_cv.notify_all();
    }
    s->executor.join();
    delete s;
    return PORO_OK;
}

const char* poro_server_last_error(poro_server* s) {
    if (!s) return g_srv_err.c_str();
    std::lock_guard<std::mutex> l(s->mu);
    return s->err.c_str();
}

poro_status poro_submit(poro_server* s, const poro_scenario* sc, uint64_t* ticket) {
    if (!s || !sc || !ticket) return sfail(s, PORO_EINVAL, "poro_submit: NULL argument");
    if (sc->n_elem <= 0 || sc->n_vert <= 0 || !sc->xyz || !sc->tet || !sc->nb || !sc->face_tag || !sc->mat ||
        sc->degree_N < 1 || sc->degree_N > poro::MAX_N || sc->max_clusters < 1 || !(sc->t_end > 0.0) ||
        (sc->n_sources > 0 && (!sc->src_xyz || !sc->src_w || !sc->src_f0 || !sc->src_t0 || !sc->src_amp)) ||
        (sc->n_receivers > 0 && !sc->rec_xyz))
        return sfail(s, PORO_EINVAL, "poro_submit: invalid scenario");
    auto r = std::make_unique<Request>();
    r->N = sc->degree_N;
    r->prec = sc->precision;
    r->C = sc->max_clusters;
    r->refine = sc->refine_sweeps;
    r->cfl = sc->cfl_c > 0.0 ? sc->cfl_c : 0.5;
    r->t_end = sc->t_end;
    r->xyz.assign(sc->xyz, sc->xyz + 3 * sc->n_vert);
    r->tet.assign(sc->tet, sc->tet + 4 * sc->n_elem);
    r->nb.assign(sc->nb, sc->nb + 4 * sc->n_elem);
    r->tag.assign(sc->face_tag, sc->face_tag + 4 * sc->n_elem);
    r->mat.assign(sc->mat, sc->mat + sc->n_elem);
    if (sc->n_sources > 0) {
        r->src_xyz.assign(sc->src_xyz, sc->src_xyz + 3 * sc->n_sources);
        r->src_w.assign(sc->src_w, sc->src_w + 13 * sc->n_sources);
        r->src_f0.assign(sc->src_f0, sc->src_f0 + sc->n_sources);
        r->src_t0.assign(sc->src_t0, sc->src_t0 + sc->n_sources);
        r->src_amp.assign(sc->src_amp, sc->src_amp + sc->n_sources);
    }
    if (sc->n_receivers > 0) r->rec_xyz.assign(sc->rec_xyz, sc->rec_xyz + 3 * sc->n_receivers);
    if (sc->Q0) r->q0.assign(sc->Q0, sc->Q0 + (size_t)sc->n_elem * poro::NQ * poro::n_modes(sc->degree_N));
    r->footprint = footprint_bytes(r->N, sc->n_elem, r->C, sc->n_receivers);
    r->t_submit = clk::now();
    std::lock_guard<std::mutex> l(s->mu);
    r->ticket = s->next++;
    *ticket = r->ticket;
    s->queue.push_back(r->ticket);
    s->reqs[r->ticket] = std::move(r);
    s->cv.notify_all();
    return PORO_OK;
}

poro_status poro_poll(poro_server* s, uint64_t ticket, int32_t* state, double* sim_time) {
    if (!s) return sfail(nullptr, PORO_EINVAL, "poro_poll: NULL server");
    std::lock_guard<std::mutex> l(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return PORO_EINVAL;
    if (state) *state = it->second->state;
    if (sim_time) *sim_time = it->second->sim_t;
    return PORO_OK;
}

poro_status poro_wait(poro_server* s, uint64_t ticket, int32_t timeout_ms, int32_t* state) {
    if (!s) return sfail(nullptr, PORO_EINVAL, "poro_wait: NULL server");
    std::unique_lock<std::mutex> l(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return PORO_EINVAL;
    Request* r = it->second.get();
    auto finished = [&] { return r->state >= PORO_REQ_DONE; };
    if (timeout_ms < 0) s->done_cv.wait(l, finished);
    else if (!s->done_cv.wait_for(l, std::chrono::milliseconds(timeout_ms), finished)) {
        if (state) *state = r->state;
        return PORO_ETIMEOUT;
    }
    if (state) *state = r->state;
    return PORO_OK;
}

poro_status poro_fetch(poro_server* s, uint64_t ticket, int32_t rec, int64_t cap, double* t_out, double* q_out,
                       int64_t* n_out) {
    if (!s) return sfail(nullptr, PORO_EINVAL, "poro_fetch: NULL server");
    std::lock_guard<std::mutex> l(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return PORO_EINVAL;
    Request* r = it->second.get();
    if (r->state != PORO_REQ_DONE) return PORO_ESTATE;
    if (rec < 0 || rec >= (int32_t)r->seis_t.size()) return PORO_EINVAL;
    const int64_t n = (int64_t)r->seis_t[rec].size();
    if (n_out) *n_out = n;
    const int64_t m = std::min(n, cap);
    if (m > 0 && (!t_out || !q_out)) return PORO_EINVAL;
    if (m > 0) {
        std::memcpy(t_out, r->seis_t[rec].data(), m * sizeof(double));
        std::memcpy(q_out, r->seis_q[rec].data(), (size_t)m * poro::NQ * sizeof(double));
    }
    return PORO_OK;
}

poro_status poro_request_times(poro_server* s, uint64_t ticket, double* queued_s, double* run_s, double* total_s) {
    if (!s) return sfail(nullptr, PORO_EINVAL, "poro_request_times: NULL server");
    std::lock_guard<std::mutex> l(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return PORO_EINVAL;
    Request* r = it->second.get();
    if (r->state < PORO_REQ_DONE) return PORO_ESTATE;
    using d = std::chrono::duration<double>;
    const bool ran = r->t_start.time_since_epoch().count() != 0;
    if (queued_s) *queued_s = d((ran ? r->t_start : r->t_done) - r->t_submit).count();
    if (run_s) *run_s = ran ? d(r->t_done - r->t_start).count() : 0.0;
    if (total_s) *total_s = d(r->t_done - r->t_submit).count();
    return PORO_OK;
}

poro_status poro_request_error(poro_server* s, uint64_t ticket, char* buf, size_t cap) {
    if (!s || !buf || cap == 0) return sfail(s, PORO_EINVAL, "poro_request_error: bad argument");
    std::lock_guard<std::mutex> l(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return PORO_EINVAL;
    std::strncpy(buf, it->second->err.c_str(), cap - 1);
    buf[cap - 1] = 0;
    return PORO_OK;
}

poro_status poro_cancel(poro_server* s, uint64_t ticket) {
    if (!s) return sfail(nullptr, PORO_EINVAL, "poro_cancel: NULL server");
    std::lock_guard<std::mutex> l(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return PORO_EINVAL;
    it->second->cancel = true;
    s->cv.notify_all();
    return PORO_OK;
}

poro_status poro_footprint_bytes(int degree_N, int64_t n_elem, int32_t max_clusters, int32_t n_receivers,
                                 size_t* bytes) {
    if (!bytes || degree_N < 1 || degree_N > poro::MAX_N || n_elem < 0 || max_clusters < 1)
        return sfail(nullptr, PORO_EINVAL, "poro_footprint_bytes: bad argument");
    *bytes = footprint_bytes(degree_N, n_elem, max_clusters, n_receivers);
    return PORO_OK;
}

}  // extern "C"
