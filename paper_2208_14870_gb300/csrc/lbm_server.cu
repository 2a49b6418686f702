// lbm_server.cu -- continuous-batching solve server.
//
// A worker thread owns two packed arenas (FP32 and FP16-shifted storage),
// each with half of the HBM budget.  Requests are copied at submission and
// queued; between chunks the worker admits queued requests whose lattice fits
// the free arena memory (first-fit, oldest first, with a bound on how long a
// request can be bypassed by later ones), runs one chunk of check_every steps
// of every resident problem (one persistent cooperative launch per arena,
// replayed from a CUDA graph), and retires problems whose residual dropped
// below their tolerance: their displacement and stress are recovered into
// host memory owned by the request, their arena memory is freed for the next
// admissions, and their latency (submission to completion) is recorded.
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
#include <vector>

#include "../../include/lbm.h"
#include "lbm_engine.cuh"

using namespace lbm;

namespace {

using clk = std::chrono::steady_clock;

enum ReqState { R_QUEUED = 0, R_RUNNING = 1, R_DONE = 2 };

struct Request {
    uint64_t ticket = 0;
    int nx = 0, ny = 0, dtype = LBM_F32;
    double lambda = 0.0, mu = 0.0, tol = 0.0;
    int64_t max_iters = 0;
    std::vector<double> gx, gy;
    std::vector<double> fields;   // 5 * nx * ny once done
    int state = R_QUEUED;
    int status = LBM_OK;
    int64_t iters = 0;
    double residual = 0.0;
    int transposed = 0;
    clk::time_point t_submit, t_admit, t_done;
    int arena = 0, slot = -1;
    int64_t bypassed = 0;         // chunks during which later requests were admitted first
    bool cancelled = false;       // running request cancelled: the worker drops it
};

double ms_between(clk::time_point a, clk::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (double)(v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - (double)i;
    return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
}

}  // namespace

struct lbm_server {
    int device = 0;
    size_t budget = 0;
    int check_every = 100;
    int tile_v = 4;
    int64_t max_bypass_chunks = 50;
    cudaStream_t stream = nullptr;
    std::unique_ptr<ArenaEngine> arena[2];  // [0] FP32, [1] FP16-shifted
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    int failed = LBM_OK;
    std::string fail_msg;
    uint64_t next_ticket = 1;
    std::map<uint64_t, std::unique_ptr<Request>> reqs;
    std::deque<uint64_t> queue;                 // admission order
    std::map<int, uint64_t> slot_owner[2];      // arena slot -> ticket
    // statistics
    int64_t submitted = 0, completed = 0, chunks = 0, lups = 0;
    double device_ms = 0.0;
    int peak_running = 0;
    int64_t memory_waits = 0;
    int64_t peak_resident = 0;
    std::vector<double> latencies_ms;
    bool any_submit = false;
    clk::time_point t_first_submit, t_last_done;

    void run();
    int admit_locked();
    void retire(int a, const std::vector<int>& slots, std::unique_lock<std::mutex>& lk);
};

void lbm_server::run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
        int rc = admit_locked();
        if (rc != LBM_OK) {
            failed = rc;
            break;
        }
        const int r0 = arena[0]->running(), r1 = arena[1]->running();
        peak_running = std::max(peak_running, r0 + r1);
        peak_resident = std::max(peak_resident, arena[0]->resident_bytes() + arena[1]->resident_bytes());
        if (r0 + r1 == 0) {
            cv_work.wait_for(lk, std::chrono::milliseconds(50));
            continue;
        }
        lk.unlock();
        std::string err;
        float ms[2] = {0.0f, 0.0f};
        for (int a = 0; a < 2 && rc == LBM_OK; ++a)
            if (arena[a]->running() > 0) rc = arena[a]->run_chunk(tile_v, &ms[a], &err);
        lk.lock();
        if (rc != LBM_OK) {
            failed = rc;
            fail_msg = err;
            break;
        }
        ++chunks;
        device_ms += ms[0] + ms[1];
        for (auto& q : queue) {
            auto it = reqs.find(q);
            if (it != reqs.end()) ++it->second->bypassed;
        }
        for (int a = 0; a < 2; ++a) {
            std::vector<int> done, dropped;
            for (auto& kv : slot_owner[a]) {
                if (reqs[kv.second]->cancelled) dropped.push_back(kv.first);
                else if (arena[a]->prob(kv.first).state == P_DONE) done.push_back(kv.first);
            }
            for (int s : dropped) {
                arena[a]->release(s);
                reqs.erase(slot_owner[a][s]);
                slot_owner[a].erase(s);
            }
            if (!done.empty()) retire(a, done, lk);
        }
    }
    if (failed != LBM_OK) {
        // fail every outstanding request so that pollers see the error
        for (auto& kv : reqs)
            if (kv.second->state != R_DONE) {
                kv.second->state = R_DONE;
                kv.second->status = failed;
            }
        cv_done.notify_all();
    }
}

// Admit queued requests that fit, oldest first.  A request that has been
// bypassed for more than max_bypass_chunks chunks blocks later admissions to
// its arena until it fits (no starvation of large lattices).
int lbm_server::admit_locked() {
    bool blocked[2] = {false, false};
    for (auto it = queue.begin(); it != queue.end();) {
        Request& r = *reqs[*it];
        const int a = r.dtype == LBM_F16S ? 1 : 0;
        if (blocked[a]) {
            ++it;
            continue;
        }
        std::string err;
        const int s = arena[a]->admit(r.nx, r.ny, r.lambda, r.mu, r.gx.data(), r.gy.data(), r.tol,
                                      r.max_iters, &err);
        if (s >= 0) {
            r.state = R_RUNNING;
            r.arena = a;
            r.slot = s;
            r.t_admit = clk::now();
            slot_owner[a][s] = r.ticket;
            std::vector<double>().swap(r.gx);  // the arena holds the force now
            std::vector<double>().swap(r.gy);
            it = queue.erase(it);
            continue;
        }
        if (s < -1) return s;  // a real error
        ++memory_waits;
        if (r.bypassed > max_bypass_chunks) blocked[a] = true;
        ++it;
    }
    return LBM_OK;
}

// Finished problems of one arena: their fields are recovered together (one
// packed copy per block of problems), then each request is completed.
void lbm_server::retire(int a, const std::vector<int>& slots, std::unique_lock<std::mutex>& lk) {
    std::vector<double*> outs;
    outs.reserve(5 * slots.size());
    for (int slot : slots) {
        Request& r = *reqs[slot_owner[a][slot]];
        const int64_t n = (int64_t)r.nx * r.ny;
        r.fields.assign((size_t)5 * n, 0.0);
        double* f = r.fields.data();
        for (int k = 0; k < 5; ++k) outs.push_back(f + k * n);
    }
    std::string err;
    lk.unlock();
    const int rc = arena[a]->recover_many((int)slots.size(), slots.data(), outs.data(), &err);
    lk.lock();
    if (rc != LBM_OK) {
        failed = rc;
        fail_msg = err;
    }
    for (int slot : slots) {
        const uint64_t t = slot_owner[a][slot];
        Request& r = *reqs[t];
        const HostProb& p = arena[a]->prob(slot);
        r.status = rc != LBM_OK ? rc : p.status;
        r.iters = p.steps;
        r.residual = p.residual;
        r.transposed = p.tr ? 1 : 0;
        lups += p.lups;
        arena[a]->release(slot);
        slot_owner[a].erase(slot);
        if (r.cancelled) {
            reqs.erase(t);
            continue;
        }
        r.state = R_DONE;
        r.t_done = clk::now();
        t_last_done = r.t_done;
        latencies_ms.push_back(ms_between(r.t_submit, r.t_done));
        ++completed;
    }
    cv_done.notify_all();
}

extern "C" {

int lbm_server_create(size_t hbm_budget_bytes, int check_every, lbm_server** out) {
    if (!out) return set_last_error(LBM_ERR_ARG, "lbm_server_create: null output");
    *out = nullptr;
    if (hbm_budget_bytes < ((size_t)1 << 20) || check_every < 2)
        return set_last_error(LBM_ERR_ARG, "lbm_server_create: need a budget >= 1 MiB and check_every >= 2");
    auto s = std::make_unique<lbm_server>();
    if (cudaGetDevice(&s->device) != cudaSuccess)
        return set_last_error(LBM_ERR_CUDA, "lbm_server_create: no CUDA device");
    s->budget = hbm_budget_bytes;
    s->check_every = check_every;
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess)
        return set_last_error(LBM_ERR_CUDA, "lbm_server_create: stream creation failed");
    // Each arena gets half of the budget; capacity in nodes from its bytes per
    // node (2 x populations + carriers + force and snapshot).
    const int64_t half = (int64_t)(hbm_budget_bytes / 2);
    const int64_t per_node[2] = {2 * 32 + 24, 2 * (16 + 8) + 24};
    const int max_probs = 4096;
    for (int a = 0; a < 2; ++a) {
        s->arena[a] = std::make_unique<ArenaEngine>();
        std::string err;
        const int64_t nodes = std::max<int64_t>(half / per_node[a] - (int64_t)max_probs * 8, 1024);
        int rc = s->arena[a]->init(a == 0 ? S_F32 : S_F16S, nodes, max_probs, check_every,
                                   s->stream, &err);
        if (rc) {
            s->arena[0].reset();
            s->arena[1].reset();
            cudaStreamDestroy(s->stream);
            return set_last_error(rc, "lbm_server_create: " + err);
        }
    }
    // the wavefront chunk by default (chunk length a multiple of 4), else
    // two-step tiles (even) or 128-column tiles, unless the autotuner cache
    // holds a choice for this chunk length
    const bool even = check_every % 2 == 0, four = check_every % 4 == 0;
    int v = autotune_lookup("server|k" + std::to_string(check_every));
    s->tile_v = (v == 1 || v == 2 || v == 4 || (v == kTileTwoStep && even) || (v == kTileWave && four))
                    ? v
                    : (four ? kTileWave : (even ? kTileTwoStep : 4));
    lbm_server* raw = s.release();
    raw->worker = std::thread([raw] { raw->run(); });
    *out = raw;
    return LBM_OK;
}

void lbm_server_destroy(lbm_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    s->arena[0].reset();
    s->arena[1].reset();
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

int lbm_server_submit(lbm_server* s, const lbm_problem* p, int dtype, double tol, int64_t max_iters,
                      uint64_t* ticket) {
    if (!s || !p || !ticket) return set_last_error(LBM_ERR_ARG, "lbm_server_submit: null pointer");
    if (dtype != LBM_F32 && dtype != LBM_F16S)
        return set_last_error(LBM_ERR_ARG, "lbm_server_submit: dtype must be LBM_F32 or LBM_F16S");
    if (p->nx < 1 || p->ny < 1 || !p->gx || !p->gy || !(p->mu > 0.0) || !(p->lambda + p->mu > 0.0) ||
        !std::isfinite(p->lambda) || !std::isfinite(p->mu) || !(tol >= 0.0) || max_iters < 1)
        return set_last_error(LBM_ERR_ARG, "lbm_server_submit: malformed request");
    const int a = dtype == LBM_F16S ? 1 : 0;
    const int64_t n = (int64_t)p->nx * p->ny;
    if (s->arena[a]->bytes_for(n) > (int64_t)(s->budget / 2))
        return set_last_error(LBM_ERR_ARG, "lbm_server_submit: lattice larger than the arena budget");
    auto r = std::make_unique<Request>();
    r->nx = p->nx;
    r->ny = p->ny;
    r->dtype = dtype;
    r->lambda = p->lambda;
    r->mu = p->mu;
    r->tol = tol;
    r->max_iters = max_iters;
    r->gx.assign(p->gx, p->gx + n);
    r->gy.assign(p->gy, p->gy + n);
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(r->gx[i]) || !std::isfinite(r->gy[i]))
            return set_last_error(LBM_ERR_ARG, "lbm_server_submit: non-finite force");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->failed != LBM_OK)
            return set_last_error(s->failed, "lbm_server_submit: server failed: " + s->fail_msg);
        r->ticket = s->next_ticket++;
        r->t_submit = clk::now();
        if (!s->any_submit) {
            s->any_submit = true;
            s->t_first_submit = r->t_submit;
        }
        *ticket = r->ticket;
        s->queue.push_back(r->ticket);
        s->reqs[r->ticket] = std::move(r);
        ++s->submitted;
    }
    s->cv_work.notify_all();
    return LBM_OK;
}

static int take_result(lbm_server* s, Request& r, lbm_result* out) {
    if (out) {
        out->status = r.status;
        out->iters = r.iters;
        out->residual = r.residual;
        out->transposed = r.transposed;
        const int64_t n = (int64_t)r.nx * r.ny;
        double* dst[5] = {out->ux, out->uy, out->sxx, out->syy, out->sxy};
        if (!r.fields.empty())
            for (int i = 0; i < 5; ++i)
                if (dst[i]) std::memcpy(dst[i], r.fields.data() + i * n, sizeof(double) * n);
    }
    s->reqs.erase(r.ticket);
    return LBM_OK;
}

int lbm_server_poll(lbm_server* s, uint64_t ticket, lbm_result* out) {
    if (!s) return set_last_error(LBM_ERR_ARG, "lbm_server_poll: null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_last_error(LBM_ERR_ARG, "lbm_server_poll: unknown ticket");
    if (it->second->state != R_DONE) return LBM_PENDING;
    return take_result(s, *it->second, out);
}

int lbm_server_wait(lbm_server* s, uint64_t ticket, double timeout_s, lbm_result* out) {
    if (!s) return set_last_error(LBM_ERR_ARG, "lbm_server_wait: null server");
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = clk::now() + std::chrono::duration_cast<clk::duration>(
                                           std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0));
    while (true) {
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return set_last_error(LBM_ERR_ARG, "lbm_server_wait: unknown ticket");
        if (it->second->state == R_DONE) return take_result(s, *it->second, out);
        if (clk::now() >= deadline) return LBM_PENDING;
        s->cv_done.wait_until(lk, deadline);
    }
}

int lbm_server_cancel(lbm_server* s, uint64_t ticket) {
    if (!s) return set_last_error(LBM_ERR_ARG, "lbm_server_cancel: null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_last_error(LBM_ERR_ARG, "lbm_server_cancel: unknown ticket");
    Request& r = *it->second;
    if (r.state == R_RUNNING) {
        r.cancelled = true;  // the worker releases its arena slot between chunks
        return LBM_OK;
    }
    if (r.state == R_QUEUED)
        s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), ticket), s->queue.end());
    s->reqs.erase(it);
    return LBM_OK;
}

int lbm_server_stats(lbm_server* s, lbm_stats* out) {
    if (!s || !out) return set_last_error(LBM_ERR_ARG, "lbm_server_stats: null pointer");
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->queued = (int64_t)s->queue.size();
    out->running = (int64_t)(s->slot_owner[0].size() + s->slot_owner[1].size());
    out->p50_ms = percentile(s->latencies_ms, 0.50);
    out->p95_ms = percentile(s->latencies_ms, 0.95);
    out->p99_ms = percentile(s->latencies_ms, 0.99);
    double sum = 0.0;
    for (double v : s->latencies_ms) sum += v;
    out->mean_ms = s->latencies_ms.empty() ? 0.0 : sum / (double)s->latencies_ms.size();
    const double span_s = s->completed ? ms_between(s->t_first_submit, s->t_last_done) / 1e3 : 0.0;
    out->solves_per_s = span_s > 0.0 ? (double)s->completed / span_s : 0.0;
    out->lattice_updates = s->lups;
    out->device_ms = s->device_ms;
    out->chunks = s->chunks;
    out->hbm_bytes = (size_t)(s->arena[0]->device_bytes() + s->arena[1]->device_bytes());
    out->peak_running = s->peak_running;
    out->memory_waits = s->memory_waits;
    out->peak_resident_bytes = (size_t)s->peak_resident;
    out->tile_v = s->tile_v;
    out->failed = s->failed;
    return LBM_OK;
}

}  // extern "C"
