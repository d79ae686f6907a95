// Continuous-batching request loop for SPME evaluations (pme_server_*).
//
// Requests name a resident plan (its mesh, influence table and buckets stay on the device across
// requests) and their own device input / output arrays. A worker thread turns pending requests into
// "waves": the admitted requests are grouped by mesh shape and each group runs as one chain of six grouped
// stage launches (group.cu) on the wave's own stream. New waves are formed while earlier ones still run, so
// requests that arrive during a wave are
// admitted as soon as a wave slot, request slots and device memory allow, and their work overlaps the
// tail of the running wave on the GPU. Admission is FIFO with two rules: a plan serves one request at a
// time (its resident buffers are single-use), and the plans of all in-flight requests must fit in the
// memory budget. A result does not depend on which wave it ran in: a system's work items are the same in
// every launch.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <tuple>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/pme.h"
#include "batch_internal.h"
#include "group.h"
#include "host_tables.h"
#include "plan_internal.h"

using namespace pme;

namespace {

constexpr int WAVE_SLOTS = 3;        // waves that may be in flight at once
constexpr int MAX_WAVE_SYSTEMS = 64;  // requests per wave

double now_us() {
    return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    pme_ticket id = 0;
    pme_plan *plan = nullptr;
    const float *pos = nullptr, *q = nullptr;
    float *forces = nullptr;
    int64_t n = 0;
    double *energy = nullptr, *virial = nullptr;
    double t_submit = 0.0;
    pme_status status = PME_PENDING;
};

struct Wave {
    WaveState st;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<Request *> reqs;
    std::vector<SysDev> sys;
    std::vector<BatchEntry> entries;
    std::vector<unsigned> count;
};

}  // namespace

struct pme_server {
    int dev = 0;
    size_t budget = 0;
    int max_slots = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    std::deque<Request *> pending;
    std::unordered_map<pme_ticket, Request *> live;
    pme_ticket next_id = 1;
    int outstanding = 0;  // queued + in flight
    std::unordered_set<pme_plan *> busy_plans;
    size_t inflight_bytes = 0;
    Wave waves[WAVE_SLOTS];
    std::vector<double> lat_us;
    int64_t completed = 0, nwaves = 0;
    pme_status fatal = PME_OK;
};

static size_t plan_bytes(const pme_plan *pl) { return pme_plan_device_bytes(pl); }

// Called with the lock held: finish a wave whose event has fired.
static void finish_wave(pme_server *sv, Wave &w) {
    const double t = now_us();
    for (size_t s = 0; s < w.reqs.size(); ++s) {
        Request *r = w.reqs[s];
        const unsigned bits = w.st.h_status[s];
        if (bits & ST_TIMEOUT) {  // rare: restore the plan's resident state before anyone reuses it
            plan_recover(r->plan, w.stream);
            cudaStreamSynchronize(w.stream);
        }
        r->status = status_from_bits(bits);
        if (r->energy) *r->energy = w.st.h_ev[8 * s];
        if (r->virial)
            for (int c = 0; c < 6; ++c) r->virial[c] = w.st.h_ev[8 * s + 1 + c];
        sv->busy_plans.erase(r->plan);
        sv->inflight_bytes -= plan_bytes(r->plan);
        sv->lat_us.push_back(t - r->t_submit);
        ++sv->completed;
    }
    w.reqs.clear();
    w.busy = false;
}

// Called with the lock held: admit pending requests into wave w and launch it. Returns true if launched.
static bool launch_wave(pme_server *sv, Wave &w) {
    if (sv->pending.empty()) return false;
    std::unordered_set<pme_plan *> chosen;
    size_t bytes = sv->inflight_bytes;
    for (auto it = sv->pending.begin(); it != sv->pending.end() && (int)w.reqs.size() < MAX_WAVE_SYSTEMS;) {
        Request *r = *it;
        const size_t pb = plan_bytes(r->plan);
        const bool ok = !sv->busy_plans.count(r->plan) && !chosen.count(r->plan) && bytes + pb <= sv->budget;
        if (ok) {
            chosen.insert(r->plan);
            bytes += pb;
            w.reqs.push_back(r);
            it = sv->pending.erase(it);
        } else {
            ++it;
        }
    }
    if (w.reqs.empty()) return false;
    const int nsys = (int)w.reqs.size();
    // Requests of one mesh shape form a group: one launch per stage covers the group (group.cu); groups
    // follow one another on the wave's stream.
    auto shape = [](const pme_plan *pl) { return std::make_tuple(pl->K[0], pl->K[1], pl->K[2], pl->p); };
    std::stable_sort(w.reqs.begin(), w.reqs.end(),
                     [&](const Request *x, const Request *y) { return shape(x->plan) < shape(y->plan); });
    w.sys.clear();
    for (int s = 0; s < nsys; ++s) {
        Request *r = w.reqs[s];
        w.sys.push_back(plan_descriptor(r->plan, r->pos, r->q, r->n, r->forces, nullptr));
        if (nsys > 1) shared_tiling(w.sys.back());
    }
    if (!w.st.dmem) {
        if (w.st.init(sv->dev, MAX_WAVE_SYSTEMS, 1) != PME_OK) {
            for (Request *r : w.reqs) sv->pending.push_front(r);
            w.reqs.clear();
            sv->fatal = PME_ENOMEM;
            return false;
        }
    }
    for (int s = 0; s < nsys; ++s) {
        w.sys[s].ev = w.st.d_ev + 8 * s;
        w.st.h_sys[s] = w.sys[s];
        sv->busy_plans.insert(w.reqs[s]->plan);
        sv->inflight_bytes += plan_bytes(w.reqs[s]->plan);
    }
    cudaError_t e = w.st.upload(0, w.stream);
    for (int g0 = 0; g0 < nsys && e == cudaSuccess;) {
        int g1 = g0 + 1, max_nbin = w.sys[g0].nbin;
        while (g1 < nsys && shape(w.reqs[g1]->plan) == shape(w.reqs[g0]->plan) && w.sys[g1].tlog == w.sys[g0].tlog) {
            max_nbin = std::max(max_nbin, w.sys[g1].nbin);
            ++g1;
        }
        e = launch_group_chain(w.st.d_sys + g0, g1 - g0, w.sys[g0], max_nbin, w.stream);
        g0 = g1;
    }
    if (e == cudaSuccess) e = launch_collect_status(w.st.d_sys, nsys, w.st.d_status, w.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w.st.h_ev, w.st.d_ev, sizeof(double) * 8 * nsys, cudaMemcpyDeviceToHost, w.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w.st.h_status, w.st.d_status, sizeof(unsigned) * nsys, cudaMemcpyDeviceToHost, w.stream);
    if (e == cudaSuccess) e = cudaEventRecord(w.done, w.stream);
    if (e != cudaSuccess) {
        for (Request *r : w.reqs) {
            r->status = PME_ECUDA;
            sv->busy_plans.erase(r->plan);
            sv->inflight_bytes -= plan_bytes(r->plan);
        }
        w.reqs.clear();
        sv->fatal = PME_ECUDA;
        sv->cv_done.notify_all();
        return false;
    }
    w.busy = true;
    ++sv->nwaves;
    return true;
}

static void worker_main(pme_server *sv) {
    cudaSetDevice(sv->dev);
    std::unique_lock<std::mutex> lk(sv->mu);
    while (true) {
        bool progress = false;
        for (Wave &w : sv->waves)
            if (w.busy && cudaEventQuery(w.done) == cudaSuccess) {
                finish_wave(sv, w);
                progress = true;
            }
        if (progress) sv->cv_done.notify_all();
        for (Wave &w : sv->waves)
            if (!w.busy && !sv->pending.empty()) progress |= launch_wave(sv, w);
        bool any_busy = false;
        for (Wave &w : sv->waves) any_busy |= w.busy;
        if (sv->fatal != PME_OK && !sv->pending.empty()) {  // cannot admit any more: fail what is queued
            for (Request *r : sv->pending) r->status = sv->fatal;
            sv->pending.clear();
            sv->cv_done.notify_all();
        }
        if (sv->stop && sv->pending.empty() && !any_busy) break;
        if (!progress) {
            if (any_busy) {
                // a wave is running: poll its event, unlocked, yielding the core between polls (a timed
                // sleep would round up to the kernel's timer slack, tens of microseconds)
                lk.unlock();
                std::this_thread::yield();
                lk.lock();
            } else {
                sv->cv_work.wait_for(lk, std::chrono::milliseconds(2));
            }
        }
    }
}

extern "C" {

pme_status pme_server_create(size_t mem_budget_bytes, int max_slots, pme_server **out) {
    if (!out) return fail(PME_EINVAL, "out is NULL");
    *out = nullptr;
    if (max_slots < 1 || mem_budget_bytes == 0) return fail(PME_EINVAL, "max_slots >= 1 and a nonzero budget required");
    pme_server *sv = lib_new<pme_server>();
    if (!sv) return fail(PME_ENOMEM, "host allocation failed");
    cudaGetDevice(&sv->dev);
    sv->budget = mem_budget_bytes;
    sv->max_slots = max_slots;
    cudaError_t e = configure_group_kernels();
    if (e != cudaSuccess) {
        delete sv;
        return cuda_fail(e, "configure grouped kernels");
    }
    for (Wave &w : sv->waves) {
        if ((e = cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming)) != cudaSuccess) {
            pme_server_destroy(sv);
            return cuda_fail(e, "stream / event creation");
        }
        pme_status st = w.st.init(sv->dev, MAX_WAVE_SYSTEMS, 1);
        if (st != PME_OK) {
            pme_server_destroy(sv);
            return st;
        }
    }
    sv->worker = std::thread(worker_main, sv);
    *out = sv;
    return PME_OK;
}

pme_status pme_submit(pme_server *sv, pme_plan *plan, const float *pos, const float *q, int64_t n, float *forces,
                      double *energy, double *virial, pme_ticket *out) {
    if (!sv || !out) return fail(PME_EINVAL, "server and out must be non-NULL");
    pme_status st = check_atoms(plan, pos, q, n, forces);
    if (st) return st;
    if (plan->dev != sv->dev) return fail(PME_EINVAL, "plan is on device %d, server on %d", plan->dev, sv->dev);
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->fatal != PME_OK) return fail(sv->fatal, "server stopped after an earlier failure");
    if (plan_bytes(plan) > sv->budget) return fail(PME_ENOMEM, "plan needs %zu bytes, budget is %zu", plan_bytes(plan), sv->budget);
    if (sv->outstanding >= sv->max_slots) return fail(PME_EAGAIN, "all %d request slots are in use", sv->max_slots);
    if (n > plan->n_cap) {
        // growing the plan's per-atom scratch is only safe while no request uses it
        if (sv->busy_plans.count(plan)) return fail(PME_EAGAIN, "plan is in flight and needs more atom capacity");
        for (Request *r : sv->pending)
            if (r->plan == plan) return fail(PME_EAGAIN, "plan has queued requests and needs more atom capacity");
        DeviceGuard g(plan->dev);
        if ((st = plan_reserve(plan, n)) != PME_OK) return st;
    }
    Request *r = lib_new<Request>();
    if (!r) return fail(PME_ENOMEM, "host allocation failed");
    r->id = sv->next_id++;
    r->plan = plan;
    r->pos = pos;
    r->q = q;
    r->n = n;
    r->forces = forces;
    r->energy = energy;
    r->virial = virial;
    r->t_submit = now_us();
    sv->pending.push_back(r);
    sv->live[r->id] = r;
    ++sv->outstanding;
    *out = r->id;
    sv->cv_work.notify_one();
    return PME_OK;
}

pme_status pme_poll(pme_server *sv, pme_ticket ticket, int block) {
    if (!sv) return fail(PME_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->live.find(ticket);
    if (it == sv->live.end()) return fail(PME_EINVAL, "unknown or already retired ticket %lld", (long long)ticket);
    Request *r = it->second;
    if (block)
        sv->cv_done.wait(lk, [&] { return r->status != PME_PENDING; });
    if (r->status == PME_PENDING) return PME_PENDING;
    const pme_status st = r->status;
    sv->live.erase(it);
    --sv->outstanding;
    delete r;
    if (st != PME_OK) return fail(st, "request %lld failed: %s", (long long)ticket, pme_strerror(st));
    return PME_OK;
}

pme_status pme_server_stats(pme_server *sv, int64_t *completed, double *p50_us, double *p99_us, int64_t *waves) {
    if (!sv) return fail(PME_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(sv->mu);
    std::vector<double> v = sv->lat_us;
    std::sort(v.begin(), v.end());
    auto pct = [&](double f) { return v.empty() ? 0.0 : v[std::min(v.size() - 1, (size_t)(f * (v.size() - 1) + 0.5))]; };
    if (completed) *completed = sv->completed;
    if (p50_us) *p50_us = pct(0.50);
    if (p99_us) *p99_us = pct(0.99);
    if (waves) *waves = sv->nwaves;
    return PME_OK;
}

void pme_server_destroy(pme_server *sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    DeviceGuard g(sv->dev);
    for (Wave &w : sv->waves) {
        if (w.stream) cudaStreamSynchronize(w.stream);
        w.st.release();
        if (w.done) cudaEventDestroy(w.done);
        if (w.stream) cudaStreamDestroy(w.stream);
    }
    for (auto &kv : sv->live) delete kv.second;
    delete sv;
}

}  // extern "C"
