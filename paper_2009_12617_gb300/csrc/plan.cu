// Single-system plans: the C ABI of pme.h for pme_create / pme_compute / pme_enqueue and friends.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "../../include/pme.h"
#include "host_tables.h"
#include "kernels.h"
#include "plan_internal.h"

namespace pme {

// ---------------------------------------------------------------------------------------------------------
// error reporting

static thread_local char g_msg[512] = "";
static thread_local pme_status g_status = PME_OK;

pme_status fail(pme_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    g_status = s;
    return s;
}

static std::atomic<long long> g_fail_countdown{0};  // > 0: the allocation that takes it to zero fails

bool alloc_injected_failure() {
    long long v = g_fail_countdown.load();
    while (v > 0)
        if (g_fail_countdown.compare_exchange_weak(v, v - 1)) return v == 1;
    return false;
}

cudaError_t lib_malloc(void **p, size_t bytes) {
    if (alloc_injected_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t lib_malloc_host(void **p, size_t bytes) {
    if (alloc_injected_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocHost(p, bytes);
}

pme_status cuda_fail(cudaError_t e, const char *what) {
    return fail(e == cudaErrorMemoryAllocation ? PME_ENOMEM : PME_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

pme_status status_from_bits(unsigned bits) {
    if (bits & ST_TIMEOUT) return fail(PME_ETIMEOUT, "a bounded device-side dependency wait gave up");
    if (bits & ST_NONFINITE)
        return fail(PME_EINVAL, "a position or charge is non-finite, |q| >= 2^22 e, or a position is absurdly far out");
    if (bits & ST_OVERFLOW) return fail(PME_EOVERFLOW, "sum |q| >= 2^22 e exceeds the fixed-point charge mesh headroom");
    if (bits & ST_INTERNAL) return fail(PME_ECUDA, "internal consistency check failed on the device");
    return PME_OK;
}

DeviceGuard::DeviceGuard(int dev) {
    cudaGetDevice(&prev_);
    if (prev_ != dev) cudaSetDevice(dev);
    dev_ = dev;
}
DeviceGuard::~DeviceGuard() {
    if (prev_ != dev_) cudaSetDevice(prev_);
}

cudaError_t ensure_configured(int dev) {
    static std::mutex mu;
    static std::vector<char> done(256, 0);
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    if (done[dev]) return cudaSuccess;
    cudaError_t e = configure_kernels();
    if (e == cudaSuccess) done[dev] = 1;
    return e;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// ---------------------------------------------------------------------------------------------------------
// plan construction

static pme_status upload_tables(pme_plan *pl) {
    const int *K = pl->K;
    const int H3 = K[2] / 2 + 1, Nh = K[2] / 2;
    std::vector<float4> bc((size_t)K[0] * K[1] * H3);
    make_influence(K, pl->p, pl->beta, pl->recip, pl->vol, bc.data());
    std::vector<float2> tw((size_t)K[0] + K[1] + Nh + Nh + 1);
    make_twiddles(K[0], K[0], tw.data());
    make_twiddles(K[1], K[1], tw.data() + K[0]);
    make_twiddles(Nh, Nh, tw.data() + K[0] + K[1]);
    make_twiddles(K[2], Nh + 1, tw.data() + K[0] + K[1] + Nh);
    cudaError_t e;
    if ((e = cudaStreamSynchronize(pl->stream)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if ((e = cudaMemcpy((void *)pl->d.bc, bc.data(), bc.size() * sizeof(float4), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpy(influence table)");
    if ((e = cudaMemcpy((void *)pl->d.tw1, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpy(twiddles)");
    return PME_OK;
}

static pme_status alloc_mesh(pme_plan *pl) {
    SysDev &d = pl->d;
    const size_t K1 = d.K1, K2 = d.K2, K3 = d.K3, H3 = d.H3, Nh = K3 / 2;
    size_t off = 0;
    const size_t o_grid = off; off = align256(off + K1 * K2 * K3 * 8);
    const size_t o_spec = off; off = align256(off + K1 * K2 * H3 * 8);
    const size_t o_phi = off;  off = align256(off + K1 * K2 * K3 * 4);
    const size_t o_bc = off;   off = align256(off + K1 * K2 * H3 * sizeof(float4));
    const size_t o_tw = off;   off = align256(off + (K1 + K2 + Nh + Nh + 1) * 8);
    const size_t o_cnt = off;  off = align256(off + bcount_bytes_max(pl->K));
    const size_t o_qs = off;   off = align256(off + QABS_BYTES);
    const size_t o_par = off;  off = align256(off + partials_bytes(d));
    const size_t o_ctl = off;  off = align256(off + sizeof(Ctl));
    cudaError_t e = lib_malloc(&pl->mesh_mem, off);
    if (e != cudaSuccess) {
        pl->mesh_mem = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? PME_ENOMEM : PME_ECUDA, "cudaMalloc(%zu bytes): %s", off, cudaGetErrorString(e));
    }
    pl->mesh_bytes = off;
    char *b = (char *)pl->mesh_mem;
    d.grid = (unsigned long long *)(b + o_grid);
    d.spec = (float2 *)(b + o_spec);
    d.phi = (float *)(b + o_phi);
    d.bc = (const float4 *)(b + o_bc);
    float2 *tw = (float2 *)(b + o_tw);
    d.tw1 = tw;
    d.tw2 = tw + K1;
    d.tw3h = tw + K1 + K2;
    d.tw3 = tw + K1 + K2 + Nh;
    d.bcount = (unsigned *)(b + o_cnt);
    d.qslot = (unsigned long long *)(b + o_qs);
    d.partials = (double *)(b + o_par);
    d.ctl = (Ctl *)(b + o_ctl);
    // The int64 mesh, bucket counts and control block start at zero; afterwards the consuming stages
    // reset them, so evaluations need no memset.
    if ((e = cudaMemset(pl->mesh_mem, 0, off)) != cudaSuccess) return cuda_fail(e, "cudaMemset(mesh)");
    return PME_OK;
}

pme_status plan_reserve(pme_plan *pl, int64_t n) {
    if (n <= pl->n_cap && pl->atom_mem) return PME_OK;
    SysDev &d = pl->d;
    const int64_t ncap = n > 0 ? n : 1;
    // tile edge from the atom density, or the one the autotuner / caller set (every tile counter is zero
    // between evaluations, so the tiling may change here; results do not depend on it)
    set_tiling(d, pl->tile_log_set ? pl->tile_log_set : choose_tile_log(ncap, pl->K, pl->sms));
    set_tiling(d, d.tlog, choose_k1_pieces(d, pl->sms));
    const int cap = bucket_capacity(ncap, d.ntiles, d.tlog);
    const size_t nb = (size_t)d.ntiles * cap;
    size_t off = 0;
    const size_t o_bka = off; off = align256(off + nb * 16);
    const size_t o_bkb = off; off = align256(off + nb * 8);
    const size_t o_ova = off; off = align256(off + (size_t)ncap * 16);
    const size_t o_ovb = off; off = align256(off + (size_t)ncap * 8);
    cudaError_t e = cudaStreamSynchronize(pl->stream);  // nothing in flight may still use the old buffers
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (pl->atom_mem) cudaFree(pl->atom_mem);
    pl->atom_mem = nullptr;
    pl->atom_bytes = 0;
    pl->n_cap = 0;
    e = lib_malloc(&pl->atom_mem, off);
    if (e != cudaSuccess) {
        pl->atom_mem = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? PME_ENOMEM : PME_ECUDA, "cudaMalloc(%zu bytes): %s", off, cudaGetErrorString(e));
    }
    char *b = (char *)pl->atom_mem;
    d.bka = (float4 *)(b + o_bka);
    d.bkb = (int2 *)(b + o_bkb);
    d.ova = (float4 *)(b + o_ova);
    d.ovb = (int2 *)(b + o_ovb);
    d.cap = cap;
    pl->atom_bytes = off;
    pl->n_cap = ncap;
    return PME_OK;
}

SysDev plan_descriptor(const pme_plan *pl, const float *pos, const float *q, int64_t n, float *forces, double *ev_dev) {
    SysDev d = pl->d;
    d.n = (int)n;
    d.nbin = (int)((n + BIN_CHUNK - 1) / BIN_CHUNK);
    d.pos = pos;
    d.q = q;
    d.forces = forces;
    d.ev = ev_dev ? ev_dev : pl->d.ctl->ev;
    d.tc_w = pl->influence_path == PME_INFLUENCE_TENSOR ? pl->tc_w : nullptr;
    return d;
}

pme_status check_atoms(const pme_plan *pl, const float *pos, const float *q, int64_t n, const float *forces) {
    if (!pl) return fail(PME_EINVAL, "plan is NULL");
    if (n < 0 || n > (int64_t)0x3fffffff) return fail(PME_EINVAL, "n = %lld out of range [0, 2^30)", (long long)n);
    if (n > 0 && (!pos || !q || !forces)) return fail(PME_EINVAL, "pos, q and forces must be non-NULL when n > 0");
    return PME_OK;
}

// Read (and clear) the device status word after the stream has drained.
pme_status collect_status(pme_plan *pl, bool copy_ctl) {
    cudaError_t e;
    if (!copy_ctl) {
        if ((e = cudaMemcpyAsync(&pl->h_ctl->status, &pl->d.ctl->status, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                 pl->stream)) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpyAsync(status)");
    }
    if ((e = cudaStreamSynchronize(pl->stream)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    const unsigned bits = pl->h_ctl->status;
    if (bits) {
        if ((e = cudaMemsetAsync(&pl->d.ctl->status, 0, sizeof(unsigned), pl->stream)) != cudaSuccess)
            return cuda_fail(e, "cudaMemsetAsync(status)");
        if ((e = cudaStreamSynchronize(pl->stream)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
        pl->h_ctl->status = 0;
    }
    return status_from_bits(bits);
}

// Device-accessible address of host memory that is page-locked (cudaHostAlloc / cudaHostRegister), or null.
static void *device_view(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Device staging for host-array calls (positions, forces, charges), at least n atoms.
static pme_status ensure_host_staging(pme_plan *pl, int64_t n) {
    if (n <= pl->host_cap && pl->host_mem) return PME_OK;
    cudaError_t e;
    if ((e = cudaStreamSynchronize(pl->stream)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (pl->host_mem) cudaFree(pl->host_mem);
    pl->host_mem = nullptr;
    pl->host_cap = 0;
    const int64_t m = n > 0 ? n : 1;
    const size_t bytes = align256((size_t)m * 12) * 2 + align256((size_t)m * 4);
    if ((e = lib_malloc(&pl->host_mem, bytes)) != cudaSuccess) {
        pl->host_mem = nullptr;
        return fail(PME_ENOMEM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    pl->host_cap = m;
    return PME_OK;
}

// Enqueue the call described by key through graph g: replay it if it was recorded for these arguments,
// record it now if the previous call (seen) had the same arguments, else enqueue directly. enqueue(stream)
// issues the call's work on a stream.
template <class F>
static cudaError_t run_call(pme_plan *pl, pme_plan::EvalGraph &g, pme_plan::EvalGraph &seen,
                            const pme_plan::EvalGraph &key, F enqueue) {
    if (g.exec && g.same(key)) return cudaGraphLaunch(g.exec, pl->stream);
    const bool repeat = seen.same(key);
    seen = key;
    if (repeat) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = pme_plan::EvalGraph();
        bool ok = pl->rec_stream || cudaStreamCreateWithFlags(&pl->rec_stream, cudaStreamNonBlocking) == cudaSuccess;
        cudaGraph_t graph = nullptr;
        if (ok) ok = cudaStreamBeginCapture(pl->rec_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            const cudaError_t r = enqueue(pl->rec_stream);
            const cudaError_t e = cudaStreamEndCapture(pl->rec_stream, &graph);
            ok = r == cudaSuccess && e == cudaSuccess;
            cudaGraphExec_t exec = nullptr;
            if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
            if (graph) cudaGraphDestroy(graph);
            if (ok) {
                g = key;
                g.exec = exec;
                return cudaGraphLaunch(g.exec, pl->stream);
            }
        }
        cudaGetLastError();  // not recordable here: enqueue directly
    }
    return enqueue(pl->stream);
}

}  // namespace pme

using namespace pme;

extern "C" {

const char *pme_strerror(pme_status s) {
    switch (s) {
        case PME_OK: return "ok";
        case PME_EINVAL: return "invalid argument";
        case PME_EUNSUPPORTED: return "unsupported parameters";
        case PME_ENOMEM: return "out of memory";
        case PME_ECUDA: return "CUDA error";
        case PME_EOVERFLOW: return "fixed-point charge mesh overflow";
        case PME_EAGAIN: return "no capacity right now; retry";
        case PME_ETIMEOUT: return "device-side wait timed out";
        case PME_PENDING: return "pending";
    }
    return "unknown status";
}

pme_status pme_debug_fail_alloc(int nth) {
    if (nth < 0) return fail(PME_EINVAL, "nth must be >= 0");
    g_fail_countdown.store(nth);
    return PME_OK;
}

pme_status pme_last_error_detail(char *buf, size_t len) {
    if (buf && len) {
        strncpy(buf, g_msg, len - 1);
        buf[len - 1] = 0;
    }
    return g_status;
}

pme_status pme_create(const int K[3], int p, double beta, const double box[9], void *cuda_stream, pme_plan **out) {
    if (!out) return fail(PME_EINVAL, "out is NULL");
    *out = nullptr;
    if (!K || !box) return fail(PME_EINVAL, "K and box must be non-NULL");
    char msg[256];
    const int v = validate_params(K, p, beta, box, msg, sizeof(msg));
    if (v == 1) return fail(PME_EINVAL, "%s", msg);
    if (v == 2) return fail(PME_EUNSUPPORTED, "%s", msg);
    double recip[9], vol;
    if (!cell_reciprocal(box, recip, &vol)) return fail(PME_EINVAL, "box is singular");
    pme_plan *pl = lib_new<pme_plan>();
    if (!pl) return fail(PME_ENOMEM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&pl->dev);
    if (e != cudaSuccess) {
        delete pl;
        return cuda_fail(e, "cudaGetDevice");
    }
    if ((e = ensure_configured(pl->dev)) != cudaSuccess) {
        delete pl;
        return cuda_fail(e, "configure kernels");
    }
    if ((e = cudaDeviceGetAttribute(&pl->sms, cudaDevAttrMultiProcessorCount, pl->dev)) != cudaSuccess) {
        delete pl;
        return cuda_fail(e, "cudaDeviceGetAttribute(SM count)");
    }
    pl->stream = (cudaStream_t)cuda_stream;
    memcpy(pl->K, K, sizeof(pl->K));
    pl->p = p;
    pl->beta = beta;
    memcpy(pl->box, box, sizeof(pl->box));
    memcpy(pl->recip, recip, sizeof(recip));
    pl->vol = vol;
    memset(&pl->d, 0, sizeof(pl->d));
    fill_geometry(pl->d, K, p, beta, recip);
    pme_status st;
    if ((st = alloc_mesh(pl)) != PME_OK || (st = upload_tables(pl)) != PME_OK || (st = plan_reserve(pl, 1)) != PME_OK) {
        pme_destroy(pl);
        return st;
    }
    if ((e = lib_malloc_host((void **)&pl->h_ctl, sizeof(Ctl))) != cudaSuccess) {
        pl->h_ctl = nullptr;
        pme_destroy(pl);
        return cuda_fail(e, "cudaMallocHost");
    }
    memset(pl->h_ctl, 0, sizeof(Ctl));
    pl->h_ctl_dev = (Ctl *)device_view(pl->h_ctl);
    *out = pl;
    return PME_OK;
}

pme_status pme_set_box(pme_plan *pl, const double box[9]) {
    if (!pl || !box) return fail(PME_EINVAL, "plan and box must be non-NULL");
    char msg[256];
    const int v = validate_params(pl->K, pl->p, pl->beta, box, msg, sizeof(msg));
    if (v) return fail(PME_EINVAL, "%s", msg);
    double recip[9], vol;
    if (!cell_reciprocal(box, recip, &vol)) return fail(PME_EINVAL, "box is singular");
    DeviceGuard g(pl->dev);
    memcpy(pl->box, box, sizeof(pl->box));
    memcpy(pl->recip, recip, sizeof(recip));
    pl->vol = vol;
    fill_geometry(pl->d, pl->K, pl->p, pl->beta, recip);
    ++pl->gen;
    return upload_tables(pl);
}

pme_status pme_reserve(pme_plan *pl, int64_t n) {
    if (!pl) return fail(PME_EINVAL, "plan is NULL");
    if (n < 0 || n > (int64_t)0x3fffffff) return fail(PME_EINVAL, "n out of range");
    DeviceGuard g(pl->dev);
    return plan_reserve(pl, n);
}

pme_status pme_enqueue(pme_plan *pl, const float *pos, const float *q, int64_t n, float *forces, double *ev_dev) {
    pme_status st = check_atoms(pl, pos, q, n, forces);
    if (st) return st;
    DeviceGuard g(pl->dev);
    if ((st = plan_reserve(pl, n)) != PME_OK) return st;
    const SysDev d = plan_descriptor(pl, pos, q, n, forces, ev_dev);
    cudaError_t e = launch_pipeline(d, pl->stream);
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return PME_OK;
}

pme_status pme_sync(pme_plan *pl) {
    if (!pl) return fail(PME_EINVAL, "plan is NULL");
    DeviceGuard g(pl->dev);
    for (cudaStream_t cs : {pl->copy_stream, pl->out_stream})  // pme_enqueue_host's copies
        if (cs) {
            cudaError_t e = cudaStreamSynchronize(cs);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
        }
    return collect_status(pl, false);
}

pme_status pme_compute(pme_plan *pl, const float *pos, const float *q, int64_t n, float *forces, double *energy,
                       double *virial) {
    return pme_compute_debug(pl, pos, q, n, forces, energy, virial, nullptr, nullptr);
}

pme_status pme_compute_debug(pme_plan *pl, const float *pos, const float *q, int64_t n, float *forces, double *energy,
                             double *virial, int64_t *mesh_dev, float *phi_dev) {
    pme_status st = check_atoms(pl, pos, q, n, forces);
    if (st) return st;
    DeviceGuard g(pl->dev);
    if ((st = plan_reserve(pl, n)) != PME_OK) return st;
    const SysDev d = plan_descriptor(pl, pos, q, n, forces, nullptr);
    DebugTaps taps = {(unsigned long long *)mesh_dev, phi_dev};
    const bool tapped = mesh_dev || phi_dev;
    auto enqueue = [&](cudaStream_t s) -> cudaError_t {
        cudaError_t r = launch_pipeline(d, s, tapped ? &taps : nullptr);
        if (r != cudaSuccess) return r;
        // energy, virial and status to the pinned host block: written by a kernel chained to the force stage
        // (a copy-engine transfer at the end of the chain measured 53.0 against 43.9 us per synchronous
        // 64^3 call), else copied
        if (pl->h_ctl_dev) return launch_copy_out(nullptr, nullptr, 0, pl->d.ctl, pl->h_ctl_dev, s);
        return cudaMemcpyAsync(pl->h_ctl, pl->d.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
    };
    cudaError_t e;
    if (tapped) {
        e = enqueue(pl->stream);
    } else {
        pme_plan::EvalGraph key;
        key.pos = pos;
        key.q = q;
        key.forces = forces;
        key.atoms = pl->atom_mem;
        key.n = n;
        key.mode = launch_mode();
        key.gen = pl->gen;
        e = run_call(pl, pl->g_dev, pl->seen_dev, key, enqueue);
    }
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    if ((st = collect_status(pl, true)) != PME_OK) return st;
    if (energy) *energy = pl->h_ctl->ev[0];
    if (virial)
        for (int c = 0; c < 6; ++c) virial[c] = pl->h_ctl->ev[1 + c];
    return PME_OK;
}

// One slot of pme_enqueue_host's device buffers: positions, forces, charges for m atoms, then the result
// (energy, virial, status: 8 doubles).
static size_t async_slot_bytes(int64_t m) { return 2 * align256((size_t)m * 12) + align256((size_t)m * 4) + 256; }

// pme_enqueue_host's two slots (device positions, charges and forces) for at least n atoms, the copy stream
// and the events.
static pme_status ensure_async_inputs(pme_plan *pl, int64_t n) {
    cudaError_t e;
    for (cudaStream_t *cs : {&pl->copy_stream, &pl->out_stream})
        if (!*cs && (e = cudaStreamCreateWithFlags(cs, cudaStreamNonBlocking)) != cudaSuccess) {
            *cs = nullptr;
            return cuda_fail(e, "cudaStreamCreate");
        }
    for (int s = 0; s < 2; ++s)
        for (cudaEvent_t *ev : {&pl->in_ready[s], &pl->in_free[s], &pl->out_done[s]})
            if (!*ev && (e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess) {
                *ev = nullptr;
                return cuda_fail(e, "cudaEventCreate");
            }
    for (cudaEvent_t &ev : pl->host_done)
        if (!ev && (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
            ev = nullptr;
            return cuda_fail(e, "cudaEventCreate");
        }
    if (n <= pl->async_cap && pl->async_mem) return PME_OK;
    for (cudaStream_t cs : {pl->stream, pl->copy_stream, pl->out_stream})
        if ((e = cudaStreamSynchronize(cs)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (pl->async_mem) cudaFree(pl->async_mem);
    pl->async_mem = nullptr;
    pl->async_cap = 0;
    const int64_t m = n > 0 ? n : 1;
    const size_t bytes = 2 * async_slot_bytes(m);
    if ((e = lib_malloc(&pl->async_mem, bytes)) != cudaSuccess) {
        pl->async_mem = nullptr;
        return fail(PME_ENOMEM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    pl->async_cap = m;
    for (pme_plan::EvalGraph &gr : pl->g_async)  // recorded for the old slots
        if (gr.exec) {
            cudaGraphExecDestroy(gr.exec);
            gr = pme_plan::EvalGraph();
        }
    return PME_OK;
}

static pme_status launch_async_graph(pme_plan *pl, const float *dpos, const float *dq, int64_t n, float *dfor,
                                     double *dres);

pme_status pme_enqueue_host(pme_plan *pl, const float *pos, const float *q, int64_t n, float *forces, double *result,
                            int64_t *ticket) {
    pme_status st = check_atoms(pl, pos, q, n, forces);
    if (st) return st;
    if (!result) return fail(PME_EINVAL, "result must be non-NULL");
    DeviceGuard g(pl->dev);
    if ((st = plan_reserve(pl, n)) != PME_OK) return st;
    if ((st = ensure_async_inputs(pl, n)) != PME_OK) return st;
    if (!device_view(result) || (n > 0 && (!device_view(pos) || !device_view(q) || !device_view(forces))))
        return fail(PME_EINVAL, "pme_enqueue_host needs page-locked pos, q, forces and result (cudaHostAlloc / cudaHostRegister)");
    // Slot s (alternating): the copy engine brings the inputs in on the copy stream once the evaluation that
    // last used the slot has finished; the plan stream waits for them (and for the slot's previous results to
    // have left) and evaluates into the slot's device forces and result (the graph of the slot, the same
    // whatever host arrays the call names); then the copy engine takes forces and result out on the output
    // stream. Each copy overlaps the evaluation running on the plan stream at the time.
    const int slot = pl->async_slot;
    pl->async_slot ^= 1;
    char *sb = (char *)pl->async_mem + (size_t)slot * async_slot_bytes(pl->async_cap);
    float *dpos = (float *)sb, *dfor = (float *)(sb + align256((size_t)pl->async_cap * 12));
    float *dq = (float *)(sb + 2 * align256((size_t)pl->async_cap * 12));
    double *dres = (double *)(sb + 2 * align256((size_t)pl->async_cap * 12) + align256((size_t)pl->async_cap * 4));
    const int64_t t = pl->host_seq;
    cudaEvent_t done = pl->host_done[t % pme_plan::HOST_TICKETS];
    cudaError_t e;
    if ((e = cudaStreamWaitEvent(pl->copy_stream, pl->in_free[slot], 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
    if (n > 0) {
        if ((e = cudaMemcpyAsync(dpos, pos, (size_t)n * 12, cudaMemcpyHostToDevice, pl->copy_stream)) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpyAsync(pos)");
        if ((e = cudaMemcpyAsync(dq, q, (size_t)n * 4, cudaMemcpyHostToDevice, pl->copy_stream)) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpyAsync(q)");
    }
    if ((e = cudaEventRecord(pl->in_ready[slot], pl->copy_stream)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    if ((e = cudaStreamWaitEvent(pl->stream, pl->in_ready[slot], 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
    if ((e = cudaStreamWaitEvent(pl->stream, pl->out_done[slot], 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
    if ((st = launch_async_graph(pl, dpos, dq, n, dfor, dres)) != PME_OK) return st;
    if ((e = cudaEventRecord(pl->in_free[slot], pl->stream)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    if ((e = cudaStreamWaitEvent(pl->out_stream, pl->in_free[slot], 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
    if (n > 0 && (e = cudaMemcpyAsync(forces, dfor, (size_t)n * 12, cudaMemcpyDeviceToHost, pl->out_stream)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync(forces)");
    if ((e = cudaMemcpyAsync(result, dres, 8 * sizeof(double), cudaMemcpyDeviceToHost, pl->out_stream)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync(result)");
    if ((e = cudaEventRecord(pl->out_done[slot], pl->out_stream)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    if ((e = cudaEventRecord(done, pl->out_stream)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    pl->host_seq = t + 1;
    if (ticket) *ticket = t;
    return PME_OK;
}

pme_status pme_host_wait(pme_plan *pl, int64_t ticket) {
    if (!pl) return fail(PME_EINVAL, "plan is NULL");
    if (ticket < 0 || ticket >= pl->host_seq) return fail(PME_EINVAL, "no pme_enqueue_host call has ticket %lld", (long long)ticket);
    DeviceGuard g(pl->dev);
    // the event of an older ticket may have been recorded again for a newer one; the copy stream runs in
    // order, so waiting for the newer one covers it
    cudaError_t e = cudaEventSynchronize(pl->host_done[ticket % pme_plan::HOST_TICKETS]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
    return PME_OK;
}

// The evaluation of pme_enqueue_host on slot buffers dpos / dq / dfor, its energy, virial and status bits
// into the slot's dres, as a graph recorded once per slot (and atom count; the four most recent kept).
static pme_status launch_async_graph(pme_plan *pl, const float *dpos, const float *dq, int64_t n, float *dfor,
                                     double *dres) {
    // the force stage's final reduction writes energy, virial and the status bits straight into dres
    SysDev d = plan_descriptor(pl, dpos, dq, n, dfor, dres);
    d.ev_status = 1;
    pme_plan::EvalGraph key;
    key.pos = dpos;
    key.q = dq;
    key.forces = dfor;
    key.atoms = pl->atom_mem;
    key.staging = pl->async_mem;
    key.result = dres;
    key.n = n;
    key.mode = launch_mode();
    key.gen = pl->gen;
    cudaError_t e;
    for (pme_plan::EvalGraph &gr : pl->g_async)
        if (gr.exec && gr.same(key)) {
            if ((e = cudaGraphLaunch(gr.exec, pl->stream)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
            return PME_OK;
        }
    // first use of this slot: record the evaluation as a graph (on the private stream, so the plan stream may
    // itself be busy), then launch it
    if (!pl->rec_stream && (e = cudaStreamCreateWithFlags(&pl->rec_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamCreate");
    if ((e = cudaStreamBeginCapture(pl->rec_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamBeginCapture");
    cudaError_t r = launch_pipeline(d, pl->rec_stream);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(pl->rec_stream, &graph);
    if (r != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(r != cudaSuccess ? r : e, "recording the evaluation");
    }
    pme_plan::EvalGraph &slot = pl->g_async[pl->g_async_next];
    pl->g_async_next = (pl->g_async_next + 1) % 4;
    if (slot.exec) cudaGraphExecDestroy(slot.exec);
    slot = key;
    slot.exec = nullptr;
    e = cudaGraphInstantiate(&slot.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        slot.exec = nullptr;
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    if ((e = cudaGraphLaunch(slot.exec, pl->stream)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return PME_OK;
}

pme_status pme_compute_host(pme_plan *pl, const float *pos, const float *q, int64_t n, float *forces, double *energy,
                            double *virial) {
    pme_status st = check_atoms(pl, pos, q, n, forces);
    if (st) return st;
    DeviceGuard g(pl->dev);
    cudaError_t e;
    if ((st = plan_reserve(pl, n)) != PME_OK) return st;
    if ((st = ensure_host_staging(pl, n)) != PME_OK) return st;
    char *b = (char *)pl->host_mem;
    float *dpos = (float *)b, *dfor = (float *)(b + align256((size_t)pl->host_cap * 12));
    float *dq = (float *)(b + 2 * align256((size_t)pl->host_cap * 12));
    const float *mpos = n > 0 ? (const float *)device_view(pos) : nullptr;
    const float *mq = n > 0 ? (const float *)device_view(q) : nullptr;
    float *mfor = n > 0 ? (float *)device_view(forces) : nullptr;
    Ctl *mctl = pl->h_ctl_dev;
    if (mpos && mq && mfor && mctl) {
        // Page-locked arrays: binning reads positions and charges in host memory directly (coalesced, over
        // the CPU-GPU link), the forces are gathered into device staging and written back with the control
        // block by one copy kernel; as a graph, the call is one launch and one wait.
        const SysDev d = plan_descriptor(pl, mpos, mq, n, dfor, nullptr);
        auto enqueue = [&](cudaStream_t s) -> cudaError_t {
            cudaError_t r = launch_pipeline(d, s);
            if (r != cudaSuccess) return r;
            return launch_copy_out(dfor, mfor, (long long)n * 3, pl->d.ctl, mctl, s);
        };
        pme_plan::EvalGraph key;
        key.pos = pos;
        key.q = q;
        key.forces = forces;
        key.atoms = pl->atom_mem;
        key.staging = pl->host_mem;
        key.n = n;
        key.mode = launch_mode();
        key.gen = pl->gen;
        if ((e = run_call(pl, pl->g_host, pl->seen_host, key, enqueue)) != cudaSuccess)
            return cuda_fail(e, "enqueueing the evaluation");
    } else {  // pageable arrays: copies to and from device staging around the six stages
        if (n > 0) {
            if ((e = cudaMemcpyAsync(dpos, pos, (size_t)n * 12, cudaMemcpyHostToDevice, pl->stream)) != cudaSuccess)
                return cuda_fail(e, "cudaMemcpyAsync(pos)");
            if ((e = cudaMemcpyAsync(dq, q, (size_t)n * 4, cudaMemcpyHostToDevice, pl->stream)) != cudaSuccess)
                return cuda_fail(e, "cudaMemcpyAsync(q)");
        }
        const SysDev d = plan_descriptor(pl, dpos, dq, n, dfor, nullptr);
        if ((e = launch_pipeline(d, pl->stream)) != cudaSuccess) return cuda_fail(e, "kernel launch");
        if (n > 0 && (e = cudaMemcpyAsync(forces, dfor, (size_t)n * 12, cudaMemcpyDeviceToHost, pl->stream)) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpyAsync(forces)");
        if ((e = cudaMemcpyAsync(pl->h_ctl, pl->d.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, pl->stream)) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpyAsync(result)");
    }
    if ((st = collect_status(pl, true)) != PME_OK) return st;
    if (energy) *energy = pl->h_ctl->ev[0];
    if (virial)
        for (int c = 0; c < 6; ++c) virial[c] = pl->h_ctl->ev[1 + c];
    return PME_OK;
}

pme_status pme_profile_stages(pme_plan *pl, const float *pos, const float *q, int64_t n, float *forces, int reps,
                              double stage_us[6]) {
    pme_status st = check_atoms(pl, pos, q, n, forces);
    if (st) return st;
    if (reps < 1 || !stage_us) return fail(PME_EINVAL, "reps must be >= 1 and stage_us non-NULL");
    DeviceGuard g(pl->dev);
    if ((st = plan_reserve(pl, n)) != PME_OK) return st;
    const SysDev d = plan_descriptor(pl, pos, q, n, forces, nullptr);
    cudaEvent_t ev[NUM_STAGES + 1];
    for (int i = 0; i <= NUM_STAGES; ++i) cudaEventCreate(&ev[i]);
    double acc[NUM_STAGES] = {0};
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        for (int s = 0; s < NUM_STAGES; ++s) {
            cudaEventRecord(ev[s], pl->stream);
            launch_stage(d, s, pl->stream);
        }
        cudaEventRecord(ev[NUM_STAGES], pl->stream);
        if ((e = cudaEventSynchronize(ev[NUM_STAGES])) != cudaSuccess) break;
        for (int s = 0; s < NUM_STAGES; ++s) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[s], ev[s + 1]);
            acc[s] += ms;
        }
    }
    for (int i = 0; i <= NUM_STAGES; ++i) cudaEventDestroy(ev[i]);
    if (e != cudaSuccess) return cuda_fail(e, "profiled launch");
    for (int s = 0; s < NUM_STAGES; ++s) stage_us[s] = 1000.0 * acc[s] / reps;
    return collect_status(pl, false);
}

pme_status pme_set_influence_path(pme_plan *pl, int path) {
    if (!pl) return fail(PME_EINVAL, "plan is NULL");
    if (path != PME_INFLUENCE_FP32 && path != PME_INFLUENCE_TENSOR)
        return fail(PME_EINVAL, "path must be PME_INFLUENCE_FP32 or PME_INFLUENCE_TENSOR");
    if (path == PME_INFLUENCE_TENSOR && pl->K[0] != 128)
        return fail(PME_EUNSUPPORTED, "the tensor-core influence stage needs K1 = 128 (K1 is %d)", pl->K[0]);
    DeviceGuard g(pl->dev);
    if (path == PME_INFLUENCE_TENSOR && !pl->tc_w) {
        std::vector<uint8_t> img;
        make_tc_w_image(img);
        cudaError_t e = lib_malloc(&pl->tc_w, img.size());
        if (e != cudaSuccess) {
            pl->tc_w = nullptr;
            return cuda_fail(e, "cudaMalloc(DFT-matrix image)");
        }
        if ((e = cudaMemcpy(pl->tc_w, img.data(), img.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpy(DFT-matrix image)");
    }
    cudaError_t e = cudaStreamSynchronize(pl->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    pl->influence_path = path;
    ++pl->gen;  // recorded graphs hold the other stage
    return PME_OK;
}

int pme_get_influence_path(const pme_plan *pl) { return pl ? pl->influence_path : -1; }

pme_status pme_set_launch_mode(int mode) {
    if (mode < 0 || mode > 3) return fail(PME_EINVAL, "launch mode must be 0, 1, 2 or 3");
    set_launch_mode(mode);
    return PME_OK;
}

pme_status pme_set_slab_split(int fwd_ctas, int inv_ctas) {
    if (set_slab_split(fwd_ctas, inv_ctas) != 0) return fail(PME_EINVAL, "slab split must be 1, 2 or 4 CTAs");
    return PME_OK;
}

size_t pme_plan_device_bytes(const pme_plan *pl) {
    if (!pl) return 0;
    size_t b = pl->mesh_bytes + pl->atom_bytes;
    if (pl->host_mem) b += align256((size_t)pl->host_cap * 12) * 2 + align256((size_t)pl->host_cap * 4);
    if (pl->async_mem) b += 2 * async_slot_bytes(pl->async_cap);
    return b;
}

void pme_destroy(pme_plan *pl) {
    if (!pl) return;
    DeviceGuard g(pl->dev);
    cudaStreamSynchronize(pl->stream);
    if (pl->g_dev.exec) cudaGraphExecDestroy(pl->g_dev.exec);
    if (pl->g_host.exec) cudaGraphExecDestroy(pl->g_host.exec);
    if (pl->g_md.exec) cudaGraphExecDestroy(pl->g_md.exec);
    for (pme_plan::EvalGraph &gr : pl->g_async)
        if (gr.exec) cudaGraphExecDestroy(gr.exec);
    if (pl->md_mem) cudaFree(pl->md_mem);
    if (pl->tc_w) cudaFree(pl->tc_w);
    if (pl->rec_stream) cudaStreamDestroy(pl->rec_stream);
    for (cudaStream_t cs : {pl->copy_stream, pl->out_stream})
        if (cs) {
            cudaStreamSynchronize(cs);
            cudaStreamDestroy(cs);
        }
    for (int s = 0; s < 2; ++s)
        for (cudaEvent_t ev : {pl->in_ready[s], pl->in_free[s], pl->out_done[s]})
            if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : pl->host_done)
        if (ev) cudaEventDestroy(ev);
    if (pl->async_mem) cudaFree(pl->async_mem);
    if (pl->mesh_mem) cudaFree(pl->mesh_mem);
    if (pl->atom_mem) cudaFree(pl->atom_mem);
    if (pl->host_mem) cudaFree(pl->host_mem);
    if (pl->h_ctl) cudaFreeHost(pl->h_ctl);
    delete pl;
}

}  // extern "C"
