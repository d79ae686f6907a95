// Batched evaluation of many independent systems in ONE persistent kernel launch.
//
// A host-built work list holds, stage by stage, the work items of every system: all binning items of all
// systems, then all spreading items, and so on. CTAs take list entries in order with one atomic; an
// entry waits until its system's previous stage has finished every item, so different systems overlap
// freely (one system's FFT runs beside another's spreading) and the only barriers are per system. Each
// entry depends only on entries earlier in the list, all of them already taken by running CTAs, so the
// launch makes progress whatever number of CTAs is resident. Waits are bounded: past the deadline a wait
// sets an error bit and an abort flag, and every later wait returns at once, so a launch always ends.
// The last CTA to leave resets every counter, which lets a CUDA graph replay the launch.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <tuple>
#include <vector>

#include "../../include/pme.h"
#include "batch_internal.h"
#include "group.h"
#include "host_tables.h"
#include "kernels.h"
#include "plan_internal.h"
#include "stages.cuh"

namespace pme {

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait (thread 0 of the CTA) until *counter >= target; false if the wait gave up or the launch aborted.
__device__ bool bounded_wait(const unsigned *counter, unsigned target, BatchCtrl *ctrl, unsigned long long limit_ns) {
    if (ld_acquire(counter) >= target) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (true) {
        if (ld_acquire(&ctrl->abort)) return false;
        if (ld_acquire(counter) >= target) return true;
        if (globaltimer_ns() - t0 > limit_ns) {
            atomicExch(&ctrl->abort, 1u);
            return false;
        }
        __nanosleep(200);
    }
}

// Each stage is a separate (not inlined) call, so the register allocation of one stage does not inflate
// the others and the persistent kernel keeps the occupancy of its most demanding stage.
__device__ __noinline__ void call_bin(const SysDev &d, int item, void *smem) { stage_bin(d, item, smem); }
template <int P>
__device__ __noinline__ void call_spread(const SysDev &d, int item, void *smem) {
    if (d.tlog == 4) stage_spread<P, 16>(d, item, smem);
    else stage_spread<P, 8>(d, item, smem);
}
__device__ __noinline__ void call_fwd(const SysDev &d, int item, void *smem) { stage_fwd(d, item, smem); }
__device__ __noinline__ void call_conv(const SysDev &d, int item, void *smem) { stage_conv(d, item, smem); }
__device__ __noinline__ void call_inv(const SysDev &d, int item, void *smem) { stage_inv(d, item, smem); }
template <int P>
__device__ __noinline__ void call_gather(const SysDev &d, int item, void *smem) {
    if (d.tlog == 4) stage_gather<P, 16>(d, item, smem);
    else stage_gather<P, 8>(d, item, smem);
}

// One kernel for every order: the order-specific stages dispatch on the system's p, and the other stage
// calls are compiled once.
__device__ __forceinline__ void run_stage(const SysDev &d, int stage, int item, void *smem) {
    switch (stage) {
        case STAGE_BIN: call_bin(d, item, smem); break;
        case STAGE_SPREAD:
            if (d.p == 4) call_spread<4>(d, item, smem);
            else if (d.p == 5) call_spread<5>(d, item, smem);
            else if (d.p == 6) call_spread<6>(d, item, smem);
            else call_spread<8>(d, item, smem);
            break;
        case STAGE_FWD: call_fwd(d, item, smem); break;
        case STAGE_CONV: call_conv(d, item, smem); break;
        case STAGE_INV: call_inv(d, item, smem); break;
        default:
            if (d.p == 4) call_gather<4>(d, item, smem);
            else if (d.p == 5) call_gather<5>(d, item, smem);
            else if (d.p == 6) call_gather<6>(d, item, smem);
            else call_gather<8>(d, item, smem);
            break;
    }
}

__global__ void __launch_bounds__(NT_BATCH, 4) k_batch(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SysDev sd;
    __shared__ int s_entry, s_ok;
    const int tid = threadIdx.x;
    while (true) {
        if (tid == 0) s_entry = (int)atomicAdd(&a.ctrl->head, 1u);
        __syncthreads();
        const int e = s_entry;
        if (e >= a.nentries) break;
        const BatchEntry w = a.entries[e];
        const int sys = w.sys, stage = w.stage;
        if (tid < (int)(sizeof(SysDev) / 4)) ((int *)&sd)[tid] = ((const int *)(a.sys + sys))[tid];
        if (tid == 0) {
            bool ok = true;
            if (stage > 0) {
                unsigned target = a.count[sys * NUM_STAGES + stage - 1];
                if (a.stall_entry == e) target += 1u;  // test hook: a dependency nothing completes
                ok = bounded_wait(&a.done[sys * NUM_STAGES + stage - 1], target, a.ctrl, a.wait_ns);
            }
            s_ok = ok;
            if (!ok) atomicOr(&a.sys[sys].ctl->status, ST_TIMEOUT);
        }
        __syncthreads();
        if (s_ok) {
            for (int it = w.begin; it < w.end; ++it) {
                run_stage(sd, stage, it, smem);
                __syncthreads();
            }
        }
        if (tid == 0) {
            __threadfence();
            atomicAdd(&a.done[sys * NUM_STAGES + stage], (unsigned)(w.end - w.begin));
        }
        __syncthreads();
    }
    // the last CTA out resets every counter for the next launch (all entries are finished by then)
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&a.ctrl->exited, 1u) == gridDim.x - 1u) {
            for (int i = 0; i < a.nsys * NUM_STAGES; ++i) a.done[i] = 0u;
            a.ctrl->head = 0u;
            a.ctrl->abort = 0u;
            __threadfence();
            a.ctrl->exited = 0u;
        }
    }
}

// ---------------------------------------------------------------------------------------------------------
// host side

int stage_items(const SysDev &d, int stage) {
    switch (stage) {
        case STAGE_BIN: return d.nbin;
        case STAGE_SPREAD: return d.ntiles + OVF_ITEMS;
        case STAGE_FWD: return d.K1;
        case STAGE_CONV: return d.nconv;
        case STAGE_INV: return d.K1;
        default: return d.ntiles + OVF_ITEMS;
    }
}

// items of one stage grouped per list entry (fewer, larger entries for the many small tile items)
static int stage_group(int stage) {
    return (stage == STAGE_SPREAD || stage == STAGE_GATHER) ? 4 : (stage == STAGE_CONV ? 2 : 1);
}

void build_work_list(const std::vector<SysDev> &sys, std::vector<BatchEntry> &entries, std::vector<unsigned> &count) {
    entries.clear();
    count.assign(sys.size() * NUM_STAGES, 0u);
    for (int stage = 0; stage < NUM_STAGES; ++stage)
        for (size_t s = 0; s < sys.size(); ++s) {
            const int n = stage_items(sys[s], stage), g = stage_group(stage);
            count[s * NUM_STAGES + stage] = (unsigned)n;
            for (int b = 0; b < n; b += g) {
                BatchEntry e;
                e.sys = (unsigned short)s;
                e.stage = (unsigned short)stage;
                e.begin = b;
                e.end = std::min(n, b + g);
                entries.push_back(e);
            }
        }
}

size_t batch_smem(const std::vector<SysDev> &sys) {
    size_t m = smem_bin(NT_BATCH);
    for (const SysDev &d : sys) {
        m = std::max(m, smem_spread(d.p, d.tlog));
        m = std::max(m, smem_gather_all(d.p, d.tlog));
        m = std::max(m, smem_slab(d.K2, d.K3));
        m = std::max(m, smem_inv(d.K2, d.K3));
        m = std::max(m, smem_conv(d.K1, NT_BATCH));
    }
    return m;
}

cudaError_t configure_batch_kernel() {
    return cudaFuncSetAttribute((const void *)k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(MAX_SMEM_BYTES - sizeof(SysDev) - 64));
}

int batch_grid(int dev, int p, size_t smem) {
    (void)p;
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k_batch, NT_BATCH, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return sms * per_sm;
}

cudaError_t launch_batch(const BatchArgs &a, int p, int grid, size_t smem, cudaStream_t s) {
    (void)p;
    k_batch<<<grid, NT_BATCH, smem, s>>>(a);
    return cudaGetLastError();
}

// first list entry that waits on a dependency (for the stall test hook)
int first_waiting_entry(const std::vector<BatchEntry> &entries) {
    for (size_t i = 0; i < entries.size(); ++i)
        if (entries[i].stage > 0) return (int)i;
    return -1;
}

// Device state of one persistent launch over up to cap_sys systems and cap_entries list entries.
pme_status WaveState::init(int dev_, int cap_sys_, size_t cap_entries_) {
    dev = dev_;
    cap_sys = cap_sys_;
    cap_entries = cap_entries_;
    size_t off = 0;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_sys = off;  off = al(off + sizeof(SysDev) * cap_sys);
    const size_t o_cnt = off;  off = al(off + sizeof(unsigned) * cap_sys * NUM_STAGES);
    const size_t o_ent = off;  off = al(off + sizeof(BatchEntry) * cap_entries);
    const size_t o_done = off; off = al(off + sizeof(unsigned) * cap_sys * NUM_STAGES);
    const size_t o_ctrl = off; off = al(off + sizeof(BatchCtrl));
    const size_t o_ev = off;   off = al(off + sizeof(double) * 8 * cap_sys);
    const size_t o_st = off;   off = al(off + sizeof(unsigned) * cap_sys);
    cudaError_t e = lib_malloc(&dmem, off);
    if (e != cudaSuccess) {
        dmem = nullptr;
        return fail(PME_ENOMEM, "cudaMalloc(%zu bytes) for a batch: %s", off, cudaGetErrorString(e));
    }
    if ((e = cudaMemset(dmem, 0, off)) != cudaSuccess) return cuda_fail(e, "cudaMemset(batch state)");
    if ((e = lib_malloc_host(&hmem, off)) != cudaSuccess) {
        hmem = nullptr;
        return cuda_fail(e, "cudaMallocHost(batch staging)");
    }
    memset(hmem, 0, off);
    bytes = off;
    char *b = (char *)dmem, *h = (char *)hmem;
    d_sys = (SysDev *)(b + o_sys);
    h_sys = (SysDev *)(h + o_sys);
    d_entries = (BatchEntry *)(b + o_ent);
    h_entries = (BatchEntry *)(h + o_ent);
    d_count = (unsigned *)(b + o_cnt);
    h_count = (unsigned *)(h + o_cnt);
    d_done = (unsigned *)(b + o_done);
    d_ctrl = (BatchCtrl *)(b + o_ctrl);
    d_ev = (double *)(b + o_ev);
    h_ev = (double *)(h + o_ev);
    d_status = (unsigned *)(b + o_st);
    h_status = (unsigned *)(h + o_st);
    head_bytes = o_ent;  // descriptors and counts; the used part of the list follows at o_ent
    return PME_OK;
}

void WaveState::release() {
    if (dmem) cudaFree(dmem);
    if (hmem) cudaFreeHost(hmem);
    dmem = hmem = nullptr;
}

cudaError_t WaveState::upload(size_t nentries, cudaStream_t s) const {
    cudaError_t e = cudaMemcpyAsync(dmem, hmem, head_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nentries)
        e = cudaMemcpyAsync(d_entries, h_entries, sizeof(BatchEntry) * nentries, cudaMemcpyHostToDevice, s);
    return e;
}

BatchArgs WaveState::args(int nsys, int nentries, unsigned long long wait_ns, int stall_entry) const {
    BatchArgs a;
    a.sys = d_sys;
    a.entries = d_entries;
    a.count = d_count;
    a.done = d_done;
    a.ctrl = d_ctrl;
    a.nsys = nsys;
    a.nentries = nentries;
    a.wait_ns = wait_ns;
    a.stall_entry = stall_entry;
    return a;
}

// Status words of every system in the wave -> h_status (device kernel, so it can sit in a graph).
__global__ void k_collect_status(const SysDev *sys, int nsys, unsigned *out) {
    for (int s = threadIdx.x; s < nsys; s += blockDim.x) {
        out[s] = sys[s].ctl->status;
        sys[s].ctl->status = 0u;
    }
}

cudaError_t launch_collect_status(const SysDev *sys, int nsys, unsigned *out, cudaStream_t s) {
    k_collect_status<<<1, 128, 0, s>>>(sys, nsys, out);
    return cudaGetLastError();
}

// Reset the resident state of a plan after an aborted launch (counters, buckets, the int64 mesh).
pme_status plan_recover(pme_plan *pl, cudaStream_t s) {
    SysDev &d = pl->d;
    cudaError_t e;
    if ((e = cudaMemsetAsync(d.grid, 0, (size_t)d.K1 * d.K2 * d.K3 * 8, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(d.bcount, 0, bcount_bytes(d.ntiles), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(d.ctl, 0, sizeof(Ctl), s)) != cudaSuccess)
        return cuda_fail(e, "cudaMemsetAsync(recover)");
    return PME_OK;
}

}  // namespace pme

using namespace pme;

struct pme_batch {
    int dev = 0;
    cudaStream_t stream = nullptr;
    std::vector<pme_plan *> plans;
    std::vector<int64_t> n, off;
    std::vector<SysDev> sys;
    std::vector<BatchEntry> entries;
    std::vector<unsigned> count;
    WaveState wave;
    size_t smem = 0;
    int grid = 0;
    // Grouped execution (the default): systems of one mesh shape form a group, evaluated by a chain of six
    // grouped stage launches; the chains run as parallel branches of the graph. order lists the systems
    // group by group; d_gsys / h_gsys hold their descriptors in that order.
    struct Group {
        int first, count, max_nbin;
    };
    std::vector<int> order;
    std::vector<Group> groups;
    SysDev *d_gsys = nullptr, *h_gsys = nullptr;
    std::vector<cudaStream_t> gstreams;
    std::vector<cudaEvent_t> gevents;
    // graph of the whole evaluation (descriptor upload, the stages, status collection) for the last
    // pointer set and mode
    cudaGraphExec_t exec = nullptr;
    const void *g_pos = nullptr, *g_q = nullptr, *g_forces = nullptr, *g_ev = nullptr;
    int stall = 0;
    int64_t stall_ns = 0;
    int strategy = PME_BATCH_AUTO;  // pme_batch_set_strategy
    int g_persistent = -1;          // whether the recorded graph is the persistent launch
    std::vector<unsigned long long> plan_gen;  // each plan's generation when its descriptor was taken
};

// The persistent work-list kernel runs when asked for, while the stall hook is on (its bounded waits are
// what that hook exercises), or when the systems cannot be grouped; otherwise the grouped stage chains.
static bool batch_use_persistent(const pme_batch *b) {
    return b->stall || b->groups.empty() || b->strategy == PME_BATCH_PERSISTENT;
}

// Grouped evaluation: one chain of six grouped stage launches per mesh shape, the chains as parallel branches.
static pme_status batch_record_grouped(pme_batch *b, const float *pos, const float *q, float *forces, double *ev_dev) {
    const int nsys = (int)b->sys.size();
    for (int i = 0; i < nsys; ++i) {
        const int s = b->order[i];
        SysDev d = b->sys[s];
        d.pos = pos + 3 * b->off[s];
        d.q = q + b->off[s];
        d.forces = forces + 3 * b->off[s];
        d.ev = ev_dev + 7 * s;
        b->h_gsys[i] = d;
    }
    cudaError_t e;
    if ((e = cudaMemcpyAsync(b->d_gsys, b->h_gsys, sizeof(SysDev) * nsys, cudaMemcpyHostToDevice, b->stream)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync(batch descriptors)");
    const int G = (int)b->groups.size();
    if ((e = cudaEventRecord(b->gevents[G], b->stream)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    for (int g = 0; g < G; ++g) {
        const pme_batch::Group &gr = b->groups[g];
        cudaStream_t gs = b->gstreams[g];
        if ((e = cudaStreamWaitEvent(gs, b->gevents[G], 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
        if ((e = launch_group_chain(b->d_gsys + gr.first, gr.count, b->h_gsys[gr.first], gr.max_nbin, gs)) != cudaSuccess)
            return cuda_fail(e, "grouped stage launch");
        if ((e = cudaEventRecord(b->gevents[g], gs)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        if ((e = cudaStreamWaitEvent(b->stream, b->gevents[g], 0)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamWaitEvent");
    }
    if ((e = launch_collect_status(b->d_gsys, nsys, b->wave.d_status, b->stream)) != cudaSuccess)
        return cuda_fail(e, "status kernel launch");
    return PME_OK;
}

// Group the systems by mesh shape, order and tile edge (a group shares its kernels and CTA shape).
static bool batch_make_groups(pme_batch *b) {
    const int nsys = (int)b->sys.size();
    std::vector<int> idx(nsys);
    for (int s = 0; s < nsys; ++s) idx[s] = s;
    auto key = [&](int s) {
        const SysDev &d = b->sys[s];
        return std::make_tuple(d.K1, d.K2, d.K3, d.p, d.tlog);
    };
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return key(x) < key(y); });
    b->order = idx;
    b->groups.clear();
    for (int i = 0; i < nsys; ++i) {
        const SysDev &d = b->sys[idx[i]];
        if (i == 0 || key(idx[i]) != key(idx[i - 1])) b->groups.push_back({i, 0, 0});
        pme_batch::Group &g = b->groups.back();
        ++g.count;
        g.max_nbin = std::max(g.max_nbin, d.nbin);
    }
    return true;
}

static void batch_release_groups(pme_batch *b) {
    for (cudaStream_t s : b->gstreams) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->gevents) cudaEventDestroy(e);
    b->gstreams.clear();
    b->gevents.clear();
    if (b->d_gsys) cudaFree(b->d_gsys);
    if (b->h_gsys) cudaFreeHost(b->h_gsys);
    b->d_gsys = b->h_gsys = nullptr;
    b->groups.clear();
}

static pme_status batch_init_groups(pme_batch *b) {
    if (!batch_make_groups(b)) return PME_OK;  // stays on the persistent path
    const int nsys = (int)b->sys.size(), G = (int)b->groups.size();
    cudaError_t e;
    if ((e = configure_group_kernels()) != cudaSuccess) return cuda_fail(e, "configure grouped kernels");
    if ((e = lib_malloc((void **)&b->d_gsys, sizeof(SysDev) * nsys)) != cudaSuccess) {
        b->d_gsys = nullptr;
        return fail(PME_ENOMEM, "cudaMalloc(batch descriptors): %s", cudaGetErrorString(e));
    }
    if ((e = lib_malloc_host((void **)&b->h_gsys, sizeof(SysDev) * nsys)) != cudaSuccess) {
        b->h_gsys = nullptr;
        return cuda_fail(e, "cudaMallocHost(batch descriptors)");
    }
    for (int g = 0; g < G; ++g) {
        cudaStream_t s;
        if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
        b->gstreams.push_back(s);
    }
    for (int g = 0; g <= G; ++g) {  // one per group, then the fork
        cudaEvent_t ev;
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
        b->gevents.push_back(ev);
    }
    return PME_OK;
}

// Re-read the plans' descriptors when any plan changed since the batch took them (a new cell from
// pme_set_box, a new tiling from the autotuner or pme_plan_set_tiling): work list, groups and graph follow.
static pme_status batch_refresh(pme_batch *b) {
    bool stale = false;
    for (size_t s = 0; s < b->plans.size(); ++s) stale = stale || b->plans[s]->gen != b->plan_gen[s];
    if (!stale) return PME_OK;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    pme_status st;
    for (size_t s = 0; s < b->plans.size(); ++s) {
        pme_plan *pl = b->plans[s];
        if ((st = plan_reserve(pl, b->n[s])) != PME_OK) return st;
        b->sys[s] = plan_descriptor(pl, nullptr, nullptr, b->n[s], nullptr, nullptr);
        if (b->plans.size() > 1) shared_tiling(b->sys[s]);
        b->plan_gen[s] = pl->gen;
    }
    build_work_list(b->sys, b->entries, b->count);
    if (b->entries.size() > b->wave.cap_entries) {
        b->wave.release();
        if ((st = b->wave.init(b->dev, (int)b->sys.size(), b->entries.size())) != PME_OK) return st;
    }
    b->smem = batch_smem(b->sys);
    b->grid = batch_grid(b->dev, b->sys[0].p, b->smem);
    batch_release_groups(b);
    if ((st = batch_init_groups(b)) != PME_OK) return st;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    return PME_OK;
}

static pme_status batch_record(pme_batch *b, const float *pos, const float *q, float *forces, double *ev_dev) {
    const int nsys = (int)b->sys.size();
    for (int s = 0; s < nsys; ++s) {
        SysDev d = b->sys[s];
        d.pos = pos + 3 * b->off[s];
        d.q = q + b->off[s];
        d.forces = forces + 3 * b->off[s];
        d.ev = ev_dev + 7 * s;
        b->wave.h_sys[s] = d;
    }
    memcpy(b->wave.h_entries, b->entries.data(), sizeof(BatchEntry) * b->entries.size());
    memcpy(b->wave.h_count, b->count.data(), sizeof(unsigned) * b->count.size());
    cudaError_t e;
    if ((e = b->wave.upload(b->entries.size(), b->stream)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync(batch descriptors)");
    const int stall_entry = b->stall ? first_waiting_entry(b->entries) : -1;
    const unsigned long long wait_ns = b->stall ? (unsigned long long)b->stall_ns : 1000000000ull;
    BatchArgs a = b->wave.args(nsys, (int)b->entries.size(), wait_ns, stall_entry);
    if ((e = launch_batch(a, b->sys[0].p, b->grid, b->smem, b->stream)) != cudaSuccess)
        return cuda_fail(e, "persistent kernel launch");
    if ((e = launch_collect_status(b->wave.d_sys, nsys, b->wave.d_status, b->stream)) != cudaSuccess)
        return cuda_fail(e, "status kernel launch");
    return PME_OK;
}

extern "C" {

pme_status pme_batch_create(int nsys, pme_plan *const *plans, const int64_t *n, void *cuda_stream, pme_batch **out) {
    if (!out) return fail(PME_EINVAL, "out is NULL");
    *out = nullptr;
    if (nsys < 1 || nsys > 4096 || !plans || !n) return fail(PME_EINVAL, "need 1..4096 systems, plans and n");
    pme_batch *b = lib_new<pme_batch>();
    if (!b) return fail(PME_ENOMEM, "host allocation failed");
    b->stream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&b->dev);
    int64_t off = 0;
    for (int s = 0; s < nsys; ++s) {
        pme_plan *pl = plans[s];
        if (!pl || n[s] < 0 || n[s] > (int64_t)0x3fffffff) {
            delete b;
            return fail(PME_EINVAL, "system %d: NULL plan or n out of range", s);
        }
        if (pl->dev != b->dev) {
            const int bdev = b->dev;
            delete b;
            return fail(PME_EINVAL, "system %d: plan lives on device %d, batch on %d", s, pl->dev, bdev);
        }
        if (pl->p != plans[0]->p) {
            delete b;
            return fail(PME_EINVAL, "system %d has B-spline order %d, system 0 has %d: one order per batch", s, pl->p,
                        plans[0]->p);
        }
        for (int t = 0; t < s; ++t)
            if (plans[t] == pl) {
                delete b;
                return fail(PME_EINVAL, "systems %d and %d share a plan; each system needs its own", t, s);
            }
        pme_status st = plan_reserve(pl, n[s]);
        if (st != PME_OK) {
            delete b;
            return st;
        }
        b->plans.push_back(pl);
        b->n.push_back(n[s]);
        b->off.push_back(off);
        b->sys.push_back(plan_descriptor(pl, nullptr, nullptr, n[s], nullptr, nullptr));
        if (nsys > 1) shared_tiling(b->sys.back());
        b->plan_gen.push_back(pl->gen);
        off += n[s];
    }
    build_work_list(b->sys, b->entries, b->count);
    pme_status st = b->wave.init(b->dev, nsys, b->entries.size());
    if (st != PME_OK) {
        b->wave.release();
        delete b;
        return st;
    }
    cudaError_t e = configure_batch_kernel();
    if (e != cudaSuccess) {
        b->wave.release();
        delete b;
        return cuda_fail(e, "configure persistent kernel");
    }
    b->smem = batch_smem(b->sys);
    b->grid = batch_grid(b->dev, b->sys[0].p, b->smem);
    if ((st = batch_init_groups(b)) != PME_OK) {
        batch_release_groups(b);
        b->wave.release();
        delete b;
        return st;
    }
    *out = b;
    return PME_OK;
}

pme_status pme_batch_enqueue(pme_batch *b, const float *pos, const float *q, float *forces, double *ev_dev) {
    if (!b) return fail(PME_EINVAL, "batch is NULL");
    if (!ev_dev) return fail(PME_EINVAL, "ev_dev must be non-NULL");
    int64_t ntot = b->off.back() + b->n.back();
    if (ntot > 0 && (!pos || !q || !forces)) return fail(PME_EINVAL, "pos, q and forces must be non-NULL");
    DeviceGuard g(b->dev);
    pme_status rst = batch_refresh(b);
    if (rst != PME_OK) return rst;
    cudaError_t e;
    const bool persistent = batch_use_persistent(b);
    if (!b->exec || b->g_pos != pos || b->g_q != q || b->g_forces != forces || b->g_ev != ev_dev ||
        b->g_persistent != (int)persistent) {
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        // capture on a private stream so the caller's stream may itself be capturing or busy
        cudaStream_t cs;
        if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
        cudaStream_t keep = b->stream;
        b->stream = cs;
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        pme_status st = PME_OK;
        if (e == cudaSuccess)
            st = persistent ? batch_record(b, pos, q, forces, ev_dev) : batch_record_grouped(b, pos, q, forces, ev_dev);
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        b->stream = keep;
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
        if (st != PME_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            return cuda_fail(e, "cudaGraphInstantiate");
        }
        b->g_pos = pos;
        b->g_q = q;
        b->g_forces = forces;
        b->g_ev = ev_dev;
        b->g_persistent = (int)persistent;
    }
    if ((e = cudaGraphLaunch(b->exec, b->stream)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return PME_OK;
}

pme_status pme_batch_sync(pme_batch *b) {
    if (!b) return fail(PME_EINVAL, "batch is NULL");
    DeviceGuard g(b->dev);
    const int nsys = (int)b->sys.size();
    cudaError_t e;
    if ((e = cudaMemcpyAsync(b->wave.h_status, b->wave.d_status, sizeof(unsigned) * nsys, cudaMemcpyDeviceToHost,
                             b->stream)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync(status)");
    if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    unsigned bits = 0;
    for (int s = 0; s < nsys; ++s) bits |= b->wave.h_status[s];
    if (bits & ST_TIMEOUT) {
        // an aborted launch skipped work whose consumers reset resident state: restore it
        for (pme_plan *pl : b->plans) plan_recover(pl, b->stream);
        cudaStreamSynchronize(b->stream);
    }
    memset(b->wave.h_status, 0, sizeof(unsigned) * nsys);
    cudaMemsetAsync(b->wave.d_status, 0, sizeof(unsigned) * nsys, b->stream);
    return status_from_bits(bits);
}

pme_status pme_batch_set_strategy(pme_batch *b, int strategy) {
    if (!b) return fail(PME_EINVAL, "batch is NULL");
    if (strategy != PME_BATCH_AUTO && strategy != PME_BATCH_GROUPED && strategy != PME_BATCH_PERSISTENT)
        return fail(PME_EINVAL, "strategy must be PME_BATCH_AUTO, PME_BATCH_GROUPED or PME_BATCH_PERSISTENT");
    if (strategy == PME_BATCH_GROUPED && b->groups.empty())
        return fail(PME_EUNSUPPORTED, "these systems cannot be grouped (a plan uses 16^3 tiles)");
    b->strategy = strategy;  // the next enqueue re-records the graph if the choice changed
    return PME_OK;
}

int pme_batch_get_strategy(const pme_batch *b) {
    if (!b) return -1;
    return batch_use_persistent(b) ? PME_BATCH_PERSISTENT : PME_BATCH_GROUPED;
}

pme_status pme_batch_autotune(pme_batch *b, const float *pos, const float *q, float *forces, double *ev_dev, int reps,
                              int *strategy, double *us_per_batch) {
    if (!b) return fail(PME_EINVAL, "batch is NULL");
    if (reps < 1 || reps > 100000) return fail(PME_EINVAL, "reps must be in [1, 100000]");
    const int64_t ntot = b->off.back() + b->n.back();
    if (!ev_dev || (ntot > 0 && (!pos || !q || !forces))) return fail(PME_EINVAL, "pos, q, forces and ev_dev must be non-NULL");
    DeviceGuard g(b->dev);
    const int nsys = (int)b->sys.size();
    struct Cand {
        int strategy, nt;
        double us;
        bool same;
    };
    std::vector<Cand> cands = {{PME_BATCH_GROUPED, 0, 0.0, true}, {PME_BATCH_GROUPED, 128, 0.0, false},
                               {PME_BATCH_GROUPED, 256, 0.0, false}, {PME_BATCH_PERSISTENT, 0, 0.0, false}};
    std::vector<float> F0((size_t)(ntot > 0 ? ntot : 1) * 3), F1(F0.size());
    std::vector<double> ev0((size_t)nsys * 7), ev1(ev0.size());
    cudaEvent_t ea, eb;
    cudaEventCreate(&ea);
    cudaEventCreate(&eb);
    pme_status st = PME_OK;
    auto apply = [&](const Cand &c) -> pme_status {
        for (int s = 0; s < nsys; ++s) {
            pme_status r = plan_retile(b->plans[s], 3, c.nt, b->n[s]);
            if (r != PME_OK) return r;
        }
        b->strategy = c.strategy;
        return PME_OK;
    };
    for (size_t c = 0; c < cands.size() && st == PME_OK; ++c) {
        if ((st = apply(cands[c])) != PME_OK) break;
        if ((st = pme_batch_enqueue(b, pos, q, forces, ev_dev)) != PME_OK || (st = pme_batch_sync(b)) != PME_OK) break;
        std::vector<float> &F = c == 0 ? F0 : F1;
        std::vector<double> &ev = c == 0 ? ev0 : ev1;
        cudaError_t e = cudaMemcpy(F.data(), forces, (size_t)ntot * 12, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(ev.data(), ev_dev, ev.size() * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "cudaMemcpy(tuning results)");
            break;
        }
        if (c > 0)
            cands[c].same = memcmp(F0.data(), F1.data(), (size_t)ntot * 12) == 0 &&
                            memcmp(ev0.data(), ev1.data(), ev0.size() * sizeof(double)) == 0;
        if (!cands[c].same) continue;
        for (int i = 0; i < 2 && st == PME_OK; ++i) st = pme_batch_enqueue(b, pos, q, forces, ev_dev);
        if (st != PME_OK) break;
        cudaEventRecord(ea, b->stream);
        for (int i = 0; i < reps && st == PME_OK; ++i) st = pme_batch_enqueue(b, pos, q, forces, ev_dev);
        cudaEventRecord(eb, b->stream);
        if (st != PME_OK || (st = pme_batch_sync(b)) != PME_OK) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ea, eb);
        cands[c].us = 1000.0 * ms / reps;
    }
    cudaEventDestroy(ea);
    cudaEventDestroy(eb);
    if (st != PME_OK) return st;
    size_t best = 0;
    for (size_t c = 1; c < cands.size(); ++c)
        if (cands[c].same && cands[c].us < cands[best].us) best = c;
    if ((st = apply(cands[best])) != PME_OK) return st;
    if (strategy) *strategy = cands[best].strategy;
    if (us_per_batch) *us_per_batch = cands[best].us;
    return PME_OK;
}

pme_status pme_batch_debug_stall(pme_batch *b, int enable, int64_t wait_limit_ns) {
    if (!b) return fail(PME_EINVAL, "batch is NULL");
    if (enable && (wait_limit_ns <= 0 || wait_limit_ns > 2000000000ll))
        return fail(PME_EINVAL, "wait_limit_ns must be in (0, 2e9]");
    b->stall = enable ? 1 : 0;
    b->stall_ns = wait_limit_ns;
    if (b->exec) {  // re-record with the new setting on the next enqueue
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    return PME_OK;
}

void pme_batch_destroy(pme_batch *b) {
    if (!b) return;
    DeviceGuard g(b->dev);
    cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    batch_release_groups(b);
    b->wave.release();
    delete b;
}

}  // extern "C"
