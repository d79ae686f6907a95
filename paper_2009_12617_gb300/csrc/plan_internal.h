// Internal definition of pme_plan and helpers shared by the plan, batch and server code.
#pragma once

#include <cuda_runtime.h>

#include <new>

#include "../../include/pme.h"
#include "common.cuh"

struct pme_plan {
    int dev = 0;
    int sms = 0;  // SMs of the device (tile edge choice)
    cudaStream_t stream = nullptr;
    int K[3] = {0, 0, 0};
    int p = 0;
    double beta = 0.0;
    double box[9] = {0};
    double recip[9] = {0};
    double vol = 0.0;
    pme::SysDev d;                  // descriptor of the resident device state (atom fields unset)
    void *mesh_mem = nullptr;       // mesh, spectrum, potential, tables, counters (fixed per plan)
    size_t mesh_bytes = 0;
    void *atom_mem = nullptr;       // tile buckets and overflow list (grows with n)
    size_t atom_bytes = 0;
    int64_t n_cap = 0;
    void *host_mem = nullptr;       // device staging for pme_compute_host
    int64_t host_cap = 0;
    pme::Ctl *h_ctl = nullptr;      // pinned host copy of the control block
    pme::Ctl *h_ctl_dev = nullptr;  // its device-side (mapped) address, or null
    unsigned long long gen = 0;     // bumped whenever the kernels' arguments change (box, tiling)
    int tile_log_set = 0;           // tile edge 2^tile_log_set chosen by the autotuner or the caller (0: default)
    int influence_path = 0;         // PME_INFLUENCE_FP32 or PME_INFLUENCE_TENSOR (single-system launches)
    void *tc_w = nullptr;           // DFT-matrix image of the tensor-core influence stage (allocated on demand)
    int tuned_apt = -1000;          // atoms-per-tile class the current tiling was tuned for (-1000: none)
    // Repeated synchronous calls replay a CUDA graph of the whole call, recorded (on a private stream, as
    // the plan stream may not be capturable) once the same arguments come twice in a row: one for device
    // arrays (pme_compute) and one for page-locked host arrays (pme_compute_host).
    struct EvalGraph {
        cudaGraphExec_t exec = nullptr;
        const void *pos = nullptr, *q = nullptr, *forces = nullptr, *atoms = nullptr, *staging = nullptr,
                   *result = nullptr;
        int64_t n = -1;
        int mode = -1;
        unsigned long long gen = ~0ull;
        bool same(const EvalGraph &o) const {
            return pos == o.pos && q == o.q && forces == o.forces && atoms == o.atoms && staging == o.staging &&
                   result == o.result && n == o.n && mode == o.mode && gen == o.gen;
        }
    };
    EvalGraph g_dev, g_host, seen_dev, seen_host;  // recorded graphs, and the previous call's arguments
    EvalGraph g_async[4];           // recorded graphs of pme_enqueue_host, most recent argument sets
    int g_async_next = 0;
    // pme_enqueue_host's input slots: two device copies of (positions, charges), filled by the copy engine on
    // copy_stream while the plan stream still runs the previous evaluation; in_ready[s] marks slot s filled,
    // in_free[s] the evaluation that read it finished
    void *async_mem = nullptr;
    int64_t async_cap = 0;
    int async_slot = 0;
    cudaStream_t copy_stream = nullptr, out_stream = nullptr;  // copies in / out
    cudaEvent_t in_ready[2] = {nullptr, nullptr}, in_free[2] = {nullptr, nullptr}, out_done[2] = {nullptr, nullptr};
    // completion of each ticket's force copy to host memory (ticket t: host_done[t % HOST_TICKETS])
    static constexpr int HOST_TICKETS = 8;
    cudaEvent_t host_done[HOST_TICKETS] = {};
    int64_t host_seq = 0;
    cudaStream_t rec_stream = nullptr;
    // multi-step loop (pme_run_steps): step counter and real-space energies, and the recorded graph of one
    // chunk of steps for the last argument set
    void *md_mem = nullptr;
    struct StepGraph {
        cudaGraphExec_t exec = nullptr;
        const void *pos = nullptr, *vel = nullptr, *q = nullptr, *inv_mass = nullptr, *forces = nullptr,
                   *ev_steps = nullptr, *rs = nullptr, *atoms = nullptr;
        int64_t n = -1;
        int chunk = 0, mode = -1;
        double dt = 0.0;
        unsigned long long gen = ~0ull, rs_gen = ~0ull;
    } g_md;
};

namespace pme {

pme_status fail(pme_status s, const char *fmt, ...);

// Every allocation of the library goes through these, so that a test can make the n-th one fail
// (pme_debug_fail_alloc): host objects, device memory and page-locked host memory.
bool alloc_injected_failure();
cudaError_t lib_malloc(void **p, size_t bytes);       // cudaMalloc
cudaError_t lib_malloc_host(void **p, size_t bytes);  // cudaMallocHost
template <class T>
T *lib_new() {
    return alloc_injected_failure() ? nullptr : new (std::nothrow) T();
}
pme_status cuda_fail(cudaError_t e, const char *what);
pme_status status_from_bits(unsigned bits);
pme_status plan_reserve(pme_plan *pl, int64_t n);
pme_status check_atoms(const pme_plan *pl, const float *pos, const float *q, int64_t n, const float *forces);
pme_status collect_status(pme_plan *pl, bool copy_ctl);
// Tile edge 2^tlog (0: default) and spread / force CTA size nt (0: density rule) for a plan; reallocates the
// per-atom buckets (for at least n atoms) when the tiling changes. Defined with the autotuner.
pme_status plan_retile(pme_plan *pl, int tlog, int nt, int64_t n);
// Real-space evaluation enqueued on a given stream (argument rules of pme_real_enqueue), its per-atom scratch
// reservation, and its device.
pme_status real_enqueue_on(pme_real *rs, cudaStream_t stream, const float *pos, const float *q, int64_t n,
                           float *forces, int accumulate, double *ev_dev);
pme_status real_reserve_n(pme_real *rs, int64_t n);
int real_device(const pme_real *rs);
unsigned long long real_gen(const pme_real *rs);  // changes whenever a recorded launch of rs would be stale
SysDev plan_descriptor(const pme_plan *pl, const float *pos, const float *q, int64_t n, float *forces, double *ev_dev);
cudaError_t ensure_configured(int dev);

class DeviceGuard {
   public:
    explicit DeviceGuard(int dev);
    ~DeviceGuard();

   private:
    int prev_ = 0, dev_ = 0;
};

}  // namespace pme
