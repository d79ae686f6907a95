// Device-resident multi-step loop: M time steps of (reciprocal-space SPME forces [+ real-space forces] ->
// leapfrog update of velocities and positions) with no host round trip between steps, the way the paper's
// long-range pipeline runs "multiple timesteps" on its FPGAs without host communication beyond
// initialization and result collection (Sec. III). One chunk of steps is recorded once as a CUDA graph and
// replayed; a device-side step counter tells each step's update kernel where to store that step's energies,
// so every chunk replays the same graph.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "../../include/pme.h"
#include "kernels.h"
#include "plan_internal.h"

namespace pme {

constexpr int MD_CHUNK = 32;   // steps per recorded graph
constexpr int MD_EV = 15;      // doubles per step in ev_steps: E_rec, virial_rec[6], E_real, E_self, virial_real[6]
constexpr size_t MD_MEM = 256; // counter (16 B) + real-space energies (8 doubles), padded

struct LeapArgs {
    float *pos, *vel;
    const float *forces, *inv_mass;
    int n;
    float dt;
    const double *ev_rec;   // the plan's energy / virial of this step (7 doubles)
    const double *ev_real;  // the real-space energies of this step (8 doubles) or null
    double *ev_steps;       // steps x MD_EV or null
    unsigned *counter;      // steps completed in this call
    int steps;
};

// v += (F / m) dt, x += v dt, each product and sum rounded once in FP32 (so a host loop of the same
// operations reproduces the trajectory bit for bit); block 0 files the step's energies and advances the
// step counter.
__global__ void __launch_bounds__(256) k_leapfrog(LeapArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.n) {
        const float im = a.inv_mass ? a.inv_mass[i] : 1.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const size_t j = 3 * (size_t)i + k;
            const float v = __fadd_rn(a.vel[j], __fmul_rn(__fmul_rn(a.forces[j], im), a.dt));
            a.vel[j] = v;
            a.pos[j] = __fadd_rn(a.pos[j], __fmul_rn(v, a.dt));
        }
    }
    if (blockIdx.x == 0) {
        __shared__ unsigned step;
        if (threadIdx.x == 0) step = *a.counter;
        __syncthreads();
        if (a.ev_steps && step < (unsigned)a.steps && threadIdx.x < MD_EV) {
            const int t = threadIdx.x;
            double v = 0.0;
            if (t < 7) v = a.ev_rec[t];
            else if (a.ev_real) v = a.ev_real[t - 7];
            a.ev_steps[(size_t)step * MD_EV + t] = v;
        }
        __syncthreads();
        if (threadIdx.x == 0) *a.counter = step + 1u;
    }
}

static cudaError_t launch_leapfrog(const LeapArgs &a, cudaStream_t s) {
    const unsigned g = (unsigned)(a.n > 0 ? (a.n + 255) / 256 : 1);
    k_leapfrog<<<g, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pme

using namespace pme;

extern "C" pme_status pme_run_steps(pme_plan *pl, pme_real *rs, float *pos, float *vel, const float *q,
                                    const float *inv_mass, int64_t n, float *forces, double dt, int steps,
                                    double *ev_steps) {
    pme_status st = check_atoms(pl, pos, q, n, forces);
    if (st) return st;
    if (n > 0 && !vel) return fail(PME_EINVAL, "vel must be non-NULL when n > 0");
    if (steps < 0 || !(dt == dt) || !isfinite(dt)) return fail(PME_EINVAL, "steps must be >= 0 and dt finite");
    if (rs && real_device(rs) != pl->dev) return fail(PME_EINVAL, "the real-space context lives on another device");
    DeviceGuard g(pl->dev);
    if ((st = plan_reserve(pl, n)) != PME_OK) return st;
    if (rs && (st = real_reserve_n(rs, n)) != PME_OK) return st;
    cudaError_t e;
    if (!pl->md_mem) {
        if ((e = lib_malloc(&pl->md_mem, MD_MEM)) != cudaSuccess) {
            pl->md_mem = nullptr;
            return fail(PME_ENOMEM, "cudaMalloc(step-loop state): %s", cudaGetErrorString(e));
        }
    }
    if (steps == 0) return PME_OK;
    unsigned *counter = (unsigned *)pl->md_mem;
    double *ev_real = (double *)((char *)pl->md_mem + 16);
    if ((e = cudaMemsetAsync(pl->md_mem, 0, MD_MEM, pl->stream)) != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");

    const SysDev d = plan_descriptor(pl, pos, q, n, forces, nullptr);
    LeapArgs la;
    la.pos = pos;
    la.vel = vel;
    la.forces = forces;
    la.inv_mass = inv_mass;
    la.n = (int)n;
    la.dt = (float)dt;
    la.ev_rec = pl->d.ctl->ev;
    la.ev_real = rs ? ev_real : nullptr;
    la.ev_steps = ev_steps;
    la.counter = counter;
    la.steps = steps;
    // one step: reciprocal forces (written), real-space forces (added), the update
    auto one_step = [&](cudaStream_t s) -> cudaError_t {
        cudaError_t r = launch_pipeline(d, s);
        if (r != cudaSuccess) return r;
        if (rs && real_enqueue_on(rs, s, pos, q, n, forces, 1, ev_real) != PME_OK) return cudaErrorLaunchFailure;
        return launch_leapfrog(la, s);
    };
    const int chunk = steps < MD_CHUNK ? steps : MD_CHUNK;
    pme_plan::StepGraph key;
    key.pos = pos;
    key.vel = vel;
    key.q = q;
    key.inv_mass = inv_mass;
    key.forces = forces;
    key.ev_steps = ev_steps;
    key.rs = rs;
    key.atoms = pl->atom_mem;
    key.n = n;
    key.chunk = chunk;
    key.mode = launch_mode();
    key.dt = dt;
    key.gen = pl->gen;
    key.rs_gen = rs ? real_gen(rs) : 0ull;
    pme_plan::StepGraph &gm = pl->g_md;
    const bool same = gm.exec && gm.pos == key.pos && gm.vel == key.vel && gm.q == key.q && gm.inv_mass == key.inv_mass &&
                      gm.forces == key.forces && gm.ev_steps == key.ev_steps && gm.rs == key.rs && gm.atoms == key.atoms &&
                      gm.n == key.n && gm.chunk == key.chunk && gm.mode == key.mode && gm.dt == key.dt && gm.gen == key.gen &&
                      gm.rs_gen == key.rs_gen;
    if (!same) {
        if (gm.exec) cudaGraphExecDestroy(gm.exec);
        gm = pme_plan::StepGraph();
        if (!pl->rec_stream && (e = cudaStreamCreateWithFlags(&pl->rec_stream, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamCreate");
        if ((e = cudaStreamBeginCapture(pl->rec_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamBeginCapture");
        cudaError_t r = cudaSuccess;
        for (int i = 0; i < chunk && r == cudaSuccess; ++i) r = one_step(pl->rec_stream);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(pl->rec_stream, &graph);
        if (r != cudaSuccess || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(r != cudaSuccess ? r : e, "recording the step loop");
        }
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate(step loop)");
        gm = key;
        gm.exec = exec;
    }
    for (int done = 0; done + chunk <= steps; done += chunk)
        if ((e = cudaGraphLaunch(gm.exec, pl->stream)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch(step loop)");
    for (int i = steps - steps % chunk; i < steps; ++i)  // the remainder, launched directly
        if ((e = one_step(pl->stream)) != cudaSuccess) return cuda_fail(e, "step launch");
    return PME_OK;
}
