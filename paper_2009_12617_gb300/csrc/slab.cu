// Slab decomposition of one system over P ranks: the paper's distributed long-range pipeline (Sec. III-A
// "FFT": slabs transform independently, an all-to-all "corner turn" regroups the data so each pipeline owns
// full pencils for the Green's-function multiply, a second corner turn returns it; Sec. III-C, IV-C).
//
// Rank r owns the mesh planes [plane0[r], plane0[r+1]) and the influence-stage items (half-spectrum columns)
// [item0[r], item0[r+1]). One evaluation is three calls with the caller's two all-to-alls in between:
//   stage 1: binning (all atoms), spreading into the own planes only (atoms whose support crosses into them,
//            as the paper's pipelines process every atom that affects them), forward slab transforms of the
//            own planes, and the packing of block (own planes x columns of s) for every rank s;
//   (all-to-all: rank s receives the blocks (planes of r x own columns) from every r)
//   stage 2: unpacking, the influence stage on the own columns (full k1 pencils), the rank's energy / virial
//            partial, and the packing of block (planes of s x own columns) for every rank s;
//   (all-to-all)
//   stage 3: unpacking into the own planes, inverse slab transforms, and force interpolation, which with the
//            potential zero outside the own planes gives each atom the part of its force from those planes.
// The caller sums the forces and the energy / virial partials over the ranks. Every launch goes to the
// rank's stream; nothing waits on another rank, so P ranks may also run one after another on one GPU.
#include <cuda_runtime.h>
#include <string.h>

#include "../../include/pme.h"
#include "host_tables.h"
#include "kernels.h"
#include "plan_internal.h"
#include "stages.cuh"

namespace pme {

struct SlabArgs {
    SysDev d;
    SlabLayout L;
    int rank;
    int first_pass;  // 1: pack / unpack of the first corner turn (own planes x others' columns), 0: the second
    float2 *buf;     // P blocks of maxS x maxW complex values
    double *ev;      // stage 2: the rank's 7 partial sums
};

// CTAs blockIdx.y = s handle the block exchanged with rank s.
__global__ void __launch_bounds__(256) k_slab_pack(SlabArgs a) {
    const int s = blockIdx.y, r = a.rank, ncol = a.d.K2 * a.d.H3;
    float2 *blk = a.buf + (size_t)s * a.L.maxS * a.L.maxW;
    const int t = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    if (a.first_pass)  // own planes x s's columns
        slab_pack(a.d.spec, ncol, a.L.plane0[r], a.L.plane0[r + 1], a.L.col0[s], a.L.col0[s + 1], blk, t, nth);
    else  // s's planes x own columns
        slab_pack(a.d.spec, ncol, a.L.plane0[s], a.L.plane0[s + 1], a.L.col0[r], a.L.col0[r + 1], blk, t, nth);
}

__global__ void __launch_bounds__(256) k_slab_unpack(SlabArgs a) {
    const int s = blockIdx.y, r = a.rank, ncol = a.d.K2 * a.d.H3;
    const float2 *blk = a.buf + (size_t)s * a.L.maxS * a.L.maxW;
    const int t = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    if (a.first_pass)  // from s: s's planes x own columns
        slab_unpack(a.d.spec, ncol, a.L.plane0[s], a.L.plane0[s + 1], a.L.col0[r], a.L.col0[r + 1], blk, t, nth);
    else  // from s: own planes x s's columns
        slab_unpack(a.d.spec, ncol, a.L.plane0[r], a.L.plane0[r + 1], a.L.col0[s], a.L.col0[s + 1], blk, t, nth);
}

__global__ void __launch_bounds__(32) k_slab_energy(SlabArgs a) {
    slab_energy(a.d, a.L.item0[a.rank], a.L.item0[a.rank + 1], a.ev, threadIdx.x);
}

static cudaError_t launch_exchange(void (*k)(SlabArgs), const SlabArgs &a, cudaStream_t s) {
    const int per = a.L.maxS * a.L.maxW;
    unsigned gx = (unsigned)((per + 255) / 256);
    if (gx > 64) gx = 64;
    k<<<dim3(gx, (unsigned)a.L.P), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pme

using namespace pme;

struct pme_slab {
    pme_plan *pl = nullptr;
    int P = 1, rank = 0;
    SlabLayout L;
    double *ev = nullptr;  // device, 8 doubles
};

extern "C" {

pme_status pme_slab_create(const int K[3], int p, double beta, const double box[9], int nranks, int rank,
                           void *cuda_stream, pme_slab **out) {
    if (!out) return fail(PME_EINVAL, "out is NULL");
    *out = nullptr;
    if (nranks < 1 || nranks > SLAB_MAX_RANKS || rank < 0 || rank >= nranks)
        return fail(PME_EINVAL, "need 1 <= nranks <= %d and 0 <= rank < nranks", SLAB_MAX_RANKS);
    pme_slab *sl = lib_new<pme_slab>();
    if (!sl) return fail(PME_ENOMEM, "host allocation failed");
    pme_status st = pme_create(K, p, beta, box, cuda_stream, &sl->pl);
    if (st != PME_OK) {
        delete sl;
        return st;
    }
    if (!make_slab_layout(sl->pl->d, nranks, sl->L)) {
        pme_slab_destroy(sl);
        return fail(PME_EUNSUPPORTED, "%d ranks cannot each own a mesh plane and an influence item of this mesh", nranks);
    }
    sl->P = nranks;
    sl->rank = rank;
    DeviceGuard g(sl->pl->dev);
    cudaError_t e = lib_malloc((void **)&sl->ev, 8 * sizeof(double));
    if (e != cudaSuccess) {
        sl->ev = nullptr;
        pme_slab_destroy(sl);
        return cuda_fail(e, "cudaMalloc(slab energies)");
    }
    *out = sl;
    return PME_OK;
}

pme_status pme_slab_layout(const pme_slab *sl, int *planes, int *columns, int64_t *block_values) {
    if (!sl) return fail(PME_EINVAL, "slab is NULL");
    if (planes) {
        planes[0] = sl->L.plane0[sl->rank];
        planes[1] = sl->L.plane0[sl->rank + 1];
    }
    if (columns) {
        columns[0] = sl->L.col0[sl->rank];
        columns[1] = sl->L.col0[sl->rank + 1];
    }
    if (block_values) *block_values = (int64_t)sl->L.maxS * sl->L.maxW;
    return PME_OK;
}

static SysDev slab_desc(pme_slab *sl, const float *pos, const float *q, int64_t n, float *forces) {
    SysDev d = plan_descriptor(sl->pl, pos, q, n, forces, nullptr);
    d.k1_lo = sl->L.plane0[sl->rank];
    d.k1_hi = sl->L.plane0[sl->rank + 1];
    d.tc_w = nullptr;  // the influence items of the layout are those of the FP32 stage
    return d;
}

pme_status pme_slab_stage1(pme_slab *sl, const float *pos, const float *q, int64_t n, float *send) {
    if (!sl) return fail(PME_EINVAL, "slab is NULL");
    pme_status st = check_atoms(sl->pl, pos, q, n, send);  // send stands in for forces (non-NULL check)
    if (st) return st;
    if (!send) return fail(PME_EINVAL, "send must be non-NULL");
    DeviceGuard g(sl->pl->dev);
    if ((st = plan_reserve(sl->pl, n)) != PME_OK) return st;
    const SysDev d = slab_desc(sl, pos, q, n, nullptr);
    const cudaStream_t s = sl->pl->stream;
    launch_stage(d, STAGE_BIN, s);
    launch_stage(d, STAGE_SPREAD, s);
    launch_stage_items(d, STAGE_FWD, sl->L.plane0[sl->rank], sl->L.plane0[sl->rank + 1] - sl->L.plane0[sl->rank], s);
    SlabArgs a;
    a.d = d;
    a.L = sl->L;
    a.rank = sl->rank;
    a.first_pass = 1;
    a.buf = (float2 *)send;
    a.ev = sl->ev;
    cudaError_t e = launch_exchange(k_slab_pack, a, s);
    if (e != cudaSuccess) return cuda_fail(e, "slab stage 1 launch");
    return PME_OK;
}

pme_status pme_slab_stage2(pme_slab *sl, const float *recv, float *send, double *ev_dev) {
    if (!sl || !recv || !send) return fail(PME_EINVAL, "slab, recv and send must be non-NULL");
    DeviceGuard g(sl->pl->dev);
    const SysDev d = slab_desc(sl, nullptr, nullptr, 0, nullptr);
    const cudaStream_t s = sl->pl->stream;
    SlabArgs a;
    a.d = d;
    a.L = sl->L;
    a.rank = sl->rank;
    a.first_pass = 1;
    a.buf = (float2 *)recv;
    a.ev = ev_dev ? ev_dev : sl->ev;
    cudaError_t e = launch_exchange(k_slab_unpack, a, s);
    if (e != cudaSuccess) return cuda_fail(e, "slab stage 2 launch");
    launch_stage_items(d, STAGE_CONV, sl->L.item0[sl->rank], sl->L.item0[sl->rank + 1] - sl->L.item0[sl->rank], s);
    k_slab_energy<<<1, 32, 0, s>>>(a);
    a.first_pass = 0;
    a.buf = (float2 *)send;
    if ((e = launch_exchange(k_slab_pack, a, s)) != cudaSuccess) return cuda_fail(e, "slab stage 2 launch");
    return PME_OK;
}

pme_status pme_slab_stage3(pme_slab *sl, const float *recv, const float *pos, const float *q, int64_t n,
                           float *forces) {
    if (!sl || !recv) return fail(PME_EINVAL, "slab and recv must be non-NULL");
    pme_status st = check_atoms(sl->pl, pos, q, n, forces);
    if (st) return st;
    DeviceGuard g(sl->pl->dev);
    if (n > sl->pl->n_cap) return fail(PME_EINVAL, "n differs from stage 1");
    const SysDev d = slab_desc(sl, pos, q, n, forces);
    const cudaStream_t s = sl->pl->stream;
    SlabArgs a;
    a.d = d;
    a.L = sl->L;
    a.rank = sl->rank;
    a.first_pass = 0;
    a.buf = (float2 *)recv;
    a.ev = sl->ev;
    cudaError_t e = launch_exchange(k_slab_unpack, a, s);
    if (e != cudaSuccess) return cuda_fail(e, "slab stage 3 launch");
    launch_stage_items(d, STAGE_INV, sl->L.plane0[sl->rank], sl->L.plane0[sl->rank + 1] - sl->L.plane0[sl->rank], s);
    launch_stage(d, STAGE_GATHER, s);
    // the overflow count is reset by the forward stage's plane 0, which only one rank runs
    if ((e = cudaMemsetAsync(&sl->pl->d.ctl->novf, 0, sizeof(unsigned), s)) != cudaSuccess)
        return cuda_fail(e, "cudaMemsetAsync(overflow count)");
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "slab stage 3 launch");
    return PME_OK;
}

pme_status pme_slab_sync(pme_slab *sl) {
    if (!sl) return fail(PME_EINVAL, "slab is NULL");
    return pme_sync(sl->pl);
}

void pme_slab_destroy(pme_slab *sl) {
    if (!sl) return;
    if (sl->pl) {
        DeviceGuard g(sl->pl->dev);
        cudaStreamSynchronize(sl->pl->stream);
        if (sl->ev) cudaFree(sl->ev);
        pme_destroy(sl->pl);
    }
    delete sl;
}

}  // extern "C"
