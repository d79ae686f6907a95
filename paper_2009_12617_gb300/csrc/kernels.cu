// CUDA kernels of the SPME pipeline: one kernel per stage for a single system, launched back to back on
// one stream. Each kernel is a thin wrapper over a stage body from stages.cuh.
#include <cuda_runtime.h>

#include "kernels.h"
#include "stages.cuh"

namespace pme {

__global__ void __launch_bounds__(NT_MESH) k_bin(SysDev d) {
    extern __shared__ __align__(16) unsigned char smem[];
    stage_bin(d, blockIdx.x, smem);
}

template <int P>
__global__ void __launch_bounds__(NT_TILE) k_spread(SysDev d) {
    extern __shared__ __align__(16) unsigned char smem[];
    stage_spread<P>(d, blockIdx.x, smem);
}

__global__ void __launch_bounds__(NT_MESH) k_fwd(SysDev d) {
    extern __shared__ __align__(16) unsigned char smem[];
    stage_fwd(d, blockIdx.x, smem);
}

__global__ void __launch_bounds__(NT_CONV) k_conv(SysDev d) {
    extern __shared__ __align__(16) unsigned char smem[];
    stage_conv(d, blockIdx.x, smem);
}

__global__ void __launch_bounds__(NT_MESH) k_inv(SysDev d) {
    extern __shared__ __align__(16) unsigned char smem[];
    stage_inv(d, blockIdx.x, smem);
}

template <int P>
__global__ void __launch_bounds__(NT_TILE) k_gather(SysDev d) {
    extern __shared__ __align__(16) unsigned char smem[];
    stage_gather<P>(d, blockIdx.x, smem);
}

static cudaError_t set_smem_limit(const void *fn, size_t bytes) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t configure_kernels() {
    const size_t big = MAX_SMEM_BYTES;
    cudaError_t e;
    if ((e = set_smem_limit((const void *)k_fwd, big)) != cudaSuccess) return e;
    if ((e = set_smem_limit((const void *)k_conv, big)) != cudaSuccess) return e;
    if ((e = set_smem_limit((const void *)k_inv, big)) != cudaSuccess) return e;
    return cudaSuccess;
}

template <int P>
static void launch_tiles_spread(const SysDev &d, cudaStream_t s) {
    k_spread<P><<<d.ntiles + OVF_ITEMS, NT_TILE, smem_spread(P), s>>>(d);
}
template <int P>
static void launch_tiles_gather(const SysDev &d, cudaStream_t s) {
    k_gather<P><<<d.ntiles + OVF_ITEMS, NT_TILE, smem_gather(P), s>>>(d);
}

void launch_stage(const SysDev &d, int stage, cudaStream_t s) {
    switch (stage) {
        case STAGE_BIN:
            k_bin<<<d.nbin > 0 ? d.nbin : 1, NT_MESH, smem_bin(NT_MESH), s>>>(d);
            break;
        case STAGE_SPREAD:
            if (d.p == 4) launch_tiles_spread<4>(d, s);
            else if (d.p == 6) launch_tiles_spread<6>(d, s);
            else launch_tiles_spread<8>(d, s);
            break;
        case STAGE_FWD:
            k_fwd<<<d.K1, NT_MESH, smem_slab(d.K2, d.K3), s>>>(d);
            break;
        case STAGE_CONV:
            k_conv<<<d.nconv, NT_CONV, smem_conv(d.K1, NT_CONV), s>>>(d);
            break;
        case STAGE_INV:
            k_inv<<<d.K1, NT_MESH, smem_slab(d.K2, d.K3), s>>>(d);
            break;
        default:
            if (d.p == 4) launch_tiles_gather<4>(d, s);
            else if (d.p == 6) launch_tiles_gather<6>(d, s);
            else launch_tiles_gather<8>(d, s);
            break;
    }
}

cudaError_t launch_pipeline(const SysDev &d, cudaStream_t s, const DebugTaps *taps) {
    const size_t mesh = (size_t)d.K1 * d.K2 * d.K3;
    cudaError_t e;
    launch_stage(d, STAGE_BIN, s);
    launch_stage(d, STAGE_SPREAD, s);
    if (taps && taps->mesh_out &&
        (e = cudaMemcpyAsync(taps->mesh_out, d.grid, mesh * 8, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return e;
    launch_stage(d, STAGE_FWD, s);
    launch_stage(d, STAGE_CONV, s);
    launch_stage(d, STAGE_INV, s);
    if (taps && taps->phi_out &&
        (e = cudaMemcpyAsync(taps->phi_out, d.phi, mesh * 4, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return e;
    launch_stage(d, STAGE_GATHER, s);
    return cudaGetLastError();
}

}  // namespace pme
