// Host-side interface of the CUDA kernels (launch configuration and entry points).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace pme {

constexpr int NT_MESH = 256;   // threads per CTA for binning and the FFT / influence stages
constexpr int NT_TILE = 128;   // threads per CTA for spreading and force interpolation
constexpr int NT_CONV = 128;   // threads per CTA for the influence stage
constexpr size_t MAX_SMEM_BYTES = 226 * 1024;  // opt-in limit is 227 KB including static shared memory

// Raise the dynamic shared-memory limit of the large-footprint kernels (once per device).
cudaError_t configure_kernels();

// Optional device-to-device copies of intermediate meshes (diagnostics).
struct DebugTaps {
    unsigned long long *mesh_out;  // fixed-point charge mesh after spreading, K1*K2*K3
    float *phi_out;                // potential mesh after the inverse FFT, K1*K2*K3
};

enum Stage { STAGE_BIN = 0, STAGE_SPREAD, STAGE_FWD, STAGE_CONV, STAGE_INV, STAGE_GATHER, NUM_STAGES };

// Enqueue one stage kernel of system d.
void launch_stage(const SysDev &d, int stage, cudaStream_t s);

// Enqueue the six stage kernels of one evaluation of system d on stream s.
cudaError_t launch_pipeline(const SysDev &d, cudaStream_t s, const DebugTaps *taps = nullptr);

}  // namespace pme
