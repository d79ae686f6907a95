// Host-side interface of the CUDA kernels (launch configuration and entry points).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace pme {

constexpr int NT_BIN = 128;    // threads per CTA for binning (BIN_CHUNK atoms per CTA)
constexpr int NT_SLAB = SLAB_THREADS;  // threads per CTA for the forward / inverse slab FFT stages
constexpr int NT_TILE = 256;   // threads per CTA for spreading and force interpolation (two per atom), at most,
constexpr int NT_TILE16 = 512; // with 8^3 / 16^3 tiles
PME_HD int tile_nt_bound(int T) { return T >= 16 ? NT_TILE16 : NT_TILE; }
// Spread / gather CTA size for a system whose binned atoms number about n_bins * BIN_CHUNK: two threads per
// atom, sized to the mean tile occupancy, so sparse 8^3 tiles (large meshes) do not leave half the CTA idle
// and twice as many CTAs fit on an SM. Dense 8^3 tiles interpolate forces on 192 threads: at 64 registers,
// five such CTAs fit on an SM, three beside an inverse-stage CTA that has not retired yet, so all tiles of
// a 64^3 mesh are dispatched at once (with 256 threads, 13-15 SMs ran a fifth tile in a second wave; 28.65
// vs 28.75 us per evaluation). 16^3 tiles (hundreds of atoms each): 512 threads for spreading, 128
// for force interpolation, whose 106 registers per thread (p = 6) leave room for four 128-thread CTAs per
// SM but only one 512-thread CTA, so all tiles of a 128^3 mesh fit in one wave (128^3, p = 6: 131.6 vs
// 133.6 us per evaluation with 256 threads, 145.4 with 512). Results do not depend on it.
inline int tile_threads(const SysDev &d, int64_t n, bool gather = false) {
    if (d.nt_tile == 128 || d.nt_tile == NT_TILE || (d.nt_tile == NT_TILE16 && d.tlog >= 4))
        return d.nt_tile;  // chosen by the autotuner or the caller
    if (d.tlog >= 4) return gather ? 128 : NT_TILE16;
    if (d.ntiles > 0 && n <= (int64_t)64 * d.ntiles) return 128;
    return gather ? 192 : NT_TILE;
}
constexpr int NT_CONV = 128;   // threads per CTA for the influence stage
constexpr size_t MAX_SMEM_BYTES = 226 * 1024;  // opt-in limit is 227 KB including static shared memory

// Cubic meshes K^3 whose lane plans get kernels (and batch stage calls) specialised at compile time.
#define PME_CUBIC_KS(X) X(16) X(20) X(24) X(32) X(40) X(48) X(64) X(80) X(96) X(128)
template <int K>
struct Cubic {
    static constexpr int PR = slab_lane_plan(K / 2, K), PC = slab_lane_plan(K, K / 2 + 1), P1 = conv_lane_plan(K);
    static_assert(PR >= 0 && PC >= 0 && P1 >= 0, "every listed cubic mesh has lane plans");
};

// Launch mode of the per-stage kernels: 0 plain, 1 programmatic dependent launch triggered at kernel entry,
// 2 triggered at CTA exit (the influence stage: right after its own wait), 3 triggered right after the
// kernel's own wait. Process-wide; affects launches recorded afterwards.
void set_launch_mode(int mode);
int launch_mode();
// The PdlScope argument of a kernel of stage `stage` in launch mode `mode`. In mode 2 the influence stage
// releases the inverse stage early: the inverse stage's K1 slab CTAs fit beside the influence CTAs and
// become resident during them (measured 30.6 vs 31.1 us per 64^3 evaluation); released early, the other
// stages' successors were slower or no faster (their CTAs then land unevenly on the SMs).
int pdl_when(int mode, int stage);

// CTAs per slab of the single-system forward and inverse slab stages: 1, or 2 / 4 (a thread-block cluster
// per slab exchanging its intermediate rows / columns through distributed shared memory; meshes with
// K2 = K3 in {32, 64, 128} at 2, 64 at 4, others keep one CTA). Process-wide, default 1; affects launches
// issued afterwards. Returns -1 for other values. Results are bitwise the same for every value.
int set_slab_split(int fwd_ctas, int inv_ctas);
int slab_split(int inverse);

// Raise the dynamic shared-memory limit of the large-footprint kernels (once per device).
cudaError_t configure_kernels();

// Optional device-to-device copies of intermediate meshes (diagnostics).
struct DebugTaps {
    unsigned long long *mesh_out;  // fixed-point charge mesh after spreading, K1*K2*K3
    float *phi_out;                // potential mesh after the inverse FFT, K1*K2*K3
};

enum Stage { STAGE_BIN = 0, STAGE_SPREAD, STAGE_FWD, STAGE_CONV, STAGE_INV, STAGE_GATHER, NUM_STAGES };

// Enqueue the copy of nf floats from device memory to page-locked host memory (dst: its device-side
// address), of the control block ctl to its host copy hctl (device-side address; may be null) and, when
// res8 (device-side address of page-locked memory) is given, of energy, virial and status bits to res8[0..7],
// after the work before it on s.
cudaError_t launch_copy_out(const float *src, float *dst, long long nf, const Ctl *ctl, Ctl *hctl, cudaStream_t s,
                            double *res8 = nullptr);

// Enqueue one stage kernel of system d.
void launch_stage(const SysDev &d, int stage, cudaStream_t s);
// The forward, influence or inverse stage over its work items [first, first + count) only (a rank's planes or
// columns in the slab decomposition).
void launch_stage_items(const SysDev &d, int stage, int first, int count, cudaStream_t s);

// Tensor-core influence stage (tc_dft.cu): kernel set-up, tiles per evaluation, launch, and the DFT-matrix
// image (three BF16 terms of the real and imaginary parts, both K halves, 128-byte swizzled K-major rows).
cudaError_t configure_tc_kernel();
int tc_tiles(const SysDev &d);
cudaError_t launch_conv_tc(const SysDev &d, const void *w_img, cudaStream_t s);
void make_tc_w_image(std::vector<uint8_t> &img);
constexpr size_t TC_W_IMAGE_BYTES = 2 * 6 * 128 * 128;

// Enqueue the six stage kernels of one evaluation of system d on stream s.
cudaError_t launch_pipeline(const SysDev &d, cudaStream_t s, const DebugTaps *taps = nullptr);

}  // namespace pme
