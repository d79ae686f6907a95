// Throughput probes of the resources the spreading stage is bound by: shared-memory 32-bit integer atomics
// (its per-contribution accumulation) and 64-bit integer reductions into global memory (its tile flush).
// The measurement code times them with CUDA events around pme_probe_launch to obtain measured peaks, so
// the spreading kernel's achieved rate can be stated as a fraction of what this GPU sustains.
#include <cuda_runtime.h>

#include "../../include/pme.h"
#include "plan_internal.h"

namespace pme {

constexpr int PROBE_THREADS = 512;
constexpr int PROBE_SMEM_INTS = 8192;  // 32 KB of counters per CTA
constexpr int PROBE_UNROLL = 8;

// Each thread adds to PROBE_UNROLL counters per round, all distinct; the 32 lanes of a warp hit 32
// distinct banks (consecutive words), so the rate is the shared-memory atomic unit's conflict-free peak.
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_smem_atomics(int rounds, unsigned *out) {
    __shared__ int s[PROBE_SMEM_INTS];
    for (int i = threadIdx.x; i < PROBE_SMEM_INTS; i += blockDim.x) s[i] = 0;
    __syncthreads();
    const int t = threadIdx.x;
    for (int r = 0; r < rounds; ++r) {
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u) atomicAdd(&s[(t + u * PROBE_THREADS) & (PROBE_SMEM_INTS - 1)], 1 + u);
    }
    __syncthreads();
    if (t == 0) {
        int acc = 0;
        for (int i = 0; i < PROBE_SMEM_INTS; ++i) acc += s[i];
        out[blockIdx.x] = (unsigned)acc;  // keeps the work observable
    }
}

// Each thread reduces into PROBE_UNROLL distinct 64-bit words per round; a warp covers 32 consecutive
// words (four 64-byte sectors), and the grid sweeps a buffer of nwords words that stays in L2.
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_global_red64(int rounds, unsigned long long *buf,
                                                                        unsigned long long nwords) {
    const unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long span = (unsigned long long)gridDim.x * blockDim.x;
    for (int r = 0; r < rounds; ++r) {
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u) {
            const unsigned long long i = (g + ((unsigned long long)r * PROBE_UNROLL + u) * span) % nwords;
            atomicAdd(buf + i, 1ull);
        }
    }
}

}  // namespace pme

using namespace pme;

extern "C" pme_status pme_probe_launch(int kind, int ctas, int rounds, void *buf, size_t buf_bytes, void *cuda_stream,
                                       double *ops) {
    if (ctas < 1 || ctas > 65536 || rounds < 1 || rounds > (1 << 20) || !buf || !ops)
        return fail(PME_EINVAL, "pme_probe_launch: need 1..65536 CTAs, 1..2^20 rounds, a buffer and ops");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const double per = (double)ctas * PROBE_THREADS * PROBE_UNROLL * rounds;
    if (kind == 0) {
        if (buf_bytes < (size_t)ctas * sizeof(unsigned)) return fail(PME_EINVAL, "buffer below 4 bytes per CTA");
        k_probe_smem_atomics<<<ctas, PROBE_THREADS, 0, s>>>(rounds, (unsigned *)buf);
    } else if (kind == 1) {
        const unsigned long long nwords = buf_bytes / 8;
        if (nwords < PROBE_THREADS) return fail(PME_EINVAL, "buffer below one CTA's words");
        k_probe_global_red64<<<ctas, PROBE_THREADS, 0, s>>>(rounds, (unsigned long long *)buf, nwords);
    } else {
        return fail(PME_EINVAL, "kind must be 0 (shared-memory atomics) or 1 (global 64-bit reductions)");
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "probe launch");
    *ops = per;
    return PME_OK;
}
