// Stage kernels over a group of systems that share one mesh shape (K1, K2, K3, p): one launch per stage
// covers every work item of every system in the group, CTA b taking item b mod ips of system b / ips. The
// stage bodies and block sizes are the single-system ones, so a system's results are bit-identical to its
// single-system evaluation. Batches run one chain of six such launches per group, the chains as parallel
// branches of one CUDA graph.
#include <cuda_runtime.h>

#include "group.h"
#include "pdl.cuh"
#include "stages.cuh"

namespace pme {

// The CTA's system descriptor, copied from the group's array into shared memory.
__device__ __forceinline__ int group_load(const GroupArgs &a, SysDev &sd) {
    const int sys = blockIdx.x / a.ips;
    const int *src = (const int *)(a.sys + sys);
    for (int i = threadIdx.x; i < (int)(sizeof(SysDev) / 4); i += blockDim.x) ((int *)&sd)[i] = src[i];
    __syncthreads();
    return blockIdx.x - sys * a.ips;
}

__global__ void __launch_bounds__(NT_BIN) k_bin_g(GroupArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SysDev sd;
    PdlScope pdl(a.late);
    const int item = group_load(a, sd);
    if (item < sd.nbin) stage_bin(sd, item, smem);
}

template <int P, int T>
__global__ void __launch_bounds__(tile_nt_bound(T)) k_spread_g(GroupArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SysDev sd;
    spread_clear<P, T>(smem);  // before the wait: shared memory only
    PdlScope pdl(a.late);
    const int item = group_load(a, sd);
    stage_spread<P, T>(sd, item, smem, true);
}

template <int PR, int PC>
__global__ void __launch_bounds__(NT_SLAB) k_fwd_g(GroupArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SysDev sd;
    PdlScope pdl(a.late);
    const int item = group_load(a, sd);
    stage_fwd<PR, PC>(sd, item, smem);
}

template <int P1>
__global__ void __launch_bounds__(NT_CONV) k_conv_g(GroupArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SysDev sd;
    PdlScope pdl(a.late);
    const int item = group_load(a, sd);
    stage_conv<P1>(sd, item, smem);
}

template <int PR, int PC>
__global__ void __launch_bounds__(NT_SLAB) k_inv_g(GroupArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SysDev sd;
    PdlScope pdl(a.late);
    const int item = group_load(a, sd);
    stage_inv<PR, PC>(sd, item, smem);
}

template <int P, int T>
__global__ void __launch_bounds__(tile_nt_bound(T)) k_gather_g(GroupArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SysDev sd;
    PdlScope pdl(a.late);
    const int item = group_load(a, sd);
    stage_gather<P, T>(sd, item, smem);
}

// The spread / force kernels of a group: order p, tile edge 2^tlog.
template <int T>
static void (*spread_g_t(int p))(GroupArgs) {
    return p == 4 ? k_spread_g<4, T> : (p == 5 ? k_spread_g<5, T> : (p == 6 ? k_spread_g<6, T> : k_spread_g<8, T>));
}
template <int T>
static void (*gather_g_t(int p))(GroupArgs) {
    return p == 4 ? k_gather_g<4, T> : (p == 5 ? k_gather_g<5, T> : (p == 6 ? k_gather_g<6, T> : k_gather_g<8, T>));
}
static void (*spread_g(const SysDev &d))(GroupArgs) { return d.tlog == 4 ? spread_g_t<16>(d.p) : spread_g_t<8>(d.p); }
static void (*gather_g(const SysDev &d))(GroupArgs) { return d.tlog == 4 ? gather_g_t<16>(d.p) : gather_g_t<8>(d.p); }

static cudaError_t set_limit(const void *fn) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(MAX_SMEM_BYTES - sizeof(SysDev) - 64));
}

cudaError_t configure_group_kernels() {
    const void *fns[] = {(const void *)k_bin_g, (const void *)k_fwd_g<-1, -1>, (const void *)k_conv_g<-1>,
                         (const void *)k_inv_g<-1, -1>};
    for (int p : {4, 5, 6, 8})
        for (const void *f : {(const void *)spread_g_t<8>(p), (const void *)spread_g_t<16>(p),
                              (const void *)gather_g_t<8>(p), (const void *)gather_g_t<16>(p)}) {
            cudaError_t e = set_limit(f);
            if (e != cudaSuccess) return e;
        }
    for (const void *f : fns) {
        cudaError_t e = set_limit(f);
        if (e != cudaSuccess) return e;
    }
#define PME_CFG_K(K)                                                                                        \
    for (const void *f : {(const void *)k_fwd_g<Cubic<K>::PR, Cubic<K>::PC>, (const void *)k_conv_g<Cubic<K>::P1>, \
                          (const void *)k_inv_g<Cubic<K>::PR, Cubic<K>::PC>}) {                               \
        cudaError_t e = set_limit(f);                                                                       \
        if (e != cudaSuccess) return e;                                                                     \
    }
    PME_CUBIC_KS(PME_CFG_K)
#undef PME_CFG_K
    return cudaSuccess;
}

int group_items(const SysDev &d, int stage) {
    switch (stage) {
        case STAGE_BIN: return d.nbin > 0 ? d.nbin : 1;
        case STAGE_SPREAD: return d.ntiles + OVF_ITEMS;
        case STAGE_FWD: return d.K1;
        case STAGE_CONV: return d.nconv;
        case STAGE_INV: return d.K1;
        default: return d.ntiles + OVF_ITEMS;
    }
}

template <class... Args>
static cudaError_t launch_ex(void (*kernel)(Args...), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                             Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = launch_mode() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

static void (*fwd_g(const SysDev &d))(GroupArgs) {
    if (d.lane_slab) {
#define PME_PICK(K) \
    if (d.lp_rows == Cubic<K>::PR && d.lp_cols == Cubic<K>::PC) return k_fwd_g<Cubic<K>::PR, Cubic<K>::PC>;
        PME_CUBIC_KS(PME_PICK)
#undef PME_PICK
    }
    return k_fwd_g<-1, -1>;
}
static void (*inv_g(const SysDev &d))(GroupArgs) {
    if (d.lane_slab) {
#define PME_PICK(K) \
    if (d.lp_rows == Cubic<K>::PR && d.lp_cols == Cubic<K>::PC) return k_inv_g<Cubic<K>::PR, Cubic<K>::PC>;
        PME_CUBIC_KS(PME_PICK)
#undef PME_PICK
    }
    return k_inv_g<-1, -1>;
}
static void (*conv_g(const SysDev &d))(GroupArgs) {
    if (d.lane_conv) {
#define PME_PICK(K) \
    if (d.lp_k1 == Cubic<K>::P1) return k_conv_g<Cubic<K>::P1>;
        PME_CUBIC_KS(PME_PICK)
#undef PME_PICK
    }
    return k_conv_g<-1>;
}

cudaError_t launch_group_chain(const SysDev *sys_dev, int nsys, const SysDev &proto, int max_nbin, cudaStream_t s) {
    GroupArgs a;
    a.sys = sys_dev;
    const SysDev &d = proto;
    cudaError_t e;
    for (int stage = 0; stage < NUM_STAGES; ++stage) {
        a.late = pdl_when(launch_mode(), stage);
        a.ips = stage == STAGE_BIN ? (max_nbin > 0 ? max_nbin : 1) : group_items(d, stage);
        const unsigned grid = (unsigned)(a.ips * nsys);
        switch (stage) {
            case STAGE_BIN: e = launch_ex(k_bin_g, grid, NT_BIN, smem_bin(NT_BIN), s, a); break;
            case STAGE_SPREAD:
                e = launch_ex(spread_g(d), grid, (unsigned)tile_threads(d, (int64_t)max_nbin * BIN_CHUNK),
                              smem_spread(d.p, d.tlog), s, a);
                break;
            case STAGE_FWD: e = launch_ex(fwd_g(d), grid, NT_SLAB, smem_slab(d.K2, d.K3), s, a); break;
            case STAGE_CONV: e = launch_ex(conv_g(d), grid, NT_CONV, smem_conv(d.K1, NT_CONV), s, a); break;
            case STAGE_INV: e = launch_ex(inv_g(d), grid, NT_SLAB, smem_inv(d.K2, d.K3), s, a); break;
            default:
                e = launch_ex(gather_g(d), grid, (unsigned)tile_threads(d, (int64_t)max_nbin * BIN_CHUNK, true),
                              smem_gather_all(d.p, d.tlog), s, a);
                break;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace pme
