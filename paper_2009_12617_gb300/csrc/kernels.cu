// CUDA kernels of the SPME pipeline: one kernel per stage for a single system, launched back to back on
// one stream. Each kernel is a thin wrapper over a stage body from stages.cuh.
#include <cuda_runtime.h>

#include "kernels.h"
#include "pdl.cuh"
#include "stages.cuh"

namespace pme {

static int g_launch_mode = 2;  // measured fastest on GB300 (late trigger)
void set_launch_mode(int mode) { g_launch_mode = mode; }
int launch_mode() { return g_launch_mode; }
int pdl_when(int mode, int stage) { return mode == 1 ? 0 : (mode == 3 || stage == STAGE_CONV ? 2 : 1); }

__global__ void __launch_bounds__(NT_BIN) k_bin(SysDev d) {
    extern __shared__ __align__(16) unsigned char smem[];
    PdlScope pdl(d.pdl_late);
    stage_bin(d, blockIdx.x, smem);
}

template <int P, int T>
__global__ void __launch_bounds__(tile_nt_bound(T)) k_spread(SysDev d) {
    extern __shared__ __align__(16) unsigned char smem[];
    // before the wait: shared memory and kernel parameters only
    spread_clear<P, T>(smem);
    int org[3] = {0, 0, 0};
    if ((int)blockIdx.x < d.ntiles) tile_origin(d, blockIdx.x, org[0], org[1], org[2]);
    PdlScope pdl(d.pdl_late);
    stage_spread<P, T>(d, blockIdx.x, smem, true, org);
}

__global__ void __launch_bounds__(NT_SLAB) k_fwd(SysDev d) {
    extern __shared__ __align__(16) unsigned char smem[];
    PdlScope pdl(d.pdl_late);
    stage_fwd(d, d.item0 + blockIdx.x, smem);
}

__global__ void __launch_bounds__(NT_CONV) k_conv(SysDev d) {
    extern __shared__ __align__(16) unsigned char smem[];
    PdlScope pdl(d.pdl_late);
    stage_conv(d, d.item0 + blockIdx.x, smem);
}

__global__ void __launch_bounds__(NT_SLAB) k_inv(SysDev d) {
    extern __shared__ __align__(16) unsigned char smem[];
    PdlScope pdl(d.pdl_late);
    stage_inv(d, d.item0 + blockIdx.x, smem);
}

// Slab and influence kernels specialised for the lane plans of the cubic meshes of PME_CUBIC_KS (kernels.h);
// each holds only its plans' code. Other meshes run the kernels above, which choose among all plans at run
// time.

template <int PR, int PC>
__global__ void __launch_bounds__(NT_SLAB) k_fwd_p(SysDev d) {
    extern __shared__ __align__(16) unsigned char smem[];
    PdlScope pdl(d.pdl_late);
    stage_fwd<PR, PC>(d, d.item0 + blockIdx.x, smem);
}

template <int P1>
__global__ void __launch_bounds__(NT_CONV) k_conv_p(SysDev d) {
    extern __shared__ __align__(16) unsigned char smem[];
    PdlScope pdl(d.pdl_late);
    stage_conv<P1>(d, d.item0 + blockIdx.x, smem);
}

template <int PR, int PC>
__global__ void __launch_bounds__(NT_SLAB) k_inv_p(SysDev d) {
    extern __shared__ __align__(16) unsigned char smem[];
    PdlScope pdl(d.pdl_late);
    stage_inv<PR, PC>(d, d.item0 + blockIdx.x, smem);
}

// Slab kernels with each slab split over a thread-block cluster of CS CTAs (slab d.item0 + blockIdx.x / CS,
// cluster rank blockIdx.x mod CS), for K2 = K3 = K. They keep the one-CTA kernels' lane plans (the same
// transforms in the same order, so the same bits), with fewer transforms per CTA.
template <int K, int CS>
struct SlabSplit {
    static constexpr int H3 = K / 2 + 1;
    static constexpr int PR = Cubic<K>::PR, PC = Cubic<K>::PC;
    static constexpr int units(int c, int ntr) { return ((ntr + 32 / plan_L(c) - 1) / (32 / plan_L(c))) * 32; }
    static constexpr int NT_FWD = units(PR, K / CS) > units(PC, (H3 + CS - 1) / CS) ? units(PR, K / CS)
                                                                                       : units(PC, (H3 + CS - 1) / CS);
    static constexpr int NT_INV = NT_FWD + 64;  // two spare warps for the side work
    static_assert(PR >= 0 && PC >= 0 && NT_INV <= 1024, "split slab plans");
};

template <int K, int CS>
__global__ void __launch_bounds__(SlabSplit<K, CS>::NT_FWD) k_fwd_c(SysDev d) {
    extern __shared__ __align__(16) unsigned char smem[];
    PdlScope pdl(d.pdl_late);
    const int c = (int)cg::this_cluster().block_rank();
    stage_fwd_cluster<SlabSplit<K, CS>::PR, SlabSplit<K, CS>::PC, CS>(d, d.item0 + blockIdx.x / CS, c, smem);
}

template <int K, int CS>
__global__ void __launch_bounds__(SlabSplit<K, CS>::NT_INV) k_inv_c(SysDev d) {
    extern __shared__ __align__(16) unsigned char smem[];
    PdlScope pdl(d.pdl_late);
    const int c = (int)cg::this_cluster().block_rank();
    stage_inv_cluster<SlabSplit<K, CS>::PR, SlabSplit<K, CS>::PC, CS>(d, d.item0 + blockIdx.x / CS, c, smem);
}

template <int P, int T>
__global__ void __launch_bounds__(tile_nt_bound(T)) k_gather(SysDev d) {
    extern __shared__ __align__(16) unsigned char smem[];
    int org[3] = {0, 0, 0};  // before the wait: kernel parameters only
    if ((int)blockIdx.x < d.ntiles) tile_origin(d, blockIdx.x, org[0], org[1], org[2]);
    PdlScope pdl(d.pdl_late);
    stage_gather<P, T>(d, blockIdx.x, smem, org);
}

static void launch_pdl(void (*kernel)(SysDev), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                       const SysDev &d0, int stage, unsigned cluster = 1) {
    SysDev d = d0;
    d.pdl_late = pdl_when(g_launch_mode, stage);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    unsigned na = 0;
    if (cluster > 1) {
        attr[na].id = cudaLaunchAttributeClusterDimension;
        attr[na].val.clusterDim.x = cluster;
        attr[na].val.clusterDim.y = 1;
        attr[na].val.clusterDim.z = 1;
        ++na;
    }
    if (g_launch_mode) {
        attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[na].val.programmaticStreamSerializationAllowed = 1;
        ++na;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    cudaLaunchKernelEx(&cfg, kernel, d);
}

// CTAs per slab of the forward and the inverse slab stages (thread-block clusters), process-wide.
static int g_slab_split[2] = {1, 1};  // split slabs measured slower in the pipelined evaluation
int set_slab_split(int fwd_ctas, int inv_ctas) {
    for (int c : {fwd_ctas, inv_ctas})
        if (c != 1 && c != 2 && c != 4) return -1;
    g_slab_split[0] = fwd_ctas;
    g_slab_split[1] = inv_ctas;
    return 0;
}
int slab_split(int inverse) { return g_slab_split[inverse ? 1 : 0]; }

// The split slab kernels instantiated: cubic meshes K, clusters of CS CTAs.
#define PME_SPLIT_KS(X) X(32, 2) X(64, 2) X(64, 4) X(128, 2)

// Launches the split forward (fwd = true) or inverse slab kernel for the items [d.item0, d.item0 + count)
// if the mesh has one for the current split, else returns false.
static bool launch_split_slab(const SysDev &d, bool fwd, int count, cudaStream_t s) {
    const int cs = g_slab_split[fwd ? 0 : 1];
    if (cs == 1 || !d.lane_slab || d.K2 != d.K3) return false;
#define PME_SPLIT_LAUNCH(K, CS)                                                                                  \
    if (d.K2 == K && cs == CS) {                                                                                 \
        if (fwd)                                                                                                 \
            launch_pdl(k_fwd_c<K, CS>, (unsigned)(count * CS), SlabSplit<K, CS>::NT_FWD, smem_slab(K, K), s, d, \
                       STAGE_FWD, CS);                                                                           \
        else                                                                                                     \
            launch_pdl(k_inv_c<K, CS>, (unsigned)(count * CS), SlabSplit<K, CS>::NT_INV, smem_inv(K, K), s, d,  \
                       STAGE_INV, CS);                                                                           \
        return true;                                                                                             \
    }
    PME_SPLIT_KS(PME_SPLIT_LAUNCH)
#undef PME_SPLIT_LAUNCH
    return false;
}

static cudaError_t set_smem_limit(const void *fn, size_t bytes) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t configure_kernels() {
    const size_t big = MAX_SMEM_BYTES;
    const void *fns[] = {(const void *)k_fwd, (const void *)k_conv, (const void *)k_inv,
                         (const void *)k_spread<4, 8>, (const void *)k_spread<5, 8>, (const void *)k_spread<6, 8>,
                         (const void *)k_spread<8, 8>, (const void *)k_spread<4, 16>, (const void *)k_spread<5, 16>,
                         (const void *)k_spread<6, 16>, (const void *)k_spread<8, 16>, (const void *)k_gather<4, 8>,
                         (const void *)k_gather<5, 8>, (const void *)k_gather<6, 8>, (const void *)k_gather<8, 8>,
                         (const void *)k_gather<4, 16>, (const void *)k_gather<5, 16>, (const void *)k_gather<6, 16>,
                         (const void *)k_gather<8, 16>};
    for (const void *f : fns) {
        cudaError_t e = set_smem_limit(f, big);
        if (e != cudaSuccess) return e;
    }
#define PME_CFG_K(K)                                                                                        \
    for (const void *f : {(const void *)k_fwd_p<Cubic<K>::PR, Cubic<K>::PC>, (const void *)k_conv_p<Cubic<K>::P1>, \
                          (const void *)k_inv_p<Cubic<K>::PR, Cubic<K>::PC>}) {                               \
        cudaError_t e = set_smem_limit(f, big);                                                             \
        if (e != cudaSuccess) return e;                                                                     \
    }
    PME_CUBIC_KS(PME_CFG_K)
#undef PME_CFG_K
#define PME_CFG_SPLIT(K, CS)                                                                \
    for (const void *f : {(const void *)k_fwd_c<K, CS>, (const void *)k_inv_c<K, CS>}) {   \
        cudaError_t e = set_smem_limit(f, big);                                             \
        if (e != cudaSuccess) return e;                                                     \
    }
    PME_SPLIT_KS(PME_CFG_SPLIT)
#undef PME_CFG_SPLIT
    return configure_tc_kernel();
}

// The specialised kernel for the system's plans, or the general one.
static void (*fwd_kernel(const SysDev &d))(SysDev) {
    if (d.lane_slab) {
#define PME_PICK(K) \
    if (d.lp_rows == Cubic<K>::PR && d.lp_cols == Cubic<K>::PC) return k_fwd_p<Cubic<K>::PR, Cubic<K>::PC>;
        PME_CUBIC_KS(PME_PICK)
#undef PME_PICK
    }
    return k_fwd;
}
static void (*inv_kernel(const SysDev &d))(SysDev) {
    if (d.lane_slab) {
#define PME_PICK(K) \
    if (d.lp_rows == Cubic<K>::PR && d.lp_cols == Cubic<K>::PC) return k_inv_p<Cubic<K>::PR, Cubic<K>::PC>;
        PME_CUBIC_KS(PME_PICK)
#undef PME_PICK
    }
    return k_inv;
}
static void (*conv_kernel(const SysDev &d))(SysDev) {
    if (d.lane_conv) {
#define PME_PICK(K) \
    if (d.lp_k1 == Cubic<K>::P1) return k_conv_p<Cubic<K>::P1>;
        PME_CUBIC_KS(PME_PICK)
#undef PME_PICK
    }
    return k_conv;
}

template <int P>
static void launch_tiles_spread(const SysDev &d, cudaStream_t s) {
    const unsigned nt = (unsigned)tile_threads(d, d.n);
    if (d.tlog == 4) launch_pdl(k_spread<P, 16>, d.ntiles + OVF_ITEMS, nt, smem_spread(P, 4), s, d, STAGE_SPREAD);
    else launch_pdl(k_spread<P, 8>, d.ntiles + OVF_ITEMS, nt, smem_spread(P, 3), s, d, STAGE_SPREAD);
}
template <int P>
static void launch_tiles_gather(const SysDev &d, cudaStream_t s) {
    const unsigned nt = (unsigned)tile_threads(d, d.n, true);
    if (d.tlog == 4) launch_pdl(k_gather<P, 16>, d.ntiles + OVF_ITEMS, nt, smem_gather_all(P, 4), s, d, STAGE_GATHER);
    else launch_pdl(k_gather<P, 8>, d.ntiles + OVF_ITEMS, nt, smem_gather_all(P, 3), s, d, STAGE_GATHER);
}

void launch_stage(const SysDev &d0, int stage, cudaStream_t s) {
    // with the tensor-core influence stage, every stage of the evaluation sees its tile count as the number
    // of influence items (the inverse stage's level-1 reduction reads that many partials)
    SysDev dt;
    if (d0.tc_w) {
        dt = d0;
        dt.nconv = tc_tiles(d0);
    }
    const SysDev &d = d0.tc_w ? dt : d0;
    switch (stage) {
        case STAGE_BIN:
            launch_pdl(k_bin, d.nbin > 0 ? d.nbin : 1, NT_BIN, smem_bin(NT_BIN), s, d, STAGE_BIN);
            break;
        case STAGE_SPREAD:
            if (d.p == 4) launch_tiles_spread<4>(d, s);
            else if (d.p == 5) launch_tiles_spread<5>(d, s);
            else if (d.p == 6) launch_tiles_spread<6>(d, s);
            else launch_tiles_spread<8>(d, s);
            break;
        case STAGE_FWD:
            if (!launch_split_slab(d, true, d.K1, s))
                launch_pdl(fwd_kernel(d), d.K1, NT_SLAB, smem_slab(d.K2, d.K3), s, d, STAGE_FWD);
            break;
        case STAGE_CONV:
            if (d.tc_w) {
                SysDev dp = d;
                dp.pdl_late = pdl_when(g_launch_mode, STAGE_CONV);
                launch_conv_tc(dp, d.tc_w, s);
            } else {
                launch_pdl(conv_kernel(d), d.nconv, NT_CONV, smem_conv(d.K1, NT_CONV), s, d, STAGE_CONV);
            }
            break;
        case STAGE_INV:
            if (!launch_split_slab(d, false, d.K1, s))
                launch_pdl(inv_kernel(d), d.K1, NT_SLAB, smem_inv(d.K2, d.K3), s, d, STAGE_INV);
            break;
        default:
            if (d.p == 4) launch_tiles_gather<4>(d, s);
            else if (d.p == 5) launch_tiles_gather<5>(d, s);
            else if (d.p == 6) launch_tiles_gather<6>(d, s);
            else launch_tiles_gather<8>(d, s);
            break;
    }
}

void launch_stage_items(const SysDev &d0, int stage, int first, int count, cudaStream_t s) {
    SysDev d = d0;
    d.item0 = first;
    if (count < 1) return;
    switch (stage) {
        case STAGE_FWD:
            launch_pdl(fwd_kernel(d), count, NT_SLAB, smem_slab(d.K2, d.K3), s, d, STAGE_FWD);
            break;
        case STAGE_CONV:
            launch_pdl(conv_kernel(d), count, NT_CONV, smem_conv(d.K1, NT_CONV), s, d, STAGE_CONV);
            break;
        case STAGE_INV:
            launch_pdl(inv_kernel(d), count, NT_SLAB, smem_inv(d.K2, d.K3), s, d, STAGE_INV);
            break;
        default:
            launch_stage(d0, stage, s);
            break;
    }
}

// Forces from device memory to page-locked host memory (coalesced 16-byte stores where both addresses
// allow) and the control block to its host copy: the last step of an evaluation on host arrays.
__global__ void __launch_bounds__(256) k_copy_out(const float *src, float *dst, long long nf, const Ctl *ctl, Ctl *hctl,
                                                  double *res8) {
    pdl_wait();
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x, nth = (long long)gridDim.x * blockDim.x;
    if (((((size_t)src) | ((size_t)dst)) & 15) == 0) {
        const long long n4 = nf >> 2;
        for (long long i = tid; i < n4; i += nth) ((float4 *)dst)[i] = __ldcg((const float4 *)src + i);
        for (long long i = (n4 << 2) + tid; i < nf; i += nth) dst[i] = __ldcg(src + i);
    } else {
        for (long long i = tid; i < nf; i += nth) dst[i] = __ldcg(src + i);
    }
    if (hctl && blockIdx.x == 0 && threadIdx.x < sizeof(Ctl) / 4)
        ((unsigned *)hctl)[threadIdx.x] = __ldcg((const unsigned *)ctl + threadIdx.x);
    if (res8 && blockIdx.x == 0 && threadIdx.x < 8)  // energy, virial[6], status bits
        res8[threadIdx.x] = threadIdx.x < 7 ? __ldcg(ctl->ev + threadIdx.x) : (double)__ldcg(&ctl->status);
}

cudaError_t launch_copy_out(const float *src, float *dst, long long nf, const Ctl *ctl, Ctl *hctl, cudaStream_t s,
                            double *res8) {
    long long blocks = (nf / 4 + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 1216) blocks = 1216;  // 152 SMs x 8
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = g_launch_mode ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_copy_out, src, dst, nf, ctl, hctl, res8);
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
