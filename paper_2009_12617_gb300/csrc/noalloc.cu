// Allocation-free single-system evaluation: pme_compute_noalloc.
//
// Who needs it: callers that must not allocate device memory themselves. An application that has
// handed all device memory to its own pool up front (a caching allocator, an arena sized at start-up)
// may have nothing left for cudaMalloc, and cudaMalloc / cudaFree synchronise the device, which a
// latency-bound caller (a request loop, a real-time controller) cannot afford on every call. Such
// callers pass only their inputs and outputs; everything else lives in a fixed static device array.
//
// How: one cooperative kernel runs every stage of the evaluation (influence-table set-up, binning,
// spreading, forward FFT, influence multiply with energy / virial, inverse FFT, force interpolation),
// separated by grid-wide barriers. The cooperative launch guarantees that all CTAs are resident, so the
// barriers always complete. All scratch is carved out of g_noalloc_scratch, a file-scope
// static __device__ array of NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until exit.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

// The single cooperative kernel keeps only the shared-memory transforms (one code path per stage keeps it
// small to build); its plans say so through choose_fft_paths(d, false).
#define PME_NO_LANE_FFT 1
#include "../../include/pme.h"
#include "host_tables.h"
#include "kernels.h"
#include "plan_internal.h"
#include "stages.cuh"

namespace cg = cooperative_groups;

namespace pme {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)4 << 20;  // 4 MiB per device
constexpr int NOALLOC_MAX_MESH_POINTS = 32768;             // K1 * K2 * K3 (e.g. 32^3)
constexpr int64_t NOALLOC_MAX_ATOMS = 16384;
constexpr int NOALLOC_THREADS = 256;

}  // namespace pme

// The scratch array. In host code this name is only a stand-in for the device symbol; its device address
// comes from cudaGetSymbolAddress in noalloc_setup().
static __device__ __align__(256) unsigned char g_noalloc_scratch[pme::NOALLOC_SCRATCH_BYTES];

namespace pme {

struct NoallocArgs {
    SysDev d;
    double recip[9];  // a*_alpha[j] at 3*alpha + j
    double vol, beta;
    double *bmod;     // |b_1|^2 (K1), |b_2|^2 (K2), |b_3|^2 (K3)
    float4 *bc;       // writable alias of d.bc
    float2 *tw;       // writable alias of the twiddle block (K1 + K2 + K3/2 + K3/2 + 1)
    unsigned long long zero_bytes;  // bytes from the scratch start that must be zero before binning
};

__device__ double dev_signed_freq(int m, int K) { return (double)(2 * m <= K ? m : m - K); }

__device__ double dev_norm2(const NoallocArgs &A, double mt1, double mt2, double mt3) {
    const double *r = A.recip;
    double mv[3];
    for (int j = 0; j < 3; ++j) mv[j] = mt1 * r[j] + mt2 * r[3 + j] + mt3 * r[6 + j];
    return mv[0] * mv[0] + mv[1] * mv[1] + mv[2] * mv[2];
}
// C(m) and the virial factor f(m) = 2 (1 / |m'|^2 + pi^2 / beta^2) from |m'|^2
__device__ double dev_influence_c(const NoallocArgs &A, double m2n) {
    const double pi = 3.14159265358979323846;
    return exp(-pi * pi * m2n / (A.beta * A.beta)) / (pi * A.vol * m2n);
}
__device__ double dev_virial_f(const NoallocArgs &A, double m2n) {
    const double pi = 3.14159265358979323846;
    return 2.0 * (1.0 / m2n + pi * pi / (A.beta * A.beta));
}

template <int P>
__global__ void __launch_bounds__(NOALLOC_THREADS) k_eval_noalloc(NoallocArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    cg::grid_group grid = cg::this_grid();
    const SysDev &d = A.d;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int gtid = blockIdx.x * nth + tid, gnth = gridDim.x * nth;

    // 0: clear what must start at zero (control block, counters, partials, charge mesh) whatever the
    //    previous call left; B-spline moduli and FFT twiddles for this mesh.
    {
        unsigned long long *z = (unsigned long long *)g_noalloc_scratch;
        for (unsigned long long i = gtid; i < A.zero_bytes / 8; i += gnth) z[i] = 0ull;
        const int Ks[3] = {d.K1, d.K2, d.K3};
        const int Ktot = d.K1 + d.K2 + d.K3;
        for (int i = gtid; i < Ktot; i += gnth) {
            const int al = i < d.K1 ? 0 : (i < d.K1 + d.K2 ? 1 : 2);
            const int m = i - (al == 0 ? 0 : (al == 1 ? d.K1 : d.K1 + d.K2));
            const int K = Ks[al];
            // M_P at the integer knots by the unnormalised recursion, then the Euler spline denominator
            double M[P + 1], prev[P + 1];
            for (int x = 0; x <= P; ++x) prev[x] = (x == 1) ? 1.0 : 0.0;
            for (int nn = 3; nn <= P; ++nn) {
                for (int x = 0; x <= P; ++x) M[x] = ((double)x * prev[x] + (double)(nn - x) * (x >= 1 ? prev[x - 1] : 0.0)) / (nn - 1);
                for (int x = 0; x <= P; ++x) prev[x] = M[x];
            }
            double sr = 0.0, si = 0.0;
            for (int k = 0; k <= P - 2; ++k) {
                double s, c;
                sincospi(2.0 * (double)((m * k) % K) / (double)K, &s, &c);
                sr += prev[k + 1] * c;
                si += prev[k + 1] * s;
            }
            A.bmod[i] = 1.0 / (sr * sr + si * si);
        }
        const int Nh = d.K3 / 2;
        const int lens[4] = {d.K1, d.K2, Nh, d.K3};
        const int counts[4] = {d.K1, d.K2, Nh, Nh + 1};
        const int ntw = d.K1 + d.K2 + Nh + Nh + 1;
        for (int i = gtid; i < ntw; i += gnth) {
            int seg = 0, k = i;
            while (k >= counts[seg]) k -= counts[seg++];
            double s, c;
            sincospi(-2.0 * (double)k / (double)lens[seg], &s, &c);
            A.tw[i] = make_float2((float)c, (float)s);
        }
    }
    grid.sync();
    // 1: influence table on the half spectrum, [m2][m1][m3] (SysDev::bc): B(m) (C(m) + C(-m)) / 2 as (hi, lo)
    // floats, then B C f(m) and, off the self-conjugate planes on a Nyquist plane, B C f(m_p)
    {
        const int H3 = d.H3;
        const int tot = d.K1 * d.K2 * H3;
        for (int i = gtid; i < tot; i += gnth) {
            const int m3 = i % H3, m1 = (i / H3) % d.K1, m2 = i / (H3 * d.K1);
            double v = 0.0, g = 0.0, gp = 0.0;
            if (m1 | m2 | m3) {
                const int mt1 = dev_signed_freq(m1, d.K1), mt2 = dev_signed_freq(m2, d.K2), mt3 = dev_signed_freq(m3, d.K3);
                const double nm = dev_norm2(A, mt1, mt2, mt3);
                const double np = dev_norm2(A, dev_signed_freq((d.K1 - m1) % d.K1, d.K1),
                                            dev_signed_freq((d.K2 - m2) % d.K2, d.K2),
                                            dev_signed_freq((d.K3 - m3) % d.K3, d.K3));
                v = A.bmod[m1] * A.bmod[d.K1 + m2] * A.bmod[d.K1 + d.K2 + m3] * 0.5 *
                    (dev_influence_c(A, nm) + dev_influence_c(A, np));
                g = v * dev_virial_f(A, nm);
                const bool self = m3 == 0 || 2 * m3 == d.K3;
                if (!self && (2 * m1 == d.K1 || 2 * m2 == d.K2))
                    gp = v * dev_virial_f(A, dev_norm2(A, 2 * m1 == d.K1 ? mt1 : -mt1, 2 * m2 == d.K2 ? mt2 : -mt2, -mt3));
            }
            const float hi = (float)v;
            A.bc[i] = make_float4(hi, (float)(v - (double)hi), (float)g, (float)gp);
        }
    }
    grid.sync();
    // 2..7: the six pipeline stages, each over its work items, with a grid barrier in between
    // A CTA that takes several items of one stage waits at a CTA barrier after each: the next item's first
    // shared-memory writes (spread_clear, the gather's region load) must not overtake warps still reading
    // the previous item's tile.
    const int nbin = d.nbin;
    for (int it = blockIdx.x; it < nbin; it += gridDim.x) {
        stage_bin(d, it, smem);
        __syncthreads();
    }
    grid.sync();
    for (int it = blockIdx.x; it < d.ntiles + OVF_ITEMS; it += gridDim.x) {
        stage_spread<P, 8>(d, it, smem);
        __syncthreads();
    }
    grid.sync();
    for (int it = blockIdx.x; it < d.K1; it += gridDim.x) {
        stage_fwd(d, it, smem);
        __syncthreads();
    }
    grid.sync();
    for (int it = blockIdx.x; it < d.nconv; it += gridDim.x) {
        stage_conv(d, it, smem);
        __syncthreads();
    }
    grid.sync();
    for (int it = blockIdx.x; it < d.K1; it += gridDim.x) {
        stage_inv(d, it, smem);
        __syncthreads();
    }
    grid.sync();
    for (int it = blockIdx.x; it < d.ntiles + OVF_ITEMS; it += gridDim.x) {
        stage_gather<P, 8>(d, it, smem);
        __syncthreads();
    }
}

struct NoallocDevice {
    bool ready = false;
    unsigned char *scratch = nullptr;  // device address of g_noalloc_scratch
    int grid[9] = {0};                 // co-resident CTAs for P = 4, 6, 8 (index P)
};

static std::mutex g_noalloc_mu;
static NoallocDevice g_noalloc_dev[64];

static size_t noalloc_smem(int K[3], int p) {
    size_t s = smem_bin(NOALLOC_THREADS);
    s = s > smem_spread(p, 3) ? s : smem_spread(p, 3);  // this path always uses 8^3 tiles
    s = s > smem_gather_all(p, 3) ? s : smem_gather_all(p, 3);
    s = s > smem_slab(K[1], K[2]) ? s : smem_slab(K[1], K[2]);
    s = s > smem_inv(K[1], K[2]) ? s : smem_inv(K[1], K[2]);
    s = s > smem_conv(K[0], NOALLOC_THREADS) ? s : smem_conv(K[0], NOALLOC_THREADS);
    return s;
}

// Once per device, with that device current: the scratch array's device address and the number of CTAs
// of each kernel variant that fit on the device at once (the cooperative grid size).
static pme_status noalloc_setup(int dev, NoallocDevice **out) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (dev < 0 || dev >= 64) return fail(PME_ECUDA, "device index %d out of range", dev);
    NoallocDevice &nd = g_noalloc_dev[dev];
    if (!nd.ready) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        int sms = 0, coop = 0;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return cuda_fail(e, "cudaDeviceGetAttribute");
        if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev)) != cudaSuccess)
            return cuda_fail(e, "cudaDeviceGetAttribute");
        if (!coop) return fail(PME_EUNSUPPORTED, "device does not support cooperative launches");
        const void *fns[3] = {(const void *)k_eval_noalloc<4>, (const void *)k_eval_noalloc<6>,
                              (const void *)k_eval_noalloc<8>};
        const int ps[3] = {4, 6, 8};
        for (int i = 0; i < 3; ++i) {
            int K[3] = {64, 64, 64};  // the largest shared-memory footprint the size limits allow
            const size_t smem = noalloc_smem(K, ps[i]);
            if ((e = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
                return cuda_fail(e, "cudaFuncSetAttribute(k_eval_noalloc)");
            int per_sm = 0;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fns[i], NOALLOC_THREADS, smem)) != cudaSuccess)
                return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
            if (per_sm < 1) return fail(PME_ECUDA, "k_eval_noalloc does not fit on an SM");
            nd.grid[ps[i]] = sms * (per_sm < 2 ? per_sm : 2);
        }
        nd.scratch = (unsigned char *)ptr;
        nd.ready = true;
    }
    *out = &nd;
    return PME_OK;
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace pme

using namespace pme;

extern "C" pme_status pme_compute_noalloc(const int K[3], int p, double beta, const double box[9], const float *pos,
                                          const float *q, int64_t n, float *forces, double *energy, double *virial,
                                          void *cuda_stream) {
    if (!K || !box) return fail(PME_EINVAL, "K and box must be non-NULL");
    char msg[256];
    const int v = validate_params(K, p, beta, box, msg, sizeof(msg));
    if (v == 1) return fail(PME_EINVAL, "%s", msg);
    if (v == 2) return fail(PME_EUNSUPPORTED, "%s", msg);
    if (p != 4 && p != 6 && p != 8) return fail(PME_EUNSUPPORTED, "pme_compute_noalloc: B-spline orders 4, 6 and 8 only");
    const int64_t mesh = (int64_t)K[0] * K[1] * K[2];
    if (mesh > NOALLOC_MAX_MESH_POINTS || K[0] > 64 || K[1] > 64 || K[2] > 64)
        return fail(PME_EINVAL, "pme_compute_noalloc: mesh %dx%dx%d exceeds its static limit (K1*K2*K3 <= %d, each K <= 64)",
                    K[0], K[1], K[2], NOALLOC_MAX_MESH_POINTS);
    if (n < 0 || n > NOALLOC_MAX_ATOMS)
        return fail(PME_EINVAL, "pme_compute_noalloc: n = %lld outside [0, %lld]", (long long)n, (long long)NOALLOC_MAX_ATOMS);
    if (n > 0 && (!pos || !q || !forces)) return fail(PME_EINVAL, "pos, q and forces must be non-NULL when n > 0");
    double recip[9], vol;
    if (!cell_reciprocal(box, recip, &vol)) return fail(PME_EINVAL, "box is singular");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    NoallocDevice *nd = nullptr;
    pme_status st = noalloc_setup(dev, &nd);
    if (st != PME_OK) return st;

    // carve the static scratch: everything that must start at zero comes first
    NoallocArgs A;
    memset(&A, 0, sizeof(A));
    SysDev &d = A.d;
    fill_geometry(d, K, p, beta, recip);
    choose_fft_paths(d, false);
    const size_t K1 = K[0], K2 = K[1], K3 = K[2], H3 = d.H3, Nh = K3 / 2;
    const int64_t ncap = n > 0 ? n : 1;
    const int cap = bucket_capacity(ncap, d.ntiles, d.tlog);
    size_t off = 0;
    const size_t o_ctl = off;  off = al256(off + sizeof(Ctl));
    const size_t o_cnt = off;  off = al256(off + bcount_bytes(d.ntiles));
    const size_t o_qs = off;   off = al256(off + QABS_BYTES);
    const size_t o_par = off;  off = al256(off + partials_bytes(d));
    const size_t o_grid = off; off = al256(off + K1 * K2 * K3 * 8);
    const size_t zero_bytes = off;
    const size_t o_bmod = off; off = al256(off + (K1 + K2 + K3) * 8);
    const size_t o_tw = off;   off = al256(off + (K1 + K2 + Nh + Nh + 1) * 8);
    const size_t o_bc = off;   off = al256(off + K1 * K2 * H3 * sizeof(float4));
    const size_t o_spec = off; off = al256(off + K1 * K2 * H3 * 8);
    const size_t o_phi = off;  off = al256(off + K1 * K2 * K3 * 4);
    const size_t o_bka = off;  off = al256(off + (size_t)d.ntiles * cap * 16);
    const size_t o_bkb = off;  off = al256(off + (size_t)d.ntiles * cap * 8);
    const size_t o_ova = off;  off = al256(off + (size_t)ncap * 16);
    const size_t o_ovb = off;  off = al256(off + (size_t)ncap * 8);
    if (off > NOALLOC_SCRATCH_BYTES)
        return fail(PME_EINVAL, "pme_compute_noalloc: this system needs %zu bytes of scratch; the static limit is %zu",
                    off, NOALLOC_SCRATCH_BYTES);
    unsigned char *b = nd->scratch;
    d.ctl = (Ctl *)(b + o_ctl);
    d.bcount = (unsigned *)(b + o_cnt);
    d.qslot = (unsigned long long *)(b + o_qs);
    d.partials = (double *)(b + o_par);
    d.grid = (unsigned long long *)(b + o_grid);
    A.bmod = (double *)(b + o_bmod);
    A.tw = (float2 *)(b + o_tw);
    d.tw1 = A.tw;
    d.tw2 = A.tw + K1;
    d.tw3h = A.tw + K1 + K2;
    d.tw3 = A.tw + K1 + K2 + Nh;
    A.bc = (float4 *)(b + o_bc);
    d.bc = A.bc;
    d.spec = (float2 *)(b + o_spec);
    d.phi = (float *)(b + o_phi);
    d.bka = (float4 *)(b + o_bka);
    d.bkb = (int2 *)(b + o_bkb);
    d.ova = (float4 *)(b + o_ova);
    d.ovb = (int2 *)(b + o_ovb);
    d.cap = cap;
    d.n = (int)n;
    d.nbin = (int)((n + BIN_CHUNK - 1) / BIN_CHUNK);
    d.pos = pos;
    d.q = q;
    d.forces = forces;
    d.ev = d.ctl->ev;
    memcpy(A.recip, recip, sizeof(recip));
    A.vol = vol;
    A.beta = beta;
    A.zero_bytes = zero_bytes;

    int Kc[3] = {K[0], K[1], K[2]};
    const size_t smem = noalloc_smem(Kc, p);
    const void *fn = p == 4 ? (const void *)k_eval_noalloc<4> : (p == 6 ? (const void *)k_eval_noalloc<6> : (const void *)k_eval_noalloc<8>);
    void *args[] = {&A};
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    e = cudaLaunchCooperativeKernel(fn, dim3(nd->grid[p]), dim3(NOALLOC_THREADS), args, smem, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaLaunchCooperativeKernel(k_eval_noalloc)");
    Ctl h;  // pageable host copy: this copy returns once the kernel and the copy are done
    if ((e = cudaMemcpyAsync(&h, d.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync(result)");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if ((st = status_from_bits(h.status)) != PME_OK) return st;
    if (energy) *energy = h.ev[0];
    if (virial)
        for (int c = 0; c < 6; ++c) virial[c] = h.ev[1 + c];
    return PME_OK;
}
