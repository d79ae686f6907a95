// Influence stage with the k1 transforms as dense matrix products on the tensor cores (tcgen05), for
// K1 = 128: the comparison path of the precision study at 128^3 (the paper lists reduced precision as
// future work, Sec. VI). The FP32 path transforms each half-spectrum column along k1 with a 128-point FFT;
// here a CTA takes 128 columns c at once and computes
//     Y^T[c, m] = sum_k X^T[c, k] W[m, k],   W[m, k] = exp(-2 pi i m k / 128),
// then Z = B C Y with the energy and virial terms (the same influence_point as the FP32 path), then the
// inverse O^T[c, k] = sum_m Z^T[c, m] conj(W[k, m]) (W is symmetric). Complex products are split into
// real ones (Yr = Xr Wr - Xi Wi, Yi = Xi Wr + Xr Wi and the conjugate for the inverse), and every real
// operand is an unevaluated sum of three BF16 numbers (hi + mid + lo, about 24 significant bits): the six
// term products whose error exceeds 2^-24 relative are kept (hh, hm, mh, hl, mm, lh), accumulated in FP32 in
// tensor memory. The tensor cores' FP32 accumulation truncates at every step, so the main product (hi x hi)
// and the five corrections go to separate accumulators, added in FP32 afterwards: the corrections, about
// 2^-8 of the result, then lose only 2^-8 of their truncation against the result.
//
// Per CTA (128 threads, one per column of the tile; one elected thread issues the MMAs):
//   A operand = the column data X^T (then Z^T): 128 rows (columns c) x 64 K, three terms x (re, im), written
//     by the threads in the 128-byte-swizzled K-major layout, one K half (64 of the 128 points) at a time;
//   B operand = W (rows n = output index, K = input index): precomputed per plan in the same layout, three
//     terms x (Wr, Wi) per K half, 96 KB, brought in with one bulk copy per half;
//   D = tensor memory: columns 0-127 re and 128-255 im of the main product, 256-511 the same for the
//     corrections; lane = c. The forward result Z goes back to the half spectrum (in place) and is read
//     again, one K half at a time, as the inverse transform's A operand.
// Every wait on an mbarrier is bounded (1 s); past it the kernel flags ST_TIMEOUT, stops issuing work,
// waits (bounded) for what it issued, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "../../include/pme.h"
#include "host_tables.h"
#include "kernels.h"
#include "pdl.cuh"
#include "plan_internal.h"
#include "stages.cuh"

namespace pme {

constexpr int TC_K1 = 128;
constexpr int TC_COLS = 128;                     // columns per tile (MMA M)
constexpr int TC_THREADS = 128;
constexpr int TC_BLOCK = 128 * 128;              // bytes of one 128-row x 64-K BF16 operand block
constexpr int TC_HALF_BYTES = 6 * TC_BLOCK;      // three terms x (re, im) of one K half: 96 KB
constexpr size_t TC_W_BYTES = 2 * (size_t)TC_HALF_BYTES;  // the W image, both K halves
static_assert(TC_W_BYTES == TC_W_IMAGE_BYTES, "W image size");
constexpr size_t TC_SMEM = 2 * (size_t)TC_HALF_BYTES + 1024 + 64;  // A and B halves, alignment, barriers

// ---- host side: the W image -----------------------------------------------------------------------------

static uint16_t bf16_bits(float f) {  // round to nearest even (finite values only)
    uint32_t u;
    memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
static double bf16_value(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}

// Byte offset of (row r, 16-byte chunk j) in a 128-row block of 128-byte rows, 128-byte swizzle.
static inline size_t sw128_offset(int r, int j) { return (size_t)(r >> 3) * 1024 + (size_t)(r & 7) * 128 + (size_t)((j ^ (r & 7)) << 4); }

// W image: [half][term][part (0: Wr, 1: Wi)] blocks, row n, K element k of the half.
void make_tc_w_image(std::vector<uint8_t> &img) {
    img.assign(TC_W_BYTES, 0);
    const double PI = 3.14159265358979323846;
    for (int h = 0; h < 2; ++h)
        for (int n = 0; n < TC_K1; ++n)
            for (int kk = 0; kk < 64; ++kk) {
                const int k = 64 * h + kk;
                const double ang = -2.0 * PI * (double)((n * k) % TC_K1) / (double)TC_K1;
                const double w[2] = {cos(ang), sin(ang)};  // Wr, Wi
                for (int part = 0; part < 2; ++part) {
                    double r = w[part];
                    for (int term = 0; term < 3; ++term) {
                        const uint16_t b = bf16_bits((float)r);
                        r -= bf16_value(b);
                        uint8_t *blk = img.data() + (size_t)h * TC_HALF_BYTES + (size_t)(2 * term + part) * TC_BLOCK;
                        const size_t off = sw128_offset(n, kk >> 3) + (size_t)(kk & 7) * 2;
                        memcpy(blk + off, &b, 2);
                    }
                }
            }
}

// ---- device side ------------------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long tc_globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait until the barrier's phase with this parity has completed; false after limit_ns.
__device__ bool mbar_wait(uint64_t *bar, unsigned parity, unsigned long long limit_ns) {
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = tc_globaltimer();
    while (!mbar_test(bar, parity)) {
        if (tc_globaltimer() - t0 > limit_ns) return false;
        __nanosleep(64);
    }
    return true;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: 128-byte swizzle, K-major, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major layouts)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                 // descriptor version
    d |= (uint64_t)2 << 61;                 // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: BF16 x BF16 -> FP32, both operands K-major, M x N, B optionally negated.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N, bool neg_b) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((neg_b ? 1u : 0u) << 14) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// x = hi + mid + lo in BF16 (each the rounded remainder of the previous).
__device__ __forceinline__ void split3(float x, uint16_t &h, uint16_t &m, uint16_t &l) {
    const __nv_bfloat16 bh = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(bh);
    const __nv_bfloat16 bm = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(bm);
    const __nv_bfloat16 bl = __float2bfloat16_rn(r2);
    h = __bfloat16_as_ushort(bh);
    m = __bfloat16_as_ushort(bm);
    l = __bfloat16_as_ushort(bl);
}

// Write this thread's row (column c of the tile) of one K half: re[k], im[k] for k < 64, as three terms.
__device__ __forceinline__ void write_a_row(uint8_t *A, int row, const float *re, const float *im) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {  // 16-byte chunk j: K elements 8j..8j+7
        uint32_t w[3][2][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            uint16_t h0, m0, l0, h1, m1, l1;
            split3(re[8 * j + e], h0, m0, l0);
            split3(re[8 * j + e + 1], h1, m1, l1);
            w[0][0][e >> 1] = (uint32_t)h0 | ((uint32_t)h1 << 16);
            w[1][0][e >> 1] = (uint32_t)m0 | ((uint32_t)m1 << 16);
            w[2][0][e >> 1] = (uint32_t)l0 | ((uint32_t)l1 << 16);
            split3(im[8 * j + e], h0, m0, l0);
            split3(im[8 * j + e + 1], h1, m1, l1);
            w[0][1][e >> 1] = (uint32_t)h0 | ((uint32_t)h1 << 16);
            w[1][1][e >> 1] = (uint32_t)m0 | ((uint32_t)m1 << 16);
            w[2][1][e >> 1] = (uint32_t)l0 | ((uint32_t)l1 << 16);
        }
        const uint32_t off = (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((j ^ (row & 7)) << 4));
#pragma unroll
        for (int t = 0; t < 3; ++t)
#pragma unroll
            for (int p = 0; p < 2; ++p)
                *(uint4 *)(A + (size_t)(2 * t + p) * TC_BLOCK + off) = make_uint4(w[t][p][0], w[t][p][1], w[t][p][2], w[t][p][3]);
    }
}

// The 96 MMAs of one K half: 4 steps of 16, 6 term pairs, 4 real products each; the main pair (hi x hi)
// into the accumulators at tmem, the corrections into those at tmem + 256. inverse selects the signs of the
// conjugate transform. first: the half that initialises the accumulators.
__device__ void issue_half(uint32_t tmem, uint32_t a_base, uint32_t b_base, bool inverse, bool first) {
    const uint32_t ip = tc_idesc(128, 128, false), in = tc_idesc(128, 128, true);
#pragma unroll 1
    for (int ks = 0; ks < 4; ++ks) {
#pragma unroll
        for (int pr = 0; pr < 6; ++pr) {
            // (data term, W term): hh, then the corrections lh, mm, hl, mh, hm (smallest first)
            const int t = pr == 0 ? 0 : pr == 1 ? 2 : pr == 2 ? 1 : pr == 3 ? 0 : pr == 4 ? 1 : 0;
            const int s = pr == 0 ? 0 : pr == 1 ? 0 : pr == 2 ? 1 : pr == 3 ? 2 : pr == 4 ? 0 : 1;
            const uint32_t d_re = tmem + (pr == 0 ? 0u : 256u), d_im = d_re + 128u;
            const uint32_t koff = (uint32_t)(ks * 32);  // 16 BF16 = 32 bytes along K inside the swizzle atom
            const uint64_t ar = sw128_desc(a_base + (uint32_t)(2 * t) * TC_BLOCK + koff);
            const uint64_t ai = sw128_desc(a_base + (uint32_t)(2 * t + 1) * TC_BLOCK + koff);
            const uint64_t br = sw128_desc(b_base + (uint32_t)(2 * s) * TC_BLOCK + koff);
            const uint64_t bi = sw128_desc(b_base + (uint32_t)(2 * s + 1) * TC_BLOCK + koff);
            const uint32_t acc = (first && ks == 0 && pr <= 1) ? 0u : 1u;  // pr 0 and 1 open their accumulators
            if (!inverse) {  // Yr = Xr Wr - Xi Wi ; Yi = Xi Wr + Xr Wi
                tc_mma(d_re, ar, br, ip, acc);
                tc_mma(d_re, ai, bi, in, 1u);
                tc_mma(d_im, ai, br, ip, acc);
                tc_mma(d_im, ar, bi, ip, 1u);
            } else {  // Or = Zr Wr + Zi Wi ; Oi = Zi Wr - Zr Wi
                tc_mma(d_re, ar, br, ip, acc);
                tc_mma(d_re, ai, bi, ip, 1u);
                tc_mma(d_im, ai, br, ip, acc);
                tc_mma(d_im, ar, bi, in, 1u);
            }
        }
    }
}

struct TcArgs {
    SysDev d;
    const uint8_t *w_img;  // TC_W_BYTES, device
    int ntiles;            // column tiles of TC_COLS
};

__global__ void __launch_bounds__(TC_THREADS, 1) k_conv_tc(TcArgs args) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const SysDev &d = args.d;
    PdlScope pdl(d.pdl_late);
    // 1024-byte alignment for the swizzled operand blocks
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *A = base;
    uint8_t *B = base + TC_HALF_BYTES;
    uint64_t *bars = (uint64_t *)(base + 2 * TC_HALF_BYTES);  // [0] B loaded, [1] MMAs done
    uint32_t *tmem_slot = (uint32_t *)(bars + 2);
    int *abort_flag = (int *)(tmem_slot + 1);
    float *red = (float *)A;  // energy / virial reduction scratch (7 x 128), used after the last MMAs
    const int tid = threadIdx.x, warp = tid >> 5;
    const unsigned long long LIMIT = 1000000000ull;

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_addr(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    const uint32_t a_s = smem_addr(A), b_s = smem_addr(B);
    unsigned ph_b = 0, ph_m = 0;  // parities of the next completion of bars[0] and bars[1]
    const int K2 = d.K2, H3 = d.H3, ncol = K2 * H3;
    const float inv_h3 = 1.0f / (float)H3;
    bool ok = true;

    for (int tile = blockIdx.x; tile < args.ntiles && ok; tile += gridDim.x) {
        const int col = tile * TC_COLS + tid;
        const bool live = col < ncol;
        const int cc = live ? col : 0;
        const int m2 = fdiv(cc, inv_h3), m3 = cc - m2 * H3;
        float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        // forward (dir 0) then inverse (dir 1), each over two K halves
        for (int dir = 0; dir < 2 && ok; ++dir) {
            for (int h = 0; h < 2 && ok; ++h) {
                if (tid == 0) {  // B half h (the same W image serves both directions)
                    mbar_arrive_expect_tx(&bars[0], (unsigned)TC_HALF_BYTES);
                    bulk_g2s(B, args.w_img + (size_t)h * TC_HALF_BYTES, (unsigned)TC_HALF_BYTES, &bars[0]);
                }
                // the column's points 64 h .. 64 h + 63 along k1: X (forward) or Z (inverse, written below)
                float re[64], im[64];
#pragma unroll
                for (int kk = 0; kk < 64; ++kk) {
                    const float2 x = live ? ldcg(d.spec + ((size_t)(64 * h + kk) * K2 + m2) * H3 + m3) : make_float2(0.f, 0.f);
                    re[kk] = x.x;
                    im[kk] = x.y;
                }
                write_a_row(A, tid, re, im);
                fence_proxy_async();
                tc_fence_before();
                __syncthreads();
                if (tid == 0) {
                    tc_fence_after();
                    if (!mbar_wait(&bars[0], ph_b, LIMIT)) {
                        *abort_flag = 1;
                    } else {
                        issue_half(tmem, a_s, b_s, dir == 1, h == 0);
                        tc_commit(&bars[1]);
                    }
                }
                ph_b ^= 1u;
                __syncthreads();
                if (*abort_flag) {
                    ok = false;
                    break;
                }
                // every thread waits for the MMAs before the next half overwrites A and B
                if (!mbar_wait(&bars[1], ph_m, LIMIT)) *abort_flag = 1;
                ph_m ^= 1u;
                tc_fence_after();
                __syncthreads();
                if (*abort_flag) ok = false;
            }
            if (!ok) break;
            // result = main + corrections; the forward result times B C (with the energy and virial terms)
            // and the inverse result back to the half spectrum, in place, index 16 q + e along k1
            const int mt2 = signed_freq(m2, K2);
#pragma unroll 1
            for (int q = 0; q < 8; ++q) {
                float a0[16], a1[16], c0[16], c1[16];
                tmem_ld16(tmem + lane_base + (uint32_t)(16 * q), a0);
                tmem_ld16(tmem + lane_base + 128u + (uint32_t)(16 * q), a1);
                tmem_ld16(tmem + lane_base + 256u + (uint32_t)(16 * q), c0);
                tmem_ld16(tmem + lane_base + 384u + (uint32_t)(16 * q), c1);
                if (live) {
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int k = 16 * q + e;
                        float2 v = make_float2(a0[e] + c0[e], a1[e] + c1[e]);
                        if (dir == 0) {
                            const float4 t = ldcg(d.bc + ((size_t)m2 * TC_K1 + k) * H3 + m3);
                            v = influence_point(d, k, m2, m3, mt2, v, t, acc);
                        }
                        d.spec[((size_t)k * K2 + m2) * H3 + m3] = v;
                    }
                }
            }
            tc_fence_before();
            __syncthreads();  // tensor memory read before the next MMAs overwrite it
            tc_fence_after();
        }
        if (!ok) break;
        // the tile's energy / virial partial: fixed-order double-float sums over the 128 columns
#pragma unroll
        for (int c = 0; c < 7; ++c) red[c * TC_THREADS + tid] = live ? acc[c] : 0.f;
        __syncthreads();
        if (tid < 7) {
            DF s;
            s.hi = red[tid * TC_THREADS];
            s.lo = 0.f;
            for (int t = 1; t < TC_THREADS; ++t) s = df_add(s, red[tid * TC_THREADS + t]);
            ((DF *)d.partials)[(size_t)tile * 8 + tid] = s;
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    if (!ok && tid == 0) atomicOr(&d.ctl->status, ST_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

cudaError_t configure_tc_kernel() {
    return cudaFuncSetAttribute((const void *)k_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
}

int tc_tiles(const SysDev &d) { return (d.K2 * d.H3 + TC_COLS - 1) / TC_COLS; }

cudaError_t launch_conv_tc(const SysDev &d, const void *w_img, cudaStream_t s) {
    TcArgs a;
    a.d = d;
    a.w_img = (const uint8_t *)w_img;
    a.ntiles = tc_tiles(d);
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)(a.ntiles < sms ? a.ntiles : sms);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = TC_SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = launch_mode() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_conv_tc, a);
}

}  // namespace pme
