// Shared definitions for the SPME stage bodies.
//
// Every stage body is written as a sequence of data-parallel phases ("for idx = tid; idx < total;
// idx += nthreads") separated by CTA barriers. Built by nvcc they are the CUDA kernels' bodies; built by
// a host C++ compiler with PME_HOST_EMULATION they run with one thread per CTA (tid = 0, nthreads = 1,
// barriers vanish), which the CPU tests use to check the index arithmetic against the FP64 oracle. The
// library itself only contains the CUDA build.
#pragma once

#include <math.h>
#include <stdint.h>

#if defined(PME_HOST_EMULATION)
#include <cuda_runtime.h>  // host-side vector types only (float2, float4, int2, ulonglong2)
#include <string.h>
#define PME_DEV inline
#define PME_TID 0
#define PME_NTH 1
#define PME_SYNC() ((void)0)
#define PME_FENCE() ((void)0)
#define PME_SHARED static
#else
#include <cuda_runtime.h>
#define PME_DEV __device__ __forceinline__
#define PME_TID ((int)threadIdx.x)
#define PME_NTH ((int)blockDim.x)
#define PME_SYNC() __syncthreads()
#define PME_FENCE() __threadfence()
#define PME_SHARED __shared__
#endif

namespace pme {

// Mesh edge of a spread / gather tile: 2^tlog with tlog 3 or 4, chosen per plan from the atom density
// (about a hundred atoms or more per tile). Atoms are binned by the tile that holds their highest support
// point; the tile's shared-memory region is (T + p - 1)^3 mesh points. Results do not depend on the choice.
constexpr int TILE_MIN_LOG = 3, TILE_MAX_LOG = 4;
// Fixed-point scale of the charge mesh: Q is accumulated as round(q theta1 theta2 theta3 * 2^40) in int64,
// so the mesh is bit-identical whatever order the atoms are added in.
constexpr float FIX_SCALE = 1099511627776.0f;            // 2^40
constexpr float FIX_INV = 9.094947017729282379150390625e-13f;  // 2^-40
// Sum |q| is accumulated in fixed point 2^24 per e. The mesh headroom is |Q| < 2^23 e; sum |q| < 2^22 e
// bounds every mesh value and every partial sum, so larger totals are refused.
constexpr float QABS_SCALE = 16777216.0f;                // 2^24
constexpr unsigned long long QABS_LIMIT = 1ull << 46;    // 2^22 e in 2^24 units
// The binning CTAs add their sums of |q| into QABS_SLOTS counters, one per 128-byte line (CTA b into
// b mod QABS_SLOTS), so no single address collects one atomic per CTA; the force stage's final reduction
// adds them up and resets them.
constexpr int QABS_SLOTS = 64;
constexpr size_t QABS_BYTES = (size_t)QABS_SLOTS * 128;
constexpr int BIN_PER_THREAD = 1;           // atoms per thread per pass of the binning stage
constexpr int BIN_CHUNK = 128 * BIN_PER_THREAD;  // atoms per binning work item
constexpr int OVF_ITEMS = 8;     // extra spread / gather work items that handle bucket-overflow atoms
constexpr int MAX_K = 128;
// Tile counters sit on separate 128-byte lines so the binning atomics spread over the L2 slices.
constexpr int BCOUNT_STRIDE = 32;
// Shared-memory accumulation splits each fixed-point contribution v into hi = rn(v / 2^20) and
// lo = rn(v - hi 2^20) in [-2^19, 2^19], summed in two int32 arrays with native 32-bit atomics. A B-spline
// weight of order >= 4 is at most 2/3, so with |q| <= Q_TILE_MAX every |v| <= 2 (2/3)^3 2^40 < 2^39, |hi|
// <= 2^19; with at most 1024 atoms per tile neither sum reaches 2^30. Atoms with larger charges take the
// 64-bit global path instead. Bucket capacity per tile: at most CAP_MAX (8^3 tiles) or CAP_MAX16 (16^3).
constexpr float Q_TILE_MAX = 2.0f;
constexpr int CAP_MAX = 512;
constexpr int CAP_MAX16 = 1024;
constexpr int cap_max_for(int tlog) { return tlog >= 4 ? CAP_MAX16 : CAP_MAX; }
// Columns m3 per influence-stage work item (shared-memory transform path).
constexpr int CONV_COLS = 8;
// Lane plans of the register-resident transforms: plan c has length LANE_L[c] * LANE_E[c], L lanes of
// E points each (fft.cuh, lane_fft). Lengths without a plan use the shared-memory Stockham path.
constexpr int LANE_PLANS = 21;
#define PME_LANE_CASES(X)                                                                               \
    X(0, 1, 4) X(1, 1, 5) X(2, 1, 6) X(3, 1, 8) X(4, 2, 4) X(5, 2, 5) X(6, 2, 6) X(7, 2, 8) X(8, 4, 4) \
        X(9, 4, 5) X(10, 4, 6) X(11, 4, 8) X(12, 8, 4) X(13, 8, 5) X(14, 8, 6) X(15, 8, 8) X(16, 16, 4) \
            X(17, 16, 5) X(18, 16, 6) X(19, 16, 8) X(20, 32, 4)
// Threads (lanes) per influence-stage work item on the register path: 128 / L columns of L lanes each.
constexpr int CONV_UNITS = 128;
// Threads of a slab-stage CTA (the register path picks its lane plans to fill about this many).
constexpr int SLAB_THREADS = 512;

#if defined(PME_HOST_EMULATION)
#define PME_HD constexpr inline
#else
#define PME_HD __host__ __device__ constexpr inline
#endif

// Lanes L and points per lane E of lane plan c.
#define PME_PLAN_L(c_, L_, E_) c == c_ ? L_:
#define PME_PLAN_E(c_, L_, E_) c == c_ ? E_:
PME_HD int plan_L(int c) { return PME_LANE_CASES(PME_PLAN_L) 1; }
PME_HD int plan_E(int c) { return PME_LANE_CASES(PME_PLAN_E) 1; }
#undef PME_PLAN_L
#undef PME_PLAN_E

// Plan for ntr transforms of length N in one slab CTA: the fewest points per lane (the shortest serial
// chain per thread) whose lanes still fit in SLAB_THREADS, else the plan with the fewest lanes; -1 when N
// has no plan.
PME_HD int slab_lane_plan(int N, int ntr) {
    int best = -1, fewest = -1;
    for (int c = 0; c < LANE_PLANS; ++c) {
        const int L = plan_L(c), E = plan_E(c);
        if (L * E != N) continue;
        const int T = 32 / L, units = ((ntr + T - 1) / T) * 32;
        if (units <= SLAB_THREADS && (best < 0 || E < plan_E(best))) best = c;
        if (fewest < 0 || L < plan_L(fewest)) fewest = c;
    }
    return best >= 0 ? best : fewest;
}

// Plan of the influence stage's K1-point transforms: the fewest points per lane, so that the work spreads
// over as many threads as possible, with at most 16 lanes per transform so that a warp spans at least two
// adjacent columns (its loads along k1 then use whole 16-byte pieces of each row).
PME_HD int conv_lane_plan(int N) {
    int best = -1;
    for (int c = 0; c < LANE_PLANS; ++c)
        if (plan_L(c) * plan_E(c) == N && plan_L(c) <= 16 && (best < 0 || plan_E(c) < plan_E(best))) best = c;
    return best;
}
// Independent global loads each thread keeps in flight when staging data into shared memory.
constexpr int LOAD_BATCH = 8;
// Slots of the fixed-order final energy / virial reduction (a power of two, >= MAX_K / 2).
constexpr int REDUCE_SLOTS = 64;

enum StatusBits : unsigned {
    ST_NONFINITE = 1u,   // a position or charge is NaN / Inf, or absurdly far outside the cell
    ST_OVERFLOW = 2u,    // sum |q| beyond the fixed-point headroom
    ST_TIMEOUT = 4u,     // a bounded dependency wait gave up
    ST_INTERNAL = 8u     // an internal consistency check failed
};

// Per-system control block in device memory. Zeroed at creation; every counter is reset by the stage
// that consumes it last, so no memset is needed between evaluations.
struct Ctl {
    unsigned status;            // StatusBits, latched until the host reads and clears it
    unsigned novf;              // atoms that did not fit in their tile's bucket
    unsigned long long unused;  // (kept for the layout the host copy expects)
    unsigned novf_gather;       // copy of novf taken by the spreading stage for the force stage
    unsigned pad[3];
    double ev[8];               // energy, virial xx yy zz xy xz yz (internal copy for synchronous calls)
};

// Everything a stage needs to know about one system, passed by value to kernels.
struct SysDev {
    int K1, K2, K3, H3;          // mesh; H3 = K3/2 + 1 (half spectrum along k3)
    int p;                       // B-spline order
    int tlog;                    // tile edge 2^tlog mesh points
    int nt1, nt2, nt3, ntiles;   // spread / gather tiles per dimension (nt1: pieces of the k1 axis)
    float rnt1;                  // 1 / nt1
    int cap;                     // bucket capacity (atoms per tile)
    int n;                       // atoms
    int nbin;                    // binning work items = ceil(n / BIN_CHUNK)
    int nchunk3;                 // influence-stage column chunks = ceil(H3 / CONV_COLS) (shared-memory path)
    int nconv;                   // influence-stage work items: K2 * nchunk3, or the register path's
                                 // ceil(K2 * H3 / columns per item)
    int lp_rows, lp_cols, lp_k1; // lane plans (PME_LANE_CASES) of the K3/2, K2 and K1 transforms, -1: none
    int lane_slab, lane_conv;    // slab stages / influence stage take the register path (1) or not (0)
    int pdl_late;                // when a stage kernel triggers its successor's launch (PdlScope, pdl.cuh)
    int nt_tile;                 // spread / force CTA threads (128 or 256) chosen by the tuner; 0: density rule
    int item0;                   // first work item of the slab / influence stage launches (slab decomposition)
    int k1_lo, k1_hi;            // spreading writes only the mesh planes k1_lo <= k1 < k1_hi (slab decomposition)
    const void *tc_w;            // non-null: single-system launches run the influence stage on the tensor
                                 // cores with this DFT-matrix image (K1 = 128; batches keep the FP32 stage)
    float kinv[3];               // 1 / K_alpha
    // u_alpha = sum_j r_j C[j][alpha], C[j][alpha] = K_alpha a*_alpha[j], as an unevaluated float sum
    // chi + clo (about 48 significant bits), index 3*j + alpha.
    float chi[9], clo[9];
    // a*_alpha[j] (index 3*j + alpha) for m' = sum_alpha mt_alpha a*_alpha, and pi^2 / beta^2.
    float rec[9];
    float pi2b2;
    // inputs / outputs (caller-owned)
    const float *pos;
    const float *q;
    float *forces;
    double *ev;
    // resident state (library-owned)
    unsigned long long *grid;    // K1*K2*K3 int64 fixed-point charge mesh, [k1][k2][k3]
    float2 *spec;                // K1*K2*H3 complex half spectrum, [k1][m2][m3]
    float *phi;                  // K1*K2*K3 potential mesh, [k1][k2][k3]
    // influence table per half-spectrum point, [m2][m1][m3]: x, y = B*C as (hi, lo) floats; z = B*C f(m) and
    // w = B*C f(m_p) with f = 2 (1 / |m'|^2 + pi^2 / beta^2), m_p the conjugate partner kept separately on
    // Nyquist planes (w = 0 elsewhere), for the virial
    const float4 *bc;
    const float2 *tw1, *tw2;     // exp(-2 pi i k / K1), exp(-2 pi i k / K2)
    const float2 *tw3h, *tw3;    // exp(-2 pi i k / (K3/2)), exp(-2 pi i k / K3) for k <= K3/2
    float4 *bka;                 // bucket records (w1, w2, w3, q), [tile][cap]
    int2 *bkb;                   // bucket records (packed base, atom index)
    unsigned *bcount;            // atoms binned per tile, at tile * BCOUNT_STRIDE
    unsigned long long *qslot;   // QABS_SLOTS sums of |q| (2^-24 e units), at slot * 16
    int ev_status;               // 1: the final reduction also stores the status bits, as a double, in ev[7]
    float4 *ova;                 // overflow records, capacity n
    int2 *ovb;
    double *partials;            // 8 double-float (hi, lo) slots per influence-stage item, then K1 level-1 slots
    Ctl *ctl;
};

// ---------------------------------------------------------------------------------------------------------
// small helpers that differ between the CUDA build and the host emulation

#if defined(PME_HOST_EMULATION)
template <class T> inline T ldcg(const T *p) { return *p; }
inline unsigned atomic_add_u32(unsigned *p, unsigned v) { unsigned o = *p; *p = o + v; return o; }
inline void atomic_add_i32(int *p, int v) { *p += v; }
inline void atomic_or_u32(unsigned *p, unsigned v) { *p |= v; }
inline void atomic_add_u64(unsigned long long *p, unsigned long long v) { *p += v; }
inline void red_add_u64(unsigned long long *p, unsigned long long v) { *p += v; }
inline float fmul_rn(float a, float b) { return a * b; }
inline float fadd_rn(float a, float b) { return a + b; }
inline float fsub_rn(float a, float b) { return a - b; }
inline long long f2ll_rn(float x) { return llrintf(x); }
inline int f2i_rd(float x) { return (int)floorf(x); }
inline int f2i_rn(float x) { return (int)rintf(x); }
#else
template <class T> __device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }
__device__ __forceinline__ unsigned atomic_add_u32(unsigned *p, unsigned v) { return atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add_i32(int *p, int v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_or_u32(unsigned *p, unsigned v) { atomicOr(p, v); }
__device__ __forceinline__ void atomic_add_u64(unsigned long long *p, unsigned long long v) { atomicAdd(p, v); }
__device__ __forceinline__ void red_add_u64(unsigned long long *p, unsigned long long v) { atomicAdd(p, v); }
__device__ __forceinline__ float fmul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fadd_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ long long f2ll_rn(float x) { return __float2ll_rn(x); }
__device__ __forceinline__ int f2i_rd(float x) { return __float2int_rd(x); }
__device__ __forceinline__ int f2i_rn(float x) { return __float2int_rn(x); }
#endif

PME_DEV int imin(int a, int b) { return a < b ? a : b; }

// floor(a / b) for 0 <= a < 2^20 and 1 <= b <= 2^12 from a precomputed float reciprocal: (a + 0.5) / b is
// at least 1/(2b) away from an integer, far more than the float rounding, so the truncation is exact.
PME_DEV int fdiv(int a, float binv) { return (int)(((float)a + 0.5f) * binv); }

// Pieces of the k1 axis for the spread / force tiles (set_tiling): piece j covers [floor(j K1 / nt1),
// floor((j + 1) K1 / nt1)); the piece holding k is floor(((k + 1) nt1 - 1) / K1). Both divisions are exact
// by fdiv (numerators below 2^16, divisors at most 256).
PME_DEV int k1_piece(const SysDev &d, int k) { return fdiv((k + 1) * d.nt1 - 1, d.kinv[0]); }
PME_DEV int k1_start(const SysDev &d, int j) { return fdiv(j * d.K1, d.rnt1); }

#if defined(PME_HOST_EMULATION)
inline unsigned long long warp_sum_u64(unsigned long long v) { return v; }
#else
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
#endif

PME_DEV float qnan_f() {
    union {
        unsigned u;
        float f;
    } v;
    v.u = 0x7fc00000u;
    return v.f;
}

// The bits of a float as an int (a register move on the GPU).
#if defined(PME_HOST_EMULATION)
inline int float_bits(float f) {
    int i;
    memcpy(&i, &f, sizeof(i));
    return i;
}
#else
__device__ __forceinline__ int float_bits(float f) { return __float_as_int(f); }
#endif

// int64 fixed point (scale 2^40) -> float. Split into a signed high word and an unsigned low word so
// only 32-bit conversions are used; the result is within one rounding of v * 2^-40.
PME_DEV float fix_to_float(long long v) {
    float hi = (float)(int)(v >> 32);
    float lo = (float)(unsigned)(v & 0xffffffffll);
    return (hi * 4294967296.0f + lo) * FIX_INV;
}

// Double-float accumulator: value = hi + lo with |lo| <= ulp(hi)/2 (Knuth's TwoSum).
struct DF {
    float hi, lo;
};
PME_DEV DF df_add(DF a, float b) {
    float s = fadd_rn(a.hi, b);
    float bb = fsub_rn(s, a.hi);
    float err = fadd_rn(fsub_rn(a.hi, fsub_rn(s, bb)), fsub_rn(b, bb));
    DF r;
    r.hi = s;
    r.lo = a.lo + err;
    return r;
}
PME_DEV DF df_add(DF a, DF b) {
    DF r = df_add(a, b.hi);
    r.lo += b.lo;
    float s = fadd_rn(r.hi, r.lo);
    r.lo = fsub_rn(r.lo, fsub_rn(s, r.hi));
    r.hi = s;
    return r;
}

// ---------------------------------------------------------------------------------------------------------
// Scaled fractional coordinate of one position along dimension al (paper Sec. III-A "Charge Spreading":
// an atom sits at a fractional position between mesh points). u = sum_j r_j C[j][al] is formed from exact
// FP32 products (TwoProd via fma) and TwoSum, so w = u - floor(u) carries no FP32 rounding of u itself
// (|u| up to ~2^23): GB300's FP64 pipe is too slow to spend on every atom. Returns false for a non-finite
// or absurdly distant position. b = floor(u) mod K, w in [0, 1].
PME_DEV bool scaled_coord(const SysDev &d, const float r[3], int al, int K, int &b, float &w) {
    float uh = 0.f, ul = 0.f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float ch = d.chi[3 * j + al], cl = d.clo[3 * j + al];
        const float p = fmul_rn(r[j], ch);
        float e = fmaf(r[j], ch, -p);  // exact error of the product
        e = fmaf(r[j], cl, e);
        const float s = fadd_rn(uh, p);
        const float bb = fsub_rn(s, uh);
        const float err = fadd_rn(fsub_rn(uh, fsub_rn(s, bb)), fsub_rn(p, bb));
        uh = s;
        ul = ul + (err + e);
    }
    const float s = fadd_rn(uh, ul);
    ul = fsub_rn(ul, fsub_rn(s, uh));
    uh = s;
    if (!(fabsf(uh) < 8388608.0f)) return false;  // |u| < 2^23 (also rejects NaN)
    float fl = floorf(uh);
    float ww = fadd_rn(fsub_rn(uh, fl), ul);
    if (ww >= 1.f) {
        ww -= 1.f;
        fl += 1.f;
    } else if (ww < 0.f) {
        ww += 1.f;
        fl -= 1.f;
    }
    // fl mod K in exact float arithmetic (|fl| <= 2^23 + 1, so fl - K floor(fl / K) is exact)
    const float qk = floorf(fl * d.kinv[al]);
    int m = (int)(fl - qk * (float)K);
    if (m < 0) m += K;
    else if (m >= K) m -= K;
    b = m;
    w = ww;
    return true;
}

// ---------------------------------------------------------------------------------------------------------
// Cardinal B-spline weights th[j] = M_P(w + j), j = 0..P-1, by the two-term recursion from the hat
// function M_2 (the "b-spline calculation" of the paper's Sec. V-C pipeline); with dth[j] = M_P'(w + j) =
// M_{P-1}(w + j) - M_{P-1}(w + j - 1) when requested. The mesh point of weight j is base - j.
//
// The recursion runs on N_n = (n-1)! M_n, whose coefficients are exact small integers, and divides once
// by (P-1)! with a correctly rounded division at the end. Multiplying by a rounded 1/(n-1) at every order
// instead would scale every atom's weights by the same relative error, a bias the energy (sixth power of
// the weights) amplifies; the remaining rounding errors here differ from atom to atom.

template <int P>
PME_DEV void bspline_order_up(float w, float *th, int n) {
    th[n - 1] = (1.0f - w) * th[n - 2];
#pragma unroll
    for (int j = n - 2; j >= 1; --j) th[j] = (w + (float)j) * th[j] + ((float)(n - j) - w) * th[j - 1];
    th[0] = w * th[0];
}

constexpr double factorial_d(int k) { return k <= 1 ? 1.0 : (double)k * factorial_d(k - 1); }

// x / k! as x * (hi + lo), the reciprocal of k! split into two floats (about 48 bits): one rounding at the
// end, so the result is unbiased (a single rounded reciprocal would scale every atom alike).
template <int K>
struct InvFact {
    static constexpr double r = 1.0 / factorial_d(K);
    static constexpr float hi = (float)r;
    static constexpr float lo = (float)(r - (double)hi);
};
template <int K>
PME_DEV float div_fact(float x) {
    return fmaf(x, InvFact<K>::hi, x * InvFact<K>::lo);
}

template <int P>
PME_DEV void bspline_w(float w, float *th) {
    th[0] = w;
    th[1] = 1.0f - w;
#pragma unroll
    for (int n = 3; n <= P; ++n) bspline_order_up<P>(w, th, n);
#pragma unroll
    for (int j = 0; j < P; ++j) th[j] = div_fact<P - 1>(th[j]);
}

template <int P>
PME_DEV void bspline_wd(float w, float *th, float *dth) {
    th[0] = w;
    th[1] = 1.0f - w;
#pragma unroll
    for (int n = 3; n <= P - 1; ++n) bspline_order_up<P>(w, th, n);
    dth[0] = div_fact<P - 2>(th[0]);
#pragma unroll
    for (int j = 1; j <= P - 2; ++j) dth[j] = div_fact<P - 2>(th[j] - th[j - 1]);
    dth[P - 1] = -div_fact<P - 2>(th[P - 2]);
    bspline_order_up<P>(w, th, P);
#pragma unroll
    for (int j = 0; j < P; ++j) th[j] = div_fact<P - 1>(th[j]);
}

}  // namespace pme
