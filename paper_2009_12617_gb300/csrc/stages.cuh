// Stage bodies of the reciprocal-space SPME pipeline (paper Sec. III-A, Fig. "LRPipe"): binning with
// B-spline set-up, charge spreading, forward 3D FFT, influence-function multiply with energy / virial,
// inverse 3D FFT, and force interpolation. Each body handles one work item of one system and is called
// both from the per-stage kernels and from the batched / cooperative kernels.
//
// Work items per system:
//   bin     nbin items          atoms [item*BIN_CHUNK, ...): fractional coordinates, tile key, bucket insert
//   spread  ntiles+OVF_ITEMS    one tile each, then bucket-overflow atoms
//   fwd     K1 items            slab k1: int64 -> float, real FFT along k3, complex FFT along k2
//   conv    K2*nchunk3 items    pencils (m2, CONV_COLS columns m3): FFT along k1, times B*C, energy /
//                               virial, inverse FFT along k1
//   inv     K1 items            slab k1: inverse FFT along k2, complex-to-real FFT along k3 -> phi
//   gather  ntiles+OVF_ITEMS    one tile each (forces), then bucket-overflow atoms
#pragma once

#include "common.cuh"
#include "fft.cuh"

// The register transforms (lane plans) need warps; the CPU emulation and builds that define
// PME_NO_LANE_FFT keep only the shared-memory transforms.
#if !defined(PME_HOST_EMULATION) && !defined(PME_NO_LANE_FFT)
#define PME_LANE_FFT 1
#endif

namespace pme {

// Tile region edge (mesh points) for spline order P and tile edge T: the tile plus the p - 1 points below.
template <int P, int T>
struct Region {
    static constexpr int R = T + P - 1;
    static constexpr int VOL = R * R * R;
};

// The two threads of an atom split its support planes j1: half 0 takes [0, H0), half 1 [H0, P), with
// H0 = ceil(P / 2) (equal halves for even orders, one plane more in half 0 for odd ones).
PME_HD int half_planes(int P) { return (P + 1) / 2; }

// Spreading region layout: R planes of R rows of R points, rows RS apart and planes PL apart.
//
// P = 4 with 8^3 tiles (spread_warp_lanes): one warp takes one atom at a time, lane (jA, j2, j3) =
// (lane / 16, lane / 4 mod 4, lane mod 4) adding the points (jA, j2, j3) and (jA + 2, j2, j3) below the
// atom's highest support point. RS and PL are padded until the 32 offsets jA PL + j2 RS + j3 fall in
// distinct banks (mod 32), so every shared-memory atomic of the warp is conflict-free wherever the atom
// sits (R = 11: RS = 12, PL = 144).
//
// Otherwise: two threads per atom split its planes (half_planes); rows are not padded (RS = R) and planes
// are padded so that the two halves (H0 planes apart) sit 16 banks apart, H0 PL = 16 (mod 32). Then the 32
// lanes of a warp (16 atoms x 2 halves) hit distinct banks whenever the atoms' base addresses differ mod
// 16, which the dealt processing order (stage_spread) arranges.
PME_HD bool spread_warp_lanes(int P, int tlog) { return P == 4 && tlog == 3; }
PME_HD bool warp_lanes_distinct(int rs, int pl) {
    unsigned seen = 0u;
    for (int ja = 0; ja < 2; ++ja)
        for (int j2 = 0; j2 < 4; ++j2)
            for (int j3 = 0; j3 < 4; ++j3) {
                const unsigned bit = 1u << ((ja * pl + j2 * rs + j3) & 31);
                if (seen & bit) return false;
                seen |= bit;
            }
    return true;
}
// the smallest RS >= R for which some PL in [R RS, R RS + 32) gives distinct lane banks, and the smallest
// such PL (RS = 4 (mod 16) with PL = 16 (mod 32) always works, so the search ends within 16 steps)
PME_HD int warp_row_stride(int R) {
    for (int rs = R; rs < R + 16; ++rs)
        for (int pl = R * rs; pl < R * rs + 32; ++pl)
            if (warp_lanes_distinct(rs, pl)) return rs;
    return -1;
}
PME_HD int warp_plane_stride(int R) {
    const int rs = warp_row_stride(R);
    for (int pl = R * rs; pl < R * rs + 32; ++pl)
        if (warp_lanes_distinct(rs, pl)) return pl;
    return -1;
}
PME_HD int spread_row(int P, int tlog) {
    const int R = (1 << tlog) + P - 1;
    return spread_warp_lanes(P, tlog) ? warp_row_stride(R) : R;
}
PME_HD int spread_plane(int P, int tlog) {
    const int R = (1 << tlog) + P - 1;
    if (spread_warp_lanes(P, tlog)) return warp_plane_stride(R);
    int pl = R * R;
    while ((half_planes(P) * pl) % 32 != 16) ++pl;
    return pl;
}
// Accumulator array length (R PL rounded up to 4 ints, so the record arrays after the two accumulators
// stay 16-byte aligned) and record bytes per atom: the warp-lane path keeps the atom's weights (three
// float4) and region index, the other the record (float4 + int2), the dealt order's key and inverse.
PME_HD int spread_vol(int P, int tlog) { return (((1 << tlog) + P - 1) * spread_plane(P, tlog) + 3) / 4 * 4; }
PME_HD int spread_rec_bytes(int P, int tlog) { return spread_warp_lanes(P, tlog) ? 3 * 16 + 4 : 16 + 8 + 4 + 4; }
template <int P, int T>
struct SpreadLayout {
    static constexpr int TLOG = T >= 16 ? 4 : 3;
    static constexpr bool WARP = spread_warp_lanes(P, TLOG);
    static constexpr int R = T + P - 1;
    static constexpr int RS = spread_row(P, TLOG);
    static constexpr int PL = spread_plane(P, TLOG);
    static constexpr int VOLP = spread_vol(P, TLOG);
    static constexpr int CAP = cap_max_for(T >= 16 ? 4 : 3);  // record slots
};

// ---------------------------------------------------------------------------------------------------------
// shared-memory sizes (bytes) of each stage for a given system and block size

inline size_t smem_bin(int nth) { return (size_t)((nth + 31) / 32) * sizeof(unsigned long long) + 16; }
inline size_t smem_tile_region(int p, int tlog) {
    const size_t r = (size_t)(1 << tlog) + p - 1;
    return r * r * r;
}
// split accumulators over the padded region (2 x spread_vol ints), cap = cap_max_for(tlog) records of
// spread_rec_bytes and 16 residue counters
inline size_t smem_spread(int p, int tlog) {
    return (size_t)2 * spread_vol(p, tlog) * sizeof(int) + (size_t)cap_max_for(tlog) * spread_rec_bytes(p, tlog) +
           16 * sizeof(unsigned);
}
inline size_t smem_gather(int p, int tlog) { return smem_tile_region(p, tlog) * sizeof(float); }
// Two K2 x H3 buffers (the register path uses one, with rows padded by up to 15), then the twiddles.
inline size_t smem_slab(int K2, int K3) {
    const int H3 = K3 / 2 + 1;
    return (2 * (size_t)K2 * H3 + 16 * (size_t)K2 + (K3 / 2) + (K3 / 2 + 1) + K2) * sizeof(float2);
}
inline size_t smem_conv(int K1, int nth) {
    size_t fft = (2 * (size_t)K1 * CONV_COLS + K1) * sizeof(float2);
    size_t red = (size_t)7 * nth * sizeof(float) + 7 * 16 * sizeof(DF);
    return fft > red ? fft : red;
}
inline size_t smem_inv(int K2, int K3) { return smem_slab(K2, K3); }
// the force stage's first overflow item also runs the final energy / virial reduction
inline size_t smem_gather_all(int p, int tlog) {
    size_t fin = (size_t)REDUCE_SLOTS * 7 * sizeof(DF);
    return smem_gather(p, tlog) > fin ? smem_gather(p, tlog) : fin;
}

// global -> shared copy of n elements with LOAD_BATCH independent loads in flight per thread
template <class T>
PME_DEV void copy_batched(T *dst, const T *src, int n) {
    const int tid = PME_TID, nth = PME_NTH;
    for (int base = tid; base < n; base += LOAD_BATCH * nth) {
        T v[LOAD_BATCH];
#pragma unroll
        for (int u = 0; u < LOAD_BATCH; ++u)
            if (base + u * nth < n) v[u] = ldcg(src + base + u * nth);
#pragma unroll
        for (int u = 0; u < LOAD_BATCH; ++u)
            if (base + u * nth < n) dst[base + u * nth] = v[u];
    }
}

// ---------------------------------------------------------------------------------------------------------
// 64-bit fixed point (scale 2^40) as (hi, lo): rn(v) = hi * 2^20 + lo with lo in [-2^19, 2^19]. The split is
// a deterministic function of the float v, and the global path adds the same integer rn(v) in one 64-bit
// step, so the mesh does not depend on which path an atom takes.

PME_DEV void fix_split(float v, int &h, int &l) {
    // Round-to-nearest by the float magic number M = 1.5 * 2^23: for |x| < 2^22, x + M carries
    // rn(x) in its low mantissa bits, so no float-to-integer conversion instruction is needed.
    // h = rn(v / 2^20) (v / 2^20 is exact), l = rn(v - h 2^20) with v - h 2^20 in [-2^19, 2^19] exact;
    // h 2^20 + l = rn(v), the same integer whatever the split.
    const float M = 12582912.0f;
    const float t = fmaf(v, 9.5367431640625e-07f, M);
    h = float_bits(t) - 0x4B400000;
    const float r = fmaf(-(t - M), 1048576.0f, v);
    l = float_bits(r + M) - 0x4B400000;
}
PME_DEV unsigned long long fix_join(long long h, long long l) { return (unsigned long long)(h * 1048576ll + l); }

// ---------------------------------------------------------------------------------------------------------
// a1: bin atoms by spread tile (replaces the paper's hardware atom reordering, Sec. III-A / V-C; with
// order-independent fixed-point accumulation the order inside a tile no longer matters)

PME_DEV void stage_bin(const SysDev &d, int item, void *smem) {
    unsigned long long *red = (unsigned long long *)smem;  // one slot per warp
    const int tid = PME_TID, nth = PME_NTH;
    const int i0 = item * BIN_CHUNK;
    const int i1 = imin(d.n, i0 + BIN_CHUNK);
    unsigned long long qacc = 0;
    unsigned bad = 0;
    // the trip count is the same for every thread of the block (lanes past the end have no atom), so the
    // warp-wide slot claim below always sees whole warps
    for (int base = i0 + tid; base - tid < i1; base += BIN_PER_THREAD * nth) {
        float r[BIN_PER_THREAD][3], qv[BIN_PER_THREAD];
#pragma unroll
        for (int k = 0; k < BIN_PER_THREAD; ++k) {  // issue every load first
            const int i = base + k * nth;
            if (i < i1) {
                r[k][0] = d.pos[3 * (size_t)i];
                r[k][1] = d.pos[3 * (size_t)i + 1];
                r[k][2] = d.pos[3 * (size_t)i + 2];
                qv[k] = d.q[i];
            }
        }
        int tile[BIN_PER_THREAD];
        float4 ra[BIN_PER_THREAD];
        int2 rb[BIN_PER_THREAD];
        int kind[BIN_PER_THREAD];  // 0: absent, 1: bucket, 2: overflow list, 3: invalid
#pragma unroll
        for (int k = 0; k < BIN_PER_THREAD; ++k) {
            const int i = base + k * nth;
            kind[k] = 0;
            if (i >= i1) continue;
            const float q = qv[k];
            int b0, b1, b2;
            float w0, w1, w2;
            bool ok = isfinite(q) && fabsf(q) < 4194304.0f;  // |q| < 2^22 e
            if (ok) ok = scaled_coord(d, r[k], 0, d.K1, b0, w0) && scaled_coord(d, r[k], 1, d.K2, b1, w1) &&
                         scaled_coord(d, r[k], 2, d.K3, b2, w2);
            if (!ok) {
                kind[k] = 3;
                continue;
            }
            qacc += (unsigned long long)f2ll_rn(fabsf(q) * QABS_SCALE);
            tile[k] = (k1_piece(d, b0) * d.nt2 + (b1 >> d.tlog)) * d.nt3 + (b2 >> d.tlog);
            ra[k] = make_float4(w0, w1, w2, q);
            rb[k] = make_int2(b0 | (b1 << 10) | (b2 << 20), i);
            kind[k] = fabsf(q) <= Q_TILE_MAX ? 1 : 2;
        }
        unsigned rank[BIN_PER_THREAD];
#pragma unroll
        for (int k = 0; k < BIN_PER_THREAD; ++k) {  // independent atomics, all in flight together
#if defined(PME_HOST_EMULATION)
            if (kind[k] == 1) rank[k] = atomic_add_u32(&d.bcount[(size_t)tile[k] * BCOUNT_STRIDE], 1u);
#else
            // lanes of a warp binning into the same tile (the atoms of a molecule, mostly) claim consecutive
            // slots with one atomic by their lowest lane: fewer same-address atomics queue at each counter
            const int key = kind[k] == 1 ? tile[k] : -1;
            const unsigned peers = __match_any_sync(0xffffffffu, key);
            const int lane = tid & 31, leader = __ffs(peers) - 1;
            unsigned first = 0;
            if (key >= 0 && lane == leader)
                first = atomic_add_u32(&d.bcount[(size_t)key * BCOUNT_STRIDE], (unsigned)__popc(peers));
            first = __shfl_sync(0xffffffffu, first, leader);
            rank[k] = first + (unsigned)__popc(peers & ((1u << lane) - 1u));
#endif
        }
#pragma unroll
        for (int k = 0; k < BIN_PER_THREAD; ++k) {
            const int i = base + k * nth;
            if (kind[k] == 3) {
                bad |= ST_NONFINITE;
                const float nan = qnan_f();
                d.forces[3 * (size_t)i] = nan;
                d.forces[3 * (size_t)i + 1] = nan;
                d.forces[3 * (size_t)i + 2] = nan;
            } else if (kind[k] == 1 && rank[k] < (unsigned)d.cap) {
                d.bka[(size_t)tile[k] * d.cap + rank[k]] = ra[k];
                d.bkb[(size_t)tile[k] * d.cap + rank[k]] = rb[k];
            } else if (kind[k] != 0) {
                const unsigned j = atomic_add_u32(&d.ctl->novf, 1u);
                if (j < (unsigned)d.n) {
                    d.ova[j] = ra[k];
                    d.ovb[j] = rb[k];
                } else {
                    bad |= ST_INTERNAL;
                }
            }
        }
    }
    if (bad) atomic_or_u32(&d.ctl->status, bad);
    // sum of |q| in fixed point (exact, so the order of the additions does not matter): warp sums, then
    // one atomic per CTA
    qacc = warp_sum_u64(qacc);
    if ((tid & 31) == 0) red[tid >> 5] = qacc;
    PME_SYNC();
    if (tid == 0) {
        unsigned long long tot = 0;
        for (int w = 0; w < (nth + 31) / 32; ++w) tot += red[w];
        if (tot >= QABS_LIMIT) atomic_or_u32(&d.ctl->status, ST_OVERFLOW);
        else if (tot) atomic_add_u64(d.qslot + (size_t)(item & (QABS_SLOTS - 1)) * 16, tot);
    }
}

// ---------------------------------------------------------------------------------------------------------
// a2: charge spreading Q(k) = sum_i q_i theta1 theta2 theta3 (paper Sec. III-A "Charge Spreading": each
// charge goes to the p^3 mesh points around it). A tile accumulates its atoms into a shared-memory region
// R^3 (R = tile edge + p - 1) as split 32-bit fixed point, then adds the region (including the p - 1 halo that
// overlaps neighbouring tiles, the analogue of the paper's atoms processed by every pipeline they touch)
// into the global int64 mesh with 64-bit integer reductions.

PME_DEV void tile_origin(const SysDev &d, int tile, int &o1, int &o2, int &o3) {
    const int t3 = tile % d.nt3, t2 = (tile / d.nt3) % d.nt2, t1 = tile / (d.nt3 * d.nt2);
    o1 = k1_start(d, t1);
    o2 = t2 << d.tlog;
    o3 = t3 << d.tlog;
}
// Width along k1 of the tile with origin o1 (the piece's end minus its start).
PME_DEV int tile_width1(const SysDev &d, int o1) { return k1_start(d, k1_piece(d, o1) + 1) - o1; }

PME_DEV int wrapk(int k, int K) { return k < 0 ? k + K : (k >= K ? k - K : k); }

template <int P>
PME_DEV void spread_atom_global(const SysDev &d, float4 ra, int2 rb) {
    float th1[P], th2[P], th3[P];
    bspline_w<P>(ra.x, th1);
    bspline_w<P>(ra.y, th2);
    bspline_w<P>(ra.z, th3);
    const int b1 = rb.x & 1023, b2 = (rb.x >> 10) & 1023, b3 = (rb.x >> 20) & 1023;
#pragma unroll
    for (int j1 = 0; j1 < P; ++j1) {
        const int k1 = wrapk(b1 - j1, d.K1);
        if (k1 < d.k1_lo || k1 >= d.k1_hi) continue;  // another rank's planes (slab decomposition)
#pragma unroll
        for (int j2 = 0; j2 < P; ++j2) {
            const int k2 = wrapk(b2 - j2, d.K2);
            // the fixed-point scale (a power of two) applied to the row factor: rn(c 2^40 th3) = rn(c th3) 2^40
            const float c = ra.w * th1[j1] * th2[j2] * FIX_SCALE;
            unsigned long long *row = d.grid + ((size_t)k1 * d.K2 + k2) * d.K3;
#pragma unroll
            for (int j3 = 0; j3 < P; ++j3) {
                // rn(v) directly in 64 bits: the same integer as the tile path's split, for any |q| < 2^22
                red_add_u64(row + wrapk(b3 - j3, d.K3), (unsigned long long)f2ll_rn(c * th3[j3]));
            }
        }
    }
}

// Shared memory of a spreading tile (sizes as smem_spread): split accumulators over the padded region, then
// per atom either its weights and region index (warp-lane path) or its record, the dealt order's key and
// inverse, and 16 residue counters.
template <int P, int T>
struct SpreadSmem {
    static constexpr int VOLP = SpreadLayout<P, T>::VOLP;
    static constexpr int CAP = SpreadLayout<P, T>::CAP;
    int *hi, *lo;
    // warp-lane path: rn(q th1[j]) 2^40 for j = 0, 2, 1, 3 (lane jA reads planes jA and jA + 2 as one pair),
    // th2, th3, and the region index of the highest support point
    float4 *u_s, *t2_s, *t3_s;
    int *ix_s;
    // two-thread path
    float4 *ra_s;    // the tile's records (16-byte aligned: VOLP is a multiple of 4)
    int2 *rb_s;
    int *key_s;      // per atom: rank << 4 | residue
    int *inv_s;      // dealt position -> atom
    unsigned *bins;  // 16 residue counters
    PME_DEV explicit SpreadSmem(void *smem) {
        hi = (int *)smem;
        lo = hi + VOLP;
        if (SpreadLayout<P, T>::WARP) {
            u_s = (float4 *)(lo + VOLP);
            t2_s = u_s + CAP;
            t3_s = t2_s + CAP;
            ix_s = (int *)(t3_s + CAP);
            bins = (unsigned *)(ix_s + CAP);
            ra_s = nullptr;
            rb_s = nullptr;
            key_s = inv_s = nullptr;
        } else {
            ra_s = (float4 *)(lo + VOLP);
            rb_s = (int2 *)(ra_s + CAP);
            key_s = (int *)(rb_s + CAP);
            inv_s = key_s + CAP;
            bins = (unsigned *)(inv_s + CAP);
            u_s = t2_s = t3_s = nullptr;
            ix_s = nullptr;
        }
    }
};

// Zero the accumulators and residue counters. It touches no global memory, so the stage kernel runs it
// before waiting for its predecessor (inside the launch window of programmatic dependent launch).
template <int P, int T>
PME_DEV void spread_clear(void *smem) {
    const SpreadSmem<P, T> s(smem);
    for (int i = PME_TID; i < 16; i += PME_NTH) s.bins[i] = 0u;
    int4 *z = (int4 *)s.hi;  // hi and lo are contiguous, 2 VOLP ints, VOLP a multiple of 4
    for (int i = PME_TID; i < SpreadSmem<P, T>::VOLP / 2; i += PME_NTH) z[i] = make_int4(0, 0, 0, 0);
}

// One lane's share of an atom on the warp-lane path: points (jA, j2, j3) and (jA + 2, j2, j3) below the
// atom's highest support point, jA = lane / 16, j2 = lane / 4 mod 4, j3 = lane mod 4. The value added is
// rn(rn(rn(q th1) 2^40 th2) th3), equal to the two-thread and global paths' rn(rn(rn(q th1) th2) 2^40 th3)
// (scaling by a power of two commutes with rounding; products too small for that to hold round to 0 in
// both). Loading and adding are separate steps so that a warp can hold two atoms' weights in flight.
struct Lane4 {
    float2 u;  // rn(q th1) 2^40 of the planes jA, jA + 2
    float t2, t3;
    int i;     // region index of the point (jA, j2, j3); on the GPU its byte address in the shared window
};
#if defined(PME_HOST_EMULATION)
template <int P, int T>
struct Lanes4 {
    const SpreadSmem<P, T> &s;
    int off;  // region offset of the lane's point below the atom's highest support point
    Lanes4(const SpreadSmem<P, T> &sm, int lane)
        : s(sm),
          off((lane >> 4) * SpreadLayout<P, T>::PL + ((lane >> 2) & 3) * SpreadLayout<P, T>::RS + (lane & 3)),
          ja(lane >> 4), j2((lane >> 2) & 3), j3(lane & 3) {}
    int ja, j2, j3;
    Lane4 load(int a) const {
        Lane4 w;
        w.u = ((const float2 *)(s.u_s + a))[ja];
        w.t2 = ((const float *)(s.t2_s + a))[j2];
        w.t3 = ((const float *)(s.t3_s + a))[j3];
        w.i = s.ix_s[a] - off;
        return w;
    }
    void add(const Lane4 &w) const {
        constexpr int PL = SpreadLayout<P, T>::PL;
        int h, l;
        fix_split((w.u.x * w.t2) * w.t3, h, l);
        s.hi[w.i] += h;
        s.lo[w.i] += l;
        fix_split((w.u.y * w.t2) * w.t3, h, l);
        s.hi[w.i - 2 * PL] += h;
        s.lo[w.i - 2 * PL] += l;
    }
};
#else
// GPU: 32-bit shared-window addresses computed once per lane, so each load or reduction costs one add
// instead of 64-bit generic pointer arithmetic
PME_DEV unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
template <int P, int T>
struct Lanes4 {
    static constexpr unsigned DLO = 4u * SpreadLayout<P, T>::VOLP;  // lo - hi, bytes
    static constexpr unsigned D2 = 8u * SpreadLayout<P, T>::PL;     // two planes, bytes
    unsigned su, st2, st3, six, shi;
    PME_DEV Lanes4(const SpreadSmem<P, T> &s, int lane) {
        const int ja = lane >> 4, j2 = (lane >> 2) & 3, j3 = lane & 3;
        su = smem_u32(s.u_s) + 8u * ja;
        st2 = smem_u32(s.t2_s) + 4u * j2;
        st3 = smem_u32(s.t3_s) + 4u * j3;
        six = smem_u32(s.ix_s);
        shi = smem_u32(s.hi) - 4u * (ja * SpreadLayout<P, T>::PL + j2 * SpreadLayout<P, T>::RS + j3);
    }
    PME_DEV Lane4 load(int a) const {
        Lane4 w;
        int ix;
        asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(w.u.x), "=f"(w.u.y) : "r"(su + 16u * a) : "memory");
        asm volatile("ld.shared.f32 %0, [%1];" : "=f"(w.t2) : "r"(st2 + 16u * a) : "memory");
        asm volatile("ld.shared.f32 %0, [%1];" : "=f"(w.t3) : "r"(st3 + 16u * a) : "memory");
        asm volatile("ld.shared.s32 %0, [%1];" : "=r"(ix) : "r"(six + 4u * a) : "memory");
        w.i = (int)(shi + 4u * (unsigned)ix);
        return w;
    }
    PME_DEV static void red(unsigned addr, int v) {
        asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
    }
    PME_DEV void add(const Lane4 &w) const {
        const unsigned ad = (unsigned)w.i;
        int h, l;
        fix_split((w.u.x * w.t2) * w.t3, h, l);
        red(ad, h);
        red(ad + DLO, l);
        fix_split((w.u.y * w.t2) * w.t3, h, l);
        red(ad - D2, h);
        red(ad + DLO - D2, l);
    }
};
#endif

// cleared: spread_clear already ran on this shared memory (and nothing has used it since). org: the tile's
// origin (tile_origin), when the caller computed it already.
template <int P, int T>
PME_DEV void stage_spread(const SysDev &d, int item, void *smem, bool cleared = false, const int *org = nullptr) {
    const int tid = PME_TID, nth = PME_NTH;
    if (item >= d.ntiles) {  // bucket-overflow atoms, straight to the global mesh
        const unsigned novf = imin((int)ldcg(&d.ctl->novf), d.n);
        // the force stage reads this copy; the forward FFT stage resets the counter for the next binning
        if (item == d.ntiles && tid == 0) d.ctl->novf_gather = novf;
        for (unsigned a = (unsigned)((item - d.ntiles) * nth + tid); a < novf; a += (unsigned)(OVF_ITEMS * nth))
            spread_atom_global<P>(d, ldcg(d.ova + a), ldcg(d.ovb + a));
        return;
    }
    constexpr int R = SpreadLayout<P, T>::R, RS = SpreadLayout<P, T>::RS, PL = SpreadLayout<P, T>::PL, H = P - 1;
    const SpreadSmem<P, T> sm(smem);
    int *hi = sm.hi, *lo = sm.lo, *key_s = sm.key_s, *inv_s = sm.inv_s;
    float4 *ra_s = sm.ra_s;
    int2 *rb_s = sm.rb_s;
    unsigned *bins = sm.bins;
    int o1, o2, o3;
    if (org) {
        o1 = org[0];
        o2 = org[1];
        o3 = org[2];
    } else {
        tile_origin(d, item, o1, o2, o3);
    }
    const float4 *A = d.bka + (size_t)item * d.cap;
    const int2 *B = d.bkb + (size_t)item * d.cap;
    // this thread's first record in flight with the count, for the threads below the mean occupancy (the
    // bucket capacity is twice it plus a margin), so that few loads land on empty slots
    const bool pf = tid < (d.cap >> 1);
    float4 ra0 = make_float4(0.f, 0.f, 0.f, 0.f);
    int2 rb0 = make_int2(0, 0);
    if (pf) {
        ra0 = ldcg(A + tid);
        rb0 = ldcg(B + tid);
    }
    const int cnt = imin((int)ldcg(&d.bcount[(size_t)item * BCOUNT_STRIDE]), d.cap);
    if (!cleared) spread_clear<P, T>(smem);
    PME_SYNC();
    if constexpr (SpreadLayout<P, T>::WARP) {
        // one thread per atom: its weights and the region index of its highest support point
        for (int a = tid; a < cnt; a += nth) {
            const bool first = pf && a == tid;
            const float4 ra = first ? ra0 : ldcg(A + a);
            const int2 rb = first ? rb0 : ldcg(B + a);
            float th1[P], th2[P], th3[P];
            bspline_w<P>(ra.x, th1);
            bspline_w<P>(ra.y, th2);
            bspline_w<P>(ra.z, th3);
            const float qs = ra.w * FIX_SCALE;  // exact: a power of two
            sm.u_s[a] = make_float4(qs * th1[0], qs * th1[2], qs * th1[1], qs * th1[3]);
            sm.t2_s[a] = make_float4(th2[0], th2[1], th2[2], th2[3]);
            sm.t3_s[a] = make_float4(th3[0], th3[1], th3[2], th3[3]);
            sm.ix_s[a] = ((rb.x & 1023) - o1 + H) * PL + (((rb.x >> 10) & 1023) - o2 + H) * RS +
                         (((rb.x >> 20) & 1023) - o3 + H);
        }
        PME_SYNC();
        // one warp per atom, its 64 points over the 32 lanes (two each, in distinct banks); each warp takes
        // the atoms w, w + nw, ... two at a time, both atoms' weights loaded before either is added
#if defined(PME_HOST_EMULATION)
        for (int a = 0; a < cnt; ++a)
            for (int lane = 0; lane < 32; ++lane) {
                const Lanes4<P, T> ln(sm, lane);
                ln.add(ln.load(a));
            }
#else
        const int nw = nth >> 5;
        const Lanes4<P, T> ln(sm, tid & 31);
        int a = tid >> 5;
        for (; a + nw < cnt; a += 2 * nw) {
            const Lane4 w0 = ln.load(a), w1 = ln.load(a + nw);
            ln.add(w0);
            ln.add(w1);
        }
        if (a < cnt) ln.add(ln.load(a));
#endif
    } else {
        // Dealt order: residue r = (base mod 16) of the atom's highest support point in the padded region;
        // round k takes the k-th atom of every residue in turn, so 16 consecutive atoms (one warp) mostly have
        // distinct residues and their shared-memory atomics do not share banks. Results do not depend on the
        // order (integer sums).
        for (int a = tid; a < cnt; a += nth) {
            const bool first = pf && a == tid;
            const float4 ra = first ? ra0 : ldcg(A + a);
            const int2 rb = first ? rb0 : ldcg(B + a);
            ra_s[a] = ra;
            rb_s[a] = rb;
            const int l1 = (rb.x & 1023) - o1 + H, l2 = ((rb.x >> 10) & 1023) - o2 + H,
                      l3 = ((rb.x >> 20) & 1023) - o3 + H;
            const int res = (l1 * PL + l2 * R + l3) & 15;
            key_s[a] = ((int)atomic_add_u32(bins + res, 1u) << 4) | res;
        }
        PME_SYNC();
        {
            unsigned nb[16];
#pragma unroll
            for (int b = 0; b < 16; ++b) nb[b] = bins[b];
            for (int a = tid; a < cnt; a += nth) {
                const int key = key_s[a], res = key & 15;
                const unsigned rk = (unsigned)(key >> 4);
                unsigned pos = 0;
#pragma unroll
                for (int b = 0; b < 16; ++b) pos += (nb[b] < rk ? nb[b] : rk) + ((b < res && nb[b] > rk) ? 1u : 0u);
                inv_s[pos] = a;
            }
        }
        PME_SYNC();
        // two threads per atom: half 0 takes the planes j1 in [0, H0), half 1 [H0, P)
        constexpr int H0 = half_planes(P);
        for (int a2 = tid; a2 < 2 * cnt; a2 += nth) {
            const int a = inv_s[a2 >> 1], half = a2 & 1;
            const float4 ra = ra_s[a];
            const int2 rb = rb_s[a];
            float th1[P], th2[P], th3[P];
            bspline_w<P>(ra.x, th1);
            bspline_w<P>(ra.y, th2);
            bspline_w<P>(ra.z, th3);
            // local index of the atom's highest support point; its points are l - j, j < P
            const int l1 = (rb.x & 1023) - o1 + H;
            const int l2 = ((rb.x >> 10) & 1023) - o2 + H;
            const int l3 = ((rb.x >> 20) & 1023) - o3 + H;
#pragma unroll
            for (int jj = 0; jj < H0; ++jj) {
                if (half && jj >= P - H0) break;  // odd P: half 1 has one plane fewer
                const int j1 = half * H0 + jj;
                const float t1 = half ? th1[H0 + jj < P ? H0 + jj : P - 1] : th1[jj];
#pragma unroll
                for (int j2 = 0; j2 < P; ++j2) {
                    // scaled row factor: rn(c 2^40 th3) = rn(c th3) 2^40 (a power of two; |v| < 2^62, and values
                    // small enough for the scaling to matter round to 0 either way), one multiply per point
                    const float c = ra.w * t1 * th2[j2] * FIX_SCALE;
                    const int row = (l1 - j1) * PL + (l2 - j2) * R + l3;
#pragma unroll
                    for (int j3 = 0; j3 < P; ++j3) {
                        int h, l;
                        fix_split(c * th3[j3], h, l);
                        atomic_add_i32(hi + row - j3, h);
                        atomic_add_i32(lo + row - j3, l);
                    }
                }
            }
        }
    }
    PME_SYNC();
    // flush: thread t < ng R^2 takes the column (i2, i3) = (c / R, c mod R), c = t mod R^2, and adds its
    // points of the planes i1 = t / R^2, t / R^2 + ng, ... below R1 (the tile's k1 width plus the halo):
    // the column's mesh address is computed once, each plane costs one add and one wrap
    constexpr int RR = R * R;
    const int R1 = tile_width1(d, o1) + H;
    const int ng = nth >= RR ? nth / RR : 1, g = nth >= RR ? tid / RR : 0;
    const size_t plane = (size_t)d.K2 * d.K3;
    if (g < ng) {
        for (int c = nth >= RR ? tid - g * RR : tid; c < RR; c += nth >= RR ? RR : nth) {
            const int i2 = c / R, i3 = c - i2 * R;
            unsigned long long *col = d.grid + (size_t)wrapk(o2 - H + i2, d.K2) * d.K3 + wrapk(o3 - H + i3, d.K3);
            const int *hc = hi + i2 * RS + i3, *lc = lo + i2 * RS + i3;
            int k1 = wrapk(o1 - H + g, d.K1);
#pragma unroll 4
            for (int i1 = g; i1 < R1; i1 += ng) {
                const int h = hc[i1 * PL], l = lc[i1 * PL];
                // k1 outside [k1_lo, k1_hi): another rank's planes (slab decomposition)
                if ((h | l) != 0 && k1 >= d.k1_lo && k1 < d.k1_hi) red_add_u64(col + k1 * plane, fix_join(h, l));
                k1 += ng;
                if (k1 >= d.K1) k1 -= d.K1;
            }
        }
    }
}

// ---------------------------------------------------------------------------------------------------------
// a3: forward slab k1 — mesh int64 -> float, real-to-complex FFT along k3 (a length K3/2 complex FFT of
// even/odd pairs plus the split step), then the complex FFT along k2 for every m3 column. (The inverse
// stage zeroes the slab of the int64 mesh for the next evaluation's spreading.)

PME_DEV void stage_fwd_smem(const SysDev &d, int k1, void *smem) {
    const int tid = PME_TID, nth = PME_NTH;
    const int K2 = d.K2, K3 = d.K3, H3 = d.H3, Nh = K3 / 2;
    const float inv_h3 = 1.0f / (float)H3;
    float2 *A = (float2 *)smem;
    float2 *B = A + K2 * H3;
    float2 *twh = B + K2 * H3;   // Nh
    float2 *tw3 = twh + Nh;      // Nh + 1
    float2 *tw2 = tw3 + Nh + 1;  // K2
    const ulonglong2 *g = (const ulonglong2 *)(d.grid + (size_t)k1 * K2 * K3);
    const int tot = K2 * Nh;
    for (int base = tid; base < tot; base += LOAD_BATCH * nth) {  // row k2 pairs (2n, 2n+1) -> complex z[n]
        ulonglong2 v[LOAD_BATCH];
#pragma unroll
        for (int u = 0; u < LOAD_BATCH; ++u)  // all loads in flight before any use
            if (base + u * nth < tot) v[u] = ldcg(g + base + u * nth);
#pragma unroll
        for (int u = 0; u < LOAD_BATCH; ++u) {
            const int i = base + u * nth;
            if (i < tot) {
                A[i] = make_float2(fix_to_float((long long)v[u].x), fix_to_float((long long)v[u].y));
            }
        }
    }
    for (int i = tid; i < Nh; i += nth) twh[i] = d.tw3h[i];
    for (int i = tid; i <= Nh; i += nth) tw3[i] = d.tw3[i];
    for (int i = tid; i < K2; i += nth) tw2[i] = d.tw2[i];
    PME_SYNC();
    float2 *Z = fft_batch<false>(A, B, Nh, K2, 1, Nh, twh);  // rows, stride Nh
    float2 *X = (Z == A) ? B : A;
    // split: X[m] = E[m] + W_K3^m O[m], E = (Z[m] + conj Z[Nh-m]) / 2, O = -i (Z[m] - conj Z[Nh-m]) / 2
    for (int i = tid; i < K2 * H3; i += nth) {
        const int k2 = fdiv(i, inv_h3), m = i - k2 * H3;
        const float2 *z = Z + k2 * Nh;
        const float2 zm = z[m == Nh ? 0 : m];
        const float2 zc = cconj(z[m == 0 ? 0 : Nh - m]);
        const float2 E = cscale(cadd(zm, zc), 0.5f);
        const float2 O = cscale(cmul_mi<false>(csub(zm, zc)), 0.5f);
        X[i] = cadd(E, cmul(tw3[m], O));
    }
    PME_SYNC();
    float2 *Y = fft_batch<false>(X, Z, K2, H3, H3, 1, tw2);  // columns m3, stride H3
    float2 *out = d.spec + (size_t)k1 * K2 * H3;
    for (int i = tid; i < K2 * H3; i += nth) out[i] = Y[i];
}

// ---------------------------------------------------------------------------------------------------------
// a4: pencils (m2, a chunk of m3 columns) — FFT along k1, multiply by the influence function B*C (the
// paper's "Green's function" step between Z and Z^-1, Sec. III-A "FFT"), reduce energy and virial, inverse
// FFT along k1.
//
// Energy and virial over the half spectrum: each m3 in (0, K3/2) stands for itself and its conjugate
// partner (weight 2), m3 = 0 and K3/2 have weight 1. Per-thread sums are double-float (about 44 bits);
// per-item partials are FP64, and the last item reduces all partials in a fixed order.

// m' = sum_alpha mt_alpha a*_alpha for the signed frequency (mt1, mt2, mt3).
PME_DEV void recip_vec(const SysDev &d, float mt1, float mt2, float mt3, float mv[3]) {
#pragma unroll
    for (int j = 0; j < 3; ++j) mv[j] = mt1 * d.rec[3 * j] + mt2 * d.rec[3 * j + 1] + mt3 * d.rec[3 * j + 2];
}

// signed frequency of index m on a K-point axis: m for m <= K/2, else m - K (K/2 maps to +K/2)
PME_DEV int signed_freq(int m, int K) { return 2 * m <= K ? m : m - K; }

#if defined(PME_HOST_EMULATION)
inline DF warp_sum_df(DF v) { return v; }
#else
__device__ __forceinline__ DF warp_sum_df(DF v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        DF other;
        other.hi = __shfl_down_sync(0xffffffffu, v.hi, o);
        other.lo = __shfl_down_sync(0xffffffffu, v.lo, o);
        v = df_add(v, other);
    }
    return v;
}
#endif

// One point m of the half spectrum: energy and virial terms of B*C |Q^(m)|^2 added to acc (E, then
// Pi xx yy zz xy xz yz), and the point multiplied by B*C. t is the point's influence-table entry (see
// SysDev::bc). With e = w B C |Q^|^2 (w = 1/2 on the self-conjugate planes m3 = 0, K3/2, else 1, the point
// standing for itself and its partner) the virial term is e (delta_ab - f m'_a m'_b), f = 2 (1 / |m'|^2 +
// pi^2 / beta^2), the table holding B*C f; on Nyquist planes the partner's m'_p differs from -m' and the
// term averages the two. m = 0 gives zero.
PME_DEV float2 influence_point(const SysDev &d, int m1, int m2, int m3, int mt2, float2 x, float4 t, float acc[7]) {
    if ((m1 | m2 | m3) == 0) return make_float2(0.f, 0.f);
    const bool self = (m3 == 0 || 2 * m3 == d.K3);
    const float wgt = self ? 0.5f : 1.0f;
    const float s2 = x.x * x.x + x.y * x.y;
    const float e = wgt * fmaf(t.x, s2, t.y * s2);
    const int mt1 = signed_freq(m1, d.K1);
    float mv[3];
    recip_vec(d, (float)mt1, (float)mt2, (float)m3, mv);
    const bool pair = t.w != 0.f;  // Nyquist plane: average with the partner
    const float G = (pair ? 0.5f : 1.0f) * wgt * s2 * t.z;
    float V[6];
    V[0] = G * mv[0] * mv[0];
    V[1] = G * mv[1] * mv[1];
    V[2] = G * mv[2] * mv[2];
    V[3] = G * mv[0] * mv[1];
    V[4] = G * mv[0] * mv[2];
    V[5] = G * mv[1] * mv[2];
    if (pair) {
        float mp[3];
        recip_vec(d, (float)(2 * m1 == d.K1 ? mt1 : -mt1), (float)(2 * m2 == d.K2 ? mt2 : -mt2), (float)(-m3), mp);
        const float Gp = 0.5f * wgt * s2 * t.w;
        V[0] = fmaf(Gp * mp[0], mp[0], V[0]);
        V[1] = fmaf(Gp * mp[1], mp[1], V[1]);
        V[2] = fmaf(Gp * mp[2], mp[2], V[2]);
        V[3] = fmaf(Gp * mp[0], mp[1], V[3]);
        V[4] = fmaf(Gp * mp[0], mp[2], V[4]);
        V[5] = fmaf(Gp * mp[1], mp[2], V[5]);
    }
    acc[0] += e;
    acc[1] += e - V[0];
    acc[2] += e - V[1];
    acc[3] += e - V[2];
    acc[4] -= V[3];
    acc[5] -= V[4];
    acc[6] -= V[5];
    x.x *= t.x;
    x.y *= t.x;
    return x;
}

PME_DEV void stage_conv_smem(const SysDev &d, int item, void *smem) {
    const int tid = PME_TID, nth = PME_NTH;
    const int K1 = d.K1, K2 = d.K2, H3 = d.H3;
    const int m2 = item / d.nchunk3;
    const int c0 = (item - m2 * d.nchunk3) * CONV_COLS;
    const int C = imin(CONV_COLS, H3 - c0);
    const float inv_c = 1.0f / (float)C;
    float2 *A = (float2 *)smem;
    float2 *B = A + K1 * CONV_COLS;
    float2 *tw1 = B + K1 * CONV_COLS;
    for (int base = tid; base < K1 * C; base += LOAD_BATCH * nth) {
        float2 v[LOAD_BATCH];
#pragma unroll
        for (int u = 0; u < LOAD_BATCH; ++u) {
            const int i = base + u * nth;
            if (i < K1 * C) {
                const int k1 = fdiv(i, inv_c), mc = i - k1 * C;
                v[u] = ldcg(d.spec + ((size_t)k1 * K2 + m2) * H3 + c0 + mc);
            }
        }
#pragma unroll
        for (int u = 0; u < LOAD_BATCH; ++u)
            if (base + u * nth < K1 * C) A[base + u * nth] = v[u];
    }
    for (int i = tid; i < K1; i += nth) tw1[i] = d.tw1[i];
    PME_SYNC();
    float2 *X = fft_batch<false>(A, B, K1, C, C, 1, tw1);
    float acc[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) acc[c] = 0.f;
    const float4 *bc = d.bc + (size_t)m2 * K1 * H3 + c0;
    const int mt2 = signed_freq(m2, K2);
    for (int i = tid; i < K1 * C; i += nth) {
        const int m1 = fdiv(i, inv_c), mc = i - m1 * C, m3 = c0 + mc;
        X[i] = influence_point(d, m1, m2, m3, mt2, X[i], bc[(size_t)m1 * H3 + mc], acc);
    }
    PME_SYNC();
    float2 *Y = fft_batch<true>(X, (X == A) ? B : A, K1, C, C, 1, tw1);
    for (int i = tid; i < K1 * C; i += nth) {
        const int k1 = fdiv(i, inv_c), mc = i - k1 * C;
        d.spec[((size_t)k1 * K2 + m2) * H3 + c0 + mc] = Y[i];
    }
    PME_SYNC();
    // Item partial of the 7 sums: each thread holds a few FP32 terms; they meet in a double-float tree
    // (16 lanes per component, then one lane), written to this item's slot. The inverse-FFT stage, which
    // starts only after every item of this stage, reduces the slots.
    float *red = (float *)smem;  // 7 x nth
    DF *red2 = (DF *)(red + 7 * nth);  // 7 x 16
#pragma unroll
    for (int c = 0; c < 7; ++c) red[c * nth + tid] = acc[c];
    PME_SYNC();
    for (int r = tid; r < 7 * 16; r += nth) {
        const int c = r >> 4, lane = r & 15;
        DF s;
        s.hi = s.lo = 0.f;
        for (int t = lane; t < nth; t += 16) s = df_add(s, red[c * nth + t]);
        red2[r] = s;
    }
    PME_SYNC();
    DF *part = (DF *)d.partials;  // 8 double-float slots per item
    for (int c = tid; c < 7; c += nth) {
        DF s = red2[c * 16];
        for (int lane = 1; lane < 16; ++lane) s = df_add(s, red2[c * 16 + lane]);
        part[(size_t)item * 8 + c] = s;
    }
}

// ---------------------------------------------------------------------------------------------------------
// Slab decomposition helpers (the corner turns of the paper's distributed 3D FFT, Sec. III-A "FFT"): copy
// the block of planes [pa, pb) x columns [ca, cb) of the half spectrum to or from a packed buffer
// (row k1 - pa of width cb - ca), with thread t of nth covering elements t, t + nth, ...

PME_DEV void slab_pack(const float2 *spec, int ncol, int pa, int pb, int ca, int cb, float2 *dst, int t, int nth) {
    const int w = cb - ca, tot = (pb - pa) * w;
    for (int i = t; i < tot; i += nth) {
        const int k = i / w, c = i - k * w;
        dst[i] = ldcg(spec + (size_t)(pa + k) * ncol + ca + c);
    }
}
PME_DEV void slab_unpack(float2 *spec, int ncol, int pa, int pb, int ca, int cb, const float2 *src, int t, int nth) {
    const int w = cb - ca, tot = (pb - pa) * w;
    for (int i = t; i < tot; i += nth) {
        const int k = i / w, c = i - k * w;
        spec[(size_t)(pa + k) * ncol + ca + c] = ldcg(src + i);
    }
}

// The energy and virial partial of the influence items [i0, i1) (this rank's columns), summed in order in
// double-float: out[c] for the 7 components (E, then Pi xx yy zz xy xz yz). Thread t < 7 sums component t.
PME_DEV void slab_energy(const SysDev &d, int i0, int i1, double *out, int t) {
    if (t >= 7) return;
    const DF *part = (const DF *)d.partials;
    DF s;
    s.hi = s.lo = 0.f;
    for (int i = i0; i < i1; ++i) s = df_add(s, part[(size_t)i * 8 + t]);
    out[t] = (double)s.hi + (double)s.lo;
}

// Energy and virial of the whole system, in two fixed-order levels off the critical path. Level 1 (inverse
// slab item k1): the influence-stage item partials k1, k1 + K1, k1 + 2 K1, ... in order -> slot k1. Level 2
// (the first overflow item of the force stage, otherwise idle when no bucket overflowed): the K1 slots in a
// fixed binary tree -> FP64 energy and virial. Neither order depends on the block size.
PME_DEV void reduce_level1(const SysDev &d, int k1, int tid, int nth) {
    const DF *part = (const DF *)d.partials;
    DF *slot = (DF *)d.partials + (size_t)d.nconv * 8;  // K1 level-1 slots of 8 after the item partials
    for (int c = tid; c < 7; c += nth) {
        DF s;
        s.hi = s.lo = 0.f;
        for (int it0 = k1; it0 < d.nconv; it0 += LOAD_BATCH * d.K1) {
            float2 p2[LOAD_BATCH];
#pragma unroll
            for (int u = 0; u < LOAD_BATCH; ++u) {
                const int it = it0 + u * d.K1;
                if (it < d.nconv) p2[u] = ldcg((const float2 *)(part + (size_t)it * 8 + c));
            }
#pragma unroll
            for (int u = 0; u < LOAD_BATCH; ++u)
                if (it0 + u * d.K1 < d.nconv) {
                    DF pv;
                    pv.hi = p2[u].x;
                    pv.lo = p2[u].y;
                    s = df_add(s, pv);
                }
        }
        slot[(size_t)k1 * 8 + c] = s;
    }
}

// Plane k1 of the int64 charge mesh back to zero for the next spreading (its reader, the forward stage,
// finished before the influence stage started); the stores overlap the inverse stage's own work.
PME_DEV void zero_mesh_plane(const SysDev &d, int k1, int tid, int nth) {
    ulonglong2 *g = (ulonglong2 *)(d.grid + (size_t)k1 * d.K2 * d.K3);
    const int tot = d.K2 * d.K3 / 2;
    for (int i = tid; i < tot; i += nth) g[i] = make_ulonglong2(0ull, 0ull);
}

// Side work of inverse slab k1, off the transforms' critical path: zero the mesh plane and run the level-1
// energy / virial reduction (every influence item has finished), on threads [t0, t0 + nt).
PME_DEV void inv_side_work(const SysDev &d, int k1, int t0, int nt) {
    const int t = PME_TID - t0;
    if (t < 0 || t >= nt) return;
    reduce_level1(d, k1, t, nt);
    zero_mesh_plane(d, k1, t, nt);
}

PME_DEV void reduce_level2(const SysDev &d, void *smem) {
    const int tid = PME_TID, nth = PME_NTH;
    const DF *slot = (const DF *)d.partials + (size_t)d.nconv * 8;
    DF *t = (DF *)smem;  // REDUCE_SLOTS x 7: slot v holds level-1 slots v, v + REDUCE_SLOTS (K1 <= 2 * REDUCE_SLOTS)
    for (int r = tid; r < REDUCE_SLOTS * 7; r += nth) {
        const int v = r / 7, c = r - v * 7;
        DF s;
        s.hi = s.lo = 0.f;
        if (v < d.K1) {
            const float2 a = ldcg((const float2 *)(slot + (size_t)v * 8 + c));
            s.hi = a.x;
            s.lo = a.y;
        }
        if (v + REDUCE_SLOTS < d.K1) {
            const float2 b = ldcg((const float2 *)(slot + (size_t)(v + REDUCE_SLOTS) * 8 + c));
            DF bv;
            bv.hi = b.x;
            bv.lo = b.y;
            s = df_add(s, bv);
        }
        t[r] = s;
    }
    PME_SYNC();
    for (int h = REDUCE_SLOTS / 2; h > 0; h >>= 1) {
        for (int r = tid; r < h * 7; r += nth) {
            const int v = r / 7, c = r - v * 7;
            t[v * 7 + c] = df_add(t[v * 7 + c], t[(v + h) * 7 + c]);
        }
        PME_SYNC();
    }
    if (tid == 0)
        for (int c = 0; c < 7; ++c) d.ev[c] = (double)t[c].hi + (double)t[c].lo;
    // the sum of |q| over the binning slots (exact integers): past the fixed-point headroom -> overflow;
    // the slots go back to zero for the next binning
    // (every stage that may set status bits but this one has completed, so with ev_status the word stored
    // in ev[7] is final)
#if defined(PME_HOST_EMULATION)
    if (tid == 0) {
        unsigned long long qa = 0;
        for (int sl = 0; sl < QABS_SLOTS; ++sl) {
            qa += d.qslot[(size_t)sl * 16];
            d.qslot[(size_t)sl * 16] = 0ull;
        }
        if (qa >= QABS_LIMIT) atomic_or_u32(&d.ctl->status, ST_OVERFLOW);
        if (d.ev_status) d.ev[7] = (double)d.ctl->status;
    }
#else
    if (tid < 32) {
        unsigned long long qa = ldcg(d.qslot + (size_t)tid * 16) + ldcg(d.qslot + (size_t)(tid + 32) * 16);
        qa = warp_sum_u64(qa);
        d.qslot[(size_t)tid * 16] = 0ull;
        d.qslot[(size_t)(tid + 32) * 16] = 0ull;
        if (tid == 0) {
            if (qa >= QABS_LIMIT) atomic_or_u32(&d.ctl->status, ST_OVERFLOW);
            if (d.ev_status) d.ev[7] = (double)(ldcg(&d.ctl->status) | (qa >= QABS_LIMIT ? (unsigned)ST_OVERFLOW : 0u));
        }
    }
#endif
    PME_SYNC();
}

// ---------------------------------------------------------------------------------------------------------
// a5: inverse slab k1 — inverse FFT along k2 per m3 column, then the complex-to-real inverse along k3
// (merge step + a length K3/2 complex FFT whose real / imaginary parts are the even / odd samples).

PME_DEV void stage_inv_smem(const SysDev &d, int k1, void *smem) {
    const int tid = PME_TID, nth = PME_NTH;
    const int K2 = d.K2, K3 = d.K3, H3 = d.H3, Nh = K3 / 2;
    const float inv_nh = 1.0f / (float)Nh;
    float2 *A = (float2 *)smem;
    float2 *B = A + K2 * H3;
    float2 *twh = B + K2 * H3;
    float2 *tw3 = twh + Nh;
    float2 *tw2 = tw3 + Nh + 1;
    const float2 *in = d.spec + (size_t)k1 * K2 * H3;
    copy_batched(A, in, K2 * H3);
    for (int i = tid; i < Nh; i += nth) twh[i] = d.tw3h[i];
    for (int i = tid; i <= Nh; i += nth) tw3[i] = d.tw3[i];
    for (int i = tid; i < K2; i += nth) tw2[i] = d.tw2[i];
    PME_SYNC();
    float2 *Y = fft_batch<true>(A, B, K2, H3, H3, 1, tw2);
    float2 *Z = (Y == A) ? B : A;
    // Z[m] = (X[m] + conj X[Nh-m]) + i (X[m] - conj X[Nh-m]) exp(+2 pi i m / K3), m < Nh
    for (int i = tid; i < K2 * Nh; i += nth) {
        const int k2 = fdiv(i, inv_nh), m = i - k2 * Nh;
        const float2 *x = Y + k2 * H3;
        const float2 xm = x[m], xc = cconj(x[Nh - m]);
        const float2 a = cadd(xm, xc);
        const float2 b = cmul(csub(xm, xc), cconj(tw3[m]));
        Z[i] = make_float2(a.x - b.y, a.y + b.x);
    }
    PME_SYNC();
    float2 *R = fft_batch<true>(Z, Y, Nh, K2, 1, Nh, twh);
    float2 *out = (float2 *)(d.phi + (size_t)k1 * K2 * K3);  // (phi[2n], phi[2n+1]) = (Re, Im) of R[n]
    for (int i = tid; i < K2 * Nh; i += nth) out[i] = R[i];
}

#if defined(PME_LANE_FFT)
}  // namespace pme
#include <cooperative_groups.h>
namespace pme {
namespace cg = cooperative_groups;
// ---------------------------------------------------------------------------------------------------------
// Register path of a3 - a5 (lane plans, fft.cuh): each transform runs in the registers of L lanes of one
// warp, reading its points straight from global memory (or from the slab buffer in shared memory) and
// writing its results straight to their destination. A slab stage has one CTA barrier (between its two
// transform directions), the influence stage none before its energy reduction. Thread counts must be
// multiples of 32; every warp runs whole loop iterations, and lanes past the end work on a valid dummy
// transform without storing, so the shuffles always see full warps.

// Unit u -> (transform t, lane j): warp u / 32 holds T = 32 / L transforms at lane ids t mod T + T j.
template <int L>
PME_DEV void lane_unit(int u, int &t, int &j) {
    constexpr int T = 32 / L;
    const int lid = u & 31;
    t = (u >> 5) * T + (lid & (T - 1));
    j = lid / T;
}

// Units covering ntr transforms of L lanes: whole warps.
template <int L>
PME_DEV int lane_units(int ntr) {
    constexpr int T = 32 / L;
    return ((ntr + T - 1) / T) * 32;
}

// Where a slab pass stores its intermediate results: the CTA's own slab buffer and, when a slab is split
// over a cluster of NB CTAs, the same offset in the other CTAs' buffers (distributed shared memory), so that
// every CTA of the cluster holds the whole intermediate slab for the second pass.
template <int NB>
struct SlabDst {
    float2 *buf[NB];
    PME_DEV void put(int i, float2 v) const {
#pragma unroll
        for (int c = 0; c < NB; ++c) buf[c][i] = v;
    }
};

// a3 rows: the packed real row k2 (z[n] = Q[2n] + i Q[2n+1], K3/2 = L E points) from the int64 mesh; the
// K3/2-point transform goes to row k2 of Z (row stride zs). Rows [t0, t0 + nt).
template <int L, int E, int NB>
PME_DEV void fwd_rows_lane(const SysDev &d, int k1, const SlabDst<NB> &Z, int zs, int t0, int nt) {
    const int K2 = d.K2, total = lane_units<L>(nt);
    for (int u = PME_TID; u < total; u += PME_NTH) {
        int t, j;
        lane_unit<L>(u, t, j);
        const bool ok = t < nt;
        t += t0;
        const ulonglong2 *g = (const ulonglong2 *)(d.grid + ((size_t)k1 * K2 + (ok ? t : t0)) * d.K3);
        ulonglong2 w[E];
#pragma unroll
        for (int n = 0; n < E; ++n) w[n] = ldcg(g + j + L * n);
        const LaneTw<L, E> tw = lane_tw<L, E, true>(d.tw3h, j);
        float2 v[E];
#pragma unroll
        for (int n = 0; n < E; ++n) v[n] = make_float2(fix_to_float((long long)w[n].x), fix_to_float((long long)w[n].y));
        lane_fft<L, E, false>(v, j, tw);
        if (ok) {
            const int r = lane_rev<L>(j);
#pragma unroll
            for (int k = 0; k < E; ++k) Z.put(t * zs + k + E * r, v[k]);
        }
    }
}

// a3 columns: the split X[m] = E[m] + W_K3^m O[m] of row transforms Z (E, O as in the shared-memory path)
// fused into the loads of column m3, then the K2-point transform along k2 into the half spectrum. tw3
// (K3/2 + 1 entries) and tw2 (K2 entries) are shared-memory copies. Columns [m0, m0 + nm).
template <int L, int E>
PME_DEV void fwd_cols_lane(const SysDev &d, int k1, const float2 *Z, int zs, const float2 *tw3, const float2 *tw2,
                           int m0, int nm) {
    const int K2 = d.K2, H3 = d.H3, Nh = d.K3 / 2, total = lane_units<L>(nm);
    float2 *out = d.spec + (size_t)k1 * K2 * H3;
    for (int u = PME_TID; u < total; u += PME_NTH) {
        int m, j;
        lane_unit<L>(u, m, j);
        const bool ok = m < nm;
        m += m0;
        const int mm = ok ? m : m0;
        const LaneTw<L, E> tw = lane_tw<L, E, false>(tw2, j);
        const float2 w3 = tw3[mm];
        const int ia = mm == Nh ? 0 : mm, ib = mm == 0 ? 0 : Nh - mm;
        float2 v[E];
#pragma unroll
        for (int n = 0; n < E; ++n) {
            const float2 *z = Z + (j + L * n) * zs;
            const float2 zm = z[ia], zc = cconj(z[ib]);
            const float2 Ev = cscale(cadd(zm, zc), 0.5f);
            const float2 Ov = cscale(cmul_mi<false>(csub(zm, zc)), 0.5f);
            v[n] = cadd(Ev, cmul(w3, Ov));
        }
        lane_fft<L, E, false>(v, j, tw);
        if (ok) {
            const int r = lane_rev<L>(j);
#pragma unroll
            for (int k = 0; k < E; ++k) out[(size_t)(k + E * r) * H3 + m] = v[k];
        }
    }
}

// a5 columns: inverse K2-point transforms of column m3 of the half spectrum into Y (row stride ys). Columns
// [m0, m0 + nm).
template <int L, int E, int NB>
PME_DEV void inv_cols_lane(const SysDev &d, int k1, const SlabDst<NB> &Y, int ys, int m0, int nm) {
    const int K2 = d.K2, H3 = d.H3, total = lane_units<L>(nm);
    const float2 *in = d.spec + (size_t)k1 * K2 * H3;
    for (int u = PME_TID; u < total; u += PME_NTH) {
        int m, j;
        lane_unit<L>(u, m, j);
        const bool ok = m < nm;
        m += m0;
        const int mm = ok ? m : m0;
        float2 v[E];
#pragma unroll
        for (int n = 0; n < E; ++n) v[n] = ldcg(in + (size_t)(j + L * n) * H3 + mm);
        const LaneTw<L, E> tw = lane_tw<L, E, true>(d.tw2, j);
        lane_fft<L, E, true>(v, j, tw);
        if (ok) {
            const int r = lane_rev<L>(j);
#pragma unroll
            for (int k = 0; k < E; ++k) Y.put((k + E * r) * ys + m, v[k]);
        }
    }
}

// a5 rows: the merge Z[m] = (X[m] + conj X[Nh-m]) + i (X[m] - conj X[Nh-m]) exp(+2 pi i m / K3) fused into
// the loads, then the inverse K3/2-point transform, whose real / imaginary parts are phi at even / odd k3.
// twh (K3/2 entries) and tw3 (K3/2 + 1) are shared-memory copies. Rows [t0, t0 + nt).
template <int L, int E>
PME_DEV void inv_rows_lane(const SysDev &d, int k1, const float2 *Y, int ys, const float2 *twh, const float2 *tw3,
                           int t0, int nt) {
    const int K2 = d.K2, Nh = d.K3 / 2, total = lane_units<L>(nt);
    float2 *out = (float2 *)(d.phi + (size_t)k1 * K2 * d.K3);
    for (int u = PME_TID; u < total; u += PME_NTH) {
        int t, j;
        lane_unit<L>(u, t, j);
        const bool ok = t < nt;
        t += t0;
        const float2 *x = Y + (ok ? t : t0) * ys;
        const LaneTw<L, E> tw = lane_tw<L, E, false>(twh, j);
        float2 v[E];
#pragma unroll
        for (int n = 0; n < E; ++n) {
            const int m = j + L * n;
            const float2 xm = x[m], xc = cconj(x[Nh - m]);
            const float2 a = cadd(xm, xc);
            const float2 b = cmul(csub(xm, xc), cconj(tw3[m]));
            v[n] = make_float2(a.x - b.y, a.y + b.x);
        }
        lane_fft<L, E, true>(v, j, tw);
        if (ok) {
            const int r = lane_rev<L>(j);
            float2 *o = out + (size_t)t * Nh;
#pragma unroll
            for (int k = 0; k < E; ++k) o[k + E * r] = v[k];
        }
    }
}

// a4 / a7 register path: work item = CONV_UNITS / L consecutive columns (m2, m3) of the half spectrum
// (flattened m2 H3 + m3). Each column: forward K1-point transform, B*C product with the energy and virial
// terms (influence_point), adjoint transform back in place. The item's energy / virial partial is a
// fixed-order double-float tree over its CONV_UNITS lanes, one component per warp, independent of the block
// size.
template <int L, int E>
PME_DEV void conv_lane(const SysDev &d, int item, void *smem) {
    constexpr int COLS = CONV_UNITS / L;
    const int tid = PME_TID, nth = PME_NTH;
    const int K1 = d.K1, K2 = d.K2, H3 = d.H3, ncol = K2 * H3;
    const float inv_h3 = 1.0f / (float)H3;
    float *red = (float *)smem;  // 7 x CONV_UNITS
    for (int u = tid; u < CONV_UNITS; u += nth) {
        int t, j;
        lane_unit<L>(u, t, j);
        const int col = item * COLS + t;
        const bool ok = col < ncol;
        const int cc = ok ? col : 0;
        const int m2 = fdiv(cc, inv_h3), m3 = cc - m2 * H3;
        const int r = lane_rev<L>(j);
        float2 v[E];
        float4 bcv[E];
#pragma unroll
        for (int n = 0; n < E; ++n) v[n] = ldcg(d.spec + ((size_t)(j + L * n) * K2 + m2) * H3 + m3);
#pragma unroll
        for (int k = 0; k < E; ++k) bcv[k] = ldcg(d.bc + ((size_t)m2 * K1 + k + E * r) * H3 + m3);
        const LaneTw<L, E> tw = lane_tw<L, E, true>(d.tw1, j);
        lane_fft<L, E, false>(v, j, tw);
        float acc[7];
#pragma unroll
        for (int c = 0; c < 7; ++c) acc[c] = 0.f;
        const int mt2 = signed_freq(m2, K2);
#pragma unroll
        for (int k = 0; k < E; ++k) v[k] = influence_point(d, k + E * r, m2, m3, mt2, v[k], bcv[k], acc);
        lane_fft_adjoint<L, E>(v, j, tw);
        if (ok) {
#pragma unroll
            for (int n = 0; n < E; ++n) d.spec[((size_t)(j + L * n) * K2 + m2) * H3 + m3] = v[n];
        }
#pragma unroll
        for (int c = 0; c < 7; ++c) red[c * CONV_UNITS + u] = ok ? acc[c] : 0.f;
    }
    PME_SYNC();
    // component c by warp c mod 4: each lane adds units lane, lane + 32, ... in double-float, then a
    // shuffle tree over the warp (lane 0 holds the fixed-order result)
    DF *part = (DF *)d.partials;
    const int nw = nth >> 5, w = tid >> 5, lane = tid & 31;
    for (int c0 = w; c0 < 7; c0 += 2 * nw) {  // components c0 and c0 + nw side by side
        const int c1 = c0 + nw < 7 ? c0 + nw : c0;
        DF s0, s1;
        s0.hi = red[c0 * CONV_UNITS + lane];
        s1.hi = red[c1 * CONV_UNITS + lane];
        s0.lo = s1.lo = 0.f;
        for (int t = lane + 32; t < CONV_UNITS; t += 32) {
            s0 = df_add(s0, red[c0 * CONV_UNITS + t]);
            s1 = df_add(s1, red[c1 * CONV_UNITS + t]);
        }
        s0 = warp_sum_df(s0);
        s1 = warp_sum_df(s1);
        if (lane == 0) {
            part[(size_t)item * 8 + c0] = s0;
            if (c1 != c0) part[(size_t)item * 8 + c1] = s1;
        }
    }
}


PME_DEV int plan_col_units(int c, int ntr) {
    const int T = 32 / plan_L(c);
    return ((ntr + T - 1) / T) * 32;
}

// Row strides (>= w) of the slab buffers, chosen so that the 16 lanes of a half-warp of the reading pass
// (T = 32 / L transforms x 16 / T lanes, float2 = two banks) fall on distinct shared-memory banks.
// Column reader (transform = column, lane j steps rows): stride = min(T, 16) mod 16.
PME_DEV int stride_col_reader(int w, int c) {
    const int L = plan_L(c);
    if (L <= 2) return w;  // a half-warp reads 16 consecutive columns of one row
    return w + ((32 / L - w) & 15);
}
// Row reader (transform = row, lane j steps along the row): stride = max(L / 2, 1) mod 16.
PME_DEV int stride_row_reader(int w, int c) {
    const int L = plan_L(c);
    if (L >= 32) return w;  // a half-warp reads 16 consecutive points of one row
    return w + (((L >= 2 ? L / 2 : 1) - w) & 15);
}

// Compile-time lanes and points of plan C.
template <int C>
struct PlanLE {
    static constexpr int L = plan_L(C), E = plan_E(C);
};

// Lane slab / influence stages with the plans fixed at compile time (PR, PC, P1 >= 0: only that plan's code
// is built into the kernel, which keeps it small enough for the instruction caches) or chosen at run time
// from the system's plans (-1).
template <int PR, int PC>
PME_DEV void stage_fwd_lane(const SysDev &d, int k1, void *smem) {
    const int Nh = d.K3 / 2, zs = stride_col_reader(Nh, d.lp_cols);
    float2 *Z = (float2 *)smem;
    float2 *tw3 = Z + d.K2 * zs;  // Nh + 1
    float2 *tw2 = tw3 + Nh + 1;   // K2
    // the column pass's tables: loads issued before the row pass, stores after it, so their latency hides
    // behind the row pass
    const int tid = PME_TID;
    const float2 a = tid <= Nh ? __ldg(d.tw3 + tid) : make_float2(0.f, 0.f);
    const float2 b = tid < d.K2 ? __ldg(d.tw2 + tid) : make_float2(0.f, 0.f);
    const SlabDst<1> Zd = {{Z}};
    if constexpr (PR >= 0) {
        fwd_rows_lane<PlanLE<PR>::L, PlanLE<PR>::E>(d, k1, Zd, zs, 0, d.K2);
    } else {
        switch (d.lp_rows) {
#define PME_ROWS(c, L, E) \
    case c: fwd_rows_lane<L, E>(d, k1, Zd, zs, 0, d.K2); break;
            PME_LANE_CASES(PME_ROWS)
#undef PME_ROWS
        }
    }
    if (tid <= Nh) tw3[tid] = a;
    if (tid < d.K2) tw2[tid] = b;
    for (int i = tid + PME_NTH; i <= Nh; i += PME_NTH) tw3[i] = d.tw3[i];
    for (int i = tid + PME_NTH; i < d.K2; i += PME_NTH) tw2[i] = d.tw2[i];
    PME_SYNC();
    if constexpr (PC >= 0) {
        fwd_cols_lane<PlanLE<PC>::L, PlanLE<PC>::E>(d, k1, Z, zs, tw3, tw2, 0, d.H3);
    } else {
        switch (d.lp_cols) {
#define PME_COLS(c, L, E) \
    case c: fwd_cols_lane<L, E>(d, k1, Z, zs, tw3, tw2, 0, d.H3); break;
            PME_LANE_CASES(PME_COLS)
#undef PME_COLS
        }
    }
}

template <int PR, int PC>
PME_DEV void stage_inv_lane(const SysDev &d, int k1, void *smem) {
    const int Nh = d.K3 / 2, ys = stride_row_reader(d.H3, d.lp_rows);
    float2 *Y = (float2 *)smem;
    float2 *twh = Y + d.K2 * ys;  // Nh
    float2 *tw3 = twh + Nh;       // Nh + 1
    // the row pass's tables: loads issued first, stores after the column pass (latency hidden behind it)
    const int tid = PME_TID;
    const float2 a = tid < Nh ? __ldg(d.tw3h + tid) : make_float2(0.f, 0.f);
    const float2 b = tid <= Nh ? __ldg(d.tw3 + tid) : make_float2(0.f, 0.f);
    // the column pass needs cu threads; warps beyond them (if any) take the side work, else everyone first
    const int cu = plan_col_units(d.lp_cols, d.H3);
    if (PME_NTH - cu >= 32) inv_side_work(d, k1, cu, PME_NTH - cu);
    else inv_side_work(d, k1, 0, PME_NTH);
    const SlabDst<1> Yd = {{Y}};
    if constexpr (PC >= 0) {
        inv_cols_lane<PlanLE<PC>::L, PlanLE<PC>::E>(d, k1, Yd, ys, 0, d.H3);
    } else {
        switch (d.lp_cols) {
#define PME_COLS(c, L, E) \
    case c: inv_cols_lane<L, E>(d, k1, Yd, ys, 0, d.H3); break;
            PME_LANE_CASES(PME_COLS)
#undef PME_COLS
        }
    }
    if (tid < Nh) twh[tid] = a;
    if (tid <= Nh) tw3[tid] = b;
    for (int i = tid + PME_NTH; i < Nh; i += PME_NTH) twh[i] = d.tw3h[i];
    for (int i = tid + PME_NTH; i <= Nh; i += PME_NTH) tw3[i] = d.tw3[i];
    PME_SYNC();
    if constexpr (PR >= 0) {
        inv_rows_lane<PlanLE<PR>::L, PlanLE<PR>::E>(d, k1, Y, ys, twh, tw3, 0, d.K2);
    } else {
        switch (d.lp_rows) {
#define PME_ROWS(c, L, E) \
    case c: inv_rows_lane<L, E>(d, k1, Y, ys, twh, tw3, 0, d.K2); break;
            PME_LANE_CASES(PME_ROWS)
#undef PME_ROWS
        }
    }
}

// Slab k1 split over a cluster of CS CTAs (rank c of the cluster), plans PR / PC at compile time: each
// CTA transforms rows [c K2 / CS, (c + 1) K2 / CS) and stores them into every CTA's slab buffer (distributed
// shared memory), the cluster barrier makes them visible, then each CTA transforms its share of the
// columns. With the plans of the one-CTA kernel these are the same transforms and stores as
// stage_fwd_lane, so the results are bitwise the same; a slab takes CS SMs instead of one.
PME_DEV void split_range(int n, int c, int cs, int &a, int &cnt) {
    const int per = (n + cs - 1) / cs;
    a = imin(n, c * per);
    cnt = imin(n, a + per) - a;
}

template <int PR, int PC, int CS>
PME_DEV void stage_fwd_cluster(const SysDev &d, int k1, int c, void *smem) {
    cg::cluster_group cl = cg::this_cluster();
    const int Nh = d.K3 / 2, zs = stride_col_reader(Nh, PC);
    float2 *Z = (float2 *)smem;
    float2 *tw3 = Z + d.K2 * zs;
    float2 *tw2 = tw3 + Nh + 1;
    const int tid = PME_TID;
    const float2 a = tid <= Nh ? __ldg(d.tw3 + tid) : make_float2(0.f, 0.f);
    const float2 b = tid < d.K2 ? __ldg(d.tw2 + tid) : make_float2(0.f, 0.f);
    if (k1 == 0 && c == 0 && tid == 0) d.ctl->novf = 0u;  // spreading (its last reader) has finished
    SlabDst<CS> Zd;
#pragma unroll
    for (int q = 0; q < CS; ++q) Zd.buf[q] = cl.map_shared_rank(Z, (unsigned)((c + q) % CS));
    int t0, nt, m0, nm;
    split_range(d.K2, c, CS, t0, nt);
    split_range(d.H3, c, CS, m0, nm);
    fwd_rows_lane<PlanLE<PR>::L, PlanLE<PR>::E, CS>(d, k1, Zd, zs, t0, nt);
    if (tid <= Nh) tw3[tid] = a;
    if (tid < d.K2) tw2[tid] = b;
    for (int i = tid + PME_NTH; i <= Nh; i += PME_NTH) tw3[i] = d.tw3[i];
    for (int i = tid + PME_NTH; i < d.K2; i += PME_NTH) tw2[i] = d.tw2[i];
    cl.sync();  // every row of Z, from every CTA of the cluster; no remote access after this point
    fwd_cols_lane<PlanLE<PC>::L, PlanLE<PC>::E>(d, k1, Z, zs, tw3, tw2, m0, nm);
}

// Inverse slab k1 split the same way: columns first (stored into every CTA's buffer), the cluster barrier,
// then each CTA's rows. The side work (zeroing the mesh plane, the level-1 energy reduction) is divided
// among the CTAs and runs on the warps the column pass leaves free (else before it).
template <int PR, int PC, int CS>
PME_DEV void stage_inv_cluster(const SysDev &d, int k1, int c, void *smem) {
    cg::cluster_group cl = cg::this_cluster();
    const int Nh = d.K3 / 2, ys = stride_row_reader(d.H3, PR);
    float2 *Y = (float2 *)smem;
    float2 *twh = Y + d.K2 * ys;
    float2 *tw3 = twh + Nh;
    const int tid = PME_TID, nth = PME_NTH;
    const float2 a = tid < Nh ? __ldg(d.tw3h + tid) : make_float2(0.f, 0.f);
    const float2 b = tid <= Nh ? __ldg(d.tw3 + tid) : make_float2(0.f, 0.f);
    int t0, nt, m0, nm;
    split_range(d.K2, c, CS, t0, nt);
    split_range(d.H3, c, CS, m0, nm);
    {
        const int cu = lane_units<PlanLE<PC>::L>(nm);
        const int s0 = nth - cu >= 32 ? cu : 0, ns = nth - s0, st = tid - s0;
        if (st >= 0) {
            if (c == 0) reduce_level1(d, k1, st, ns);
            ulonglong2 *g = (ulonglong2 *)(d.grid + (size_t)k1 * d.K2 * d.K3);
            int z0, nz;
            split_range(d.K2 * d.K3 / 2, c, CS, z0, nz);
            for (int i = st; i < nz; i += ns) g[z0 + i] = make_ulonglong2(0ull, 0ull);
        }
    }
    SlabDst<CS> Yd;
#pragma unroll
    for (int q = 0; q < CS; ++q) Yd.buf[q] = cl.map_shared_rank(Y, (unsigned)((c + q) % CS));
    inv_cols_lane<PlanLE<PC>::L, PlanLE<PC>::E, CS>(d, k1, Yd, ys, m0, nm);
    if (tid < Nh) twh[tid] = a;
    if (tid <= Nh) tw3[tid] = b;
    for (int i = tid + nth; i < Nh; i += nth) twh[i] = d.tw3h[i];
    for (int i = tid + nth; i <= Nh; i += nth) tw3[i] = d.tw3[i];
    cl.sync();  // every column of Y, from every CTA of the cluster; no remote access after this point
    inv_rows_lane<PlanLE<PR>::L, PlanLE<PR>::E>(d, k1, Y, ys, twh, tw3, t0, nt);
}

template <int P1>
PME_DEV void stage_conv_lane(const SysDev &d, int item, void *smem) {
    if constexpr (P1 >= 0) {
        conv_lane<PlanLE<P1>::L, PlanLE<P1>::E>(d, item, smem);
    } else {
        switch (d.lp_k1) {
#define PME_K1(c, L, E) \
    case c: conv_lane<L, E>(d, item, smem); break;
            PME_LANE_CASES(PME_K1)
#undef PME_K1
        }
    }
}
#endif  // PME_LANE_FFT

// Stage entry points: the register path where the plan has lane plans, else the shared-memory path. With
// plans given at compile time (a kernel specialised for one mesh), only the register path is built in; such
// a kernel runs only for systems with exactly those plans.
template <int PR = -1, int PC = -1>
PME_DEV void stage_fwd(const SysDev &d, int k1, void *smem) {
    if (k1 == 0 && PME_TID == 0) d.ctl->novf = 0u;  // spreading (its last reader) has finished
#if defined(PME_LANE_FFT)
    if constexpr (PR >= 0) {
        stage_fwd_lane<PR, PC>(d, k1, smem);
    } else {
        if (d.lane_slab) stage_fwd_lane<-1, -1>(d, k1, smem);
        else stage_fwd_smem(d, k1, smem);
    }
#else
    stage_fwd_smem(d, k1, smem);
#endif
}

template <int P1 = -1>
PME_DEV void stage_conv(const SysDev &d, int item, void *smem) {
#if defined(PME_LANE_FFT)
    if constexpr (P1 >= 0) {
        stage_conv_lane<P1>(d, item, smem);
    } else {
        if (d.lane_conv) stage_conv_lane<-1>(d, item, smem);
        else stage_conv_smem(d, item, smem);
    }
#else
    stage_conv_smem(d, item, smem);
#endif
}

template <int PR = -1, int PC = -1>
PME_DEV void stage_inv(const SysDev &d, int k1, void *smem) {
#if defined(PME_LANE_FFT)
    if constexpr (PR >= 0) {
        stage_inv_lane<PR, PC>(d, k1, smem);
    } else {
        if (d.lane_slab) {
            stage_inv_lane<-1, -1>(d, k1, smem);
        } else {
            inv_side_work(d, k1, 0, PME_NTH);
            stage_inv_smem(d, k1, smem);
        }
    }
#else
    inv_side_work(d, k1, 0, PME_NTH);
    stage_inv_smem(d, k1, smem);
#endif
}

// ---------------------------------------------------------------------------------------------------------
// a6: force interpolation F_i = -q_i sum_k grad(theta1 theta2 theta3) phi(k) (paper Sec. III-A "Force
// Interpolation": B-spline derivatives times the potential mesh, summed over the p^3 neighbourhood). A
// tile stages its phi region (with the p - 1 halo) in shared memory; each thread interpolates one atom
// and writes its force at the atom's input index.

template <int P>
PME_DEV void force_from_grad(const SysDev &d, float q, int idx, float g1, float g2, float g3) {
#pragma unroll
    for (int j = 0; j < 3; ++j)
        d.forces[3 * (size_t)idx + j] = -q * (d.chi[3 * j] * g1 + d.chi[3 * j + 1] * g2 + d.chi[3 * j + 2] * g3);
}

// Bucket-overflow atoms read phi from global memory but sum exactly like the tile path (two halves of the
// j1 planes, then half 0 + half 1), so an atom's force has the same bits whichever path it takes.
template <int P>
PME_DEV void gather_atom_global(const SysDev &d, float4 ra, int2 rb) {
    float th1[P], th2[P], th3[P], dth1[P], dth2[P], dth3[P];
    bspline_wd<P>(ra.x, th1, dth1);
    bspline_wd<P>(ra.y, th2, dth2);
    bspline_wd<P>(ra.z, th3, dth3);
    const int b1 = rb.x & 1023, b2 = (rb.x >> 10) & 1023, b3 = (rb.x >> 20) & 1023;
    constexpr int H0 = half_planes(P);
    float gh[2][3];
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        float g1 = 0.f, g2 = 0.f, g3 = 0.f;
#pragma unroll
        for (int jj = 0; jj < (half ? P - H0 : H0); ++jj) {
            const int j1 = half * H0 + jj;
            const int k1 = wrapk(b1 - j1, d.K1);
#pragma unroll
            for (int j2 = 0; j2 < P; ++j2) {
                const int k2 = wrapk(b2 - j2, d.K2);
                const float *row = d.phi + ((size_t)k1 * d.K2 + k2) * d.K3;
                float s = 0.f, ds = 0.f;
#pragma unroll
                for (int j3 = 0; j3 < P; ++j3) {
                    const float ph = ldcg(row + wrapk(b3 - j3, d.K3));
                    s = fmaf(th3[j3], ph, s);
                    ds = fmaf(dth3[j3], ph, ds);
                }
                g1 = fmaf(dth1[j1] * th2[j2], s, g1);
                g2 = fmaf(th1[j1] * dth2[j2], s, g2);
                g3 = fmaf(th1[j1] * th2[j2], ds, g3);
            }
        }
        gh[half][0] = g1;
        gh[half][1] = g2;
        gh[half][2] = g3;
    }
    force_from_grad<P>(d, ra.w, rb.y, gh[0][0] + gh[1][0], gh[0][1] + gh[1][1], gh[0][2] + gh[1][2]);
}

// org: the tile's origin (tile_origin), when the caller computed it already.
template <int P, int T>
PME_DEV void stage_gather(const SysDev &d, int item, void *smem, const int *org = nullptr) {
    const int tid = PME_TID, nth = PME_NTH;
    if (item >= d.ntiles) {
        if (item == d.ntiles) reduce_level2(d, smem);  // every inverse-slab item has finished
        const unsigned novf = imin((int)ldcg(&d.ctl->novf_gather), d.n);
        for (unsigned a = (unsigned)((item - d.ntiles) * nth + tid); a < novf; a += (unsigned)(OVF_ITEMS * nth))
            gather_atom_global<P>(d, ldcg(d.ova + a), ldcg(d.ovb + a));
    } else {
        constexpr int R = Region<P, T>::R, H = P - 1;
        float *reg = (float *)smem;
        int o1, o2, o3;
        if (org) {
            o1 = org[0];
            o2 = org[1];
            o3 = org[2];
        } else {
            tile_origin(d, item, o1, o2, o3);
        }
        const float4 *A = d.bka + (size_t)item * d.cap;
        const int2 *B = d.bkb + (size_t)item * d.cap;
        // the count and this thread's first two records in flight with the region loads (the record slots
        // are always inside the bucket; each is used only if it holds an atom)
        const int cnt = imin((int)ldcg(&d.bcount[(size_t)item * BCOUNT_STRIDE]), d.cap);
        const int a0 = imin(tid >> 1, d.cap - 1), a1 = imin((tid + nth) >> 1, d.cap - 1);
        const float4 ra0 = ldcg(A + a0), ra1 = ldcg(A + a1);
        const int2 rb0 = ldcg(B + a0), rb1 = ldcg(B + a1);
        const int R1 = tile_width1(d, o1) + H;  // planes of the region the tile's atoms reach
        if (nth >= R) {
            // thread t < ng R loads point i3 = t mod R of rows t / R, t / R + ng, ... (ng = nth / R row
            // groups): the k3 index is computed once, each row costs two wraps
            const int ng = nth / R, rg = tid / R, i3 = tid - rg * R;
            if (rg < ng) {
                const int k3 = wrapk(o3 - H + i3, d.K3);
                for (int r0 = rg; r0 < R1 * R; r0 += LOAD_BATCH * ng) {
                    float v[LOAD_BATCH];
#pragma unroll
                    for (int u = 0; u < LOAD_BATCH; ++u) {
                        const int r = r0 + u * ng;
                        if (r < R1 * R) {
                            const int i1 = r / R, i2 = r - i1 * R;
                            const int k1 = wrapk(o1 - H + i1, d.K1), k2 = wrapk(o2 - H + i2, d.K2);
                            v[u] = ldcg(d.phi + ((size_t)k1 * d.K2 + k2) * d.K3 + k3);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < LOAD_BATCH; ++u)
                        if (r0 + u * ng < R1 * R) reg[(r0 + u * ng) * R + i3] = v[u];
                }
            }
        } else {
            for (int i = tid; i < R1 * R * R; i += nth) {
                const int i3 = i % R, i2 = (i / R) % R, i1 = i / (R * R);
                const int k1 = wrapk(o1 - H + i1, d.K1), k2 = wrapk(o2 - H + i2, d.K2), k3 = wrapk(o3 - H + i3, d.K3);
                reg[i] = ldcg(d.phi + ((size_t)k1 * d.K2 + k2) * d.K3 + k3);
            }
        }
        PME_SYNC();
        if (tid == 0) d.bcount[(size_t)item * BCOUNT_STRIDE] = 0u;  // consumed: ready for the next binning
#if defined(PME_HOST_EMULATION)
        float e1 = 0.f, e2 = 0.f, e3 = 0.f;  // the even half's partial sums, combined on the odd half
#endif
        // two threads per atom (adjacent lanes): half 0 sums the planes j1 in [0, H0), half 1 [H0, P); the
        // halves are added in a fixed order, so both lanes hold the same total
        constexpr int H0 = half_planes(P);
        for (int a2 = tid; a2 < 2 * cnt; a2 += nth) {
            const int a = a2 >> 1, half = a2 & 1;
            const bool first = a2 == tid, second = a2 == tid + nth;
            const float4 ra = first ? ra0 : (second ? ra1 : ldcg(A + a));
            const int2 rb = first ? rb0 : (second ? rb1 : ldcg(B + a));
            float th1[P], th2[P], th3[P], dth1[P], dth2[P], dth3[P];
            bspline_wd<P>(ra.x, th1, dth1);
            bspline_wd<P>(ra.y, th2, dth2);
            bspline_wd<P>(ra.z, th3, dth3);
            const int l1 = (rb.x & 1023) - o1 + H;
            const int l2 = ((rb.x >> 10) & 1023) - o2 + H;
            const int l3 = ((rb.x >> 20) & 1023) - o3 + H;
            float g1 = 0.f, g2 = 0.f, g3 = 0.f;
#pragma unroll
            for (int jj = 0; jj < H0; ++jj) {
                if (half && jj >= P - H0) break;  // odd P: half 1 has one plane fewer
                const int j1 = half * H0 + jj;
                const int jh = H0 + jj < P ? H0 + jj : P - 1;
                const float t1 = half ? th1[jh] : th1[jj];
                const float dt1 = half ? dth1[jh] : dth1[jj];
#pragma unroll
                for (int j2 = 0; j2 < P; ++j2) {
                    const float *row = reg + ((l1 - j1) * R + (l2 - j2)) * R + l3;
                    float s = 0.f, ds = 0.f;
#pragma unroll
                    for (int j3 = 0; j3 < P; ++j3) {
                        const float ph = row[-j3];
                        s = fmaf(th3[j3], ph, s);
                        ds = fmaf(dth3[j3], ph, ds);
                    }
                    g1 = fmaf(dt1 * th2[j2], s, g1);
                    g2 = fmaf(t1 * dth2[j2], s, g2);
                    g3 = fmaf(t1 * th2[j2], ds, g3);
                }
            }
#if defined(PME_HOST_EMULATION)
            if (!half) {
                e1 = g1;
                e2 = g2;
                e3 = g3;
                continue;
            }
            g1 = e1 + g1;
            g2 = e2 + g2;
            g3 = e3 + g3;
            force_from_grad<P>(d, ra.w, rb.y, g1, g2, g3);
#else
            const unsigned mask = __activemask();  // both lanes of every pair are active together
            const float o1f = __shfl_xor_sync(mask, g1, 1), o2f = __shfl_xor_sync(mask, g2, 1),
                        o3f = __shfl_xor_sync(mask, g3, 1);
            if (!half) force_from_grad<P>(d, ra.w, rb.y, g1 + o1f, g2 + o2f, g3 + o3f);
#endif
        }
    }
}

}  // namespace pme
