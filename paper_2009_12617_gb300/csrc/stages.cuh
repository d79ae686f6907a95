// Stage bodies of the reciprocal-space SPME pipeline (paper Sec. III-A, Fig. "LRPipe"): binning with
// B-spline set-up, charge spreading, forward 3D FFT, influence-function multiply with energy / virial,
// inverse 3D FFT, and force interpolation. Each body handles one work item of one system and is called
// both from the per-stage kernels and from the persistent batched kernel.
//
// Work items per system:
//   bin     nbin items        atoms [item*BIN_CHUNK, ...): fractional coordinates, tile key, bucket insert
//   spread  ntiles+OVF_ITEMS  one tile each, then bucket-overflow atoms
//   fwd     K1 items          slab k1: int64 -> float, real FFT along k3, complex FFT along k2
//   conv    K2 items          pencils m2: FFT along k1, times B*C, energy / virial, inverse FFT along k1
//   inv     K1 items          slab k1: inverse FFT along k2, complex-to-real FFT along k3 -> phi
//   gather  ntiles+OVF_ITEMS  one tile each (forces), then bucket-overflow atoms
#pragma once

#include "common.cuh"
#include "fft.cuh"

namespace pme {

// ---------------------------------------------------------------------------------------------------------
// shared-memory sizes (bytes) of each stage for a given system and block size

inline size_t smem_bin(int nth) { return (size_t)nth * sizeof(unsigned long long); }
inline size_t smem_tile_region(int p) { return (size_t)(TILE + p - 1) * (TILE + p - 1) * (TILE + p - 1); }
inline size_t smem_spread(int p) { return smem_tile_region(p) * sizeof(unsigned long long); }
inline size_t smem_gather(int p) { return smem_tile_region(p) * sizeof(float); }
inline size_t smem_slab(int K2, int K3) {
    const int H3 = K3 / 2 + 1;
    return (2 * (size_t)K2 * H3 + (K3 / 2) + (K3 / 2 + 1) + K2) * sizeof(float2);
}
inline size_t smem_conv(int K1, int K3, int nth) {
    const int H3 = K3 / 2 + 1;
    size_t fft = (2 * (size_t)K1 * H3 + K1) * sizeof(float2);
    size_t red = (size_t)nth * 7 * sizeof(DF);
    return fft > red ? fft : red;
}

// ---------------------------------------------------------------------------------------------------------
// a1: bin atoms by spread tile (replaces the paper's hardware atom reordering, Sec. III-A / V-C; with
// order-independent fixed-point accumulation the order inside a tile no longer matters)

PME_DEV void stage_bin(const SysDev &d, int item, void *smem) {
    unsigned long long *red = (unsigned long long *)smem;
    const int tid = PME_TID, nth = PME_NTH;
    const int i0 = item * BIN_CHUNK;
    const int i1 = imin(d.n, i0 + BIN_CHUNK);
    unsigned long long qacc = 0;
    unsigned bad = 0;
    for (int i = i0 + tid; i < i1; i += nth) {
        const float r[3] = {d.pos[3 * (size_t)i], d.pos[3 * (size_t)i + 1], d.pos[3 * (size_t)i + 2]};
        const float q = d.q[i];
        int b[3];
        float w[3];
        bool ok = isfinite(q) && fabsf(q) < 4194304.0f;  // |q| < 2^22 e
        if (ok) ok = scaled_coord(d, r, 0, d.K1, b[0], w[0]) && scaled_coord(d, r, 1, d.K2, b[1], w[1]) &&
                     scaled_coord(d, r, 2, d.K3, b[2], w[2]);
        if (!ok) {
            bad |= ST_NONFINITE;
            const float nan = qnan_f();
            d.forces[3 * (size_t)i] = nan;
            d.forces[3 * (size_t)i + 1] = nan;
            d.forces[3 * (size_t)i + 2] = nan;
            continue;
        }
        qacc += (unsigned long long)f2ll_rn(fabsf(q) * QABS_SCALE);
        const int tile = ((b[0] / TILE) * d.nt2 + (b[1] / TILE)) * d.nt3 + (b[2] / TILE);
        const float4 ra = make_float4(w[0], w[1], w[2], q);
        const int2 rb = make_int2(b[0] | (b[1] << 10) | (b[2] << 20), i);
        const unsigned rank = atomic_add_u32(&d.bcount[tile], 1u);
        if (rank < (unsigned)d.cap) {
            d.bka[(size_t)tile * d.cap + rank] = ra;
            d.bkb[(size_t)tile * d.cap + rank] = rb;
        } else {
            const unsigned j = atomic_add_u32(&d.ctl->novf, 1u);
            if (j < (unsigned)d.n) {
                d.ova[j] = ra;
                d.ovb[j] = rb;
            } else {
                bad |= ST_INTERNAL;
            }
        }
    }
    if (bad) atomic_or_u32(&d.ctl->status, bad);
    // CTA sum of |q| (fixed point, so the total is exact and order-independent)
    red[tid] = qacc;
    PME_SYNC();
    for (int s = nth / 2; s > 0; s >>= 1) {
        if (tid < s) red[tid] += red[tid + s];
        PME_SYNC();
    }
    if (tid == 0 && red[0]) {
        if (red[0] >= QABS_LIMIT) atomic_or_u32(&d.ctl->status, ST_OVERFLOW);
        else atomic_add_u64(&d.ctl->qabs, red[0]);
    }
}

// ---------------------------------------------------------------------------------------------------------
// a2: charge spreading Q(k) = sum_i q_i theta1 theta2 theta3 (paper Sec. III-A "Charge Spreading": each
// charge goes to the p^3 mesh points around it). A tile accumulates its atoms into a shared-memory region
// (TILE + p - 1)^3 with 64-bit fixed-point atomics, then adds the region (including the p - 1 halo that
// overlaps neighbouring tiles, the analogue of the paper's atoms processed by every pipeline they touch)
// into the global mesh with 64-bit integer reductions.

struct TileGeom {
    int o1, o2, o3;   // tile origin
    int R1, R2, R3;   // region extents (tile extent + p - 1)
};

PME_DEV TileGeom tile_geom(const SysDev &d, int tile) {
    TileGeom g;
    const int t3 = tile % d.nt3, t2 = (tile / d.nt3) % d.nt2, t1 = tile / (d.nt3 * d.nt2);
    g.o1 = t1 * TILE;
    g.o2 = t2 * TILE;
    g.o3 = t3 * TILE;
    g.R1 = imin(TILE, d.K1 - g.o1) + d.p - 1;
    g.R2 = imin(TILE, d.K2 - g.o2) + d.p - 1;
    g.R3 = imin(TILE, d.K3 - g.o3) + d.p - 1;
    return g;
}

PME_DEV int wrapk(int k, int K) { return k < 0 ? k + K : (k >= K ? k - K : k); }

template <int P>
PME_DEV void spread_atom_global(const SysDev &d, float4 ra, int2 rb) {
    float th1[P], th2[P], th3[P];
    bspline_w<P>(ra.x, th1);
    bspline_w<P>(ra.y, th2);
    bspline_w<P>(ra.z, th3);
    const int b1 = rb.x & 1023, b2 = (rb.x >> 10) & 1023, b3 = (rb.x >> 20) & 1023;
    for (int j1 = 0; j1 < P; ++j1) {
        const int k1 = wrapk(b1 - j1, d.K1);
        for (int j2 = 0; j2 < P; ++j2) {
            const int k2 = wrapk(b2 - j2, d.K2);
            const float c = ra.w * th1[j1] * th2[j2];
            unsigned long long *row = d.grid + ((size_t)k1 * d.K2 + k2) * d.K3;
#pragma unroll
            for (int j3 = 0; j3 < P; ++j3)
                red_add_u64(row + wrapk(b3 - j3, d.K3), (unsigned long long)f2ll_rn(c * th3[j3] * FIX_SCALE));
        }
    }
}

template <int P>
PME_DEV void stage_spread(const SysDev &d, int item, void *smem) {
    const int tid = PME_TID, nth = PME_NTH;
    if (item >= d.ntiles) {  // bucket-overflow atoms, straight to the global mesh
        const unsigned novf = imin((int)ldcg(&d.ctl->novf), d.n);
        for (unsigned a = (unsigned)((item - d.ntiles) * nth + tid); a < novf; a += (unsigned)(OVF_ITEMS * nth))
            spread_atom_global<P>(d, ldcg(d.ova + a), ldcg(d.ovb + a));
        return;
    }
    unsigned long long *reg = (unsigned long long *)smem;
    const TileGeom g = tile_geom(d, item);
    const int vol = g.R1 * g.R2 * g.R3;
    for (int i = tid; i < vol; i += nth) reg[i] = 0ull;
    const int cnt = imin((int)ldcg(&d.bcount[item]), d.cap);
    PME_SYNC();
    const float4 *A = d.bka + (size_t)item * d.cap;
    const int2 *B = d.bkb + (size_t)item * d.cap;
    for (int a = tid; a < cnt; a += nth) {
        const float4 ra = ldcg(A + a);
        const int2 rb = ldcg(B + a);
        float th1[P], th2[P], th3[P];
        bspline_w<P>(ra.x, th1);
        bspline_w<P>(ra.y, th2);
        bspline_w<P>(ra.z, th3);
        // local index of the atom's highest support point; its points are l - j, j < P
        const int l1 = (rb.x & 1023) - g.o1 + P - 1;
        const int l2 = ((rb.x >> 10) & 1023) - g.o2 + P - 1;
        const int l3 = ((rb.x >> 20) & 1023) - g.o3 + P - 1;
#pragma unroll
        for (int j1 = 0; j1 < P; ++j1) {
#pragma unroll
            for (int j2 = 0; j2 < P; ++j2) {
                const float c = ra.w * th1[j1] * th2[j2];
                unsigned long long *row = reg + ((l1 - j1) * g.R2 + (l2 - j2)) * g.R3 + l3;
#pragma unroll
                for (int j3 = 0; j3 < P; ++j3)
                    atomic_add_u64(row - j3, (unsigned long long)f2ll_rn(c * th3[j3] * FIX_SCALE));
            }
        }
    }
    PME_SYNC();
    const int H = P - 1;
    for (int i = tid; i < vol; i += nth) {
        const unsigned long long v = reg[i];
        if (v == 0ull) continue;
        const int i3 = i % g.R3, i2 = (i / g.R3) % g.R2, i1 = i / (g.R3 * g.R2);
        const int k1 = wrapk(g.o1 - H + i1, d.K1), k2 = wrapk(g.o2 - H + i2, d.K2), k3 = wrapk(g.o3 - H + i3, d.K3);
        red_add_u64(d.grid + ((size_t)k1 * d.K2 + k2) * d.K3 + k3, v);
    }
}

// ---------------------------------------------------------------------------------------------------------
// a3: forward slab k1 — mesh int64 -> float, real-to-complex FFT along k3 (a length K3/2 complex FFT of
// even/odd pairs plus the split step), then the complex FFT along k2 for every m3 column. The slab of
// the int64 mesh is zeroed after it is read, ready for the next evaluation's spreading.

PME_DEV void stage_fwd(const SysDev &d, int k1, void *smem) {
    const int tid = PME_TID, nth = PME_NTH;
    const int K2 = d.K2, K3 = d.K3, H3 = d.H3, Nh = K3 / 2;
    float2 *A = (float2 *)smem;
    float2 *B = A + K2 * H3;
    float2 *twh = B + K2 * H3;   // Nh
    float2 *tw3 = twh + Nh;      // Nh + 1
    float2 *tw2 = tw3 + Nh + 1;  // K2
    ulonglong2 *g = (ulonglong2 *)(d.grid + (size_t)k1 * K2 * K3);
    for (int i = tid; i < K2 * Nh; i += nth) {  // row k2 pairs (2n, 2n+1) -> complex z[n]
        const ulonglong2 v = ldcg(g + i);
        A[i] = make_float2(fix_to_float((long long)v.x), fix_to_float((long long)v.y));
        g[i] = make_ulonglong2(0ull, 0ull);
    }
    for (int i = tid; i < Nh; i += nth) twh[i] = d.tw3h[i];
    for (int i = tid; i <= Nh; i += nth) tw3[i] = d.tw3[i];
    for (int i = tid; i < K2; i += nth) tw2[i] = d.tw2[i];
    PME_SYNC();
    float2 *Z = fft_batch<false>(A, B, Nh, K2, 1, Nh, twh);  // rows, stride Nh
    float2 *X = (Z == A) ? B : A;
    // split: X[m] = E[m] + W_K3^m O[m], E = (Z[m] + conj Z[Nh-m]) / 2, O = -i (Z[m] - conj Z[Nh-m]) / 2
    for (int i = tid; i < K2 * H3; i += nth) {
        const int k2 = i / H3, m = i - k2 * H3;
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
// a4: pencils m2 — FFT along k1, multiply by the influence function B*C (the paper's "Green's function"
// step between Z and Z^-1, Sec. III-A "FFT"), reduce energy and virial, inverse FFT along k1.
//
// Energy and virial over the half spectrum: each m3 in (0, K3/2) stands for itself and its conjugate
// partner (weight 2), m3 = 0 and K3/2 have weight 1. Per-thread sums are double-float (about 44 bits);
// per-item partials are FP64, and the last item reduces all partials in a fixed order.

// Virial weight W_ab = delta_ab - 2 (1 + pi^2 |m'|^2 / beta^2) m'_a m'_b / |m'|^2 for the signed
// frequency (mt1, mt2, mt3), m' = sum_alpha mt_alpha a*_alpha. Order xx yy zz xy xz yz.
PME_DEV void virial_weights(const SysDev &d, float mt1, float mt2, float mt3, float W[6]) {
    float mv[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) mv[j] = mt1 * d.rec[3 * j] + mt2 * d.rec[3 * j + 1] + mt3 * d.rec[3 * j + 2];
    const float m2n = mv[0] * mv[0] + mv[1] * mv[1] + mv[2] * mv[2];
    const float f = 2.0f * (1.0f / m2n + d.pi2b2);
    W[0] = 1.0f - f * mv[0] * mv[0];
    W[1] = 1.0f - f * mv[1] * mv[1];
    W[2] = 1.0f - f * mv[2] * mv[2];
    W[3] = -f * mv[0] * mv[1];
    W[4] = -f * mv[0] * mv[2];
    W[5] = -f * mv[1] * mv[2];
}

// signed frequency of index m on a K-point axis: m for m <= K/2, else m - K (K/2 maps to +K/2)
PME_DEV int signed_freq(int m, int K) { return 2 * m <= K ? m : m - K; }

PME_DEV void stage_conv(const SysDev &d, int m2, void *smem) {
    const int tid = PME_TID, nth = PME_NTH;
    const int K1 = d.K1, K2 = d.K2, K3 = d.K3, H3 = d.H3;
    float2 *A = (float2 *)smem;
    float2 *B = A + K1 * H3;
    float2 *tw1 = B + K1 * H3;
    for (int i = tid; i < K1 * H3; i += nth) {
        const int k1 = i / H3, m3 = i - k1 * H3;
        A[i] = ldcg(d.spec + ((size_t)k1 * K2 + m2) * H3 + m3);
    }
    for (int i = tid; i < K1; i += nth) tw1[i] = d.tw1[i];
    PME_SYNC();
    float2 *X = fft_batch<false>(A, B, K1, H3, H3, 1, tw1);
    DF acc[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) acc[c].hi = acc[c].lo = 0.f;
    const float2 *bc = d.bc + (size_t)m2 * K1 * H3;
    const int mt2 = signed_freq(m2, K2);
    for (int i = tid; i < K1 * H3; i += nth) {
        const int m1 = i / H3, m3 = i - m1 * H3;
        const float2 t = bc[i];  // B*C as hi + lo
        float2 x = X[i];
        if ((m1 | m2 | m3) != 0) {
            const bool self = (m3 == 0 || 2 * m3 == K3);  // conjugate partner is another point of this plane
            const float s2 = x.x * x.x + x.y * x.y;
            const float e = (self ? 0.5f : 1.0f) * fmaf(t.x, s2, t.y * s2);
            const int mt1 = signed_freq(m1, K1);
            float W[6];
            virial_weights(d, (float)mt1, (float)mt2, (float)m3, W);
            if (!self && (2 * m1 == K1 || 2 * m2 == K2)) {
                // the partner -m keeps +K/2 on a Nyquist axis, so its m' is not -m': average the two
                float Wp[6];
                virial_weights(d, (float)(2 * m1 == K1 ? mt1 : -mt1), (float)(2 * m2 == K2 ? mt2 : -mt2),
                               (float)(-m3), Wp);
#pragma unroll
                for (int c = 0; c < 6; ++c) W[c] = 0.5f * (W[c] + Wp[c]);
            }
            acc[0] = df_add(acc[0], e);
#pragma unroll
            for (int c = 0; c < 6; ++c) acc[1 + c] = df_add(acc[1 + c], e * W[c]);
            x.x *= t.x;
            x.y *= t.x;
        } else {
            x = make_float2(0.f, 0.f);
        }
        X[i] = x;
    }
    PME_SYNC();
    float2 *Y = fft_batch<true>(X, (X == A) ? B : A, K1, H3, H3, 1, tw1);
    for (int i = tid; i < K1 * H3; i += nth) {
        const int k1 = i / H3, m3 = i - k1 * H3;
        d.spec[((size_t)k1 * K2 + m2) * H3 + m3] = Y[i];
    }
    PME_SYNC();
    // CTA reduction of the 7 double-float sums (fixed tree order)
    DF *red = (DF *)smem;
#pragma unroll
    for (int c = 0; c < 7; ++c) red[c * nth + tid] = acc[c];
    PME_SYNC();
    for (int s = nth / 2; s > 0; s >>= 1) {
        if (tid < s) {
#pragma unroll
            for (int c = 0; c < 7; ++c) red[c * nth + tid] = df_add(red[c * nth + tid], red[c * nth + tid + s]);
        }
        PME_SYNC();
    }
    PME_SHARED unsigned last_flag;
    if (tid == 0) {
        for (int c = 0; c < 7; ++c) d.partials[(size_t)m2 * 8 + c] = (double)red[c * nth].hi + (double)red[c * nth].lo;
        PME_FENCE();
        const unsigned done = atomic_add_u32(&d.ctl->conv_done, 1u);
        last_flag = (done == (unsigned)K2 - 1u) ? 1u : 0u;
    }
    PME_SYNC();
    if (last_flag) {
        // last item: FP64 sum over the K2 partials in a fixed two-level order
        PME_FENCE();
        double *dred = (double *)smem;  // 7 x 8 partial sums
        for (int r = tid; r < 56; r += nth) {
            const int c = r >> 3, part = r & 7;
            double s = 0.0;
            for (int it = part; it < K2; it += 8) s += ldcg(d.partials + (size_t)it * 8 + c);
            dred[r] = s;
        }
        PME_SYNC();
        if (tid == 0) {
            for (int c = 0; c < 7; ++c) {
                double s = 0.0;
                for (int part = 0; part < 8; ++part) s += dred[c * 8 + part];
                d.ev[c] = s;
            }
            if (ldcg(&d.ctl->qabs) >= QABS_LIMIT) atomic_or_u32(&d.ctl->status, ST_OVERFLOW);
            d.ctl->qabs = 0ull;
            d.ctl->conv_done = 0u;
        }
    }
}

// ---------------------------------------------------------------------------------------------------------
// a5: inverse slab k1 — inverse FFT along k2 per m3 column, then the complex-to-real inverse along k3
// (merge step + a length K3/2 complex FFT whose real / imaginary parts are the even / odd samples).

PME_DEV void stage_inv(const SysDev &d, int k1, void *smem) {
    const int tid = PME_TID, nth = PME_NTH;
    const int K2 = d.K2, K3 = d.K3, H3 = d.H3, Nh = K3 / 2;
    float2 *A = (float2 *)smem;
    float2 *B = A + K2 * H3;
    float2 *twh = B + K2 * H3;
    float2 *tw3 = twh + Nh;
    float2 *tw2 = tw3 + Nh + 1;
    const float2 *in = d.spec + (size_t)k1 * K2 * H3;
    for (int i = tid; i < K2 * H3; i += nth) A[i] = ldcg(in + i);
    for (int i = tid; i < Nh; i += nth) twh[i] = d.tw3h[i];
    for (int i = tid; i <= Nh; i += nth) tw3[i] = d.tw3[i];
    for (int i = tid; i < K2; i += nth) tw2[i] = d.tw2[i];
    PME_SYNC();
    float2 *Y = fft_batch<true>(A, B, K2, H3, H3, 1, tw2);
    float2 *Z = (Y == A) ? B : A;
    // Z[m] = (X[m] + conj X[Nh-m]) + i (X[m] - conj X[Nh-m]) exp(+2 pi i m / K3), m < Nh
    for (int i = tid; i < K2 * Nh; i += nth) {
        const int k2 = i / Nh, m = i - k2 * Nh;
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

template <int P>
PME_DEV void gather_atom_global(const SysDev &d, float4 ra, int2 rb) {
    float th1[P], th2[P], th3[P], dth1[P], dth2[P], dth3[P];
    bspline_wd<P>(ra.x, th1, dth1);
    bspline_wd<P>(ra.y, th2, dth2);
    bspline_wd<P>(ra.z, th3, dth3);
    const int b1 = rb.x & 1023, b2 = (rb.x >> 10) & 1023, b3 = (rb.x >> 20) & 1023;
    float g1 = 0.f, g2 = 0.f, g3 = 0.f;
    for (int j1 = 0; j1 < P; ++j1) {
        const int k1 = wrapk(b1 - j1, d.K1);
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
    force_from_grad<P>(d, ra.w, rb.y, g1, g2, g3);
}

template <int P>
PME_DEV void stage_gather(const SysDev &d, int item, void *smem) {
    const int tid = PME_TID, nth = PME_NTH;
    if (item >= d.ntiles) {
        const unsigned novf = imin((int)ldcg(&d.ctl->novf), d.n);
        for (unsigned a = (unsigned)((item - d.ntiles) * nth + tid); a < novf; a += (unsigned)(OVF_ITEMS * nth))
            gather_atom_global<P>(d, ldcg(d.ova + a), ldcg(d.ovb + a));
    } else {
        float *reg = (float *)smem;
        const TileGeom g = tile_geom(d, item);
        const int vol = g.R1 * g.R2 * g.R3;
        const int H = P - 1;
        for (int i = tid; i < vol; i += nth) {
            const int i3 = i % g.R3, i2 = (i / g.R3) % g.R2, i1 = i / (g.R3 * g.R2);
            const int k1 = wrapk(g.o1 - H + i1, d.K1), k2 = wrapk(g.o2 - H + i2, d.K2), k3 = wrapk(g.o3 - H + i3, d.K3);
            reg[i] = ldcg(d.phi + ((size_t)k1 * d.K2 + k2) * d.K3 + k3);
        }
        const int cnt = imin((int)ldcg(&d.bcount[item]), d.cap);
        PME_SYNC();
        if (tid == 0) d.bcount[item] = 0u;  // consumed: ready for the next evaluation's binning
        const float4 *A = d.bka + (size_t)item * d.cap;
        const int2 *B = d.bkb + (size_t)item * d.cap;
        for (int a = tid; a < cnt; a += nth) {
            const float4 ra = ldcg(A + a);
            const int2 rb = ldcg(B + a);
            float th1[P], th2[P], th3[P], dth1[P], dth2[P], dth3[P];
            bspline_wd<P>(ra.x, th1, dth1);
            bspline_wd<P>(ra.y, th2, dth2);
            bspline_wd<P>(ra.z, th3, dth3);
            const int l1 = (rb.x & 1023) - g.o1 + H;
            const int l2 = ((rb.x >> 10) & 1023) - g.o2 + H;
            const int l3 = ((rb.x >> 20) & 1023) - g.o3 + H;
            float g1 = 0.f, g2 = 0.f, g3 = 0.f;
#pragma unroll
            for (int j1 = 0; j1 < P; ++j1) {
#pragma unroll
                for (int j2 = 0; j2 < P; ++j2) {
                    const float *row = reg + ((l1 - j1) * g.R2 + (l2 - j2)) * g.R3 + l3;
                    float s = 0.f, ds = 0.f;
#pragma unroll
                    for (int j3 = 0; j3 < P; ++j3) {
                        const float ph = row[-j3];
                        s = fmaf(th3[j3], ph, s);
                        ds = fmaf(dth3[j3], ph, ds);
                    }
                    g1 = fmaf(dth1[j1] * th2[j2], s, g1);
                    g2 = fmaf(th1[j1] * dth2[j2], s, g2);
                    g3 = fmaf(th1[j1] * th2[j2], ds, g3);
                }
            }
            force_from_grad<P>(d, ra.w, rb.y, g1, g2, g3);
        }
    }
    PME_SYNC();
    if (tid == 0) {
        PME_FENCE();
        const unsigned done = atomic_add_u32(&d.ctl->gather_done, 1u);
        if (done == (unsigned)(d.ntiles + OVF_ITEMS) - 1u) {  // every gather item has read novf
            d.ctl->novf = 0u;
            d.ctl->gather_done = 0u;
        }
    }
}

}  // namespace pme
