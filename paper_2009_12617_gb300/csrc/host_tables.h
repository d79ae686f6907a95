// Host-side set-up of a system: argument validation, cell geometry, FFT twiddles and the influence table.
// Plain C++ (no CUDA calls), shared by the library's plan code and the CPU emulation build.
#pragma once

#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include <vector>

#include "common.cuh"

namespace pme {

constexpr double PI_D = 3.14159265358979323846;

// 2, 3, 5-smooth
inline bool smooth235(int k) {
    if (k <= 0) return false;
    for (int f : {2, 3, 5})
        while (k % f == 0) k /= f;
    return k == 1;
}

// Returns 0 (ok), 1 (invalid) or 2 (valid SPME input this build does not implement); msg gets a reason.
inline int validate_params(const int K[3], int p, double beta, const double box[9], char *msg, size_t len) {
    for (int a = 0; a < 3; ++a) {
        if (K[a] < 8 || K[a] > MAX_K || (K[a] & 1) || !smooth235(K[a])) {
            snprintf(msg, len, "K[%d] = %d: each mesh edge must be even, in [8, %d] and 2,3,5-smooth", a, K[a], MAX_K);
            return 1;
        }
    }
    if (p < 2 || p > K[0] || p > K[1] || p > K[2]) {
        snprintf(msg, len, "p = %d must be in [2, min(K)]", p);
        return 1;
    }
    if (p != 4 && p != 5 && p != 6 && p != 8) {
        snprintf(msg, len, "p = %d: only B-spline orders 4, 5, 6, 8 are implemented", p);
        return 2;
    }
    if (!(beta > 0.0) || !isfinite(beta)) {
        snprintf(msg, len, "beta must be positive and finite");
        return 1;
    }
    for (int i = 0; i < 9; ++i)
        if (!isfinite(box[i])) {
            snprintf(msg, len, "box has a non-finite entry");
            return 1;
        }
    return 0;
}

// recip[3*alpha + j] = component j of a*_alpha (a*_alpha . a_beta = delta), vol = |det|. false if singular.
inline bool cell_reciprocal(const double box[9], double recip[9], double *vol) {
    const double *a = box, *b = box + 3, *c = box + 6;
    const double bxc[3] = {b[1] * c[2] - b[2] * c[1], b[2] * c[0] - b[0] * c[2], b[0] * c[1] - b[1] * c[0]};
    const double cxa[3] = {c[1] * a[2] - c[2] * a[1], c[2] * a[0] - c[0] * a[2], c[0] * a[1] - c[1] * a[0]};
    const double axb[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    const double det = a[0] * bxc[0] + a[1] * bxc[1] + a[2] * bxc[2];
    double scale = 0.0;
    for (int i = 0; i < 9; ++i) scale = fmax(scale, fabs(box[i]));
    if (!(fabs(det) > 1e-12 * scale * scale * scale)) return false;
    for (int j = 0; j < 3; ++j) {
        recip[j] = bxc[j] / det;
        recip[3 + j] = cxa[j] / det;
        recip[6 + j] = axb[j] / det;
    }
    *vol = fabs(det);
    return true;
}

// Tile edge 2^tlog: tiles per dimension and their count. Needs d.K1..K3. Along k2 and k3 the tiles are
// 2^tlog wide (the last one ragged); along k1 the mesh is cut into np1 >= ceil(K1 / 2^tlog) pieces, piece j
// starting at floor(j K1 / np1) (k1_piece / k1_start), so every piece is at most 2^tlog wide (np1 = 0: the
// fewest pieces, which for K1 a multiple of the edge are the plain 2^tlog slabs).
inline void set_tiling(SysDev &d, int tlog, int np1 = 0) {
    const int T = 1 << tlog;
    const int base = (d.K1 + T - 1) / T;
    d.tlog = tlog;
    d.nt1 = np1 > base ? np1 : base;
    d.rnt1 = 1.0f / (float)d.nt1;
    d.nt2 = (d.K2 + T - 1) / T;
    d.nt3 = (d.K3 + T - 1) / T;
    d.ntiles = d.nt1 * d.nt2 * d.nt3;
}

// Descriptor of a system that shares the GPU with others (batches, server waves of several systems): the
// fewest k1 pieces, since balancing one system's tiles over the SMs is moot there and thinner pieces only add
// halo. Uses the plan's buckets as they are (fewer tiles of at most the same capacity).
inline void shared_tiling(SysDev &d) { set_tiling(d, d.tlog, 0); }

// Pieces along k1 for one system on `sms` SMs. When a single system has more tiles than SMs, all of them
// are resident at once and the SMs holding one tile more than the others set the stage time (at 64^3:
// 512 tiles on 152 SMs, 64 SMs with four and 88 with three). Cutting k1 into a few more, thinner pieces can
// lower the busiest SM's work, ceil(tiles / SMs) x (atoms + halo share) per tile, at the price of a little
// more halo: 64^3 at p = 4 takes 9 pieces (576 tiles, at most four per SM, each 7/8 as heavy).
inline int choose_k1_pieces(const SysDev &d, int sms) {
    const int T = 1 << d.tlog;
    const int base = (d.K1 + T - 1) / T;
    const int64_t cols = (int64_t)((d.K2 + T - 1) / T) * ((d.K3 + T - 1) / T);
    if (sms <= 0 || base * cols < sms) return base;
    int best = base;
    double best_cost = 0.0;
    for (int np = base; np <= 2 * base; ++np) {
        const int64_t per_sm = (np * cols + sms - 1) / sms;
        const double cost = (double)per_sm * ((double)d.K1 / np + 0.5 * (d.p - 1));
        if (np == base || cost < best_cost - 1e-9) {
            best = np;
            best_cost = cost;
        }
    }
    return best;
}

// Tile edge for n atoms on a GPU with `sms` SMs. 16^3 tiles halve the halo each tile adds to the global
// mesh (a region of (16 + p - 1)^3 points per 4096 instead of (8 + p - 1)^3 per 512) and hold enough atoms
// per residue class for the dealt order to avoid shared-memory bank conflicts, but there are 8 times fewer
// of them. They pay when there are still at least two per SM and they hold about 256 atoms or more (128^3,
// 262144 atoms, p = 6: 144 vs 151 us per evaluation on GB300); otherwise 8^3 tiles (many light CTAs) are
// faster. Results do not depend on the edge.
inline int choose_tile_log(int64_t n, const int K[3], int sms) {
    const int64_t t16 = (int64_t)((K[0] + 15) / 16) * ((K[1] + 15) / 16) * ((K[2] + 15) / 16);
    if (sms > 0 && t16 >= 2 * (int64_t)sms && n >= 256 * t16) return TILE_MAX_LOG;
    return TILE_MIN_LOG;
}

// Transform paths: the register path (lane plans) wherever both transforms of a slab stage, or the K1
// transform of the influence stage, have a plan; the shared-memory Stockham path otherwise. The CPU
// emulation of the stage bodies (one thread per CTA) has no lanes and always takes the shared-memory path.
inline void choose_fft_paths(SysDev &d, bool lanes) {
    d.lp_rows = lanes ? slab_lane_plan(d.K3 / 2, d.K2) : -1;
    d.lp_cols = lanes ? slab_lane_plan(d.K2, d.H3) : -1;
    d.lp_k1 = lanes ? conv_lane_plan(d.K1) : -1;
    d.lane_slab = (d.lp_rows >= 0 && d.lp_cols >= 0) ? 1 : 0;
    d.lane_conv = d.lp_k1 >= 0 ? 1 : 0;
    d.nchunk3 = (d.H3 + CONV_COLS - 1) / CONV_COLS;
    if (d.lane_conv) {
        const int cols = CONV_UNITS / plan_L(d.lp_k1);  // columns per work item
        d.nconv = (d.K2 * d.H3 + cols - 1) / cols;
    } else {
        d.nconv = d.K2 * d.nchunk3;
    }
}

#if defined(PME_HOST_EMULATION)
constexpr bool LANE_FFT_DEFAULT = false;
#else
constexpr bool LANE_FFT_DEFAULT = true;
#endif

// Mesh geometry, coordinate transform and tiling of a system.
inline void fill_geometry(SysDev &d, const int K[3], int p, double beta, const double recip[9]) {
    d.K1 = K[0];
    d.K2 = K[1];
    d.K3 = K[2];
    d.H3 = K[2] / 2 + 1;
    d.p = p;
    d.item0 = 0;
    d.k1_lo = 0;
    d.k1_hi = K[0];
    d.ev_status = 0;
    set_tiling(d, TILE_MIN_LOG);
    choose_fft_paths(d, LANE_FFT_DEFAULT);
    for (int a = 0; a < 3; ++a) d.kinv[a] = 1.0f / (float)K[a];
    for (int j = 0; j < 3; ++j)
        for (int al = 0; al < 3; ++al) {
            const double c = (double)K[al] * recip[3 * al + j];  // K_alpha a*_alpha[j]
            const float hi = (float)c;
            d.chi[3 * j + al] = hi;
            d.clo[3 * j + al] = (float)(c - (double)hi);
            d.rec[3 * j + al] = (float)recip[3 * al + j];
        }
    d.pi2b2 = (float)(PI_D * PI_D / (beta * beta));
}

// out[k] = exp(-2 pi i k / L), k < count
inline void make_twiddles(int L, int count, float2 *out) {
    for (int k = 0; k < count; ++k) {
        const double a = -2.0 * PI_D * (double)k / (double)L;
        out[k].x = (float)cos(a);
        out[k].y = (float)sin(a);
    }
}

// M_p at the integer knots 0..p by the recursion M_n(x) = [x M_{n-1}(x) + (n - x) M_{n-1}(x - 1)] / (n - 1).
inline std::vector<double> bspline_knots(int p) {
    std::vector<double> M(p + 1, 0.0), prev(p + 1, 0.0);
    prev[1] = 1.0;  // M_2(1) = 1
    for (int n = 3; n <= p; ++n) {
        for (int x = 0; x <= p; ++x) M[x] = ((double)x * prev[x] + (double)(n - x) * (x >= 1 ? prev[x - 1] : 0.0)) / (n - 1);
        prev = M;
    }
    return prev;
}

// |b(m)|^2 = 1 / |sum_{k=0}^{p-2} M_p(k+1) exp(2 pi i m k / K)|^2 (the Euler exponential-spline factor).
// For odd p the denominator vanishes at m = K/2 (symmetric knot values, alternating sum); there it is taken
// as the mean of the denominators at K/2 - 1 and K/2 + 1.
inline std::vector<double> bspline_moduli(int K, int p) {
    const std::vector<double> M = bspline_knots(p);
    std::vector<double> den(K), b(K);
    for (int m = 0; m < K; ++m) {
        double sr = 0.0, si = 0.0;
        for (int k = 0; k <= p - 2; ++k) {
            const double a = 2.0 * PI_D * (double)((int64_t)m * k % K) / (double)K;
            sr += M[k + 1] * cos(a);
            si += M[k + 1] * sin(a);
        }
        den[m] = sr * sr + si * si;
    }
    if ((p & 1) && (K & 1) == 0 && K >= 4) den[K / 2] = 0.5 * (den[K / 2 - 1] + den[K / 2 + 1]);
    for (int m = 0; m < K; ++m) b[m] = 1.0 / den[m];
    return b;
}

inline int signed_freq_h(int m, int K) { return 2 * m <= K ? m : m - K; }

// Influence table on the half spectrum, [m2][m1][m3] with m3 <= K3/2 (layout of SysDev::bc): the even part
// B(m) (C(m) + C(-m)) / 2 of B*C as (hi, lo) floats of its FP64 value (the two halves differ only on Nyquist
// axes of non-orthogonal cells, because index K/2 always means frequency +K/2; C(0) = 0), and the virial factors B C f(m), B C f(m_p) in FP64 rounded
// once, f = 2 (1 / |m'|^2 + pi^2 / beta^2). m_p (the point's conjugate partner, whose frequencies keep +K/2 on
// a Nyquist axis) gets its own factor only where it differs from -m: off the self-conjugate planes m3 = 0,
// K3/2 and on a Nyquist plane m1 = K1/2 or m2 = K2/2; elsewhere w = 0.
inline void make_influence(const int K[3], int p, double beta, const double recip[9], double vol, float4 *out) {
    const std::vector<double> b1 = bspline_moduli(K[0], p), b2 = bspline_moduli(K[1], p), b3 = bspline_moduli(K[2], p);
    const int H3 = K[2] / 2 + 1;
    const double fac = PI_D * PI_D / (beta * beta);
    auto norm2 = [&](int mt1, int mt2, int mt3) {
        double mv[3];
        for (int j = 0; j < 3; ++j) mv[j] = mt1 * recip[j] + mt2 * recip[3 + j] + mt3 * recip[6 + j];
        return mv[0] * mv[0] + mv[1] * mv[1] + mv[2] * mv[2];
    };
    auto C = [&](double m2n) { return exp(-fac * m2n) / (PI_D * vol * m2n); };
    auto f = [&](double m2n) { return 2.0 * (1.0 / m2n + fac); };
    for (int m2 = 0; m2 < K[1]; ++m2)
        for (int m1 = 0; m1 < K[0]; ++m1)
            for (int m3 = 0; m3 < H3; ++m3) {
                double v = 0.0, g = 0.0, gp = 0.0;
                if (m1 | m2 | m3) {
                    const int mt1 = signed_freq_h(m1, K[0]), mt2 = signed_freq_h(m2, K[1]), mt3 = signed_freq_h(m3, K[2]);
                    const double nm = norm2(mt1, mt2, mt3);
                    const double np = norm2(signed_freq_h((K[0] - m1) % K[0], K[0]), signed_freq_h((K[1] - m2) % K[1], K[1]),
                                            signed_freq_h((K[2] - m3) % K[2], K[2]));
                    v = b1[m1] * b2[m2] * b3[m3] * 0.5 * (C(nm) + C(np));
                    g = v * f(nm);
                    const bool self = m3 == 0 || 2 * m3 == K[2];
                    if (!self && (2 * m1 == K[0] || 2 * m2 == K[1])) {
                        const double npart = norm2(2 * m1 == K[0] ? mt1 : -mt1, 2 * m2 == K[1] ? mt2 : -mt2, -mt3);
                        gp = v * f(npart);
                    }
                }
                float4 &o = out[((size_t)m2 * K[0] + m1) * H3 + m3];
                o.x = (float)v;
                o.y = (float)(v - (double)o.x);
                o.z = (float)g;
                o.w = (float)gp;
            }
}

// Slab decomposition of one system over P ranks (the paper's distributed FFT, Sec. III-A "FFT", III-C):
// rank r owns the mesh planes [plane0[r], plane0[r+1]) along k1 for spreading and the slab transforms, and
// the influence-stage work items [item0[r], item0[r+1]), which cover the half-spectrum columns (m2, m3)
// flattened as c = m2 H3 + m3 in [col0[r], col0[r+1]). The two corner turns move, between every pair
// (r, s), the block of r's planes x s's columns: at most maxS x maxW complex values.
constexpr int SLAB_MAX_RANKS = 64;
struct SlabLayout {
    int P;
    int plane0[SLAB_MAX_RANKS + 1], item0[SLAB_MAX_RANKS + 1], col0[SLAB_MAX_RANKS + 1];
    int maxS, maxW;
};

// First half-spectrum column of influence-stage item i (items cover consecutive columns).
inline int conv_item_col(const SysDev &d, int i) {
    const int ncol = d.K2 * d.H3;
    if (i >= d.nconv) return ncol;
    int c;
    if (d.lane_conv) {
        c = i * (CONV_UNITS / plan_L(d.lp_k1));
    } else {
        const int m2 = i / d.nchunk3, ch = i - m2 * d.nchunk3;
        c = m2 * d.H3 + ch * CONV_COLS;
    }
    return c < ncol ? c : ncol;
}

// Even split of the planes and of the influence items; false when a rank would own no plane or no item.
inline bool make_slab_layout(const SysDev &d, int P, SlabLayout &L) {
    if (P < 1 || P > SLAB_MAX_RANKS || P > d.K1 || P > d.nconv) return false;
    L.P = P;
    L.maxS = L.maxW = 0;
    for (int r = 0; r <= P; ++r) {
        L.plane0[r] = (int)((int64_t)r * d.K1 / P);
        L.item0[r] = (int)((int64_t)r * d.nconv / P);
        L.col0[r] = conv_item_col(d, L.item0[r]);
    }
    for (int r = 0; r < P; ++r) {
        const int S = L.plane0[r + 1] - L.plane0[r], W = L.col0[r + 1] - L.col0[r];
        if (S < 1 || W < 1) return false;
        L.maxS = S > L.maxS ? S : L.maxS;
        L.maxW = W > L.maxW ? W : L.maxW;
    }
    return true;
}

// Bucket capacity per tile for n atoms in tiles of edge 2^tlog: twice the mean occupancy plus a margin, a
// multiple of 32, at most cap_max_for(tlog). Atoms beyond it go to the overflow list (handled by
// global-memory paths), so this only tunes speed.
inline int bucket_capacity(int64_t n, int ntiles, int tlog) {
    const int cmax = cap_max_for(tlog);
    const double mean = (double)n / (double)ntiles;
    const double want = 2.0 * mean + 32.0;
    int cap = want > (double)cmax ? cmax : (int)want;
    cap = (cap + 31) / 32 * 32;
    return cap < 32 ? 32 : (cap > cmax ? cmax : cap);
}

// Bytes of the padded tile-counter array and of the influence-stage partials.
inline size_t bcount_bytes(int ntiles) { return (size_t)ntiles * BCOUNT_STRIDE * sizeof(unsigned); }
// counters for the finest tiling (the most tiles any choice can need: 8-point tiles, twice the k1 pieces)
inline size_t bcount_bytes_max(const int K[3]) {
    return bcount_bytes(2 * ((K[0] + 7) / 8) * ((K[1] + 7) / 8) * ((K[2] + 7) / 8));
}
inline size_t partials_bytes(const SysDev &d) { return ((size_t)d.nconv + d.K1) * 8 * sizeof(float2); }

}  // namespace pme
