/*
 * FP64 CPU oracle for the reciprocal-space Smooth Particle Mesh Ewald (SPME) evaluation.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * legs may load this library. It shares no code, header, table or constant with the CUDA path.
 *
 * What it computes. The paper (Sec. II; Sec. III-A "Charge Spreading", "FFT", "Force Interpolation") uses
 * SPME [Essmann et al. 1995] but describes it only in words: order-p cardinal B-splines spread each
 * charge onto a p x p x p neighbourhood of mesh points (4x4x4 in the paper), a forward 3D FFT, a multiply
 * by the "Green's function", an inverse 3D FFT, and forces from B-spline derivatives times the potential
 * mesh. The equations below are the standard SPME definitions of those steps, written out plainly:
 *
 *   (1) a*_alpha . a_beta = delta_alpha,beta ; V = |det box| ; s_i,alpha = frac(a*_alpha . r_i) ;
 *       u_i,alpha = K_alpha s_i,alpha.
 *   (2) M_2(x) = 1 - |x - 1| on [0,2], else 0 ;  M_p(x) = [x M_{p-1}(x) + (p - x) M_{p-1}(x - 1)] / (p - 1) ;
 *       M_p'(x) = M_{p-1}(x) - M_{p-1}(x - 1).
 *   (3) Q(k) = sum_i q_i prod_alpha sum_{n in Z} M_p(u_i,alpha - k_alpha - n K_alpha).
 *   (4) Qhat(m) = sum_k Q(k) exp(+2 pi i sum_alpha m_alpha k_alpha / K_alpha)   (direct, unnormalised).
 *   (5) |b_alpha(m)|^2 = 1 / |sum_{k=0}^{p-2} M_p(k+1) exp(2 pi i m k / K_alpha)|^2 ; B(m) = prod |b_alpha|^2
 *       (odd p: at m = K/2, where the sum vanishes, the mean of the neighbouring denominators).
 *   (6) m' = sum_alpha mt_alpha a*_alpha with mt = m for m <= K/2 else m - K ;
 *       C(m) = exp(-pi^2 |m'|^2 / beta^2) / (pi V |m'|^2), C(0) = 0.
 *   (7) E = 1/2 sum_m B C |Qhat|^2.
 *   (8) Pi_ab = 1/2 sum_m B C |Qhat|^2 (delta_ab - 2 (1 + pi^2 |m'|^2 / beta^2) m'_a m'_b / |m'|^2).
 *   (9) phi(k) = sum_m B(m) C(m) Qhat(m) exp(-2 pi i m.k/K)  (unnormalised inverse; real).
 *  (10) F_i = -q_i sum_k sum_alpha K_alpha a*_alpha M_p'(u_i,alpha - k_alpha) prod_{beta != alpha} M_p(...) phi(k).
 *  (11) Ewald comparison terms: brute-force reciprocal k-sum, real-space erfc image sum, self term.
 *
 * Units: e, Angstrom, Coulomb constant 1 (energy in e^2/A). Box = rows a, b, c (box[3*alpha + j]).
 * Mesh arrays are row-major [k1][k2][k3] with k3 fastest.
 *
 * Every routine is a plain loop over the definition: no blocking, fusion or fast transform.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* Threads. Where a loop runs in parallel (built with OpenMP), each output element is computed by exactly
 * one thread with the same operations in the same order as the serial loop, so results do not depend on
 * the thread count; sums over many atoms or mesh points that feed one output stay serial. */
void oracle_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}
int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------------------------------------ */
/* (1) cell geometry                                                                                       */

/* Reciprocal vectors: recip[3*alpha + j] = component j of a*_alpha, with a*_alpha . a_beta = delta.
 * Returns 0, or -1 for a singular box. *vol = |det box|. */
int oracle_recip(const double box[9], double recip[9], double *vol) {
    const double *a = box, *b = box + 3, *c = box + 6;
    double det = a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
                 a[2] * (b[0] * c[1] - b[1] * c[0]);
    if (det == 0.0 || !isfinite(det)) return -1;
    /* a* = (b x c)/det, b* = (c x a)/det, c* = (a x b)/det */
    recip[0] = (b[1] * c[2] - b[2] * c[1]) / det;
    recip[1] = (b[2] * c[0] - b[0] * c[2]) / det;
    recip[2] = (b[0] * c[1] - b[1] * c[0]) / det;
    recip[3] = (c[1] * a[2] - c[2] * a[1]) / det;
    recip[4] = (c[2] * a[0] - c[0] * a[2]) / det;
    recip[5] = (c[0] * a[1] - c[1] * a[0]) / det;
    recip[6] = (a[1] * b[2] - a[2] * b[1]) / det;
    recip[7] = (a[2] * b[0] - a[0] * b[2]) / det;
    recip[8] = (a[0] * b[1] - a[1] * b[0]) / det;
    *vol = fabs(det);
    return 0;
}

/* u_alpha = K_alpha * frac(a*_alpha . r), for one position. */
static void scaled_coords(const double r[3], const int K[3], const double recip[9], double u[3]) {
    for (int al = 0; al < 3; ++al) {
        double s = recip[3 * al + 0] * r[0] + recip[3 * al + 1] * r[1] + recip[3 * al + 2] * r[2];
        s -= floor(s);
        u[al] = K[al] * s;
    }
}

void oracle_scaled_coords(int64_t n, const double *pos, const int K[3], const double box[9], double *u) {
    double recip[9], vol;
    oracle_recip(box, recip, &vol);
    for (int64_t i = 0; i < n; ++i) scaled_coords(pos + 3 * i, K, recip, u + 3 * i);
}

/* ------------------------------------------------------------------------------------------------------ */
/* (2) cardinal B-splines by the recursion                                                                 */

double oracle_bspline(int p, double x) {
    if (p < 2) return 0.0;
    if (p == 2) return (x >= 0.0 && x <= 2.0) ? 1.0 - fabs(x - 1.0) : 0.0;
    if (x <= 0.0 || x >= (double)p) return 0.0;
    return (x * oracle_bspline(p - 1, x) + ((double)p - x) * oracle_bspline(p - 1, x - 1.0)) / (double)(p - 1);
}

double oracle_bspline_deriv(int p, double x) {
    return oracle_bspline(p - 1, x) - oracle_bspline(p - 1, x - 1.0);
}

static int64_t pmod(int64_t a, int64_t m) {
    int64_t r = a % m;
    return r < 0 ? r + m : r;
}

/* ------------------------------------------------------------------------------------------------------ */
/* (3) charge spreading                                                                                    */

/* Q (K1*K2*K3 doubles) = eq. (3). For each atom and dimension, every integer t with 0 < u - t < p is a
 * support point (M_p vanishes elsewhere); the mesh index is t mod K, which sums the periodic images. */
void oracle_spread(int64_t n, const double *pos, const double *q, const int K[3], int p, const double box[9],
                   double *Q) {
    double recip[9], vol;
    oracle_recip(box, recip, &vol);
    const int64_t K1 = K[0], K2 = K[1], K3 = K[2];
    memset(Q, 0, sizeof(double) * K1 * K2 * K3);
    double *w[3];
    int64_t *idx[3];
    for (int al = 0; al < 3; ++al) {
        w[al] = (double *)malloc(sizeof(double) * (p + 1));
        idx[al] = (int64_t *)malloc(sizeof(int64_t) * (p + 1));
    }
    int cnt[3];
    for (int64_t i = 0; i < n; ++i) {
        double u[3];
        scaled_coords(pos + 3 * i, K, recip, u);
        for (int al = 0; al < 3; ++al) {
            cnt[al] = 0;
            for (int64_t t = (int64_t)floor(u[al]) - p; t <= (int64_t)floor(u[al]) + 1; ++t) {
                double x = u[al] - (double)t;
                if (x > 0.0 && x < (double)p) {
                    w[al][cnt[al]] = oracle_bspline(p, x);
                    idx[al][cnt[al]] = pmod(t, K[al]);
                    cnt[al]++;
                }
            }
        }
        for (int a = 0; a < cnt[0]; ++a)
            for (int b = 0; b < cnt[1]; ++b)
                for (int c = 0; c < cnt[2]; ++c)
                    Q[(idx[0][a] * K2 + idx[1][b]) * K3 + idx[2][c]] += q[i] * w[0][a] * w[1][b] * w[2][c];
    }
    for (int al = 0; al < 3; ++al) {
        free(w[al]);
        free(idx[al]);
    }
}

/* ------------------------------------------------------------------------------------------------------ */
/* (4)/(9) direct discrete Fourier transforms                                                              */

/* exp(sign * 2 pi i j / K) with the exponent reduced modulo K first (exact argument). */
static void twiddle(int64_t j, int64_t K, int sign, double *re, double *im) {
    double ang = 2.0 * OR_PI * (double)pmod(j, K) / (double)K;
    *re = cos(ang);
    *im = sign * sin(ang);
}

/* Table of exp(sign * 2 pi i j / K), j = 0..K-1, so a line sum reads exp(sign 2 pi i m k / K) as entry
 * (m k) mod K instead of calling cos/sin per term. Same values as twiddle(). */
static void twiddle_table(int64_t K, int sign, double *re, double *im) {
    for (int64_t j = 0; j < K; ++j) twiddle(j, K, sign, &re[j], &im[j]);
}

/* Separable direct 3D DFT: out(m) = sum_k in(k) exp(sign 2 pi i sum m_a k_a / K_a), one dimension at a
 * time (k3, then k2, then k1), each a plain O(K^2) sum per line. in/out may not alias. */
void oracle_dft3(const int K[3], int sign, const double *in_re, const double *in_im, double *out_re,
                 double *out_im) {
    const int64_t K1 = K[0], K2 = K[1], K3 = K[2], tot = K1 * K2 * K3;
    double *ar = (double *)malloc(sizeof(double) * tot), *ai = (double *)malloc(sizeof(double) * tot);
    double *br = (double *)malloc(sizeof(double) * tot), *bi = (double *)malloc(sizeof(double) * tot);
    for (int64_t x = 0; x < tot; ++x) {
        ar[x] = in_re[x];
        ai[x] = in_im ? in_im[x] : 0.0;
    }
    double *tK1r = (double *)malloc(sizeof(double) * K1), *tK1i = (double *)malloc(sizeof(double) * K1);
    double *tK2r = (double *)malloc(sizeof(double) * K2), *tK2i = (double *)malloc(sizeof(double) * K2);
    double *tK3r = (double *)malloc(sizeof(double) * K3), *tK3i = (double *)malloc(sizeof(double) * K3);
    twiddle_table(K1, sign, tK1r, tK1i);
    twiddle_table(K2, sign, tK2r, tK2i);
    twiddle_table(K3, sign, tK3r, tK3i);
    /* along k3 */
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t a = 0; a < K1; ++a)
        for (int64_t b = 0; b < K2; ++b)
            for (int64_t m = 0; m < K3; ++m) {
                double sr = 0.0, si = 0.0;
                for (int64_t k = 0; k < K3; ++k) {
                    double c = tK3r[(m * k) % K3], s = tK3i[(m * k) % K3];
                    int64_t x = (a * K2 + b) * K3 + k;
                    sr += ar[x] * c - ai[x] * s;
                    si += ar[x] * s + ai[x] * c;
                }
                br[(a * K2 + b) * K3 + m] = sr;
                bi[(a * K2 + b) * K3 + m] = si;
            }
    /* along k2 */
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t a = 0; a < K1; ++a)
        for (int64_t c3 = 0; c3 < K3; ++c3)
            for (int64_t m = 0; m < K2; ++m) {
                double sr = 0.0, si = 0.0;
                for (int64_t k = 0; k < K2; ++k) {
                    double c = tK2r[(m * k) % K2], s = tK2i[(m * k) % K2];
                    int64_t x = (a * K2 + k) * K3 + c3;
                    sr += br[x] * c - bi[x] * s;
                    si += br[x] * s + bi[x] * c;
                }
                ar[(a * K2 + m) * K3 + c3] = sr;
                ai[(a * K2 + m) * K3 + c3] = si;
            }
    /* along k1 */
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t b = 0; b < K2; ++b)
        for (int64_t c3 = 0; c3 < K3; ++c3)
            for (int64_t m = 0; m < K1; ++m) {
                double sr = 0.0, si = 0.0;
                for (int64_t k = 0; k < K1; ++k) {
                    double c = tK1r[(m * k) % K1], s = tK1i[(m * k) % K1];
                    int64_t x = (k * K2 + b) * K3 + c3;
                    sr += ar[x] * c - ai[x] * s;
                    si += ar[x] * s + ai[x] * c;
                }
                out_re[(m * K2 + b) * K3 + c3] = sr;
                out_im[(m * K2 + b) * K3 + c3] = si;
            }
    free(ar);
    free(ai);
    free(br);
    free(bi);
    free(tK1r);
    free(tK1i);
    free(tK2r);
    free(tK2i);
    free(tK3r);
    free(tK3i);
}

/* Non-separable direct 3D DFT, O(K^6): the full triple sum per output point. Only for tiny meshes,
 * where it pins the separable version. */
void oracle_dft3_full(const int K[3], int sign, const double *in_re, const double *in_im, double *out_re,
                      double *out_im) {
    const int64_t K1 = K[0], K2 = K[1], K3 = K[2];
    for (int64_t m1 = 0; m1 < K1; ++m1)
        for (int64_t m2 = 0; m2 < K2; ++m2)
            for (int64_t m3 = 0; m3 < K3; ++m3) {
                double sr = 0.0, si = 0.0;
                for (int64_t k1 = 0; k1 < K1; ++k1)
                    for (int64_t k2 = 0; k2 < K2; ++k2)
                        for (int64_t k3 = 0; k3 < K3; ++k3) {
                            double ang = 2.0 * OR_PI *
                                         ((double)pmod(m1 * k1, K1) / (double)K1 +
                                          (double)pmod(m2 * k2, K2) / (double)K2 +
                                          (double)pmod(m3 * k3, K3) / (double)K3);
                            double c = cos(ang), s = sign * sin(ang);
                            int64_t x = (k1 * K2 + k2) * K3 + k3;
                            double xr = in_re[x], xi = in_im ? in_im[x] : 0.0;
                            sr += xr * c - xi * s;
                            si += xr * s + xi * c;
                        }
                out_re[(m1 * K2 + m2) * K3 + m3] = sr;
                out_im[(m1 * K2 + m2) * K3 + m3] = si;
            }
}

/* ------------------------------------------------------------------------------------------------------ */
/* (5)/(6) B-spline moduli and influence function                                                          */

/* The denominator |sum_{k=0}^{p-2} M_p(k+1) exp(2 pi i m k / K)|^2 of eq. (5). */
static double bmod_denominator(int K, int p, int m) {
    double sr = 0.0, si = 0.0;
    for (int k = 0; k <= p - 2; ++k) {
        double c, s;
        twiddle((int64_t)m * k, K, +1, &c, &s);
        double M = oracle_bspline(p, (double)(k + 1));
        sr += M * c;
        si += M * s;
    }
    return sr * sr + si * si;
}

/* |b(m)|^2 for one dimension of length K, eq. (5). For odd p and even K the denominator vanishes at
 * m = K/2 (the knot values M_p(1..p-1) are symmetric, so their alternating sum is zero); there the
 * denominator is taken as the mean of its two neighbours m = K/2 - 1 and K/2 + 1 (the paper is silent: it
 * uses p = 4 only; this is the usual convention of SPME codes for odd orders). */
double oracle_bmod2(int K, int p, int m) {
    if ((p & 1) && (K & 1) == 0 && 2 * m == K && K >= 4)
        return 1.0 / (0.5 * (bmod_denominator(K, p, m - 1) + bmod_denominator(K, p, m + 1)));
    return 1.0 / bmod_denominator(K, p, m);
}

static int64_t signed_freq(int64_t m, int64_t K) { return (m <= K / 2) ? m : m - K; }

/* m' = sum_alpha mt_alpha a*_alpha for the full-mesh index m. */
static void recip_vector(const int64_t m[3], const int K[3], const double recip[9], double mv[3]) {
    for (int j = 0; j < 3; ++j) mv[j] = 0.0;
    for (int al = 0; al < 3; ++al) {
        double mt = (double)signed_freq(m[al], K[al]);
        for (int j = 0; j < 3; ++j) mv[j] += mt * recip[3 * al + j];
    }
}

/* BC (K1*K2*K3) = B(m) C(m), eqs. (5)-(6), on the full mesh of m. */
void oracle_influence(const int K[3], int p, double beta, const double box[9], double *BC) {
    double recip[9], vol;
    oracle_recip(box, recip, &vol);
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t m1 = 0; m1 < K[0]; ++m1)
        for (int64_t m2 = 0; m2 < K[1]; ++m2)
            for (int64_t m3 = 0; m3 < K[2]; ++m3) {
                int64_t m[3] = {m1, m2, m3};
                int64_t x = (m1 * K[1] + m2) * K[2] + m3;
                if (m1 == 0 && m2 == 0 && m3 == 0) {
                    BC[x] = 0.0;
                    continue;
                }
                double mv[3];
                recip_vector(m, K, recip, mv);
                double m2n = mv[0] * mv[0] + mv[1] * mv[1] + mv[2] * mv[2];
                double B = oracle_bmod2(K[0], p, (int)m1) * oracle_bmod2(K[1], p, (int)m2) *
                           oracle_bmod2(K[2], p, (int)m3);
                double C = exp(-OR_PI * OR_PI * m2n / (beta * beta)) / (OR_PI * vol * m2n);
                BC[x] = B * C;
            }
}

/* ------------------------------------------------------------------------------------------------------ */
/* (3)-(10) the full SPME reciprocal evaluation                                                            */

/* Outputs: *energy; virial[6] = xx, yy, zz, xy, xz, yz; forces (n*3). Optional (NULL to skip): Q_out and
 * phi_out (K1*K2*K3 each), and e_phi = 1/2 sum_k Q(k) phi(k), which must equal *energy.
 * Returns 0, or -1 for invalid arguments. */
int oracle_spme(int64_t n, const double *pos, const double *q, const int K[3], int p, double beta,
                const double box[9], double *energy, double virial[6], double *forces, double *Q_out,
                double *phi_out, double *e_phi) {
    double recip[9], vol;
    if (p < 2 || K[0] < 1 || K[1] < 1 || K[2] < 1 || !(beta > 0.0)) return -1;
    if (oracle_recip(box, recip, &vol) != 0) return -1;
    const int64_t tot = (int64_t)K[0] * K[1] * K[2];
    double *Q = (double *)malloc(sizeof(double) * tot);
    double *Fr = (double *)malloc(sizeof(double) * tot), *Fi = (double *)malloc(sizeof(double) * tot);
    double *BC = (double *)malloc(sizeof(double) * tot);
    double *phr = (double *)malloc(sizeof(double) * tot), *phi_ = (double *)malloc(sizeof(double) * tot);

    oracle_spread(n, pos, q, K, p, box, Q);                   /* eq. (3) */
    oracle_dft3(K, +1, Q, NULL, Fr, Fi);                      /* eq. (4) */
    oracle_influence(K, p, beta, box, BC);                    /* eqs. (5)-(6) */

    double E = 0.0, vir[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t m1 = 0; m1 < K[0]; ++m1)                     /* eqs. (7)-(8) over all m */
        for (int64_t m2 = 0; m2 < K[1]; ++m2)
            for (int64_t m3 = 0; m3 < K[2]; ++m3) {
                int64_t x = (m1 * K[1] + m2) * K[2] + m3;
                if (x == 0) continue;
                double s2 = Fr[x] * Fr[x] + Fi[x] * Fi[x];
                double e = 0.5 * BC[x] * s2;
                int64_t m[3] = {m1, m2, m3};
                double mv[3];
                recip_vector(m, K, recip, mv);
                double m2n = mv[0] * mv[0] + mv[1] * mv[1] + mv[2] * mv[2];
                double f = 2.0 * (1.0 + OR_PI * OR_PI * m2n / (beta * beta)) / m2n;
                E += e;
                vir[0] += e * (1.0 - f * mv[0] * mv[0]);
                vir[1] += e * (1.0 - f * mv[1] * mv[1]);
                vir[2] += e * (1.0 - f * mv[2] * mv[2]);
                vir[3] += e * (-f * mv[0] * mv[1]);
                vir[4] += e * (-f * mv[0] * mv[2]);
                vir[5] += e * (-f * mv[1] * mv[2]);
            }

    for (int64_t x = 0; x < tot; ++x) {                       /* B C Qhat */
        Fr[x] *= BC[x];
        Fi[x] *= BC[x];
    }
    oracle_dft3(K, -1, Fr, Fi, phr, phi_);                    /* eq. (9): phi = Re(...) */

    if (e_phi) {
        double s = 0.0;
        for (int64_t x = 0; x < tot; ++x) s += Q[x] * phr[x];
        *e_phi = 0.5 * s;
    }

    /* eq. (10): forces, visiting the same support points as the spreading step */
    const int64_t K2 = K[1], K3 = K[2];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double u[3];
        scaled_coords(pos + 3 * i, K, recip, u);
        double w[3][16], dw[3][16];
        int64_t idx[3][16];
        int cnt[3];
        for (int al = 0; al < 3; ++al) {
            cnt[al] = 0;
            for (int64_t t = (int64_t)floor(u[al]) - p; t <= (int64_t)floor(u[al]) + 1; ++t) {
                double xx = u[al] - (double)t;
                if (xx > 0.0 && xx < (double)p && cnt[al] < 16) {
                    w[al][cnt[al]] = oracle_bspline(p, xx);
                    dw[al][cnt[al]] = oracle_bspline_deriv(p, xx);
                    idx[al][cnt[al]] = pmod(t, K[al]);
                    cnt[al]++;
                }
            }
        }
        double g[3] = {0, 0, 0}; /* dE/du_alpha / q_i */
        for (int a = 0; a < cnt[0]; ++a)
            for (int b = 0; b < cnt[1]; ++b)
                for (int c = 0; c < cnt[2]; ++c) {
                    double ph = phr[(idx[0][a] * K2 + idx[1][b]) * K3 + idx[2][c]];
                    g[0] += dw[0][a] * w[1][b] * w[2][c] * ph;
                    g[1] += w[0][a] * dw[1][b] * w[2][c] * ph;
                    g[2] += w[0][a] * w[1][b] * dw[2][c] * ph;
                }
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int al = 0; al < 3; ++al) s += K[al] * recip[3 * al + j] * g[al];
            forces[3 * i + j] = -q[i] * s;
        }
    }

    *energy = E;
    for (int j = 0; j < 6; ++j) virial[j] = vir[j];
    if (Q_out) memcpy(Q_out, Q, sizeof(double) * tot);
    if (phi_out) memcpy(phi_out, phr, sizeof(double) * tot);
    free(Q);
    free(Fr);
    free(Fi);
    free(BC);
    free(phr);
    free(phi_);
    return 0;
}

/* ------------------------------------------------------------------------------------------------------ */
/* (11) Ewald comparison terms                                                                             */

/* Brute-force Ewald reciprocal sum over all m != 0 with |m'| <= mcut (A^-1):
 *   E = 1/(2 pi V) sum exp(-pi^2 |m'|^2/beta^2)/|m'|^2 |S(m)|^2,  S(m) = sum_j q_j exp(2 pi i m'.r_j),
 *   F_j = (2 q_j / V) sum f(m) m' (Re S sin(th_j) - Im S cos(th_j)),  th_j = 2 pi m'.r_j,
 *   virial as eq. (8) with B C |Qhat|^2 replaced by f(m)|S|^2/(pi V). */
int oracle_ewald_recip(int64_t n, const double *pos, const double *q, double beta, const double box[9],
                       double mcut, double *energy, double virial[6], double *forces) {
    double recip[9], vol;
    if (oracle_recip(box, recip, &vol) != 0) return -1;
    /* |m_alpha| <= mcut * |a_alpha| bounds every m with |m'| <= mcut (m_alpha = m' . a_alpha). */
    int64_t mmax[3];
    for (int al = 0; al < 3; ++al) {
        const double *a = box + 3 * al;
        mmax[al] = (int64_t)ceil(mcut * sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]));
    }
    double E = 0.0, vir[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t i = 0; i < 3 * n; ++i) forces[i] = 0.0;
    double *th = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    for (int64_t m1 = -mmax[0]; m1 <= mmax[0]; ++m1)
        for (int64_t m2 = -mmax[1]; m2 <= mmax[1]; ++m2)
            for (int64_t m3 = -mmax[2]; m3 <= mmax[2]; ++m3) {
                if (m1 == 0 && m2 == 0 && m3 == 0) continue;
                double mv[3];
                for (int j = 0; j < 3; ++j)
                    mv[j] = (double)m1 * recip[j] + (double)m2 * recip[3 + j] + (double)m3 * recip[6 + j];
                double m2n = mv[0] * mv[0] + mv[1] * mv[1] + mv[2] * mv[2];
                if (m2n > mcut * mcut) continue;
                double f = exp(-OR_PI * OR_PI * m2n / (beta * beta)) / m2n;
                double sr = 0.0, si = 0.0;
                for (int64_t j = 0; j < n; ++j) {
                    th[j] = 2.0 * OR_PI * (mv[0] * pos[3 * j] + mv[1] * pos[3 * j + 1] + mv[2] * pos[3 * j + 2]);
                    sr += q[j] * cos(th[j]);
                    si += q[j] * sin(th[j]);
                }
                double e = f * (sr * sr + si * si) / (2.0 * OR_PI * vol);
                double fv = 2.0 * (1.0 + OR_PI * OR_PI * m2n / (beta * beta)) / m2n;
                E += e;
                vir[0] += e * (1.0 - fv * mv[0] * mv[0]);
                vir[1] += e * (1.0 - fv * mv[1] * mv[1]);
                vir[2] += e * (1.0 - fv * mv[2] * mv[2]);
                vir[3] += e * (-fv * mv[0] * mv[1]);
                vir[4] += e * (-fv * mv[0] * mv[2]);
                vir[5] += e * (-fv * mv[1] * mv[2]);
                for (int64_t j = 0; j < n; ++j) {
                    double c = (2.0 * q[j] / vol) * f * (sr * sin(th[j]) - si * cos(th[j]));
                    forces[3 * j] += c * mv[0];
                    forces[3 * j + 1] += c * mv[1];
                    forces[3 * j + 2] += c * mv[2];
                }
            }
    free(th);
    *energy = E;
    for (int j = 0; j < 6; ++j) virial[j] = vir[j];
    return 0;
}

/* Real-space Ewald term E = 1/2 sum_{i,j,n}' q_i q_j erfc(beta r)/r over all lattice images n with
 * r = |r_i - r_j + n| <= rcut (the primed sum skips i == j at n = 0), and its forces
 * F_i = sum q_i q_j [erfc(beta r)/r + 2 beta/sqrt(pi) exp(-beta^2 r^2)] (r_i - r_j + n) / r^2, and (when
 * virial is not NULL) its virial Pi_ab = -dE/d eps_ab = 1/2 sum' s_ij d_a d_b with s_ij the scalar factor of
 * the force above and d = r_i - r_j + n (the pair potential depends on the strain only through |d|). */
int oracle_ewald_real(int64_t n, const double *pos, const double *q, double beta, const double box[9],
                      double rcut, double *energy, double *forces, double *virial) {
    double recip[9], vol;
    if (oracle_recip(box, recip, &vol) != 0) return -1;
    /* image range: n_alpha with |n_alpha| <= ceil(rcut * |a*_alpha|) + 1 covers every image within rcut
     * of any pair inside one cell (plane spacing along alpha is 1/|a*_alpha|). */
    int64_t nmax[3];
    for (int al = 0; al < 3; ++al) {
        const double *r = recip + 3 * al;
        nmax[al] = (int64_t)ceil(rcut * sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2])) + 1;
    }
    double E = 0.0;
    for (int64_t i = 0; i < 3 * n; ++i) forces[i] = 0.0;
    const double c2 = 2.0 * beta / sqrt(OR_PI);
    /* per-atom partial energies Ei and virials Wi (one thread per atom i), summed over i in order afterwards */
    double *Ei = (double *)calloc(n > 0 ? (size_t)n : 1, sizeof(double));
    double *Wi = (double *)calloc(n > 0 ? (size_t)(6 * n) : 6, sizeof(double));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j)
            for (int64_t a = -nmax[0]; a <= nmax[0]; ++a)
                for (int64_t b = -nmax[1]; b <= nmax[1]; ++b)
                    for (int64_t c = -nmax[2]; c <= nmax[2]; ++c) {
                        if (i == j && a == 0 && b == 0 && c == 0) continue;
                        double d[3];
                        for (int k = 0; k < 3; ++k)
                            d[k] = pos[3 * i + k] - pos[3 * j + k] + a * box[k] + b * box[3 + k] + c * box[6 + k];
                        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        if (r2 > rcut * rcut) continue;
                        double r = sqrt(r2);
                        double qq = q[i] * q[j];
                        Ei[i] += 0.5 * qq * erfc(beta * r) / r;
                        double s = qq * (erfc(beta * r) / r + c2 * exp(-beta * beta * r2)) / r2;
                        for (int k = 0; k < 3; ++k) forces[3 * i + k] += s * d[k];
                        Wi[6 * i + 0] += 0.5 * s * d[0] * d[0];
                        Wi[6 * i + 1] += 0.5 * s * d[1] * d[1];
                        Wi[6 * i + 2] += 0.5 * s * d[2] * d[2];
                        Wi[6 * i + 3] += 0.5 * s * d[0] * d[1];
                        Wi[6 * i + 4] += 0.5 * s * d[0] * d[2];
                        Wi[6 * i + 5] += 0.5 * s * d[1] * d[2];
                    }
    for (int64_t i = 0; i < n; ++i) E += Ei[i];
    if (virial) {
        for (int k = 0; k < 6; ++k) virial[k] = 0.0;
        for (int64_t i = 0; i < n; ++i)
            for (int k = 0; k < 6; ++k) virial[k] += Wi[6 * i + k];
    }
    free(Ei);
    free(Wi);
    *energy = E;
    return 0;
}

/* The same real-space sum restricted to the listed atoms: for each i = rows[k], e_rows[k] = sum_{j,n}' q_i q_j
 * erfc(beta r)/r (so E_real = 1/2 sum_i e_i) and f_rows[3k..3k+2] = F_i, with the loops of oracle_ewald_real.
 * For checking single atoms of systems too large for the full double sum. */
int oracle_ewald_real_rows(int64_t n, const double *pos, const double *q, double beta, const double box[9],
                           double rcut, int64_t nrows, const int64_t *rows, double *e_rows, double *f_rows) {
    double recip[9], vol;
    if (oracle_recip(box, recip, &vol) != 0) return -1;
    int64_t nmax[3];
    for (int al = 0; al < 3; ++al) {
        const double *r = recip + 3 * al;
        nmax[al] = (int64_t)ceil(rcut * sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2])) + 1;
    }
    const double c2 = 2.0 * beta / sqrt(OR_PI);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < nrows; ++k) {
        const int64_t i = rows[k];
        double e = 0.0, f[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; ++j)
            for (int64_t a = -nmax[0]; a <= nmax[0]; ++a)
                for (int64_t b = -nmax[1]; b <= nmax[1]; ++b)
                    for (int64_t c = -nmax[2]; c <= nmax[2]; ++c) {
                        if (i == j && a == 0 && b == 0 && c == 0) continue;
                        double d[3];
                        for (int m = 0; m < 3; ++m)
                            d[m] = pos[3 * i + m] - pos[3 * j + m] + a * box[m] + b * box[3 + m] + c * box[6 + m];
                        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        if (r2 > rcut * rcut) continue;
                        double r = sqrt(r2);
                        double qq = q[i] * q[j];
                        e += qq * erfc(beta * r) / r;
                        double s = qq * (erfc(beta * r) / r + c2 * exp(-beta * beta * r2)) / r2;
                        for (int m = 0; m < 3; ++m) f[m] += s * d[m];
                    }
        e_rows[k] = e;
        for (int m = 0; m < 3; ++m) f_rows[3 * k + m] = f[m];
    }
    return 0;
}

/* Self term E_self = -(beta / sqrt(pi)) sum q_i^2. */
double oracle_ewald_self(int64_t n, const double *q, double beta) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += q[i] * q[i];
    return -beta / sqrt(OR_PI) * s;
}
