// Batched complex FFTs in shared memory (Stockham auto-sort, mixed radix 2/3/4/5/8).
//
// The paper builds its 3D FFT from pipelined radix-2 1D FFT units (Sec. III-B, Sec. IV-A). On a GPU the
// 1D transforms of a slab or pencil instead live in shared memory: each stage reads R points at stride
// N/R, applies the twiddles W_{Ns R}^{r k}, does a radix-R DFT in registers, and writes the R outputs at
// stride Ns, ping-ponging between two buffers. Input and output are in natural order, so no bit-reversal
// pass and no permuted tables are needed. Lengths are any product of 2, 3, 5 up to 128.
//
// Sign convention: forward = exp(-2 pi i jk/N), inverse = exp(+2 pi i jk/N), both unnormalised.
#pragma once

#include "common.cuh"

namespace pme {

PME_DEV float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
PME_DEV float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
PME_DEV float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
PME_DEV float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
PME_DEV float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
PME_DEV float2 cmul_mi(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <int R, bool INV>
PME_DEV void dft_small(float2 *v);

template <>
PME_DEV void dft_small<2, false>(float2 *v) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}
template <>
PME_DEV void dft_small<2, true>(float2 *v) {
    dft_small<2, false>(v);
}

template <bool INV>
PME_DEV void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3) {
    float2 s02 = cadd(a0, a2), d02 = csub(a0, a2);
    float2 s13 = cadd(a1, a3), d13 = cmul_mi<INV>(csub(a1, a3));
    a0 = cadd(s02, s13);
    a2 = csub(s02, s13);
    a1 = cadd(d02, d13);
    a3 = csub(d02, d13);
}

template <>
PME_DEV void dft_small<4, false>(float2 *v) {
    dft4<false>(v[0], v[1], v[2], v[3]);
}
template <>
PME_DEV void dft_small<4, true>(float2 *v) {
    dft4<true>(v[0], v[1], v[2], v[3]);
}

template <bool INV>
PME_DEV void dft8(float2 *v) {
    // even / odd split into two length-4 DFTs, then the W8^k combine
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    const float h = 0.70710678118654752440f;
    // W8^1 = (h, -h) forward, (h, h) inverse; W8^2 = -i / +i; W8^3 = (-h, -h) forward, (-h, h) inverse
    float2 t1 = INV ? make_float2(h * (o1.x - o1.y), h * (o1.x + o1.y)) : make_float2(h * (o1.x + o1.y), h * (o1.y - o1.x));
    float2 t2 = cmul_mi<INV>(o2);
    float2 t3 = INV ? make_float2(-h * (o3.x + o3.y), h * (o3.x - o3.y)) : make_float2(h * (o3.y - o3.x), -h * (o3.x + o3.y));
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, t1);
    v[5] = csub(e1, t1);
    v[2] = cadd(e2, t2);
    v[6] = csub(e2, t2);
    v[3] = cadd(e3, t3);
    v[7] = csub(e3, t3);
}
template <>
PME_DEV void dft_small<8, false>(float2 *v) {
    dft8<false>(v);
}
template <>
PME_DEV void dft_small<8, true>(float2 *v) {
    dft8<true>(v);
}

template <bool INV>
PME_DEV void dft3(float2 *v) {
    const float c = -0.5f, s = 0.86602540378443864676f;  // cos(2 pi/3), sin(2 pi/3)
    float2 a0 = v[0], t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
    float2 m = make_float2(a0.x + c * t1.x, a0.y + c * t1.y);
    float2 r = cmul_mi<INV>(cscale(t2, s));  // -i s t2 (forward)
    v[0] = cadd(a0, t1);
    v[1] = cadd(m, r);
    v[2] = csub(m, r);
}
template <>
PME_DEV void dft_small<3, false>(float2 *v) {
    dft3<false>(v);
}
template <>
PME_DEV void dft_small<3, true>(float2 *v) {
    dft3<true>(v);
}

template <bool INV>
PME_DEV void dft5(float2 *v) {
    const float c1 = 0.30901699437494742410f, s1 = 0.95105651629515357212f;   // cos, sin(2 pi/5)
    const float c2 = -0.80901699437494742410f, s2 = 0.58778525229247312917f;  // cos, sin(4 pi/5)
    float2 a0 = v[0];
    float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    float2 t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    float2 m1 = make_float2(a0.x + c1 * t1.x + c2 * t2.x, a0.y + c1 * t1.y + c2 * t2.y);
    float2 m2 = make_float2(a0.x + c2 * t1.x + c1 * t2.x, a0.y + c2 * t1.y + c1 * t2.y);
    float2 r1 = cmul_mi<INV>(make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y));
    float2 r2 = cmul_mi<INV>(make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y));
    v[0] = cadd(a0, cadd(t1, t2));
    v[1] = cadd(m1, r1);
    v[4] = csub(m1, r1);
    v[2] = cadd(m2, r2);
    v[3] = csub(m2, r2);
}
template <>
PME_DEV void dft_small<5, false>(float2 *v) {
    dft5<false>(v);
}
template <>
PME_DEV void dft_small<5, true>(float2 *v) {
    dft5<true>(v);
}

// Length 6 as 3 x 2 (Cooley-Tukey): DFT3 of the even and of the odd points, twiddles W6^k, then DFT2.
template <bool INV>
PME_DEV void dft6(float2 *v) {
    float2 a[3] = {v[0], v[2], v[4]}, b[3] = {v[1], v[3], v[5]};
    dft3<INV>(a);
    dft3<INV>(b);
    const float s = 0.86602540378443864676f;  // sin(pi / 3)
    // W6^1 = (1/2, -s) forward, (1/2, s) inverse; W6^2 = (-1/2, -s) forward, (-1/2, s) inverse
    const float sg = INV ? s : -s;
    b[1] = cmul(b[1], make_float2(0.5f, sg));
    b[2] = cmul(b[2], make_float2(-0.5f, sg));
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        v[k] = cadd(a[k], b[k]);
        v[k + 3] = csub(a[k], b[k]);
    }
}
template <>
PME_DEV void dft_small<6, false>(float2 *v) {
    dft6<false>(v);
}
template <>
PME_DEV void dft_small<6, true>(float2 *v) {
    dft6<true>(v);
}

// Radix chosen for the remaining length rem = N / Ns: 8, then 4, 2, 3, 5.
PME_DEV int fft_radix(int rem) {
    if (rem % 8 == 0) return 8;
    if (rem % 4 == 0) return 4;
    if (rem % 2 == 0) return 2;
    if (rem % 3 == 0) return 3;
    return 5;
}

// One Stockham stage of radix R over ntr transforms of length N (element e of transform t at
// t*bs + e*es in both buffers). tw[k] = exp(-2 pi i k / N), k < N.
template <int R, bool INV>
PME_DEV void fft_stage(const float2 *src, float2 *dst, int N, int Ns, int ntr, int es, int bs, const float2 *tw) {
    const int nb = N / R;           // butterflies per transform
    const int total = ntr * nb;
    const int tstep = nb / Ns;      // = N / (Ns R): twiddle index step
    const float inv_nb = 1.0f / (float)nb, inv_ntr = 1.0f / (float)ntr, inv_ns = 1.0f / (float)Ns;
    for (int idx = PME_TID; idx < total; idx += PME_NTH) {
        int t, j;
        if (es == 1) {  // rows contiguous: consecutive threads walk one transform
            t = fdiv(idx, inv_nb);
            j = idx - t * nb;
        } else {        // columns: consecutive threads walk consecutive transforms
            j = fdiv(idx, inv_ntr);
            t = idx - j * ntr;
        }
        const float2 *s = src + t * bs;
        float2 *o = dst + t * bs;
        const int jq = fdiv(j, inv_ns);
        const int k = j - jq * Ns;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = s[(j + r * nb) * es];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = tw[r * k * tstep];
                if (INV) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        dft_small<R, INV>(v);
        const int od = jq * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) o[(od + r * Ns) * es] = v[r];
    }
}

// Full transforms; returns the buffer (a or b) that holds the result. Ends with a barrier.
template <bool INV>
PME_DEV float2 *fft_batch(float2 *a, float2 *b, int N, int ntr, int es, int bs, const float2 *tw) {
    int Ns = 1;
    while (Ns < N) {
        const int R = fft_radix(N / Ns);
        switch (R) {
            case 8: fft_stage<8, INV>(a, b, N, Ns, ntr, es, bs, tw); break;
            case 4: fft_stage<4, INV>(a, b, N, Ns, ntr, es, bs, tw); break;
            case 2: fft_stage<2, INV>(a, b, N, Ns, ntr, es, bs, tw); break;
            case 3: fft_stage<3, INV>(a, b, N, Ns, ntr, es, bs, tw); break;
            default: fft_stage<5, INV>(a, b, N, Ns, ntr, es, bs, tw); break;
        }
        PME_SYNC();
        float2 *t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

#if !defined(PME_HOST_EMULATION)
// ---------------------------------------------------------------------------------------------------------
// Lane-distributed transforms in registers, for lengths N = L * E with L in {1, 2, 4, 8, 16} and
// E in {4, 5, 6, 8} (every lane plan below). The L lanes of one transform sit in one warp at lane ids
// t + T j (T = 32 / L transforms per warp, j = 0 .. L - 1), so a transform's lanes exchange values with
// shuffles and no CTA barrier. Lane j holds the E points x[j + L n], n < E, and the four-step
// factorisation N = E x L runs as:
//   1. an E-point DFT in each lane over n:          y_j[k] = sum_n x[j + L n] W_E^{n k}
//   2. twiddles:                                    y_j[k] *= W_N^{j k}
//   3. an L-point DFT across lanes over j, as log2 L radix-2 decimation-in-frequency rounds: the lane
//      with bit h of j clear keeps a + b, its partner (bit h set) keeps (a - b) W_{2h}^{j mod h}.
// Afterwards lane j holds X[k + E rev(j)], k < E, where rev reverses the log2 L bits of j. Inverse
// transforms conjugate every twiddle. lane_fft_adjoint applies the conjugate transpose of the whole
// sequence, which takes the bit-reversed distribution back to x[j + L n] and is the unnormalised
// inverse DFT: a forward transform, a pointwise product and the adjoint need no reordering in between.

template <int L>
PME_DEV int lane_rev(int j) {
    int r = 0;
#pragma unroll
    for (int b = 1; b < L; b <<= 1) r = (r << 1) | ((j & b) ? 1 : 0);
    return r;
}

template <int L>
struct Log2 {
    static constexpr int v = L <= 1 ? 0 : 1 + Log2<L / 2>::v;
};
template <>
struct Log2<1> {
    static constexpr int v = 0;
};

// The twiddles one lane needs (forward sign), loaded once so their latency overlaps the data loads and
// the inverse / adjoint transforms reuse them: w[k - 1] = W_N^{j k}, k = 1 .. E - 1, and r[i] =
// W_{2h}^{j mod h} for the cross-lane round h = L / 2^(i + 1).
template <int L, int E>
struct LaneTw {
    float2 w[E > 1 ? E - 1 : 1];
    float2 r[Log2<L>::v > 0 ? Log2<L>::v : 1];
};

// tw[t] = exp(-2 pi i t / N), t < N, in global (read-only path) or shared memory.
template <int L, int E, bool GLOBAL>
PME_DEV LaneTw<L, E> lane_tw(const float2 *tw, int j) {
    constexpr int N = L * E;
    LaneTw<L, E> t;
    if (L > 1) {
#pragma unroll
        for (int k = 1; k < E; ++k) t.w[k - 1] = GLOBAL ? __ldg(tw + j * k) : tw[j * k];
#pragma unroll
        for (int i = 0, h = L / 2; h >= 1; ++i, h >>= 1) {
            const int idx = (j & (h - 1)) * (N / (2 * h));
            t.r[i] = GLOBAL ? __ldg(tw + idx) : tw[idx];
        }
    }
    return t;
}

PME_DEV float2 shfl_xor_c(float2 v, int mask) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, mask), __shfl_xor_sync(0xffffffffu, v.y, mask));
}

PME_DEV float2 cmul_c(float2 a, float2 w, bool conj) { return conj ? cmul(a, cconj(w)) : cmul(a, w); }

template <int L, int E, bool INV>
PME_DEV void lane_fft(float2 (&v)[E], int j, const LaneTw<L, E> &tw) {
    constexpr int T = 32 / L;
    dft_small<E, INV>(v);
    if (L > 1) {
#pragma unroll
        for (int k = 1; k < E; ++k) v[k] = cmul_c(v[k], tw.w[k - 1], INV);
#pragma unroll
        for (int i = 0, h = L / 2; h >= 1; ++i, h >>= 1) {
            const bool up = (j & h) != 0;
#pragma unroll
            for (int k = 0; k < E; ++k) {
                const float2 p = shfl_xor_c(v[k], h * T);
                v[k] = up ? (h > 1 ? cmul_c(csub(p, v[k]), tw.r[i], INV) : csub(p, v[k])) : cadd(v[k], p);
            }
        }
    }
}

template <int L, int E>
PME_DEV void lane_fft_adjoint(float2 (&v)[E], int j, const LaneTw<L, E> &tw) {
    constexpr int T = 32 / L;
    if (L > 1) {
#pragma unroll
        for (int i = Log2<L>::v - 1, h = 1; h < L; --i, h <<= 1) {
            const bool up = (j & h) != 0;
            if (up && h > 1) {
#pragma unroll
                for (int k = 0; k < E; ++k) v[k] = cmul_c(v[k], tw.r[i], true);
            }
#pragma unroll
            for (int k = 0; k < E; ++k) {
                const float2 p = shfl_xor_c(v[k], h * T);
                v[k] = up ? csub(p, v[k]) : cadd(v[k], p);
            }
        }
#pragma unroll
        for (int k = 1; k < E; ++k) v[k] = cmul_c(v[k], tw.w[k - 1], true);
    }
    dft_small<E, true>(v);
}
#endif  // !PME_HOST_EMULATION

}  // namespace pme
