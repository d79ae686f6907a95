// Real-space and self terms of Ewald electrostatics on the GPU: with the reciprocal-space SPME evaluation
// (the paper's long-range pipeline) they make up the full Ewald sum the paper splits its electrostatics
// into (Sec. II; the short-range part runs on its own pipelines beside the long-range one, Sec. III):
//   E_real = 1/2 sum_{i,j,n}' q_i q_j erfc(beta r) / r   over images with r = |r_i - r_j + n| <= rcut,
//   F_i    = sum_{j,n}' q_i q_j [erfc(beta r) / r + 2 beta / sqrt(pi) exp(-beta^2 r^2)] d / r^2,
//   Pi_ab  = 1/2 sum' s_ij d_a d_b   (s_ij the scalar factor of the force, d = r_i - r_j + n),
//   E_self = -beta / sqrt(pi) sum_i q_i^2.
//
// Design. Cell list in fractional coordinates: the cell grid has nc_alpha = floor(1 / (rcut |a*_alpha|))
// cells along alpha (at least 1), so every image within rcut of an atom lies in the neighbouring cells
// -R..R along each axis (R = 1 unless the cell is narrower than rcut). Atoms are counted per cell, the counts
// scanned, the atoms scattered, and then each cell's atoms put in input-index order (a rank count inside the
// cell), so every sum below runs in an order that depends only on the inputs: results are bit-reproducible.
// One thread per (sorted) atom walks the (2R+1)^3 neighbour cells and sums its own force, energy and virial:
// each pair is visited from both ends, so no atom is written by two threads and no atomics are needed. The
// displacement is formed from the raw input positions and an integer image shift, r_i - r_j - sum m_alpha
// a_alpha, with the difference taken exactly (TwoSum) and the cell vectors as (hi, lo) floats, so it carries
// only FP32 rounding of its own size. Energies are summed per atom in double-float and across atoms in FP64
// by a fixed-order two-level reduction.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "../../include/pme.h"
#include "common.cuh"
#include "host_tables.h"
#include "plan_internal.h"

namespace pme {

constexpr int RS_THREADS = 128;
constexpr int RS_SCAN_THREADS = 1024;
constexpr int RS_RED_BLOCKS = 152;  // first reduction level: one block per SM, atoms in contiguous chunks
constexpr int RS_MAX_R = 4;         // neighbour cells -R..R per axis (rcut up to 4 cell widths)
constexpr int RS_MAX_CELLS = 1 << 22;

struct RealCtl {
    unsigned status;  // StatusBits
    unsigned pad[3];
    double res[8];    // E_real, E_self, virial xx yy zz xy xz yz
};

struct RealDev {
    int n;
    int nc[3], R[3], ncells;
    float rec[9];          // a*_alpha[j] at 3 alpha + j (cell assignment)
    float ahi[9], alo[9];  // a_alpha[k] at 3 alpha + k as (hi, lo) floats (image shifts)
    float rc2, beta, c2;   // rcut^2, beta, 2 beta / sqrt(pi)
    double beta_d;
    int accumulate;        // forces += (1) or = (0)
    const float *pos, *q;
    float *forces;
    double *ev;            // optional device destination of RealCtl::res (8 doubles)
    unsigned *count;       // ncells, zero between calls (reset by the scan)
    unsigned *start;       // ncells + 1
    unsigned *fill;        // ncells, zero between calls (reset by the rank kernel)
    int *cell;             // n: cell of input atom i
    int4 *img;             // n: floor of input atom i's fractional coordinates
    float4 *arec;          // n: scattered (x, y, z, q), arrival order inside a cell
    int4 *aidx;            // n: scattered (N1, N2, N3, input index)
    float4 *srec;          // n: (x, y, z, q) in cell order, input order inside a cell
    int4 *sidx;            // n: (N1, N2, N3, input index) likewise
    double *e_atom;        // n: per sorted atom, sum_j q_i q_j erfc(beta r) / r
    float *w_atom;         // 6 n: per sorted atom, 1/2 sum_j s d_a d_b
    double *partials;      // RS_RED_BLOCKS x 8
    RealCtl *ctl;
};

__device__ __forceinline__ int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// 1: cell of every atom, its image index N = floor(s), and the per-cell counts.
__global__ void __launch_bounds__(256) k_rs_bin(RealDev d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const float x = d.pos[3 * i], y = d.pos[3 * i + 1], z = d.pos[3 * i + 2], qq = d.q[i];
    int c[3], N[3];
    bool bad = !(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(qq));
#pragma unroll
    for (int al = 0; al < 3; ++al) {
        const float s = fmaf(x, d.rec[3 * al], fmaf(y, d.rec[3 * al + 1], z * d.rec[3 * al + 2]));
        if (!(fabsf(s) < 1048576.0f)) bad = true;  // also catches NaN: absurdly far out
        const float fl = bad ? 0.0f : floorf(s);
        const float f = bad ? 0.0f : s - fl;  // exact: s and floor(s) are within one of each other
        N[al] = (int)fl;
        int ci = (int)(f * (float)d.nc[al]);
        c[al] = ci < 0 ? 0 : (ci >= d.nc[al] ? d.nc[al] - 1 : ci);
    }
    if (bad) atomicOr(&d.ctl->status, ST_NONFINITE);
    const int cid = (c[0] * d.nc[1] + c[1]) * d.nc[2] + c[2];
    d.cell[i] = cid;
    d.img[i] = make_int4(N[0], N[1], N[2], 0);
    atomicAdd(d.count + cid, 1u);
}

// 2: exclusive scan of the counts into start[] (one CTA; thread t owns a contiguous run of cells), counts
// reset for the next call.
__global__ void __launch_bounds__(RS_SCAN_THREADS) k_rs_scan(RealDev d) {
    __shared__ unsigned part[RS_SCAN_THREADS];
    const int t = threadIdx.x, per = (d.ncells + RS_SCAN_THREADS - 1) / RS_SCAN_THREADS;
    const int b = t * per, e = min(d.ncells, b + per);
    unsigned s = 0;
    for (int c = b; c < e; ++c) s += d.count[c];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < RS_SCAN_THREADS; off <<= 1) {  // inclusive Hillis-Steele scan of the run sums
        const unsigned v = t >= off ? part[t - off] : 0u;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    unsigned run = part[t] - s;
    for (int c = b; c < e; ++c) {
        const unsigned k = d.count[c];
        d.start[c] = run;
        run += k;
        d.count[c] = 0u;
    }
    if (t == RS_SCAN_THREADS - 1) d.start[d.ncells] = part[t];
}

// 3: scatter into cell ranges (arrival order inside a cell).
__global__ void __launch_bounds__(256) k_rs_scatter(RealDev d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const int c = d.cell[i];
    const unsigned slot = d.start[c] + atomicAdd(d.fill + c, 1u);
    const int4 N = d.img[i];
    d.arec[slot] = make_float4(d.pos[3 * i], d.pos[3 * i + 1], d.pos[3 * i + 2], d.q[i]);
    d.aidx[slot] = make_int4(N.x, N.y, N.z, i);
}

// 4: inside each cell, input-index order: the record at slot k moves to start + (number of the cell's atoms
// with a smaller input index).
__global__ void __launch_bounds__(256) k_rs_rank(RealDev d) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.n) return;
    const int4 me = d.aidx[k];
    const int c = d.cell[me.w];
    const unsigned b = d.start[c], e = d.start[c + 1];
    unsigned r = 0;
    for (unsigned j = b; j < e; ++j) r += (unsigned)(d.aidx[j].w < me.w);
    d.srec[b + r] = d.arec[k];
    d.sidx[b + r] = me;
    if (r == 0) d.fill[c] = 0u;  // every arrival in this cell has happened (previous kernel)
}

// d = r_i - r_j - sum_alpha m_alpha a_alpha, component k: the coordinate difference exactly (TwoSum), the
// image shift against the (hi, lo) cell vectors.
__device__ __forceinline__ float disp(const RealDev &d, float ri, float rj, int k, float m0, float m1, float m2) {
    const float t = __fsub_rn(ri, rj);
    const float bb = __fsub_rn(t, ri);
    const float e = __fadd_rn(__fsub_rn(ri, __fsub_rn(t, bb)), __fsub_rn(-rj, bb));
    float acc = fmaf(-m0, d.ahi[k], t);
    acc = fmaf(-m1, d.ahi[3 + k], acc);
    acc = fmaf(-m2, d.ahi[6 + k], acc);
    const float corr = e - (m0 * d.alo[k] + m1 * d.alo[3 + k] + m2 * d.alo[6 + k]);
    return acc + corr;
}

// 5: one thread per sorted atom: force (written at the input index), energy and virial over all neighbours.
__global__ void __launch_bounds__(RS_THREADS) k_rs_pairs(RealDev d) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= d.n) return;
    const float4 ri = d.srec[a];
    const int4 ii = d.sidx[a];
    const int cid = d.cell[ii.w];
    const int c2_ = cid % d.nc[2], c1_ = (cid / d.nc[2]) % d.nc[1], c0_ = cid / (d.nc[2] * d.nc[1]);
    float fx = 0.f, fy = 0.f, fz = 0.f;
    float w[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    DF en = {0.f, 0.f};
    const float beta = d.beta, b2 = d.beta * d.beta;
    for (int o0 = -d.R[0]; o0 <= d.R[0]; ++o0) {
        const int u0 = c0_ + o0, w0 = floordiv(u0, d.nc[0]), cc0 = u0 - w0 * d.nc[0];
        for (int o1 = -d.R[1]; o1 <= d.R[1]; ++o1) {
            const int u1 = c1_ + o1, w1 = floordiv(u1, d.nc[1]), cc1 = u1 - w1 * d.nc[1];
            for (int o2 = -d.R[2]; o2 <= d.R[2]; ++o2) {
                const int u2 = c2_ + o2, w2 = floordiv(u2, d.nc[2]), cc2 = u2 - w2 * d.nc[2];
                const int nb = (cc0 * d.nc[1] + cc1) * d.nc[2] + cc2;
                const bool home = (w0 | w1 | w2) == 0;
                const unsigned b = d.start[nb], e = d.start[nb + 1];
                for (unsigned j = b; j < e; ++j) {
                    if (home && (int)j == a) continue;
                    const float4 rj = d.srec[j];
                    const int4 jj = d.sidx[j];
                    // image of j: its own image index, then the cell wrap
                    const float m0 = (float)(ii.x - jj.x + w0), m1 = (float)(ii.y - jj.y + w1), m2 = (float)(ii.z - jj.z + w2);
                    const float dx = disp(d, ri.x, rj.x, 0, m0, m1, m2);
                    const float dy = disp(d, ri.y, rj.y, 1, m0, m1, m2);
                    const float dz = disp(d, ri.z, rj.z, 2, m0, m1, m2);
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    if (r2 > d.rc2 || r2 == 0.f) continue;
                    const float rinv = rsqrtf(r2);
                    const float r = r2 * rinv;
                    const float qq = ri.w * rj.w;
                    const float ec = erfcf(beta * r);
                    const float er = qq * ec * rinv;
                    const float s = (er + qq * d.c2 * expf(-b2 * r2)) * (rinv * rinv);
                    en = df_add(en, er);
                    fx = fmaf(s, dx, fx);
                    fy = fmaf(s, dy, fy);
                    fz = fmaf(s, dz, fz);
                    const float hs = 0.5f * s;
                    w[0] = fmaf(hs * dx, dx, w[0]);
                    w[1] = fmaf(hs * dy, dy, w[1]);
                    w[2] = fmaf(hs * dz, dz, w[2]);
                    w[3] = fmaf(hs * dx, dy, w[3]);
                    w[4] = fmaf(hs * dx, dz, w[4]);
                    w[5] = fmaf(hs * dy, dz, w[5]);
                }
            }
        }
    }
    float *F = d.forces + 3 * (size_t)ii.w;
    if (d.accumulate) {
        F[0] += fx;
        F[1] += fy;
        F[2] += fz;
    } else {
        F[0] = fx;
        F[1] = fy;
        F[2] = fz;
    }
    d.e_atom[a] = (double)en.hi + (double)en.lo;
#pragma unroll
    for (int k = 0; k < 6; ++k) d.w_atom[6 * (size_t)a + k] = w[k];
}

// FP64 block sum of 8 values per thread in a fixed tree (warp shuffles, then the warps' results in order).
__device__ void block_sum8(double v[8], double *out) {
    __shared__ double wsum[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
        if (lane == 0) wsum[k][warp] = v[k];
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += wsum[threadIdx.x][w];
        out[threadIdx.x] = s;
    }
}

// 6: per block, a contiguous chunk of sorted atoms: sum e, q^2 and the six virial components.
__global__ void __launch_bounds__(256) k_rs_reduce1(RealDev d) {
    const int chunk = (d.n + gridDim.x - 1) / gridDim.x;
    const int b = blockIdx.x * chunk, e = min(d.n, b + chunk);
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int a = b + (int)threadIdx.x; a < e; a += blockDim.x) {
        v[0] += d.e_atom[a];
        const double qa = (double)d.srec[a].w;
        v[1] += qa * qa;
#pragma unroll
        for (int k = 0; k < 6; ++k) v[2 + k] += (double)d.w_atom[6 * (size_t)a + k];
    }
    block_sum8(v, d.partials + 8 * blockIdx.x);
}

// 7: the block sums in order; energies, self term and virial to the control block (and to d.ev).
__global__ void __launch_bounds__(256) k_rs_reduce2(RealDev d, int nparts) {
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int p = threadIdx.x; p < nparts; p += blockDim.x)
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] += d.partials[8 * p + k];
    __shared__ double tot[8];
    block_sum8(v, tot);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double sqrt_pi = 1.7724538509055160273;
        double r[8];
        r[0] = 0.5 * tot[0];
        r[1] = -d.beta_d / sqrt_pi * tot[1];
        for (int k = 0; k < 6; ++k) r[2 + k] = tot[2 + k];
        for (int k = 0; k < 8; ++k) d.ctl->res[k] = r[k];
        if (d.ev)
            for (int k = 0; k < 8; ++k) d.ev[k] = r[k];
    }
}

}  // namespace pme

using namespace pme;

struct pme_real {
    int dev = 0;
    cudaStream_t stream = nullptr;
    double box[9] = {0}, recip[9] = {0}, vol = 0.0, beta = 0.0, rcut = 0.0;
    RealDev d;
    void *cell_mem = nullptr;  // counts, starts, fills, partials, control block (per box)
    size_t cell_bytes = 0;
    void *atom_mem = nullptr;  // per-atom scratch (grows with n)
    size_t atom_bytes = 0;
    int64_t n_cap = 0;
    RealCtl *h_ctl = nullptr;
    unsigned long long gen = 0;  // bumped whenever the kernels' arguments change (cell, scratch)
};

static size_t al256r(size_t x) { return (x + 255) & ~(size_t)255; }

// Cell grid and float constants for a box; PME_EUNSUPPORTED when rcut needs more than RS_MAX_R cells per
// axis or the grid has more than RS_MAX_CELLS cells.
static pme_status real_geometry(pme_real *rs, const double box[9]) {
    double recip[9], vol;
    if (!cell_reciprocal(box, recip, &vol)) return fail(PME_EINVAL, "box is singular");
    int nc[3], R[3];
    long long ncells = 1;
    for (int al = 0; al < 3; ++al) {
        const double astar = sqrt(recip[3 * al] * recip[3 * al] + recip[3 * al + 1] * recip[3 * al + 1] +
                                  recip[3 * al + 2] * recip[3 * al + 2]);
        const double wfrac = rs->rcut * astar * (1.0 + 1e-6);  // cutoff in fractional units, with slack
        nc[al] = wfrac < 1.0 ? (int)floor(1.0 / wfrac) : 1;
        if (nc[al] < 1) nc[al] = 1;
        R[al] = (int)ceil(wfrac * nc[al] - 1e-12);
        if (R[al] < 1) R[al] = 1;
        if (R[al] > RS_MAX_R)
            return fail(PME_EUNSUPPORTED, "rcut %.3g A spans %d cell widths along axis %d (at most %d)", rs->rcut, R[al], al,
                        RS_MAX_R);
        ncells *= nc[al];
    }
    if (ncells > RS_MAX_CELLS) return fail(PME_EUNSUPPORTED, "%lld cells (at most %d): rcut too small for this box", ncells, RS_MAX_CELLS);
    memcpy(rs->box, box, sizeof(rs->box));
    memcpy(rs->recip, recip, sizeof(recip));
    rs->vol = vol;
    RealDev &d = rs->d;
    for (int al = 0; al < 3; ++al) {
        d.nc[al] = nc[al];
        d.R[al] = R[al];
        for (int j = 0; j < 3; ++j) {
            d.rec[3 * al + j] = (float)recip[3 * al + j];
            const double a = box[3 * al + j];
            d.ahi[3 * al + j] = (float)a;
            d.alo[3 * al + j] = (float)(a - (double)(float)a);
        }
    }
    d.ncells = (int)ncells;
    return PME_OK;
}

static pme_status real_alloc_cells(pme_real *rs) {
    const size_t nc = (size_t)rs->d.ncells;
    size_t off = 0;
    const size_t o_cnt = off;  off = al256r(off + nc * 4);
    const size_t o_fill = off; off = al256r(off + nc * 4);
    const size_t o_st = off;   off = al256r(off + (nc + 1) * 4);
    const size_t o_par = off;  off = al256r(off + RS_RED_BLOCKS * 8 * sizeof(double));
    const size_t o_ctl = off;  off = al256r(off + sizeof(RealCtl));
    if (off > rs->cell_bytes) {
        if (rs->cell_mem) cudaFree(rs->cell_mem);
        rs->cell_mem = nullptr;
        rs->cell_bytes = 0;
        cudaError_t e = lib_malloc(&rs->cell_mem, off);
        if (e != cudaSuccess) {
            rs->cell_mem = nullptr;
            return fail(PME_ENOMEM, "cudaMalloc(%zu bytes): %s", off, cudaGetErrorString(e));
        }
        rs->cell_bytes = off;
    }
    cudaError_t e = cudaMemsetAsync(rs->cell_mem, 0, rs->cell_bytes, rs->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(cells)");
    char *b = (char *)rs->cell_mem;
    RealDev &d = rs->d;
    d.count = (unsigned *)(b + o_cnt);
    d.fill = (unsigned *)(b + o_fill);
    d.start = (unsigned *)(b + o_st);
    d.partials = (double *)(b + o_par);
    d.ctl = (RealCtl *)(b + o_ctl);
    return PME_OK;
}

static pme_status real_reserve(pme_real *rs, int64_t n) {
    if (n <= rs->n_cap && rs->atom_mem) return PME_OK;
    const size_t m = (size_t)(n > 0 ? n : 1);
    size_t off = 0;
    const size_t o_cell = off; off = al256r(off + m * 4);
    const size_t o_img = off;  off = al256r(off + m * 16);
    const size_t o_arec = off; off = al256r(off + m * 16);
    const size_t o_aidx = off; off = al256r(off + m * 16);
    const size_t o_srec = off; off = al256r(off + m * 16);
    const size_t o_sidx = off; off = al256r(off + m * 16);
    const size_t o_e = off;    off = al256r(off + m * 8);
    const size_t o_w = off;    off = al256r(off + m * 24);
    cudaError_t e = cudaStreamSynchronize(rs->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (rs->atom_mem) cudaFree(rs->atom_mem);
    rs->atom_mem = nullptr;
    rs->atom_bytes = 0;
    rs->n_cap = 0;
    if ((e = lib_malloc(&rs->atom_mem, off)) != cudaSuccess) {
        rs->atom_mem = nullptr;
        return fail(PME_ENOMEM, "cudaMalloc(%zu bytes): %s", off, cudaGetErrorString(e));
    }
    char *b = (char *)rs->atom_mem;
    RealDev &d = rs->d;
    d.cell = (int *)(b + o_cell);
    d.img = (int4 *)(b + o_img);
    d.arec = (float4 *)(b + o_arec);
    d.aidx = (int4 *)(b + o_aidx);
    d.srec = (float4 *)(b + o_srec);
    d.sidx = (int4 *)(b + o_sidx);
    d.e_atom = (double *)(b + o_e);
    d.w_atom = (float *)(b + o_w);
    rs->atom_bytes = off;
    rs->n_cap = (int64_t)m;
    ++rs->gen;
    return PME_OK;
}

static cudaError_t real_launch(const RealDev &d, cudaStream_t s) {
    const unsigned g = (unsigned)((d.n + 255) / 256);
    if (d.n > 0) {
        k_rs_bin<<<g, 256, 0, s>>>(d);
        k_rs_scan<<<1, RS_SCAN_THREADS, 0, s>>>(d);
        k_rs_scatter<<<g, 256, 0, s>>>(d);
        k_rs_rank<<<g, 256, 0, s>>>(d);
        k_rs_pairs<<<(unsigned)((d.n + RS_THREADS - 1) / RS_THREADS), RS_THREADS, 0, s>>>(d);
    }
    k_rs_reduce1<<<RS_RED_BLOCKS, 256, 0, s>>>(d);
    k_rs_reduce2<<<1, 256, 0, s>>>(d, RS_RED_BLOCKS);
    return cudaGetLastError();
}

extern "C" {

pme_status pme_real_create(const double box[9], double beta, double rcut, void *cuda_stream, pme_real **out) {
    if (!out) return fail(PME_EINVAL, "out is NULL");
    *out = nullptr;
    if (!box) return fail(PME_EINVAL, "box is NULL");
    if (!(beta > 0.0) || !isfinite(beta) || !(rcut > 0.0) || !isfinite(rcut))
        return fail(PME_EINVAL, "beta and rcut must be positive and finite");
    for (int i = 0; i < 9; ++i)
        if (!isfinite(box[i])) return fail(PME_EINVAL, "box has a non-finite entry");
    pme_real *rs = lib_new<pme_real>();
    if (!rs) return fail(PME_ENOMEM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&rs->dev);
    if (e != cudaSuccess) {
        delete rs;
        return cuda_fail(e, "cudaGetDevice");
    }
    rs->stream = (cudaStream_t)cuda_stream;
    rs->beta = beta;
    rs->rcut = rcut;
    memset(&rs->d, 0, sizeof(rs->d));
    rs->d.rc2 = (float)(rcut * rcut);
    rs->d.beta = (float)beta;
    rs->d.beta_d = beta;
    rs->d.c2 = (float)(2.0 * beta / 1.7724538509055160273);
    pme_status st;
    if ((st = real_geometry(rs, box)) != PME_OK || (st = real_alloc_cells(rs)) != PME_OK ||
        (st = real_reserve(rs, 1)) != PME_OK) {
        pme_real_destroy(rs);
        return st;
    }
    if ((e = lib_malloc_host((void **)&rs->h_ctl, sizeof(RealCtl))) != cudaSuccess) {
        rs->h_ctl = nullptr;
        pme_real_destroy(rs);
        return cuda_fail(e, "cudaMallocHost");
    }
    memset(rs->h_ctl, 0, sizeof(RealCtl));
    if ((e = cudaStreamSynchronize(rs->stream)) != cudaSuccess) {
        pme_real_destroy(rs);
        return cuda_fail(e, "cudaStreamSynchronize");
    }
    *out = rs;
    return PME_OK;
}

pme_status pme_real_set_box(pme_real *rs, const double box[9]) {
    if (!rs || !box) return fail(PME_EINVAL, "real-space context and box must be non-NULL");
    for (int i = 0; i < 9; ++i)
        if (!isfinite(box[i])) return fail(PME_EINVAL, "box has a non-finite entry");
    DeviceGuard g(rs->dev);
    cudaError_t e = cudaStreamSynchronize(rs->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    pme_status st = real_geometry(rs, box);
    if (st != PME_OK) return st;
    ++rs->gen;
    if ((st = real_alloc_cells(rs)) != PME_OK) return st;
    if ((e = cudaStreamSynchronize(rs->stream)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return PME_OK;
}

pme_status pme_real_reserve(pme_real *rs, int64_t n) {
    if (!rs) return fail(PME_EINVAL, "real-space context is NULL");
    if (n < 0 || n > (int64_t)0x3fffffff) return fail(PME_EINVAL, "n out of range");
    DeviceGuard g(rs->dev);
    return real_reserve(rs, n);
}

pme_status pme_real_enqueue(pme_real *rs, const float *pos, const float *q, int64_t n, float *forces, int accumulate,
                            double *ev_dev) {
    if (!rs) return fail(PME_EINVAL, "real-space context is NULL");
    return real_enqueue_on(rs, rs->stream, pos, q, n, forces, accumulate, ev_dev);
}

}  // extern "C"

// The same on a given stream (the multi-step loop runs everything on its plan's stream).
pme_status pme::real_enqueue_on(pme_real *rs, cudaStream_t stream, const float *pos, const float *q, int64_t n,
                                float *forces, int accumulate, double *ev_dev) {
    if (n < 0 || n > (int64_t)0x3fffffff) return fail(PME_EINVAL, "n = %lld out of range [0, 2^30)", (long long)n);
    if (n > 0 && (!pos || !q || !forces)) return fail(PME_EINVAL, "pos, q and forces must be non-NULL when n > 0");
    DeviceGuard g(rs->dev);
    pme_status st = real_reserve(rs, n);
    if (st != PME_OK) return st;
    RealDev d = rs->d;
    d.n = (int)n;
    d.pos = pos;
    d.q = q;
    d.forces = forces;
    d.accumulate = accumulate ? 1 : 0;
    d.ev = ev_dev;
    const cudaError_t e = real_launch(d, stream);
    if (e != cudaSuccess) return cuda_fail(e, "real-space kernel launch");
    return PME_OK;
}

pme_status pme::real_reserve_n(pme_real *rs, int64_t n) {
    DeviceGuard g(rs->dev);
    return real_reserve(rs, n);
}

int pme::real_device(const pme_real *rs) { return rs->dev; }
unsigned long long pme::real_gen(const pme_real *rs) { return rs->gen; }

extern "C" {

pme_status pme_real_compute(pme_real *rs, const float *pos, const float *q, int64_t n, float *forces,
                            double *e_real, double *e_self, double *virial) {
    pme_status st = pme_real_enqueue(rs, pos, q, n, forces, 0, nullptr);
    if (st != PME_OK) return st;
    DeviceGuard g(rs->dev);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(rs->h_ctl, rs->d.ctl, sizeof(RealCtl), cudaMemcpyDeviceToHost, rs->stream)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync(result)");
    if ((e = cudaStreamSynchronize(rs->stream)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    const unsigned bits = rs->h_ctl->status;
    if (bits) {
        cudaMemsetAsync(&rs->d.ctl->status, 0, sizeof(unsigned), rs->stream);
        cudaStreamSynchronize(rs->stream);
        return status_from_bits(bits);
    }
    if (e_real) *e_real = rs->h_ctl->res[0];
    if (e_self) *e_self = rs->h_ctl->res[1];
    if (virial)
        for (int k = 0; k < 6; ++k) virial[k] = rs->h_ctl->res[2 + k];
    return PME_OK;
}

void pme_real_destroy(pme_real *rs) {
    if (!rs) return;
    DeviceGuard g(rs->dev);
    cudaStreamSynchronize(rs->stream);
    if (rs->cell_mem) cudaFree(rs->cell_mem);
    if (rs->atom_mem) cudaFree(rs->atom_mem);
    if (rs->h_ctl) cudaFreeHost(rs->h_ctl);
    delete rs;
}

}  // extern "C"
