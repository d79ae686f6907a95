// CPU emulation of the SPME stage bodies, for tests only.
//
// Compiles the library's stage bodies (paper_2009_12617_gb300/csrc/stages.cuh) as plain C++ with
// PME_HOST_EMULATION: every work item runs as one CTA of one thread, items run in order, and CTA barriers
// vanish. Each phase of a stage body is a data-parallel loop, so this executes exactly the index
// arithmetic and the FP32 math of the kernels (without fma contraction or GPU atomics ordering), which
// lets CPU tests compare the pipeline with the FP64 oracle before any GPU run. Not part of the library.
#define PME_HOST_EMULATION 1
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../paper_2009_12617_gb300/csrc/host_tables.h"
#include "../../paper_2009_12617_gb300/csrc/stages.cuh"

using namespace pme;

struct EmuState {
    SysDev d;
    std::vector<unsigned long long> grid;
    std::vector<float2> spec, tw;
    std::vector<float4> bc;
    std::vector<float> phi;
    std::vector<unsigned> bcount;
    std::vector<unsigned long long> qslot;
    std::vector<double> partials;
    std::vector<float4> bka, ova;
    std::vector<int2> bkb, ovb;
    Ctl ctl;
    std::vector<unsigned char> smem;
};

// Tile items alternate between the two ways the library calls the tile bodies: as the per-stage kernels do
// (shared memory cleared and the tile origin decoded before the programmatic-launch wait, then passed in) and
// as the batch and allocation-free paths do (the body does both itself). Results must not depend on it.
template <int P, int T>
static void spread_item(const SysDev &d, int it, void *sp) {
    if (it % 2 == 0) {
        spread_clear<P, T>(sp);
        int org[3] = {0, 0, 0};
        if (it < d.ntiles) tile_origin(d, it, org[0], org[1], org[2]);
        stage_spread<P, T>(d, it, sp, true, org);
    } else {
        stage_spread<P, T>(d, it, sp);
    }
}
template <int P, int T>
static void gather_item(const SysDev &d, int it, void *sp) {
    if (it % 2 == 0) {
        int org[3] = {0, 0, 0};
        if (it < d.ntiles) tile_origin(d, it, org[0], org[1], org[2]);
        stage_gather<P, T>(d, it, sp, org);
    } else {
        stage_gather<P, T>(d, it, sp);
    }
}

// Pieces of the k1 axis for the tiles of later emu_setup calls (0: the fewest, as set_tiling's default).
static int g_k1_pieces = 0;

// The emulated resident state of one system (as pme_create + pme_reserve build it on the device).
// Returns 0, or -1 / -2 for invalid / unsupported input.
static int emu_setup(EmuState &s, int64_t n, const int K[3], int p, double beta, const double box[9], int cap_override,
                     int tile_log) {
    char msg[256];
    int v = validate_params(K, p, beta, box, msg, sizeof(msg));
    if (v) return -v;
    double recip[9], vol;
    if (!cell_reciprocal(box, recip, &vol)) return -1;
    memset(&s.d, 0, sizeof(s.d));
    memset(&s.ctl, 0, sizeof(s.ctl));
    SysDev &d = s.d;
    fill_geometry(d, K, p, beta, recip);
    const size_t K1 = K[0], K2 = K[1], K3 = K[2], H3 = d.H3, Nh = K3 / 2;
    s.grid.assign(K1 * K2 * K3, 0ull);
    s.spec.assign(K1 * K2 * H3, make_float2(0, 0));
    s.phi.assign(K1 * K2 * K3, 0.f);
    s.bc.resize(K1 * K2 * H3);
    make_influence(K, p, beta, recip, vol, s.bc.data());
    s.tw.resize(K1 + K2 + Nh + Nh + 1);
    make_twiddles(K[0], K[0], s.tw.data());
    make_twiddles(K[1], K[1], s.tw.data() + K1);
    make_twiddles((int)Nh, (int)Nh, s.tw.data() + K1 + K2);
    make_twiddles(K[2], (int)Nh + 1, s.tw.data() + K1 + K2 + Nh);
    set_tiling(d, tile_log > 0 ? tile_log : choose_tile_log(n > 0 ? n : 1, K, 0), g_k1_pieces);
    s.bcount.assign(bcount_bytes(d.ntiles) / sizeof(unsigned), 0u);
    s.qslot.assign(QABS_BYTES / sizeof(unsigned long long), 0ull);
    s.partials.assign(partials_bytes(d) / sizeof(double), 0.0);
    const int cap = cap_override > 0 ? cap_override : bucket_capacity(n > 0 ? n : 1, d.ntiles, d.tlog);
    s.bka.resize((size_t)d.ntiles * cap);
    s.bkb.resize((size_t)d.ntiles * cap);
    s.ova.resize(n > 0 ? n : 1);
    s.ovb.resize(n > 0 ? n : 1);
    size_t sm = std::max({smem_bin(1), smem_spread(p, d.tlog), smem_gather_all(p, d.tlog), smem_slab(K[1], K[2]), smem_inv(K[1], K[2]), smem_conv(K[0], 1)});
    s.smem.assign(sm, 0);
    d.grid = s.grid.data();
    d.spec = s.spec.data();
    d.phi = s.phi.data();
    d.bc = s.bc.data();
    d.tw1 = s.tw.data();
    d.tw2 = s.tw.data() + K1;
    d.tw3h = s.tw.data() + K1 + K2;
    d.tw3 = s.tw.data() + K1 + K2 + Nh;
    d.bcount = s.bcount.data();
    d.qslot = s.qslot.data();
    d.partials = s.partials.data();
    d.ctl = &s.ctl;
    d.bka = s.bka.data();
    d.bkb = s.bkb.data();
    d.ova = s.ova.data();
    d.ovb = s.ovb.data();
    d.cap = cap;
    return 0;
}

extern "C" {

void emu_set_k1_pieces(int n) { g_k1_pieces = n; }

// Spreading region layout for order p and tile edge 2^tlog: row stride, plane stride, accumulator length
// (ints) and whether one warp spreads one atom at a time.
void emu_spread_layout(int p, int tlog, int *out) {
    out[0] = spread_row(p, tlog);
    out[1] = spread_plane(p, tlog);
    out[2] = spread_vol(p, tlog);
    out[3] = spread_warp_lanes(p, tlog) ? 1 : 0;
}

// One or more evaluations (repeat >= 1, same inputs) of the emulated pipeline. Outputs: forces (n*3),
// ev[7], and optionally the fixed-point mesh as spread (grid_out, K1*K2*K3 int64) and phi (K1*K2*K3).
// Returns the device status bits of the last evaluation, or -1 / -2 for invalid / unsupported input.
int emu_spme(int64_t n, const float *pos, const float *q, const int K[3], int p, double beta, const double box[9],
             int cap_override, int repeat, float *forces, double *ev, long long *grid_out, float *phi_out,
             int tile_log) {
    EmuState s;
    const int rc = emu_setup(s, n, K, p, beta, box, cap_override, tile_log);
    if (rc) return rc;
    SysDev &d = s.d;
    d.n = (int)n;
    d.nbin = (int)((n + BIN_CHUNK - 1) / BIN_CHUNK);
    d.pos = pos;
    d.q = q;
    d.forces = forces;
    d.ev = s.ctl.ev;
    void *sp = s.smem.data();
    unsigned status = 0;
    for (int rep = 0; rep < (repeat > 0 ? repeat : 1); ++rep) {
        for (int it = 0; it < (d.nbin > 0 ? d.nbin : 1); ++it) stage_bin(d, it, sp);
        for (int it = 0; it < d.ntiles + OVF_ITEMS; ++it) {
            const int key = p * 10 + d.tlog;
            switch (key) {
                case 43: spread_item<4, 8>(d, it, sp); break;
                case 53: spread_item<5, 8>(d, it, sp); break;
                case 54: spread_item<5, 16>(d, it, sp); break;
                case 63: spread_item<6, 8>(d, it, sp); break;
                case 83: spread_item<8, 8>(d, it, sp); break;
                case 44: spread_item<4, 16>(d, it, sp); break;
                case 64: spread_item<6, 16>(d, it, sp); break;
                default: spread_item<8, 16>(d, it, sp); break;
            }
        }
        if (grid_out) memcpy(grid_out, s.grid.data(), s.grid.size() * 8);
        for (int it = 0; it < K[0]; ++it) stage_fwd(d, it, sp);
        for (int it = 0; it < d.nconv; ++it) stage_conv(d, it, sp);
        for (int it = 0; it < K[0]; ++it) stage_inv(d, it, sp);
        for (int it = 0; it < d.ntiles + OVF_ITEMS; ++it) {
            const int key = p * 10 + d.tlog;
            switch (key) {
                case 43: gather_item<4, 8>(d, it, sp); break;
                case 53: gather_item<5, 8>(d, it, sp); break;
                case 54: gather_item<5, 16>(d, it, sp); break;
                case 63: gather_item<6, 8>(d, it, sp); break;
                case 83: gather_item<8, 8>(d, it, sp); break;
                case 44: gather_item<4, 16>(d, it, sp); break;
                case 64: gather_item<6, 16>(d, it, sp); break;
                default: gather_item<8, 16>(d, it, sp); break;
            }
        }
        status = s.ctl.status;
        s.ctl.status = 0;
    }
    for (int c = 0; c < 7; ++c) ev[c] = s.ctl.ev[c];
    if (phi_out) memcpy(phi_out, s.phi.data(), s.phi.size() * 4);
    // every self-resetting counter must be back at zero after an evaluation
    bool clean = s.ctl.novf == 0;
    for (unsigned long long v : s.qslot) clean = clean && v == 0;
    for (unsigned c : s.bcount) clean = clean && c == 0;
    for (unsigned long long g : s.grid) clean = clean && g == 0;
    if (!clean) status |= 0x100u;
    return (int)status;
}


// Slab decomposition (the library's pme_slab_* calls), one rank of P: the same stage bodies with the rank's
// plane window and item ranges, the corner-turn blocks packed and unpacked by the library's own helpers.
struct EmuSlab {
    EmuState s;
    SlabLayout L;
    int rank = 0;
};

static void emu_spread_all(EmuState &s, int p) {
    SysDev &d = s.d;
    void *sp = s.smem.data();
    for (int it = 0; it < d.ntiles + OVF_ITEMS; ++it) {
        switch (p * 10 + d.tlog) {
            case 43: spread_item<4, 8>(d, it, sp); break;
            case 53: spread_item<5, 8>(d, it, sp); break;
            case 63: spread_item<6, 8>(d, it, sp); break;
            case 83: spread_item<8, 8>(d, it, sp); break;
            case 44: spread_item<4, 16>(d, it, sp); break;
            case 54: spread_item<5, 16>(d, it, sp); break;
            case 64: spread_item<6, 16>(d, it, sp); break;
            default: spread_item<8, 16>(d, it, sp); break;
        }
    }
}

static void emu_gather_all(EmuState &s, int p) {
    SysDev &d = s.d;
    void *sp = s.smem.data();
    for (int it = 0; it < d.ntiles + OVF_ITEMS; ++it) {
        switch (p * 10 + d.tlog) {
            case 43: gather_item<4, 8>(d, it, sp); break;
            case 53: gather_item<5, 8>(d, it, sp); break;
            case 63: gather_item<6, 8>(d, it, sp); break;
            case 83: gather_item<8, 8>(d, it, sp); break;
            case 44: gather_item<4, 16>(d, it, sp); break;
            case 54: gather_item<5, 16>(d, it, sp); break;
            case 64: gather_item<6, 16>(d, it, sp); break;
            default: gather_item<8, 16>(d, it, sp); break;
        }
    }
}

void *emu_slab_create(int64_t n, const int K[3], int p, double beta, const double box[9], int P, int rank) {
    EmuSlab *e = new EmuSlab();
    if (emu_setup(e->s, n, K, p, beta, box, 0, 0) != 0 || !make_slab_layout(e->s.d, P, e->L) || rank < 0 || rank >= P) {
        delete e;
        return nullptr;
    }
    e->rank = rank;
    e->s.d.k1_lo = e->L.plane0[rank];
    e->s.d.k1_hi = e->L.plane0[rank + 1];
    return e;
}

void emu_slab_destroy(void *h) { delete (EmuSlab *)h; }

// block_values, and the rank's planes and columns
int64_t emu_slab_layout(void *h, int *planes, int *cols) {
    EmuSlab *e = (EmuSlab *)h;
    planes[0] = e->L.plane0[e->rank];
    planes[1] = e->L.plane0[e->rank + 1];
    cols[0] = e->L.col0[e->rank];
    cols[1] = e->L.col0[e->rank + 1];
    return (int64_t)e->L.maxS * e->L.maxW;
}

int emu_slab_stage1(void *h, int64_t n, const float *pos, const float *q, float *send) {
    EmuSlab *e = (EmuSlab *)h;
    SysDev &d = e->s.d;
    const int r = e->rank, p = d.p, ncol = d.K2 * d.H3;
    d.n = (int)n;
    d.nbin = (int)((n + BIN_CHUNK - 1) / BIN_CHUNK);
    d.pos = pos;
    d.q = q;
    void *sp = e->s.smem.data();
    for (int it = 0; it < (d.nbin > 0 ? d.nbin : 1); ++it) stage_bin(d, it, sp);
    emu_spread_all(e->s, p);
    for (int k1 = e->L.plane0[r]; k1 < e->L.plane0[r + 1]; ++k1) stage_fwd(d, k1, sp);
    float2 *buf = (float2 *)send;
    for (int s = 0; s < e->L.P; ++s)
        slab_pack(d.spec, ncol, e->L.plane0[r], e->L.plane0[r + 1], e->L.col0[s], e->L.col0[s + 1],
                  buf + (size_t)s * e->L.maxS * e->L.maxW, 0, 1);
    return (int)e->s.ctl.status;
}

int emu_slab_stage2(void *h, const float *recv, float *send, double *ev7) {
    EmuSlab *e = (EmuSlab *)h;
    SysDev &d = e->s.d;
    const int r = e->rank, ncol = d.K2 * d.H3;
    void *sp = e->s.smem.data();
    const float2 *in = (const float2 *)recv;
    for (int s = 0; s < e->L.P; ++s)
        slab_unpack(d.spec, ncol, e->L.plane0[s], e->L.plane0[s + 1], e->L.col0[r], e->L.col0[r + 1],
                    in + (size_t)s * e->L.maxS * e->L.maxW, 0, 1);
    for (int it = e->L.item0[r]; it < e->L.item0[r + 1]; ++it) stage_conv(d, it, sp);
    for (int c = 0; c < 7; ++c) slab_energy(d, e->L.item0[r], e->L.item0[r + 1], ev7, c);
    float2 *out = (float2 *)send;
    for (int s = 0; s < e->L.P; ++s)
        slab_pack(d.spec, ncol, e->L.plane0[s], e->L.plane0[s + 1], e->L.col0[r], e->L.col0[r + 1],
                  out + (size_t)s * e->L.maxS * e->L.maxW, 0, 1);
    return 0;
}

int emu_slab_stage3(void *h, const float *recv, float *forces) {
    EmuSlab *e = (EmuSlab *)h;
    SysDev &d = e->s.d;
    const int r = e->rank, ncol = d.K2 * d.H3;
    void *sp = e->s.smem.data();
    const float2 *in = (const float2 *)recv;
    for (int s = 0; s < e->L.P; ++s)
        slab_unpack(d.spec, ncol, e->L.plane0[r], e->L.plane0[r + 1], e->L.col0[s], e->L.col0[s + 1],
                    in + (size_t)s * e->L.maxS * e->L.maxW, 0, 1);
    for (int k1 = e->L.plane0[r]; k1 < e->L.plane0[r + 1]; ++k1) stage_inv(d, k1, sp);
    d.forces = forces;
    d.ev = e->s.ctl.ev;
    emu_gather_all(e->s, d.p);
    e->s.ctl.novf = 0;
    const unsigned st = e->s.ctl.status;
    e->s.ctl.status = 0;
    return (int)st;
}

}  // extern "C"
