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

extern "C" {

// One or more evaluations (repeat >= 1, same inputs) of the emulated pipeline. Outputs: forces (n*3),
// ev[7], and optionally the fixed-point mesh as spread (grid_out, K1*K2*K3 int64) and phi (K1*K2*K3).
// Returns the device status bits of the last evaluation, or -1 / -2 for invalid / unsupported input.
int emu_spme(int64_t n, const float *pos, const float *q, const int K[3], int p, double beta, const double box[9],
             int cap_override, int repeat, float *forces, double *ev, long long *grid_out, float *phi_out,
             int tile_log) {
    char msg[256];
    int v = validate_params(K, p, beta, box, msg, sizeof(msg));
    if (v) return -v;
    double recip[9], vol;
    if (!cell_reciprocal(box, recip, &vol)) return -1;
    EmuState s;
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
    set_tiling(d, tile_log > 0 ? tile_log : choose_tile_log(n > 0 ? n : 1, K));
    s.bcount.assign(bcount_bytes(d.ntiles) / sizeof(unsigned), 0u);
    s.partials.assign(partials_bytes(d) / sizeof(double), 0.0);
    const int cap = cap_override > 0 ? cap_override : bucket_capacity(n > 0 ? n : 1, d.ntiles);
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
    d.partials = s.partials.data();
    d.ctl = &s.ctl;
    d.bka = s.bka.data();
    d.bkb = s.bkb.data();
    d.ova = s.ova.data();
    d.ovb = s.ovb.data();
    d.cap = cap;
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
    bool clean = s.ctl.novf == 0 && s.ctl.qabs == 0;
    for (unsigned c : s.bcount) clean = clean && c == 0;
    for (unsigned long long g : s.grid) clean = clean && g == 0;
    if (!clean) status |= 0x100u;
    return (int)status;
}

}  // extern "C"
