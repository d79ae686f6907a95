// Shared definitions of the persistent batched kernel, used by the batch API and the server.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/pme.h"
#include "common.cuh"
#include "kernels.h"

namespace pme {

constexpr int NT_BATCH = NT_CONV;  // same CTA size as the single-system influence stage: identical sums

struct BatchEntry {
    unsigned short sys, stage;  // system index in the launch, stage
    int begin, end;             // the stage's work items [begin, end), run one after another
};

struct BatchCtrl {
    unsigned head;    // next list entry to take
    unsigned exited;  // CTAs that found the list empty
    unsigned abort;   // a wait gave up: every later wait returns at once
    unsigned pad;
};

struct BatchArgs {
    SysDev *sys;                // nsys descriptors with absolute atom pointers
    const BatchEntry *entries;  // nentries
    const unsigned *count;      // work items per (system, stage)
    unsigned *done;             // finished work items per (system, stage)
    BatchCtrl *ctrl;
    int nsys, nentries;
    unsigned long long wait_ns;  // bound of every dependency wait
    int stall_entry;             // test hook: this entry waits on a count nothing reaches (-1: off)
};

// Device + pinned host state of one persistent launch.
struct WaveState {
    int dev = 0, cap_sys = 0;
    size_t cap_entries = 0, bytes = 0, head_bytes = 0;
    void *dmem = nullptr, *hmem = nullptr;
    SysDev *d_sys = nullptr, *h_sys = nullptr;
    BatchEntry *d_entries = nullptr, *h_entries = nullptr;
    unsigned *d_count = nullptr, *h_count = nullptr, *d_done = nullptr;
    BatchCtrl *d_ctrl = nullptr;
    double *d_ev = nullptr, *h_ev = nullptr;
    unsigned *d_status = nullptr, *h_status = nullptr;

    pme_status init(int dev, int cap_sys, size_t cap_entries);
    void release();
    cudaError_t upload(size_t nentries, cudaStream_t s) const;  // descriptors, counts, used list entries
    BatchArgs args(int nsys, int nentries, unsigned long long wait_ns, int stall_entry) const;
};

int stage_items(const SysDev &d, int stage);
void build_work_list(const std::vector<SysDev> &sys, std::vector<BatchEntry> &entries, std::vector<unsigned> &count);
size_t batch_smem(const std::vector<SysDev> &sys);
cudaError_t configure_batch_kernel();
int batch_grid(int dev, int p, size_t smem);
cudaError_t launch_batch(const BatchArgs &a, int p, int grid, size_t smem, cudaStream_t s);
int first_waiting_entry(const std::vector<BatchEntry> &entries);
cudaError_t launch_collect_status(const SysDev *sys, int nsys, unsigned *out, cudaStream_t s);
pme_status plan_recover(pme_plan *pl, cudaStream_t s);

}  // namespace pme
