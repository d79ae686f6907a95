// Host interface of the grouped stage kernels (group.cu): every system of a group has the same mesh shape
// and B-spline order, so one launch per stage covers the whole group.
#pragma once

#include <cuda_runtime.h>

#include "kernels.h"

namespace pme {

struct GroupArgs {
    const SysDev *sys;  // the group's descriptors (device memory, nsys entries)
    int ips;            // work items per system of the launched stage
    int late;           // when the programmatic launch of the successor is triggered (PdlScope)
};

// Raise the dynamic shared-memory limits of the grouped kernels (once per device).
cudaError_t configure_group_kernels();

// Work items of one system in a stage (binning: of this system's atoms).
int group_items(const SysDev &d, int stage);

// Enqueue the six stages for nsys systems whose descriptors are at sys_dev (device), all shaped like
// proto; max_nbin is the largest binning item count among them.
cudaError_t launch_group_chain(const SysDev *sys_dev, int nsys, const SysDev &proto, int max_nbin, cudaStream_t s);

}  // namespace pme
