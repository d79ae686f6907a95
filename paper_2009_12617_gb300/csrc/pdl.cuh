// Programmatic dependent launch helpers shared by the stage kernels.
#pragma once

namespace pme {

// A stage kernel launched with programmatic stream serialisation (launch modes 1-3) waits for its
// predecessor to complete, with its memory visible, before touching any data, and lets its successor start
// launching at its own start (mode 1: the successor's CTAs may then become resident in a cascade down the
// whole chain), right after its own wait (mode 3: the successor's CTAs become resident and wait while this
// kernel works, one level deep) or once each CTA has finished its work (mode 2), so the successor's launch
// latency overlaps this kernel. Without the launch attribute (mode 0) both instructions are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
// when: 0 trigger before the wait, 1 at CTA exit, 2 right after the wait
struct PdlScope {
    int when;
    __device__ explicit PdlScope(int w) : when(w) {
        if (when == 0) pdl_trigger();
        pdl_wait();
        if (when == 2) pdl_trigger();
    }
    __device__ ~PdlScope() {
        if (when == 1) pdl_trigger();
    }
};

}  // namespace pme
