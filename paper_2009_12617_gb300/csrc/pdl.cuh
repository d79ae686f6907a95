// Programmatic dependent launch helpers shared by the stage kernels.
#pragma once

namespace pme {

// A stage kernel launched with programmatic stream serialisation (launch modes 1 and 2) waits for its
// predecessor to complete, with its memory visible, before touching any data, and lets its successor start
// launching either at its own start (mode 1) or once each CTA has finished its work (mode 2), so the
// successor's launch latency overlaps this kernel. Without the launch attribute (mode 0) both instructions
// are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
struct PdlScope {  // trigger at entry (early) or at exit (late); the kernel argument picks
    bool late;
    __device__ explicit PdlScope(bool l) : late(l) {
        if (!late) pdl_trigger();
        pdl_wait();
    }
    __device__ ~PdlScope() {
        if (late) pdl_trigger();
    }
};

}  // namespace pme
