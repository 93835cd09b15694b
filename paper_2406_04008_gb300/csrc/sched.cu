// Device side of the captured level schedule (Sec. 4.3: the coarse-to-fine loop over the resolution
// pyramid).  collage_run_schedule captures the whole run as one CUDA graph: per level, the level
// switch (container raster and the distribution term's tile lists), then a conditional WHILE node
// whose body is a few iterations (a divisor of the level's count).  The loop condition is decided
// on the device: these kernels compare
// the iterations completed in this run (Adam step count now against the count when the run began)
// with the run's cumulative target through the level, and stop the loop once the status word has
// latched a bin overflow or non-finite params, so that the host can resume from exactly the
// iteration that did not complete.
#include "internal.h"

namespace collage {

// The Adam step count when the run began.
__global__ void k_sched_begin(Dev d) { *d.sched_base = *d.step; }

// Sets the level's loop condition: 1 while fewer than `target` iterations of this run have
// completed and nothing has latched.  Launched once before the WHILE node (so a level of zero
// iterations runs no body) and as the last kernel of each body.
__global__ void k_sched_cond(Dev d, cudaGraphConditionalHandle cond, int target) {
  const int done = *d.step - *d.sched_base;
  const bool ok = (*d.status & (kStatusVoid | kStatusInternal)) == 0;
  cudaGraphSetConditional(cond, ok && done < target ? 1u : 0u);
}

cudaError_t launch_sched_begin(const Dev& d, cudaStream_t s) {
  k_sched_begin<<<1, 1, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_sched_cond(const Dev& d, cudaStream_t s, cudaGraphConditionalHandle cond, int target) {
  k_sched_cond<<<1, 1, 0, s>>>(d, cond, target);
  return cudaGetLastError();
}

}  // namespace collage
