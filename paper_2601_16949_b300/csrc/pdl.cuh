// Programmatic dependent launch inside the step graph.
//
// The propagation step is captured once as a CUDA graph whose consecutive
// kernel nodes are joined by programmatic edges: a kernel may be launched
// (its CTAs made resident) while the kernel before it is still running, so
// the launch latency of each of the step's few dozen nodes overlaps the
// previous node's execution.  Every kernel that can sit in that graph
// therefore begins with pdl_entry(): griddepcontrol.wait blocks until the
// preceding grid has completed and its writes are visible (a no-op when the
// kernel was launched with an ordinary dependency), and only then does
// griddepcontrol.launch_dependents allow the next grid to be launched.  The
// wait is the hardware's own grid-completion dependency, not a spin on a
// flag; the trigger after the wait keeps at most two grids in flight, and
// completion is transitive along the chain.
#pragma once

__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
