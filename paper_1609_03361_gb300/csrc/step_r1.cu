// Step-kernel instantiations for stencil radius 1 (space order 2).
#include "fdw_internal.h"
#include "fdw_step.cuh"

namespace fdw {

const void* step_kernel_r1(int tile, bool grad) {
  switch (tile) {
    case 0: return grad ? (const void*)&step_kernel<1, 1, 8, true> : (const void*)&step_kernel<1, 1, 8, false>;
    case 1: return grad ? (const void*)&step_kernel<1, 2, 8, true> : (const void*)&step_kernel<1, 2, 8, false>;
    case 2: return grad ? (const void*)&step_kernel<1, 2, 4, true> : (const void*)&step_kernel<1, 2, 4, false>;
    case 3: return grad ? (const void*)&step_kernel<1, 1, 1, true> : (const void*)&step_kernel<1, 1, 1, false>;
    default: return nullptr;
  }
}

}  // namespace fdw
