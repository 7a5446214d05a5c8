// Step-kernel instantiations for stencil radius 6 (space order 12).
#include "fdw_internal.h"
#include "fdw_step.cuh"

namespace fdw {

const void* step_kernel_r6(int tile, bool grad) {
  switch (tile) {
    case 0: return grad ? (const void*)&step_kernel<6, 1, 8, true> : (const void*)&step_kernel<6, 1, 8, false>;
    case 1: return grad ? (const void*)&step_kernel<6, 2, 8, true> : (const void*)&step_kernel<6, 2, 8, false>;
    case 2: return grad ? (const void*)&step_kernel<6, 2, 4, true> : (const void*)&step_kernel<6, 2, 4, false>;
    case 3: return grad ? (const void*)&step_kernel<6, 1, 1, true> : (const void*)&step_kernel<6, 1, 1, false>;
    default: return nullptr;
  }
}

}  // namespace fdw
