// Step-kernel instantiations for stencil radius 4 (space order 8).
#include "fdw_internal.h"
#include "fdw_step.cuh"

namespace fdw {

const void* step_kernel_r4(int tile, bool grad) {
  switch (tile) {
    case 0: return grad ? (const void*)&step_kernel<4, 1, 4, true, true>
                          : (const void*)&step_kernel<4, 1, 4, false, true>;
    case 1: return grad ? (const void*)&step_kernel<4, 2, 4, true, false>
                          : (const void*)&step_kernel<4, 2, 4, false, false>;
    case 2: return grad ? (const void*)&step_kernel<4, 1, 8, true, true>
                          : (const void*)&step_kernel<4, 1, 8, false, true>;
    case 3: return grad ? (const void*)&step_kernel<4, 1, 1, true, false>
                          : (const void*)&step_kernel<4, 1, 1, false, false>;
    case 4: return grad ? (const void*)&step_kernel<4, 1, 4, true, false>
                          : (const void*)&step_kernel<4, 1, 4, false, false>;
    case 5: return grad ? (const void*)&step_kernel<4, 2, 2, true, false>
                          : (const void*)&step_kernel<4, 2, 2, false, false>;
    case 6: return grad ? (const void*)&step_kernel<4, 1, 4, true, false>
                          : (const void*)&step_kernel<4, 1, 4, false, false, true>;
    case 7: return grad ? (const void*)&step_kernel<4, 1, 4, true, false, true, true>
                          : (const void*)&step_kernel<4, 1, 4, false, false, false, true>;
    case 8: return grad ? (const void*)&step_kernel<4, 1, 4, true, false, true, true>
                          : (const void*)&step_kernel<4, 1, 4, false, false, true, true>;
    case 9: return grad ? (const void*)&step_kernel<4, 1, 4, true, false, false, true, true>
                          : (const void*)&step_kernel<4, 1, 4, false, false, false, true, true>;
    default: return nullptr;
  }
}

}  // namespace fdw
