// Device-side primitives for sm_103a: mbarrier pipeline and TMA tensor loads
// written as inline PTX.  Every wait is bounded: it gives up after a clock
// budget and the caller records an error instead of spinning forever.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "fdw_types.h"

namespace fdw {

// Clock budget of one wait (about 2 s at 2 GHz).
constexpr long long kWaitBudget = 4000000000LL;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// As mbar_try_wait, but the thread may be suspended in hardware for up to
// `hint_ns` while the phase is incomplete (woken when it completes), instead
// of returning at once and spinning in issue slots.
__device__ __forceinline__ bool mbar_try_wait_suspend(uint32_t bar, uint32_t parity,
                                                      uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* m) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(m)) : "memory");
}

// 3D / 4D tiled tensor loads into shared memory, completing on an mbarrier.
// The innermost coordinate c0 must be a multiple of 16 bytes / element size.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* m, int c0, int c1,
                                            int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* m, int c0, int c1,
                                            int c2, int c3, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

// Cross-CTA completion counters in global memory (gpu scope).
__device__ __forceinline__ int ld_relaxed_gpu(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void fence_acq_rel_gpu() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}
__device__ __forceinline__ void red_release_add_gpu(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Orders this thread's view of global memory (generic proxy, e.g. values made
// visible by an acquire) before its later tensor (async proxy) loads.
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Named barrier among the first `nthreads` threads (consumer warps only).
__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// ---------------------------------------------------------------- tensor memory
// Tensor memory (TMEM, 128 lanes x 512 columns of 32 bits per SM) used as a
// per-thread store: in the 32x32b access shape, warp w of a warpgroup reaches
// lanes 32 (w % 4) .. + 31, one lane per thread, so each thread owns one row
// of columns of the CTA's allocation.  All of these are warp-collective
// (.sync.aligned): every lane of the warp executes them together.

// Allocate ncols columns (a power of two, 32..512) for the CTA; one warp
// executes it and the address is written to shared memory at dst.  Every CTA
// that allocates frees the same columns before it exits (tmem_dealloc).
__device__ __forceinline__ void tmem_alloc(uint32_t dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// Order tensor-memory accesses around a CTA-wide thread barrier.
__device__ __forceinline__ void tmem_fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Four 32-bit values of the thread into columns taddr .. taddr + 3 of its lane.
__device__ __forceinline__ void tmem_st4(uint32_t taddr, float4 v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
               "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y)), "r"(__float_as_uint(v.z)),
               "r"(__float_as_uint(v.w))
               : "memory");
}

__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// N (8, 16, 32 or 64) consecutive columns of the thread's lane from taddr,
// after every earlier tensor-memory store of the thread has completed; the
// values are valid when the call returns (the load and its wait are one
// statement, so no use of them can be scheduled before the wait).
#define FDW_TMEM_R8(i) "=r"(d[i + 0]), "=r"(d[i + 1]), "=r"(d[i + 2]), "=r"(d[i + 3]), \
    "=r"(d[i + 4]), "=r"(d[i + 5]), "=r"(d[i + 6]), "=r"(d[i + 7])
template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t (&d)[N]);
template <>
__device__ __forceinline__ void tmem_ld<8>(uint32_t taddr, uint32_t (&d)[8]) {
  asm volatile(
      "tcgen05.wait::st.sync.aligned;\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : FDW_TMEM_R8(0)
      : "r"(taddr)
      : "memory");
}
template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t taddr, uint32_t (&d)[16]) {
  asm volatile(
      "tcgen05.wait::st.sync.aligned;\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : FDW_TMEM_R8(0), FDW_TMEM_R8(8)
      : "r"(taddr)
      : "memory");
}
template <>
__device__ __forceinline__ void tmem_ld<32>(uint32_t taddr, uint32_t (&d)[32]) {
  asm volatile(
      "tcgen05.wait::st.sync.aligned;\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : FDW_TMEM_R8(0), FDW_TMEM_R8(8), FDW_TMEM_R8(16), FDW_TMEM_R8(24)
      : "r"(taddr)
      : "memory");
}
template <>
__device__ __forceinline__ void tmem_ld<64>(uint32_t taddr, uint32_t (&d)[64]) {
  asm volatile(
      "tcgen05.wait::st.sync.aligned;\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, "
      "%45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, "
      "%62, %63}, [%64];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : FDW_TMEM_R8(0), FDW_TMEM_R8(8), FDW_TMEM_R8(16), FDW_TMEM_R8(24), FDW_TMEM_R8(32),
        FDW_TMEM_R8(40), FDW_TMEM_R8(48), FDW_TMEM_R8(56)
      : "r"(taddr)
      : "memory");
}
#undef FDW_TMEM_R8

// Issue-only loads: the values arrive asynchronously; tmem_wait_ld(d) must
// come before any use (it names the registers, so no use can move above it).
#define FDW_TMEM_R8(i) "=r"(d[i + 0]), "=r"(d[i + 1]), "=r"(d[i + 2]), "=r"(d[i + 3]), \
    "=r"(d[i + 4]), "=r"(d[i + 5]), "=r"(d[i + 6]), "=r"(d[i + 7])
#define FDW_TMEM_W8(i) "+r"(d[i + 0]), "+r"(d[i + 1]), "+r"(d[i + 2]), "+r"(d[i + 3]), \
    "+r"(d[i + 4]), "+r"(d[i + 5]), "+r"(d[i + 6]), "+r"(d[i + 7])
template <int N>
__device__ __forceinline__ void tmem_ld_issue(uint32_t taddr, uint32_t (&d)[N]);
template <int N>
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&d)[N]);
template <>
__device__ __forceinline__ void tmem_ld_issue<8>(uint32_t taddr, uint32_t (&d)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : FDW_TMEM_R8(0)
               : "r"(taddr)
               : "memory");
}
template <>
__device__ __forceinline__ void tmem_wait_ld<8>(uint32_t (&d)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : FDW_TMEM_W8(0)
               :
               : "memory");
}
template <>
__device__ __forceinline__ void tmem_ld_issue<16>(uint32_t taddr, uint32_t (&d)[16]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
               : FDW_TMEM_R8(0), FDW_TMEM_R8(8)
               : "r"(taddr)
               : "memory");
}
template <>
__device__ __forceinline__ void tmem_wait_ld<16>(uint32_t (&d)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : FDW_TMEM_W8(0), FDW_TMEM_W8(8)
               :
               : "memory");
}
template <>
__device__ __forceinline__ void tmem_ld_issue<32>(uint32_t taddr, uint32_t (&d)[32]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
               : FDW_TMEM_R8(0), FDW_TMEM_R8(8), FDW_TMEM_R8(16), FDW_TMEM_R8(24)
               : "r"(taddr)
               : "memory");
}
template <>
__device__ __forceinline__ void tmem_wait_ld<32>(uint32_t (&d)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : FDW_TMEM_W8(0), FDW_TMEM_W8(8), FDW_TMEM_W8(16), FDW_TMEM_W8(24)
               :
               : "memory");
}
template <>
__device__ __forceinline__ void tmem_ld_issue<64>(uint32_t taddr, uint32_t (&d)[64]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];"
               : FDW_TMEM_R8(0), FDW_TMEM_R8(8), FDW_TMEM_R8(16), FDW_TMEM_R8(24), FDW_TMEM_R8(32), FDW_TMEM_R8(40), FDW_TMEM_R8(48), FDW_TMEM_R8(56)
               : "r"(taddr)
               : "memory");
}
template <>
__device__ __forceinline__ void tmem_wait_ld<64>(uint32_t (&d)[64]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : FDW_TMEM_W8(0), FDW_TMEM_W8(8), FDW_TMEM_W8(16), FDW_TMEM_W8(24), FDW_TMEM_W8(32), FDW_TMEM_W8(40), FDW_TMEM_W8(48), FDW_TMEM_W8(56)
               :
               : "memory");
}
#undef FDW_TMEM_R8
#undef FDW_TMEM_W8

// The 8 R columns of an x window of radius R as separate loads in flight:
// TmemWindow<R>::issue(addr) then wait() before reading v(i).
template <int R>
struct TmemWindow {
  static constexpr int N = 8 * R;
  static constexpr int C64 = N >= 64 ? 64 : 0;
  static constexpr int C32 = (N - C64) >= 32 ? 32 : 0;
  static constexpr int C16 = (N - C64 - C32) >= 16 ? 16 : 0;
  static constexpr int C8 = N - C64 - C32 - C16;  // 0 or 8
  uint32_t a[C64 ? 64 : 1], b[C32 ? 32 : 1], c[C16 ? 16 : 1], e[C8 ? 8 : 1];
  __device__ __forceinline__ void issue(uint32_t taddr) {
    if constexpr (C64 > 0) tmem_ld_issue<64>(taddr, a);
    if constexpr (C32 > 0) tmem_ld_issue<32>(taddr + C64, b);
    if constexpr (C16 > 0) tmem_ld_issue<16>(taddr + C64 + C32, c);
    if constexpr (C8 > 0) tmem_ld_issue<8>(taddr + C64 + C32 + C16, e);
  }
  __device__ __forceinline__ void wait() {
    if constexpr (C64 > 0) tmem_wait_ld<64>(a);
    if constexpr (C32 > 0) tmem_wait_ld<32>(b);
    if constexpr (C16 > 0) tmem_wait_ld<16>(c);
    if constexpr (C8 > 0) tmem_wait_ld<8>(e);
  }
  __device__ __forceinline__ float v(int i) const {
    if (i < C64) return __uint_as_float(a[i]);
    i -= C64;
    if (i < C32) return __uint_as_float(b[i]);
    i -= C32;
    if (i < C16) return __uint_as_float(c[i]);
    return __uint_as_float(e[i - C16]);
  }
};

// The 8 R columns (2 R planes of four values) of an x window of radius R
// (1..8) from taddr, in chunks of the load shapes above.
template <int N>
__device__ __forceinline__ void tmem_ld_f(uint32_t taddr, float* w) {
  uint32_t d[N];
  tmem_ld<N>(taddr, d);
#pragma unroll
  for (int i = 0; i < N; ++i) w[i] = __uint_as_float(d[i]);
}
template <int R>
__device__ __forceinline__ void tmem_window(uint32_t taddr, float (&w)[8 * R]) {
  constexpr int N = 8 * R;
  static_assert(R >= 1 && R <= 8, "radius 1..8");
  constexpr int C64 = N >= 64 ? 64 : 0;
  constexpr int C32 = (N - C64) >= 32 ? 32 : 0;
  constexpr int C16 = (N - C64 - C32) >= 16 ? 16 : 0;
  constexpr int C8 = N - C64 - C32 - C16;  // 0 or 8
  if constexpr (C64 > 0) tmem_ld_f<64>(taddr, w);
  if constexpr (C32 > 0) tmem_ld_f<32>(taddr + C64, w + C64);
  if constexpr (C16 > 0) tmem_ld_f<16>(taddr + C64 + C32, w + C64 + C32);
  if constexpr (C8 > 0) tmem_ld_f<8>(taddr + C64 + C32 + C16, w + C64 + C32 + C16);
}

__device__ __forceinline__ float load_m(const void* base, int mtype, long long i) {
  if (mtype == kF16) return __half2float(static_cast<const __half*>(base)[i]);
  if (mtype == kBF16) return __bfloat162float(static_cast<const __nv_bfloat16*>(base)[i]);
  return static_cast<const float*>(base)[i];
}

__device__ __forceinline__ float smem_m(const unsigned char* sm, int mtype, int i) {
  if (mtype == kF16) return __half2float(reinterpret_cast<const __half*>(sm)[i]);
  if (mtype == kBF16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(sm)[i]);
  return reinterpret_cast<const float*>(sm)[i];
}

}  // namespace fdw
