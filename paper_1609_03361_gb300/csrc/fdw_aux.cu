// Auxiliary kernels of libfdwave: per-call work around the time loop.
//  - sampling of the last time level (grid-to-point, Sec. 5.2),
//  - model set-up (edge extension into the layer, s = 1/m, storage-type conversion),
//  - damping-field set-up,
//  - checkpoint snapshots: absolute maximum, pack to 16 bits with a scale,
//    unpack,
//  - gradient output (scaling and folding of the layer onto the edges),
//  - copy of a pitched field to a dense array.
// All index arithmetic is 64-bit; grid-stride loops cover any size.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "fdw_device.cuh"
#include "fdw_internal.h"

namespace fdw {
namespace {

constexpr int kThreads = 256;

__host__ __device__ inline long long dense_points(const Geom& g) {
  return (long long)g.nx * g.ny * g.nz;
}

__device__ inline long long pitched(const Geom& g, long long i) {
  // dense index (x, y, z) -> pitched offset
  const long long z = i % g.nz;
  const long long xy = i / g.nz;
  return xy * g.nzp + z;
}

inline int blocks_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  if (b > 152LL * 32) b = 152LL * 32;
  if (b < 1) b = 1;
  return (int)b;
}

__global__ void sample_kernel(const ShotDesc* shots, int slot, int row) {
  const ShotDesc& d = shots[blockIdx.y];
  const float* u = d.u + (long long)slot * d.uslot;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d.smp_n; j += gridDim.x * blockDim.x) {
    const int bx = d.pt_base[3 * j], by = d.pt_base[3 * j + 1], bz = d.pt_base[3 * j + 2];
    const float* w = d.pt_w + 8 * j;
    float acc = 0.f;
    for (int c = 0; c < 8; ++c) {
      const float wc = w[c];
      if (wc != 0.f) {
        const long long off =
            ((long long)(bx + ((c >> 2) & 1)) * d.ny + (by + ((c >> 1) & 1))) * d.nzp + bz + (c & 1);
        acc = fmaf(wc, u[off], acc);
      }
    }
    d.smp_out[(long long)row * d.smp_ld + j] = acc;
  }
}

// The field may be an x slab of a larger grid: local plane x is plane x + xoff
// of the full computational grid of nxg planes (xoff = 0, nxg = g.nx for a
// whole grid); planes beyond the full grid take the nearest edge plane.
__global__ void model_kernel(const float* in, int layout, int px, int py, int pz, int nbl,
                             int ndim, void* out, int mtype, Geom g, int xoff, int nxg) {
  const long long n = dense_points(g);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long z = i % g.nz;
    const long long y = (i / g.nz) % g.ny;
    long long x = i / ((long long)g.nz * g.ny) + xoff;
    x = x < 0 ? 0 : (x > nxg - 1 ? nxg - 1 : x);
    float v;
    if (layout == 0) {  // physical: clamp each computational index into the physical range
      long long cx = x - nbl, cy = (ndim == 3) ? y - nbl : 0, cz = z - nbl;
      cx = cx < 0 ? 0 : (cx > px - 1 ? px - 1 : cx);
      cy = cy < 0 ? 0 : (cy > py - 1 ? py - 1 : cy);
      cz = cz < 0 ? 0 : (cz > pz - 1 ? pz - 1 : cz);
      v = in[(cx * py + cy) * pz + cz];
    } else {
      v = in[(x * g.ny + y) * g.nz + z];
    }
    const long long o = pitched(g, i);
    const float sv = 1.0f / v;  // stored as s = 1/m (squared velocity)
    if (mtype == kF16) static_cast<__half*>(out)[o] = __float2half_rn(sv);
    else if (mtype == kBF16) static_cast<__nv_bfloat16*>(out)[o] = __float2bfloat16_rn(sv);
    else static_cast<float*>(out)[o] = sv;
  }
}

__global__ void eta_field_kernel(const float* in, float scale, float* out, Geom g, int xoff,
                                 int nxg) {
  const long long n = dense_points(g);
  const long long pl = (long long)g.ny * g.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    long long x = i / pl + xoff;
    x = x < 0 ? 0 : (x > nxg - 1 ? nxg - 1 : x);
    out[pitched(g, i)] = in[x * pl + i % pl] * scale;
  }
}

// Snapshot kernels work on whole pitched fields, four floats per access: the
// padding past nz is zero in every wavefield, so it packs and unpacks to zero.

// max(|a|, |b|) over a pair of pitched fields, per shot (blockIdx.y).
__global__ void absmax_kernel(const AuxShot* shots) {
  const AuxShot& s = shots[blockIdx.y];
  const long long n4 = s.n / 4;
  const float4* a = reinterpret_cast<const float4*>(s.a);
  const float4* b = reinterpret_cast<const float4*>(s.b);
  float m = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
       i += (long long)gridDim.x * blockDim.x) {
    const float4 x = a[i], y = b[i];
    m = fmaxf(m, fmaxf(fmaxf(fabsf(x.x), fabsf(x.y)), fmaxf(fabsf(x.z), fabsf(x.w))));
    m = fmaxf(m, fmaxf(fmaxf(fabsf(y.x), fabsf(y.y)), fmaxf(fabsf(y.z), fabsf(y.w))));
  }
  for (int k = 16; k > 0; k >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, k));
  __shared__ float red[kThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    atomicMax(s.amax, __float_as_uint(m));  // non-negative floats order like their bits
  }
}

// Scale that maps the pair's maximum to 2^14 (16-bit storage), 1 otherwise.
__device__ inline float snap_scale(const unsigned int* amax, int stype) {
  if (stype == kF32) return 1.f;
  const float m = __uint_as_float(*amax);
  return m > 0.f ? 16384.f / m : 1.f;
}

template <typename H>
__device__ inline uint2 to16x4(float4 v, float sc);
template <>
__device__ inline uint2 to16x4<__half>(float4 v, float sc) {
  const __half2 lo = __floats2half2_rn(v.x * sc, v.y * sc);
  const __half2 hi = __floats2half2_rn(v.z * sc, v.w * sc);
  return make_uint2(*reinterpret_cast<const unsigned*>(&lo), *reinterpret_cast<const unsigned*>(&hi));
}
template <>
__device__ inline uint2 to16x4<__nv_bfloat16>(float4 v, float sc) {
  const __nv_bfloat162 lo = __floats2bfloat162_rn(v.x * sc, v.y * sc);
  const __nv_bfloat162 hi = __floats2bfloat162_rn(v.z * sc, v.w * sc);
  return make_uint2(*reinterpret_cast<const unsigned*>(&lo), *reinterpret_cast<const unsigned*>(&hi));
}

template <typename H>
__device__ inline float4 from16x4(uint2 r, float inv);
template <>
__device__ inline float4 from16x4<__half>(uint2 r, float inv) {
  const float2 lo = __half22float2(*reinterpret_cast<const __half2*>(&r.x));
  const float2 hi = __half22float2(*reinterpret_cast<const __half2*>(&r.y));
  return make_float4(lo.x * inv, lo.y * inv, hi.x * inv, hi.y * inv);
}
template <>
__device__ inline float4 from16x4<__nv_bfloat16>(uint2 r, float inv) {
  const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r.x));
  const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r.y));
  return make_float4(lo.x * inv, lo.y * inv, hi.x * inv, hi.y * inv);
}

template <typename H>
__global__ void pack16_kernel(const AuxShot* shots) {
  const AuxShot& s = shots[blockIdx.y];
  const long long n4 = s.n / 4;
  const float sc = snap_scale(s.amax, kF16);
  const float4* a = reinterpret_cast<const float4*>(s.a);
  const float4* b = reinterpret_cast<const float4*>(s.b);
  uint2* h = static_cast<uint2*>(s.snap);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
       i += (long long)gridDim.x * blockDim.x) {
    h[i] = to16x4<H>(a[i], sc);
    h[n4 + i] = to16x4<H>(b[i], sc);
  }
}

template <typename H>
__global__ void unpack16_kernel(const AuxShot* shots) {
  const AuxShot& s = shots[blockIdx.y];
  const long long n4 = s.n / 4;
  const float inv = 1.f / snap_scale(s.amax, kF16);
  float4* a = reinterpret_cast<float4*>(s.a);
  float4* b = reinterpret_cast<float4*>(s.b);
  const uint2* h = static_cast<const uint2*>(s.snap);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
       i += (long long)gridDim.x * blockDim.x) {
    a[i] = from16x4<H>(h[i], inv);
    b[i] = from16x4<H>(h[n4 + i], inv);
  }
}

// FP32 snapshots: plain copies in either direction (dir 0: fields -> snapshot).
__global__ void copy32_kernel(const AuxShot* shots, int dir) {
  const AuxShot& s = shots[blockIdx.y];
  const long long n4 = s.n / 4;
  float4* a = reinterpret_cast<float4*>(s.a);
  float4* b = reinterpret_cast<float4*>(s.b);
  float4* h = static_cast<float4*>(s.snap);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
       i += (long long)gridDim.x * blockDim.x) {
    if (dir == 0) {
      h[i] = a[i];
      h[n4 + i] = b[i];
    } else {
      a[i] = h[i];
      b[i] = h[n4 + i];
    }
  }
}

// Injection of one step's data into u^{n+1} as a launch of its own (the
// adjoint step's receiver residuals: thousands of nodes, which spread over
// every SM here instead of queueing at the tails of the few units that hold
// them).  Per node the same arithmetic as the step kernel's unit tail:
// u^{n+1} += dt^2 sum_t w_t a_j / (m + eta dt/2) with s = 1/m, and with grad
// the accumulator's share fwd * delta.  Nodes are unique, so no atomics.
__global__ void inject_kernel(const ShotDesc* shots, const InjNode* nodes, const int* node_shot,
                              const InjTerm* terms, int nnodes, int row, int out, int fslot,
                              float dt2, int diff, int grad, int etaf) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nnodes; i += gridDim.x * blockDim.x) {
    const InjNode nd = nodes[i];
    const ShotDesc& d = shots[node_shot[i]];
    const float* A = d.inj_a + (long long)row * d.inj_ld;
    const float* B = diff ? d.inj_b + (long long)row * d.inj_ld : nullptr;
    // the terms in order, the first one from the node record itself
    float sum = 0.f;
    if (nd.tend > nd.tbeg) {
      sum = fmaf(nd.w0, B ? A[nd.j0] - B[nd.j0] : A[nd.j0], sum);
      for (int t = nd.tbeg + 1; t < nd.tend; ++t) {
        const InjTerm tm = terms[t];
        const float v = B ? A[tm.j] - B[tm.j] : A[tm.j];
        sum = fmaf(tm.w, v, sum);
      }
    }
    const long long off = ((long long)nd.x * d.ny + nd.y) * d.nzp + nd.z;
    const float sv = load_m(d.m, d.mtype, off);
    const float e = etaf ? d.etaf[off] : d.eta[nd.x] + d.eta[d.nx + nd.y] + d.eta[d.nx + d.ny + nd.z];
    const float delta = dt2 * sum * sv / (1.f + e * sv);
    float* uo = d.u + (long long)out * d.uslot;
    uo[off] = uo[off] + delta;
    if (grad) d.acc[off] = fmaf(d.fwd[(long long)fslot * d.fslot + off], delta, d.acc[off]);
  }
}

// Gradient output.  layout 1: computational shape, out = scale * acc.
// layout 0: physical shape, each physical cell sums the computational cells
// whose clamped index is that cell (the adjoint of the edge extension).
__global__ void grad_out_kernel(const float* acc, Geom g, float scale, float* out, int layout,
                                int nbl, int ndim, int px, int py, int pz) {
  if (layout == 1) {
    const long long n = dense_points(g);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
      out[i] = scale * acc[pitched(g, i)];
    return;
  }
  const long long n = (long long)px * py * pz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i % pz);
    const int j = (int)((i / pz) % py);
    const int l = (int)(i / ((long long)pz * py));
    // computational ranges mapping onto (l, j, k)
    int xl = l + nbl, xh = l + nbl;
    if (l == 0) xl = 0;
    if (l == px - 1) xh = px - 1 + 2 * nbl;
    int yl = 0, yh = 0;
    if (ndim == 3) {
      yl = j + nbl; yh = j + nbl;
      if (j == 0) yl = 0;
      if (j == py - 1) yh = py - 1 + 2 * nbl;
    }
    int zl = k + nbl, zh = k + nbl;
    if (k == 0) zl = 0;
    if (k == pz - 1) zh = pz - 1 + 2 * nbl;
    double s = 0.0;
    for (int x = xl; x <= xh; ++x)
      for (int y = yl; y <= yh; ++y)
        for (int z = zl; z <= zh; ++z) s += acc[((long long)x * g.ny + y) * g.nzp + z];
    out[i] = (float)(scale * s);
  }
}

__global__ void copy_out_kernel(const float* f, Geom g, float* out) {
  const long long n = dense_points(g);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = f[pitched(g, i)];
}

}  // namespace

cudaError_t launch_sample(const ShotDesc* shots, int nshots, int maxpts, int slot, int row,
                          cudaStream_t s) {
  if (maxpts <= 0 || nshots <= 0) return cudaSuccess;
  dim3 grid((maxpts + kThreads - 1) / kThreads, nshots);
  sample_kernel<<<grid, kThreads, 0, s>>>(shots, slot, row);
  return cudaGetLastError();
}

cudaError_t launch_model(const float* in, int layout, int px, int py, int pz, int nbl, int ndim,
                         void* out, int mtype, Geom g, cudaStream_t s, int xoff, int nxg) {
  model_kernel<<<blocks_for(dense_points(g)), kThreads, 0, s>>>(
      in, layout, px, py, pz, nbl, ndim, out, mtype, g, xoff, nxg > 0 ? nxg : g.nx);
  return cudaGetLastError();
}

cudaError_t launch_eta_field(const float* in, float scale, float* out, Geom g, cudaStream_t s,
                             int xoff, int nxg) {
  eta_field_kernel<<<blocks_for(dense_points(g)), kThreads, 0, s>>>(in, scale, out, g, xoff,
                                                                    nxg > 0 ? nxg : g.nx);
  return cudaGetLastError();
}

// Grid of a snapshot kernel: float4 units of the largest field, at most 8
// blocks of 256 threads per SM.
static dim3 snap_grid(long long maxn, int nshots) {
  long long b = (maxn / 4 + kThreads - 1) / kThreads;
  b = std::max(1LL, std::min(b, 152LL * 8));
  return dim3((unsigned)b, (unsigned)nshots);
}

cudaError_t launch_absmax(const AuxShot* shots, int nshots, long long maxn, cudaStream_t s) {
  absmax_kernel<<<snap_grid(maxn, nshots), kThreads, 0, s>>>(shots);
  return cudaGetLastError();
}

cudaError_t launch_pack(const AuxShot* shots, int nshots, long long maxn, int stype,
                        cudaStream_t s) {
  const dim3 g = snap_grid(maxn, nshots);
  if (stype == kF16) pack16_kernel<__half><<<g, kThreads, 0, s>>>(shots);
  else if (stype == kBF16) pack16_kernel<__nv_bfloat16><<<g, kThreads, 0, s>>>(shots);
  else copy32_kernel<<<g, kThreads, 0, s>>>(shots, 0);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const AuxShot* shots, int nshots, long long maxn, int stype,
                          cudaStream_t s) {
  const dim3 g = snap_grid(maxn, nshots);
  if (stype == kF16) unpack16_kernel<__half><<<g, kThreads, 0, s>>>(shots);
  else if (stype == kBF16) unpack16_kernel<__nv_bfloat16><<<g, kThreads, 0, s>>>(shots);
  else copy32_kernel<<<g, kThreads, 0, s>>>(shots, 1);
  return cudaGetLastError();
}

cudaError_t launch_inject(const ShotDesc* shots, const InjNode* nodes, const int* node_shot,
                          const InjTerm* terms, int nnodes, int row, int out, int fslot, float dt2,
                          bool diff, bool grad, bool etaf, cudaStream_t s) {
  if (nnodes <= 0) return cudaSuccess;
  const int blocks = std::min((nnodes + kThreads - 1) / kThreads, 152 * 8);
  inject_kernel<<<blocks, kThreads, 0, s>>>(shots, nodes, node_shot, terms, nnodes, row, out, fslot,
                                            dt2, diff ? 1 : 0, grad ? 1 : 0, etaf ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_grad_out(const float* acc, Geom g, float scale, float* out, int layout,
                            int nbl, int ndim, int px, int py, int pz, cudaStream_t s) {
  const long long n = layout == 1 ? dense_points(g) : (long long)px * py * pz;
  grad_out_kernel<<<blocks_for(n), kThreads, 0, s>>>(acc, g, scale, out, layout, nbl, ndim, px,
                                                      py, pz);
  return cudaGetLastError();
}

cudaError_t launch_copy_out(const float* field, Geom g, float* out, cudaStream_t s) {
  copy_out_kernel<<<blocks_for(dense_points(g)), kThreads, 0, s>>>(field, g, out);
  return cudaGetLastError();
}

}  // namespace fdw
