// 2D diffusion u_t = alpha (u_xx + u_yy) (Sec. 4, Eq. 1): forward Euler in
// time, 3-point second differences per axis, boundary rows and columns held at
// their initial values (only interior points are updated, Sec. 4.1).
//
// One update is
//     u'(i,j) = wc u(i,j) + wx (u(i-1,j) + u(i+1,j)) + wy (u(i,j-1) + u(i,j+1)),
//     wx = dt alpha / dx^2, wy = dt alpha / dy^2, wc = 1 - 2 wx - 2 wy,
// so at the Eq. 2 limit with dx = dy the centre weight is 0 and the neighbour
// weights 1/4, the constants of the generated code of Sec. 4.
//
// Kernel: each warp owns a band of 128 columns (y, contiguous; four per lane)
// and a chunk of rows (x), and streams the rows of its chunk top to bottom.
// T time levels are carried at once: level l of row r is computed as soon as
// level l-1 holds rows r-1, r, r+1, from a three-row window of each level kept
// in registers, with the y neighbours of a lane's outer columns taken from the
// adjacent lanes by shuffles.  Each level loses one valid column at either end
// of the band and needs one more row above and below the chunk, so a band
// writes its 128 - 2T inner columns and a chunk reads T extra rows on each side:
// one pass over memory advances the field by T steps.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "fdwave.h"

namespace {

struct DiffCoef {
  float wc, wx, wy;
};

constexpr int kBand = 128;        // columns loaded per warp
constexpr int kWarps = 4;         // warps per CTA
constexpr int kAhead = 4;         // rows fetched ahead of use

template <int T>
__global__ void __launch_bounds__(kWarps * 32)
diffusion_kernel(const float* __restrict__ in, float* __restrict__ out, long long nx,
                 long long ny, int chunk, int nbands, long long nwork, DiffCoef k) {
  constexpr int W = kBand - 2 * T;  // columns written per band
  const int lane = threadIdx.x & 31;
  const long long wk = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (wk >= nwork) return;
  const int band = (int)(wk % nbands);
  const long long i0 = (wk / nbands) * chunk;
  const long long i1 = nx < i0 + chunk ? nx : i0 + chunk;
  const long long jl = (long long)band * W - T + 4 * lane;  // first column of the lane

  bool jin[4], jbnd[4], jout[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const long long j = jl + e;
    jin[e] = j >= 0 && j < ny;
    jbnd[e] = j == 0 || j == ny - 1;
    const long long jo = j - ((long long)band * W);
    jout[e] = jin[e] && jo >= 0 && jo < W;
  }

  // win[l][q][e]: level l (0 = input), rows (r - l - 1, r - l, r - l + 1) for q = 0, 1, 2
  float win[T][3][4];
#pragma unroll
  for (int l = 0; l < T; ++l)
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int e = 0; e < 4; ++e) win[l][q][e] = 0.f;

  // input rows are fetched kAhead rows before they are used, so that several
  // loads of a warp are in flight while it computes
  auto fetch = [&](long long r, float* v) {
    const bool rin = r >= 0 && r < nx;
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = (rin && jin[e]) ? in[r * ny + jl + e] : 0.f;
  };
  float pf[kAhead][4];
#pragma unroll
  for (int a = 0; a < kAhead; ++a) fetch(i0 - T + a, pf[a]);

#pragma unroll 1
  for (long long r = i0 - T; r < i1 + T; ++r) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      win[0][0][e] = win[0][1][e];
      win[0][1][e] = win[0][2][e];
      win[0][2][e] = pf[0][e];
    }
#pragma unroll
    for (int a = 0; a + 1 < kAhead; ++a)
#pragma unroll
      for (int e = 0; e < 4; ++e) pf[a][e] = pf[a + 1][e];
    fetch(r + kAhead, pf[kAhead - 1]);
#pragma unroll
    for (int l = 1; l <= T; ++l) {
      const long long rr = r - l;  // row of level l computed now
      const bool rbnd = rr <= 0 || rr >= nx - 1;
      const float* up = win[l - 1][0];
      const float* c = win[l - 1][1];
      const float* dn = win[l - 1][2];
      const float left = __shfl_up_sync(0xffffffffu, c[3], 1);
      const float right = __shfl_down_sync(0xffffffffu, c[0], 1);
      float nv[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float ym = e == 0 ? left : c[e - 1];
        const float yp = e == 3 ? right : c[e + 1];
        const float s = fmaf(k.wx, up[e] + dn[e], fmaf(k.wy, ym + yp, k.wc * c[e]));
        nv[e] = (rbnd || jbnd[e]) ? c[e] : s;
      }
      if (l < T) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          win[l][0][e] = win[l][1][e];
          win[l][1][e] = win[l][2][e];
          win[l][2][e] = nv[e];
        }
      } else if (rr >= i0 && rr < i1) {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (jout[e]) out[rr * ny + jl + e] = nv[e];
      }
    }
  }
}

template <int T>
cudaError_t launch_pass(const float* in, float* out, long long nx, long long ny, DiffCoef k,
                        cudaStream_t s) {
  constexpr int W = kBand - 2 * T;
  const int nbands = (int)((ny + W - 1) / W);
  // rows per warp: 4T (the 2T rows of overlap a minor share) unless the grid
  // is too small to give each SM 16 warps, then down to 2T; on large grids
  // longer chunks, capped at 64 warps per SM
  auto warps = [&](long long c) { return ((nx + c - 1) / c) * nbands; };
  long long chunk = std::max<long long>(4 * T, 16);
  while (chunk > std::max<long long>(2 * T, 8) && warps(chunk) < 152LL * 16) chunk /= 2;
  while (chunk < nx && warps(chunk) > 152LL * 64) chunk *= 2;
  const long long nwork = ((nx + chunk - 1) / chunk) * nbands;
  const long long blocks = (nwork + kWarps - 1) / kWarps;
  diffusion_kernel<T><<<(unsigned)blocks, kWarps * 32, 0, s>>>(in, out, nx, ny, (int)chunk, nbands,
                                                               nwork, k);
  return cudaGetLastError();
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" fdw_status fdw_diffusion2d(float* u, float* tmp, int64_t nx, int64_t ny, double dx,
                                      double dy, double alpha, double dt, int steps,
                                      int steps_per_pass, void* stream) {
  if (!u || !tmp || u == tmp || nx < 3 || ny < 3 || steps < 0) return FDW_ERR_ARG;
  if (!(dx > 0) || !(dy > 0) || !(alpha > 0) || !(dt > 0)) return FDW_ERR_ARG;
  if (nx > (1LL << 31) || ny > (1LL << 31)) return FDW_ERR_SHAPE;
  if (steps_per_pass == 0) steps_per_pass = 4;
  if (steps_per_pass != 1 && steps_per_pass != 2 && steps_per_pass != 4 && steps_per_pass != 8)
    return FDW_ERR_ARG;
  const double limit = dx * dx * dy * dy / (2.0 * alpha * (dx * dx + dy * dy));  // Eq. 2
  if (dt > limit * (1.0 + 1e-12)) return FDW_ERR_CFL;
  if (!on_device(u) || !on_device(tmp)) return FDW_ERR_ARG;
  if (steps == 0) return FDW_OK;
  const double wx = dt * alpha / (dx * dx), wy = dt * alpha / (dy * dy);
  const DiffCoef k{(float)(1.0 - 2.0 * wx - 2.0 * wy), (float)wx, (float)wy};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const float* in = u;
  float* out = tmp;
  int left = steps;
  while (left > 0) {
    cudaError_t e;
    int t;
    if (left >= 8 && steps_per_pass == 8) { e = launch_pass<8>(in, out, nx, ny, k, s); t = 8; }
    else if (left >= 4 && steps_per_pass >= 4) { e = launch_pass<4>(in, out, nx, ny, k, s); t = 4; }
    else if (left >= 2 && steps_per_pass >= 2) { e = launch_pass<2>(in, out, nx, ny, k, s); t = 2; }
    else { e = launch_pass<1>(in, out, nx, ny, k, s); t = 1; }
    if (e != cudaSuccess) return FDW_ERR_CUDA;
    left -= t;
    float* next = const_cast<float*>(in);
    in = out;
    out = next;
  }
  if (in != u &&
      cudaMemcpyAsync(u, in, sizeof(float) * (size_t)nx * (size_t)ny, cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess)
    return FDW_ERR_CUDA;
  return FDW_OK;
}
