// Host-side pieces of libfdwave shared by the context runtime (fdw_runtime.cu)
// and the allocation-free forward entry point (fdw_static.cu), so that each
// reading of the method exists once: the stencil weights and the stability
// limit, the location and multilinear weights of a sparse point, the built-in
// damping profile, the work-unit tiles, the grouping of injection terms by
// grid node and of sampled points by unit, the shared-memory layout of a step
// launch, tensor-map encoding, the step-kernel registry, the kernel's
// shared-memory limit and the meaning of the device error word.
//
// Nothing here allocates: every routine writes into arrays its caller owns.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "fdw_internal.h"
#include "fdwave.h"

namespace fdw {

// ---------------------------------------------------------------- stencil

inline bool valid_order(int p) { return p >= 2 && p <= 16 && p % 2 == 0; }

// Second-derivative weights c_0..c_r of the 2r+1 point central stencil of
// order p (r = p/2; c holds r+1 values), by Fornberg's recursion (Math. Comp.
// 51, 1988) on the nodes 0, 1, -1, 2, -2, ...; unscaled (times 1/h^2).
inline void fd_weights(int p, double* c) {
  const int r = p / 2, N = 2 * r + 1, M = 2;
  double x[2 * kMaxR + 1];
  double d[M + 1][2 * kMaxR + 1][2 * kMaxR + 1];
  std::memset(d, 0, sizeof(d));
  x[0] = 0.0;
  for (int j = 1; j <= r; ++j) {
    x[2 * j - 1] = j;
    x[2 * j] = -j;
  }
  d[0][0][0] = 1.0;
  double c1 = 1.0;
  for (int n = 1; n < N; ++n) {
    double c2 = 1.0;
    for (int v = 0; v < n; ++v) {
      const double c3 = x[n] - x[v];
      c2 *= c3;
      for (int m = 0; m <= std::min(n, M); ++m) {
        const double lower = m ? d[m - 1][n - 1][v] : 0.0;
        d[m][n][v] = (x[n] * d[m][n - 1][v] - m * lower) / c3;
      }
    }
    for (int m = 0; m <= std::min(n, M); ++m) {
      const double lower = m ? d[m - 1][n - 1][n - 1] : 0.0;
      d[m][n][n] = c1 / c2 * (m * lower - x[n - 1] * d[m][n - 1][n - 1]);
    }
    c1 = c2;
  }
  c[0] = d[M][N - 1][0];
  for (int j = 1; j <= r; ++j) c[j] = 0.5 * (d[M][N - 1][2 * j - 1] + d[M][N - 1][2 * j]);
}

// Largest |symbol| of the 1-D stencil times h^2, reached at the Nyquist
// wavenumber: |c_0 + 2 sum_j (-1)^j c_j|.
inline double symbol_max(int p) {
  double c[kMaxR + 1];
  fd_weights(p, c);
  double s = c[0];
  for (int j = 1; j <= p / 2; ++j) s += 2.0 * ((j % 2) ? -1.0 : 1.0) * c[j];
  return std::fabs(s);
}

// Leapfrog stability limit dt_max = 2 / (vmax sqrt(sum_a S / h_a^2)) over the
// ndim axes of `spacing` (user axis order).
inline double dt_limit(int ndim, const double* spacing, int p, double vmax) {
  const double S = symbol_max(p);
  double acc = 0.0;
  for (int a = 0; a < ndim; ++a) acc += S / (spacing[a] * spacing[a]);
  return 2.0 / (vmax * std::sqrt(acc));
}

// ---------------------------------------------------------------- grid

// One problem's grid on the internal axes (x, y, z); a 2D problem (x, z) has
// a single y point.  phys: physical points per axis; h: spacing.
struct GridGeom {
  int ndim = 3;
  int64_t phys[3] = {1, 1, 1};
  double h[3] = {1.0, 1.0, 1.0};
  int nbl = 0;
  bool active(int a) const { return !(ndim == 2 && a == 1); }
  // user axis of internal axis a (2D: x -> 0, z -> 1)
  int user_axis(int a) const { return (ndim == 2 && a == 2) ? 1 : a; }
};

inline GridGeom grid_geom(int ndim, const int64_t* shape, const double* spacing, int nbl) {
  GridGeom g;
  g.ndim = ndim;
  g.nbl = nbl;
  if (ndim == 3) {
    for (int a = 0; a < 3; ++a) {
      g.phys[a] = shape[a];
      g.h[a] = spacing[a];
    }
  } else {
    g.phys[0] = shape[0];
    g.phys[2] = shape[1];
    g.h[0] = spacing[0];
    g.h[2] = spacing[1];
  }
  return g;
}

// Base node (computational indices on the internal axes; 0 on an inactive
// axis) and fractional offsets of the point xyz (metres, user axis order,
// relative to the physical origin): on each axis i = floor(x/h) clamped to
// [0, N-2] (a point on the last grid line gets f = 1), plus nbl.  Returns -1
// when the point lies in [0, (N-1) h] on every axis, else the first user
// axis on which it does not.
inline int locate_point(const GridGeom& g, const double* xyz, int b[3], double f[3]) {
  for (int a = 0; a < 3; ++a) {
    b[a] = 0;
    f[a] = 0.0;
    if (!g.active(a)) continue;
    const int ua = g.user_axis(a);
    const double xv = xyz[ua];
    const double top = (double)(g.phys[a] - 1) * g.h[a];
    if (!(xv >= 0.0) || !(xv <= top)) return ua;
    const double xi = xv / g.h[a];
    long long i = (long long)std::floor(xi);
    if (i < 0) i = 0;
    if (i > g.phys[a] - 2) i = g.phys[a] - 2;
    b[a] = (int)i + g.nbl;
    f[a] = xi - (double)i;
  }
  return -1;
}

// Multilinear weight of corner cc (x bit 2, y bit 1, z bit 0) of the cell at
// the point's base node; corners with the y bit set weigh 0 in 2D.
inline float corner_weight(const GridGeom& g, const double f[3], int cc) {
  const int bx = (cc >> 2) & 1, by = (cc >> 1) & 1, bz = cc & 1;
  double w = (bx ? f[0] : 1.0 - f[0]) * (bz ? f[2] : 1.0 - f[2]);
  if (g.ndim == 3) w *= by ? f[1] : 1.0 - f[1];
  else if (by) w = 0.0;
  return (float)w;
}

// Built-in damping at computational index i of internal axis a, as eta dt/2:
// eta = 3 ln(1000) / (2 nbl h_a vmax) (d/nbl)^2 with d the distance in cells
// into the layer (0 in the physical domain and on an inactive axis).
inline float damping_half_dt(const GridGeom& g, int a, long long i, double vmax, double dt) {
  double e = 0.0;
  if (g.active(a) && g.nbl > 0) {
    const long long lo = g.nbl - i, hi = i - (g.nbl + g.phys[a] - 1);
    const long long d = lo > 0 ? lo : (hi > 0 ? hi : 0);
    const double emax = 3.0 * std::log(1000.0) / (2.0 * g.nbl * g.h[a] * vmax);
    const double fr = (double)d / g.nbl;
    e = emax * fr * fr;
  }
  return (float)(e * dt * 0.5);
}

// ---------------------------------------------------------------- work units

// Column tiles of a grid with ny x nz points: cy rows of TY and cz of kTZ.
inline void column_tiles(int ny, int nz, int TY, int* cy, int* cz) {
  *cy = (ny + TY - 1) / TY;
  *cz = (nz + kTZ - 1) / kTZ;
}

// The unit that streams column tile `li` (row-major over cy x cz tiles) of
// shot `shot` along the x planes [x0, x1).
inline Unit make_unit(int shot, int x0, int x1, int li, int cz, int TY) {
  Unit u;
  std::memset(&u, 0, sizeof(u));
  u.shot = shot;
  u.x0 = x0;
  u.x1 = x1;
  u.y0 = (li / cz) * TY;
  u.z0 = (li % cz) * kTZ;
  return u;
}

// One injected term: point j adds weight w times its sample into node
// (x, y, z), which unit `unit` updates.
struct Corner {
  int unit, x, y, z, j;
  float w;
};

// Groups n terms into injection nodes: sorts them by (unit, x, y, z, point)
// and writes one InjNode per distinct (unit, x, y, z) with its terms in point
// order (nodes[], terms[] hold up to n entries) and inj_ptr[U + 1], the nodes
// of unit u being [inj_ptr[u], inj_ptr[u+1]).  The sums at the unit tails
// then run in a fixed order.  Returns the number of nodes.
inline int group_corners(Corner* c, int n, int U, InjNode* nodes, InjTerm* terms, int* inj_ptr) {
  std::sort(c, c + n, [](const Corner& a, const Corner& b) {
    if (a.unit != b.unit) return a.unit < b.unit;
    if (a.x != b.x) return a.x < b.x;
    if (a.y != b.y) return a.y < b.y;
    if (a.z != b.z) return a.z < b.z;
    return a.j < b.j;
  });
  std::fill(inj_ptr, inj_ptr + U + 1, 0);
  int nn = 0;
  for (int i = 0; i < n; ++i) {
    const Corner& e = c[i];
    terms[i].j = e.j;
    terms[i].w = e.w;
    const bool fresh = i == 0 || e.unit != c[i - 1].unit || e.x != c[i - 1].x ||
                       e.y != c[i - 1].y || e.z != c[i - 1].z;
    if (fresh) {
      InjNode& nd = nodes[nn++];
      std::memset(&nd, 0, sizeof(nd));
      nd.x = e.x;
      nd.y = e.y;
      nd.z = e.z;
      nd.tbeg = i;
      nd.j0 = e.j;
      nd.w0 = e.w;
      inj_ptr[e.unit + 1]++;
    }
    nodes[nn - 1].tend = i + 1;
  }
  for (int u = 0; u < U; ++u) inj_ptr[u + 1] += inj_ptr[u];
  return nn;
}

// Sampled points by the unit that records them (unit_of[j] < 0: none):
// ptr[U + 1] and pts[] (up to n entries) with the points of unit u, in point
// order, at [ptr[u], ptr[u+1]).  Returns the number of listed points.
inline int bucket_points(const int* unit_of, int n, int U, int* ptr, int* pts) {
  std::fill(ptr, ptr + U + 1, 0);
  for (int j = 0; j < n; ++j)
    if (unit_of[j] >= 0) ptr[unit_of[j] + 1]++;
  for (int u = 0; u < U; ++u) ptr[u + 1] += ptr[u];
  for (int j = 0; j < n; ++j)
    if (unit_of[j] >= 0) pts[ptr[unit_of[j]]++] = j;  // ptr[u] becomes the end of unit u
  for (int u = U; u > 0; --u) ptr[u] = ptr[u - 1];
  ptr[0] = 0;
  return ptr[U];
}

// ---------------------------------------------------------------- launches

// Shared-memory stages of a step launch.  The forward and adjoint steps stage
// each plane's tiles with its halo plane; the gradient step, whose tiles are
// twice the halo plane, keeps them in a second ring of stages that is only
// occupied while they are in flight (the halo ring also holds the r planes of
// the x stencil ahead of the plane being updated).
struct StageLayout {
  int off_p, off_m, off_f, off_a, off_e;  // tile offsets inside their stage
  int off_c;    // centre tile of plane x + r (tiles with `ca`; 0 otherwise)
  int bytes;    // halo-ring stage
  int cbytes;   // second-ring stage (0: no second ring)
  int r;
};

inline int round128(int x) { return (x + 127) & ~127; }

// Stages of the second ring for `stages` halo stages: the tiles of plane x
// are issued with the halo plane x + r, so at most stages - r are in flight.
inline int second_ring_stages(const StageLayout& L, int stages) {
  return L.cbytes ? std::max(2, stages - L.r) : 0;
}

inline StageLayout stage_layout(int r, int tile, int mt_bytes, bool grad, bool etaf) {
  // the gradient step's tiles go to the second ring, except in tiles whose
  // stages hold one plane's reads (ca), where they are part of that plane
  const bool split = (grad && !kTiles[tile].ca) || kTiles[tile].split;
  const int TY = tile_rows(kTiles[tile]);
  const int R4 = (r + 3) & ~3;
  const int ZW = kTZ + 2 * R4, YW = TY + 2 * r;
  StageLayout L;
  L.r = r;
  const int halo = round128(YW * ZW * 4);
  int off = split ? 0 : halo;
  L.off_p = off;
  off += round128(TY * kTZ * 4);
  L.off_m = off;
  off += round128(TY * kTZ * mt_bytes);
  L.off_f = off;
  if (grad) off += round128(TY * kTZ * 4);
  L.off_a = off;
  if (grad) off += round128(TY * kTZ * 4);
  L.off_e = off;
  if (etaf) off += round128(TY * kTZ * 4);
  L.off_c = 0;
  if (!split && kTiles[tile].ca) {
    L.off_c = off;
    off += round128(TY * kTZ * 4);
  }
  L.bytes = split ? halo : off;
  L.cbytes = split ? off : 0;
  return L;
}

// Fewest pipeline stages of a tile: the halo plane of plane x stays staged
// until x is updated while planes up to x + r are read ahead, unless the
// centre values come in tiles of their own (then any two stages pipeline).
inline int min_stages(int r, int tile) { return kTiles[tile].ca ? 2 : r + 2; }

// Dynamic shared memory of a launch: the stages of both rings, their full
// and empty barriers, the consumers' unit-tail barrier and 128 bytes of
// alignment slack.
inline size_t smem_bytes(const StageLayout& L, int stages) {
  const int sc = second_ring_stages(L, stages);
  return (size_t)stages * L.bytes + (size_t)sc * L.cbytes + (size_t)(2 * stages + 2 * sc + 1) * 8 +
         128;
}

// The step kernel of radius r, tile and role (kernel registry).
inline const void* step_fn(int r, int tile, bool grad) {
  switch (r) {
    case 1: return step_kernel_r1(tile, grad);
    case 2: return step_kernel_r2(tile, grad);
    case 3: return step_kernel_r3(tile, grad);
    case 4: return step_kernel_r4(tile, grad);
    case 5: return step_kernel_r5(tile, grad);
    case 6: return step_kernel_r6(tile, grad);
    case 7: return step_kernel_r7(tile, grad);
    case 8: return step_kernel_r8(tile, grad);
  }
  return nullptr;
}

// Lets `fn` launch with `smem` bytes of dynamic shared memory on the current
// device.  The limit is a property of the kernel function, shared by every
// caller in the process, so it is only ever raised: a launch prepared for a
// larger limit stays valid whatever configuration another caller sets up
// later.  Also asks for all of the unified L1 / shared memory as shared
// memory (the pipeline stages are the working set).
inline cudaError_t raise_smem_limit(const void* fn, size_t smem) {
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, fn);
  if (e != cudaSuccess) return e;
  if ((size_t)a.maxDynamicSharedSizeBytes < smem) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                              (int)cudaSharedmemCarveoutMaxShared);
}

// cuTensorMapEncodeTiled from the driver (through the runtime's entry-point
// query, so the library does not link the driver); null if unavailable.
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p) {
      cudaGetLastError();
      return nullptr;
    }
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Tensor map of pitched field(s) [slots][nx][ny][nzp] of element type dt
// (rank 3 when slots == 0) with a box of box_z x box_y points of one plane;
// loads outside the grid fill zeros.
inline CUresult encode_field_map(CUtensorMap* map, CUtensorMapDataType dt, int esize,
                                 const void* base, int nx, int ny, int nz, int nzp, int slots,
                                 long long slot_elems, int box_z, int box_y) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return CUDA_ERROR_NOT_FOUND;
  cuuint64_t dims[4] = {(cuuint64_t)nz, (cuuint64_t)ny, (cuuint64_t)nx,
                        (cuuint64_t)(slots ? slots : 1)};
  cuuint64_t strides[3] = {(cuuint64_t)nzp * esize, (cuuint64_t)nzp * ny * esize,
                           (cuuint64_t)slot_elems * esize};
  cuuint32_t box[4] = {(cuuint32_t)box_z, (cuuint32_t)box_y, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  return enc(map, dt, slots ? 4 : 3, const_cast<void*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

// True for device or managed memory of the CUDA runtime.
inline bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Status of a non-zero device error word: a bounded wait that gave up is
// FDW_ERR_TIMEOUT; any other bit would be an internal fault, FDW_ERR_CUDA.
inline fdw_status device_error_status(int e) {
  if (e == 0) return FDW_OK;
  if ((e & ~(kErrTimeoutFull | kErrTimeoutEmpty)) == 0) return FDW_ERR_TIMEOUT;
  return FDW_ERR_CUDA;
}

}  // namespace fdw
