// Forward modelling that allocates nothing: fdw_forward_static.
//
// Some callers cannot call cudaMalloc: code running under a device-memory
// budget owned by another allocator, plugins whose host application forbids
// allocation after start-up, or real-time loops that must not hit the
// allocator.  This entry point runs the same time-step kernel as fdw_forward
// on a small problem, with every piece of scratch (wavefields, model, damping
// profiles, point tables, work-unit lists, the shot descriptor) in one
// file-scope device array of fixed size.  The caller passes the model, the
// wavelets and the trace buffer; nothing is allocated on the device or on the
// host heap.
//
// Limits (FDW_ERR_SHAPE beyond them): computational grid <= kMaxAxis points
// per axis and <= kMaxField pitched points per field (rows padded to 32), at
// most kMaxPoints sources and kMaxPoints receivers, at most kMaxUnits work
// units.  The array takes kStaticBytes of device memory on every GPU that
// loads the library, until the process exits.
//
// Every call shares the array: it is rewritten (and the wavefields cleared)
// at the start of each call, and calls that overlap on the GPU (different
// streams, or several host threads) race on it.  The host-side tables are
// likewise static, so the function is not reentrant.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "fdw_internal.h"
#include "fdwave.h"

namespace fdw {
namespace {

constexpr long long kMaxField = 1LL << 20;   // pitched points per field (4 MiB as float)
constexpr int kMaxAxis = 4096;
constexpr int kMaxPoints = 4096;
constexpr int kMaxUnits = 8192;
constexpr int kMaxNodes = 8 * kMaxPoints;
constexpr size_t kStaticBytes = 16u << 20;    // 16 MiB

__device__ __align__(256) unsigned char g_static[kStaticBytes];

// Byte layout of g_static (each region 256-byte aligned).
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffDesc = 0;
constexpr size_t kOffErr = align256(kOffDesc + sizeof(ShotDesc));
constexpr size_t kOffUnits = align256(kOffErr + sizeof(int));
constexpr size_t kOffInjPtr = align256(kOffUnits + sizeof(Unit) * kMaxUnits);
constexpr size_t kOffNodes = align256(kOffInjPtr + sizeof(int) * (kMaxUnits + 1));
constexpr size_t kOffTerms = align256(kOffNodes + sizeof(InjNode) * kMaxNodes);
constexpr size_t kOffSmpPtr = align256(kOffTerms + sizeof(InjTerm) * kMaxNodes);
constexpr size_t kOffSmpPts = align256(kOffSmpPtr + sizeof(int) * (kMaxUnits + 1));
constexpr size_t kOffPtBase = align256(kOffSmpPts + sizeof(int) * kMaxPoints);
constexpr size_t kOffPtW = align256(kOffPtBase + sizeof(int) * 3 * kMaxPoints);
constexpr size_t kOffEta = align256(kOffPtW + sizeof(float) * 8 * kMaxPoints);
constexpr size_t kOffModel = align256(kOffEta + sizeof(float) * 3 * kMaxAxis);
constexpr size_t kOffU = align256(kOffModel + sizeof(float) * kMaxField);
constexpr size_t kEnd = kOffU + sizeof(float) * 2 * kMaxField;
static_assert(kEnd <= kStaticBytes, "static scratch layout exceeds the array");

// Device address of g_static per device, looked up once per device with that
// device current (the host-side symbol is only a stand-in, not an address).
constexpr int kMaxDevices = 64;
unsigned char* g_dev_ptr[kMaxDevices] = {nullptr};

// Host-side tables, fixed size (no heap).
struct Corner {
  int unit, x, y, z, j;
  float w;
};
Corner h_corner[kMaxNodes];
Unit h_units[kMaxUnits];
int h_inj_ptr[kMaxUnits + 1];
InjNode h_nodes[kMaxNodes];
InjTerm h_terms[kMaxNodes];
int h_smp_ptr[kMaxUnits + 1];
int h_smp_unit[kMaxPoints];
int h_smp_pts[kMaxPoints];
int h_pt_base[3 * kMaxPoints];
float h_pt_w[8 * kMaxPoints];
float h_eta[3 * kMaxAxis];
ShotDesc h_desc;

// Second-derivative weights at offsets 0..r by Fornberg's recursion
// (Math. Comp. 51, 1988) on the nodes 0, 1, -1, 2, -2, ...
void weights(int p, double* c) {
  const int r = p / 2, N = 2 * r + 1, M = 2;
  double x[17];
  double d[3][17][17];
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
      for (int m = 0; m <= std::min(n, M); ++m)
        d[m][n][v] = (x[n] * d[m][n - 1][v] - m * (m ? d[m - 1][n - 1][v] : 0.0)) / c3;
    }
    for (int m = 0; m <= std::min(n, M); ++m)
      d[m][n][n] = c1 / c2 * (m * (m ? d[m - 1][n - 1][n - 1] : 0.0) - x[n - 1] * d[m][n - 1][n - 1]);
    c1 = c2;
  }
  c[0] = d[M][N - 1][0];
  for (int j = 1; j <= r; ++j) c[j] = 0.5 * (d[M][N - 1][2 * j - 1] + d[M][N - 1][2 * j]);
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

bool map(CUtensorMap* m, const void* base, int nx, int ny, int nz, int nzp, int slots,
         long long slot, int bz, int by) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[4] = {(cuuint64_t)nz, (cuuint64_t)ny, (cuuint64_t)nx, (cuuint64_t)(slots ? slots : 1)};
  cuuint64_t strides[3] = {(cuuint64_t)nzp * 4, (cuuint64_t)nzp * ny * 4, (cuuint64_t)slot * 4};
  cuuint32_t box[4] = {(cuuint32_t)bz, (cuuint32_t)by, 1, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, slots ? 4 : 3, const_cast<void*>(base), dims,
             strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace
}  // namespace fdw

using namespace fdw;

extern "C" fdw_status fdw_forward_static(int ndim, const int64_t* shape, const double* spacing,
                                         int space_order, int nbl, double dt, int nt, double vmax,
                                         const float* m, int nsrc, const double* src_xyz,
                                         const float* q, int nrec, const double* rec_xyz,
                                         float* rec, void* stream) {
  // ---- arguments and limits (host only)
  if (ndim != 2 && ndim != 3) return FDW_ERR_SHAPE;
  if (!shape || !spacing || !m) return FDW_ERR_ARG;
  if (space_order < 2 || space_order > 16 || space_order % 2) return FDW_ERR_ORDER;
  if (nbl < 0 || nt < 1 || !(dt > 0) || !(vmax > 0) || nsrc < 0 || nrec < 0) return FDW_ERR_ARG;
  if ((nsrc > 0 && (!src_xyz || !q)) || (nrec > 0 && (!rec_xyz || !rec))) return FDW_ERR_ARG;
  if (nsrc > kMaxPoints || nrec > kMaxPoints) return FDW_ERR_SHAPE;
  long long phys[3];
  double h[3];
  if (ndim == 3) {
    for (int a = 0; a < 3; ++a) { phys[a] = shape[a]; h[a] = spacing[a]; }
  } else {
    phys[0] = shape[0]; phys[1] = 1; phys[2] = shape[1];
    h[0] = spacing[0]; h[1] = 1.0; h[2] = spacing[1];
  }
  for (int a = 0; a < 3; ++a) {
    if (ndim == 2 && a == 1) continue;
    if (phys[a] < 2) return FDW_ERR_SHAPE;
    if (!(h[a] > 0)) return FDW_ERR_ARG;
  }
  const int nx = (int)std::min<long long>(phys[0] + 2LL * nbl, 1LL << 30);
  const int ny = ndim == 3 ? (int)std::min<long long>(phys[1] + 2LL * nbl, 1LL << 30) : 1;
  const int nz = (int)std::min<long long>(phys[2] + 2LL * nbl, 1LL << 30);
  if (nx > kMaxAxis || ny > kMaxAxis || nz > kMaxAxis) return FDW_ERR_SHAPE;
  const int nzp = (nz + 31) & ~31;
  const long long slot = (long long)nx * ny * nzp;
  if (slot > kMaxField) return FDW_ERR_SHAPE;
  const int r = space_order / 2;
  double c[9];
  weights(space_order, c);
  {
    double S = c[0];
    for (int j = 1; j <= r; ++j) S += 2.0 * ((j % 2) ? -1.0 : 1.0) * c[j];
    S = std::fabs(S);
    double acc = 0.0;
    for (int a = 0; a < 3; ++a)
      if (!(ndim == 2 && a == 1)) acc += S / (h[a] * h[a]);
    if (dt > 2.0 / (vmax * std::sqrt(acc))) return FDW_ERR_CFL;
  }

  // ---- the static array on this device (set-up once per device)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FDW_ERR_CUDA;
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static) != cudaSuccess || !p) {
      cudaGetLastError();
      return FDW_ERR_CUDA;
    }
    g_dev_ptr[dev] = static_cast<unsigned char*>(p);
  }
  unsigned char* base = g_dev_ptr[dev];
  float* d_u = reinterpret_cast<float*>(base + kOffU);
  float* d_model = reinterpret_cast<float*>(base + kOffModel);
  float* d_eta = reinterpret_cast<float*>(base + kOffEta);
  int* d_err = reinterpret_cast<int*>(base + kOffErr);

  // ---- tiling: the library's default tiles, one x chunk of up to 64 planes
  const int tile = (ny == 1) ? 3 : 0;
  const int TY = tile_rows(kTiles[tile]);
  const int lx = std::min(nx, 64);
  const int stages = r + 3;
  const int cx = (nx + lx - 1) / lx, cy = (ny + TY - 1) / TY, cz = (nz + kTZ - 1) / kTZ;
  const long long nunits = (long long)cx * cy * cz;
  if (nunits > kMaxUnits) return FDW_ERR_SHAPE;
  int U = 0;
  for (int i = 0; i < cx; ++i)
    for (int j = 0; j < cy; ++j)
      for (int k = 0; k < cz; ++k) {
        Unit& un = h_units[U++];
        std::memset(&un, 0, sizeof(un));
        un.shot = 0;
        un.x0 = i * lx;
        un.x1 = std::min(nx, (i + 1) * lx);
        un.y0 = j * TY;
        un.z0 = k * kTZ;
      }
  auto unit_of = [&](int x, int y, int z) { return ((x / lx) * cy + y / TY) * cz + z / kTZ; };

  // ---- points: base node and multilinear weights (same rule as fdw_set_*)
  auto locate = [&](const double* xyz, int j, int* b, double* f) -> bool {
    for (int a = 0; a < 3; ++a) {
      b[a] = 0;
      f[a] = 0.0;
      if (ndim == 2 && a == 1) continue;
      const int ua = (ndim == 2 && a == 2) ? 1 : a;
      const double xv = xyz[(size_t)j * ndim + ua];
      const double top = (double)(phys[a] - 1) * h[a];
      if (!(xv >= 0.0) || !(xv <= top)) return false;
      const double xi = xv / h[a];
      long long i = (long long)std::floor(xi);
      if (i < 0) i = 0;
      if (i > phys[a] - 2) i = phys[a] - 2;
      b[a] = (int)i + nbl;
      f[a] = xi - (double)i;
    }
    if (ndim == 2) b[1] = 0;
    return true;
  };
  auto corner_w = [&](const double* f, int cc) {
    const int bx = (cc >> 2) & 1, by = (cc >> 1) & 1, bz = cc & 1;
    double w = (bx ? f[0] : 1.0 - f[0]) * (bz ? f[2] : 1.0 - f[2]);
    if (ndim == 3) w *= by ? f[1] : 1.0 - f[1];
    else if (by) w = 0.0;
    return (float)w;
  };
  // receivers: sampled by the unit holding their base node
  for (int j = 0; j < nrec; ++j) {
    int b[3];
    double f[3];
    if (!locate(rec_xyz, j, b, f)) return FDW_ERR_OUT_OF_DOMAIN;
    for (int a = 0; a < 3; ++a) h_pt_base[3 * j + a] = b[a];
    for (int cc = 0; cc < 8; ++cc) h_pt_w[8 * j + cc] = corner_w(f, cc);
    h_smp_unit[j] = unit_of(b[0], b[1], b[2]);
  }
  std::fill(h_smp_ptr, h_smp_ptr + U + 1, 0);
  for (int j = 0; j < nrec; ++j) h_smp_ptr[h_smp_unit[j] + 1]++;
  for (int u = 0; u < U; ++u) h_smp_ptr[u + 1] += h_smp_ptr[u];
  {
    int fill[kMaxUnits];
    for (int u = 0; u < U; ++u) fill[u] = h_smp_ptr[u];
    for (int j = 0; j < nrec; ++j) h_smp_pts[fill[h_smp_unit[j]]++] = j;
  }
  // sources: one entry per (node, source) with a non-zero weight, grouped by
  // node in (unit, x, y, z, source) order
  int ncorner = 0;
  for (int j = 0; j < nsrc; ++j) {
    int b[3];
    double f[3];
    if (!locate(src_xyz, j, b, f)) return FDW_ERR_OUT_OF_DOMAIN;
    for (int cc = 0; cc < 8; ++cc) {
      const float w = corner_w(f, cc);
      if (w == 0.f) continue;
      Corner& e = h_corner[ncorner++];
      e.x = b[0] + ((cc >> 2) & 1);
      e.y = b[1] + ((cc >> 1) & 1);
      e.z = b[2] + (cc & 1);
      e.unit = unit_of(e.x, e.y, e.z);
      e.j = j;
      e.w = w;
    }
  }
  std::sort(h_corner, h_corner + ncorner, [](const Corner& a, const Corner& b) {
    if (a.unit != b.unit) return a.unit < b.unit;
    if (a.x != b.x) return a.x < b.x;
    if (a.y != b.y) return a.y < b.y;
    if (a.z != b.z) return a.z < b.z;
    return a.j < b.j;
  });
  int nnodes = 0;
  std::fill(h_inj_ptr, h_inj_ptr + U + 1, 0);
  for (int i = 0; i < ncorner; ++i) {
    const Corner& e = h_corner[i];
    h_terms[i].j = e.j;
    h_terms[i].w = e.w;
    const bool fresh = i == 0 || e.unit != h_corner[i - 1].unit || e.x != h_corner[i - 1].x ||
                       e.y != h_corner[i - 1].y || e.z != h_corner[i - 1].z;
    if (fresh) {
      InjNode& nd = h_nodes[nnodes++];
      std::memset(&nd, 0, sizeof(nd));
      nd.x = e.x;
      nd.y = e.y;
      nd.z = e.z;
      nd.tbeg = i;
      h_inj_ptr[e.unit + 1]++;
    }
    h_nodes[nnodes - 1].tend = i + 1;
  }
  for (int u = 0; u < U; ++u) h_inj_ptr[u + 1] += h_inj_ptr[u];

  // ---- damping profiles eta*dt/2 (built-in quadratic profile)
  const int n3[3] = {nx, ny, nz};
  int off = 0;
  for (int a = 0; a < 3; ++a) {
    for (int i = 0; i < n3[a]; ++i) {
      double e = 0.0;
      if (!(ndim == 2 && a == 1) && nbl > 0) {
        const long long lo = nbl - i, hi = i - (nbl + phys[a] - 1);
        const long long dd = lo > 0 ? lo : (hi > 0 ? hi : 0);
        const double emax = 3.0 * std::log(1000.0) / (2.0 * nbl * h[a] * vmax);
        const double fr = (double)dd / nbl;
        e = emax * fr * fr;
      }
      h_eta[off + i] = (float)(e * dt * 0.5);
    }
    off += n3[a];
  }

  // ---- shot descriptor
  std::memset(&h_desc, 0, sizeof(h_desc));
  const int R4 = (r + 3) & ~3;
  if (!map(&h_desc.tm_uh, d_u, nx, ny, nz, nzp, 2, slot, kTZ + 2 * R4, TY + 2 * r) ||
      !map(&h_desc.tm_uc, d_u, nx, ny, nz, nzp, 2, slot, kTZ, TY) ||
      !map(&h_desc.tm_m, d_model, nx, ny, nz, nzp, 0, slot, kTZ, TY))
    return FDW_ERR_CUDA;
  h_desc.u = d_u;
  h_desc.uslot = slot;
  h_desc.m = d_model;
  h_desc.eta = d_eta;
  h_desc.nx = nx; h_desc.ny = ny; h_desc.nz = nz; h_desc.nzp = nzp;
  h_desc.mtype = kF32;
  h_desc.smp_n = nrec;
  h_desc.inj_a = q;
  h_desc.inj_ld = nsrc;
  h_desc.smp_out = rec;
  h_desc.smp_ld = nrec;
  h_desc.pt_base = reinterpret_cast<const int*>(base + kOffPtBase);
  h_desc.pt_w = reinterpret_cast<const float*>(base + kOffPtW);

  // ---- upload, clear, model
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto put = [&](size_t o, const void* src, size_t bytes) {
    return bytes == 0 || cudaMemcpyAsync(base + o, src, bytes, cudaMemcpyHostToDevice, s) == cudaSuccess;
  };
  bool ok = put(kOffDesc, &h_desc, sizeof(h_desc)) && put(kOffUnits, h_units, sizeof(Unit) * U) &&
            put(kOffInjPtr, h_inj_ptr, sizeof(int) * (U + 1)) &&
            put(kOffNodes, h_nodes, sizeof(InjNode) * nnodes) &&
            put(kOffTerms, h_terms, sizeof(InjTerm) * ncorner) &&
            put(kOffSmpPtr, h_smp_ptr, sizeof(int) * (U + 1)) &&
            put(kOffSmpPts, h_smp_pts, sizeof(int) * nrec) &&
            put(kOffPtBase, h_pt_base, sizeof(int) * 3 * nrec) &&
            put(kOffPtW, h_pt_w, sizeof(float) * 8 * nrec) &&
            put(kOffEta, h_eta, sizeof(float) * (nx + ny + nz));
  ok = ok && cudaMemsetAsync(d_u, 0, sizeof(float) * 2 * slot, s) == cudaSuccess &&
       cudaMemsetAsync(d_model, 0, sizeof(float) * slot, s) == cudaSuccess &&
       cudaMemsetAsync(d_err, 0, sizeof(int), s) == cudaSuccess;
  ok = ok && launch_model(m, 0, (int)phys[0], (int)phys[1], (int)phys[2], nbl, ndim, d_model, kF32,
                          Geom{nx, ny, nz, nzp}, s) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return FDW_ERR_CUDA;
  }

  // ---- time loop: the forward step kernel of fdw_forward, one launch per step
  const void* fn = nullptr;
  switch (r) {
    case 1: fn = step_kernel_r1(tile, false); break;
    case 2: fn = step_kernel_r2(tile, false); break;
    case 3: fn = step_kernel_r3(tile, false); break;
    case 4: fn = step_kernel_r4(tile, false); break;
    case 5: fn = step_kernel_r5(tile, false); break;
    case 6: fn = step_kernel_r6(tile, false); break;
    case 7: fn = step_kernel_r7(tile, false); break;
    case 8: fn = step_kernel_r8(tile, false); break;
  }
  const int ZW = kTZ + 2 * R4, YW = TY + 2 * r;
  auto r128 = [](int x) { return (x + 127) & ~127; };
  StepParams P;
  std::memset(&P, 0, sizeof(P));
  P.shots = reinterpret_cast<const ShotDesc*>(base + kOffDesc);
  P.units = reinterpret_cast<const Unit*>(base + kOffUnits);
  P.nunits = U;
  P.flags = (nsrc > 0 ? kInject : 0) | (nrec > 0 ? kSample : 0);
  P.inj_ptr = reinterpret_cast<const int*>(base + kOffInjPtr);
  P.inj_nodes = reinterpret_cast<const InjNode*>(base + kOffNodes);
  P.inj_terms = reinterpret_cast<const InjTerm*>(base + kOffTerms);
  P.smp_ptr = reinterpret_cast<const int*>(base + kOffSmpPtr);
  P.smp_pts = reinterpret_cast<const int*>(base + kOffSmpPts);
  P.stages = stages;
  P.off_p = r128(YW * ZW * 4);
  P.off_m = P.off_p + r128(TY * kTZ * 4);
  P.off_f = P.off_m + r128(TY * kTZ * 4);
  P.off_e = P.off_f;
  P.stage_bytes = P.off_f;
  P.dt2 = (float)(dt * dt);
  double csum = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double sc = (ndim == 2 && a == 1) ? 0.0 : dt * dt / (h[a] * h[a]);
    for (int k = 0; k <= kMaxR; ++k) P.w[a][k] = (k <= r) ? (float)(c[k] * sc) : 0.f;
    csum += c[0] * sc;
  }
  P.csum = (float)csum;
  P.err = d_err;
  const size_t smem = (size_t)stages * P.stage_bytes + (size_t)(2 * stages + 1) * 8 + 128;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return FDW_ERR_CUDA;
  }
  const int threads = (kTiles[tile].warps + 1) * 32;
  int nb = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return FDW_ERR_CUDA;
  }
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(std::max(1, std::min(U, std::max(nb, 1) * sms)));
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  for (int n = 0; n + 1 < nt; ++n) {
    P.cur = n & 1;
    P.prev = P.out = (n + 1) & 1;
    P.inj_row = n;
    P.smp_row = n;
    void* args[] = {&P};
    if (cudaLaunchKernelExC(&cfg, fn, args) != cudaSuccess) {
      cudaGetLastError();
      return FDW_ERR_CUDA;
    }
  }
  if (nrec > 0 && launch_sample(P.shots, 1, nrec, (nt - 1) & 1, nt - 1, s) != cudaSuccess) {
    cudaGetLastError();
    return FDW_ERR_CUDA;
  }
  // report the device-side error word of this call
  int err = 0;
  if (cudaStreamSynchronize(s) != cudaSuccess ||
      cudaMemcpy(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return FDW_ERR_CUDA;
  }
  return err ? FDW_ERR_TIMEOUT : FDW_OK;
}
