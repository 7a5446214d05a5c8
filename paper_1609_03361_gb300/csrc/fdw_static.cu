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
//
// The readings of the method (stencil weights, stability limit, point
// location and weights, damping profile, tiles, injection and sampling lists,
// stage layout) come from fdw_host.h, the same code the context runtime uses,
// so this path computes bit for bit what fdw_forward computes with the same
// tiling (tile 0 in 3D, tile 3 in 2D, x chunks of 64 planes, r + 3 stages).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "fdw_host.h"
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

bool map_f32(CUtensorMap* m, const void* base, int nx, int ny, int nz, int nzp, int slots,
             long long slot, int bz, int by) {
  return encode_field_map(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, nx, ny, nz, nzp, slots,
                          slot, bz, by) == CUDA_SUCCESS;
}

}  // namespace
}  // namespace fdw

using namespace fdw;

extern "C" fdw_status fdw_forward_static(int ndim, const int64_t* shape, const double* spacing,
                                         int space_order, int nbl, double dt, int nt, double vmax,
                                         const float* m, int nsrc, const double* src_xyz,
                                         const float* q, int nrec, const double* rec_xyz,
                                         float* rec, void* stream) {
  // ---- arguments, limits, stability and points: host only, before any CUDA call
  if (ndim != 2 && ndim != 3) return FDW_ERR_SHAPE;
  if (!shape || !spacing || !m) return FDW_ERR_ARG;
  if (!valid_order(space_order)) return FDW_ERR_ORDER;
  if (nbl < 0 || nt < 1 || !(dt > 0) || !(vmax > 0) || nsrc < 0 || nrec < 0) return FDW_ERR_ARG;
  if ((nsrc > 0 && (!src_xyz || !q)) || (nrec > 0 && (!rec_xyz || !rec))) return FDW_ERR_ARG;
  if (nsrc > kMaxPoints || nrec > kMaxPoints) return FDW_ERR_SHAPE;
  const GridGeom g = grid_geom(ndim, shape, spacing, nbl);
  for (int a = 0; a < ndim; ++a) {
    if (shape[a] < 2) return FDW_ERR_SHAPE;
    if (!(spacing[a] > 0)) return FDW_ERR_ARG;
  }
  long long n3[3];
  for (int a = 0; a < 3; ++a) n3[a] = g.active(a) ? g.phys[a] + 2LL * nbl : 1;
  if (n3[0] > kMaxAxis || n3[1] > kMaxAxis || n3[2] > kMaxAxis) return FDW_ERR_SHAPE;
  const int nx = (int)n3[0], ny = (int)n3[1], nz = (int)n3[2];
  const int nzp = (nz + 31) & ~31;
  const long long slot = (long long)nx * ny * nzp;
  if (slot > kMaxField) return FDW_ERR_SHAPE;
  if (dt > dt_limit(ndim, spacing, space_order, vmax)) return FDW_ERR_CFL;
  const int r = space_order / 2;

  // tiling: tile 0 (3D) or 3 (2D), x chunks of up to 64 planes, r + 3 stages
  const int tile = (ny == 1) ? 3 : 0;
  const int TY = tile_rows(kTiles[tile]);
  const int lx = std::min(nx, 64);
  const int stages = r + 3;
  const int cx = (nx + lx - 1) / lx;
  int cy = 0, cz = 0;
  column_tiles(ny, nz, TY, &cy, &cz);
  const long long nunits = (long long)cx * cy * cz;
  if (nunits > kMaxUnits) return FDW_ERR_SHAPE;
  const int U = (int)nunits;
  for (int i = 0; i < cx; ++i)
    for (int li = 0; li < cy * cz; ++li)
      h_units[i * cy * cz + li] = make_unit(0, i * lx, std::min(nx, (i + 1) * lx), li, cz, TY);
  auto unit_of = [&](int x, int y, int z) { return ((x / lx) * cy + y / TY) * cz + z / kTZ; };

  // receivers: sampled by the unit holding their base node
  for (int j = 0; j < nrec; ++j) {
    int b[3];
    double f[3];
    if (locate_point(g, rec_xyz + (size_t)j * ndim, b, f) >= 0) return FDW_ERR_OUT_OF_DOMAIN;
    for (int a = 0; a < 3; ++a) h_pt_base[3 * j + a] = b[a];
    for (int cc = 0; cc < 8; ++cc) h_pt_w[8 * j + cc] = corner_weight(g, f, cc);
    h_smp_unit[j] = unit_of(b[0], b[1], b[2]);
  }
  bucket_points(h_smp_unit, nrec, U, h_smp_ptr, h_smp_pts);
  // sources: one term per (node, source) with a non-zero weight, grouped by node
  int ncorner = 0;
  for (int j = 0; j < nsrc; ++j) {
    int b[3];
    double f[3];
    if (locate_point(g, src_xyz + (size_t)j * ndim, b, f) >= 0) return FDW_ERR_OUT_OF_DOMAIN;
    for (int cc = 0; cc < 8; ++cc) {
      const float w = corner_weight(g, f, cc);
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
  const int nnodes = group_corners(h_corner, ncorner, U, h_nodes, h_terms, h_inj_ptr);

  // damping profiles eta*dt/2 (built-in quadratic profile)
  {
    int off = 0;
    for (int a = 0; a < 3; ++a) {
      for (int i = 0; i < (int)n3[a]; ++i) h_eta[off + i] = damping_half_dt(g, a, i, vmax, dt);
      off += (int)n3[a];
    }
  }

  // ---- device arrays of the caller: device (or managed) memory only; a host
  // pointer would reach the kernels as a global address
  if (!is_device_ptr(m) || (nsrc > 0 && !is_device_ptr(q)) || (nrec > 0 && !is_device_ptr(rec)))
    return FDW_ERR_ARG;

  // ---- the static array on this device (set-up once per device)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return FDW_ERR_CUDA;
  }
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

  // ---- shot descriptor
  std::memset(&h_desc, 0, sizeof(h_desc));
  const int R4 = (r + 3) & ~3;
  if (!map_f32(&h_desc.tm_uh, d_u, nx, ny, nz, nzp, 2, slot, kTZ + 2 * R4, TY + 2 * r) ||
      !map_f32(&h_desc.tm_uc, d_u, nx, ny, nz, nzp, 2, slot, kTZ, TY) ||
      !map_f32(&h_desc.tm_m, d_model, nx, ny, nz, nzp, 0, slot, kTZ, TY))
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
  ok = ok && launch_model(m, 0, (int)g.phys[0], (int)g.phys[1], (int)g.phys[2], nbl, ndim, d_model,
                          kF32, Geom{nx, ny, nz, nzp}, s) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return FDW_ERR_CUDA;
  }

  // ---- time loop: the forward step kernel of fdw_forward, one launch per step
  const void* fn = step_fn(r, tile, false);
  const StageLayout L = stage_layout(r, tile, 4, false, false);
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
  P.stage_bytes = L.bytes;
  P.off_p = L.off_p;
  P.off_m = L.off_m;
  P.off_f = L.off_f;
  P.off_a = L.off_a;
  P.off_e = L.off_e;
  P.dt2 = (float)(dt * dt);
  {
    double c[kMaxR + 1];
    fd_weights(space_order, c);
    double csum = 0.0;
    for (int a = 0; a < 3; ++a) {
      const double sc = g.active(a) ? dt * dt / (g.h[a] * g.h[a]) : 0.0;
      for (int k = 0; k <= kMaxR; ++k) P.w[a][k] = (k <= r) ? (float)(c[k] * sc) : 0.f;
      csum += c[0] * sc;
    }
    P.csum = (float)csum;
  }
  P.err = d_err;
  const size_t smem = smem_bytes(L, stages);
  const int threads = (kTiles[tile].warps + 1) * 32;
  int nb = 0, sms = 0;
  if (raise_smem_limit(fn, smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess ||
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
  return device_error_status(err);
}
