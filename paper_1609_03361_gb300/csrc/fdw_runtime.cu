// Host runtime and C ABI of libfdwave.
//
// A context (fdw_ctx) owns one shot: its grid, model, damping, wavefield
// buffers, sparse points and checkpoint store.  A plan (Plan) turns one or more
// contexts into what the time-step kernel walks: a table of work units (one
// column tile of a shot streamed along an x chunk), per-unit injection and
// sampling lists for each role (forward, adjoint, recompute) and per-shot
// descriptors with TMA tensor maps.  Time loops are captured once into CUDA
// graphs and replayed.  Each step launch gets its own unit-ticket counter
// (CTAs take units in table order as they become free); adjoint steps inject
// their data in a separate launch.  The gradient pass replays either one
// checkpoint pair per k steps or a binomial schedule under a memory budget; a
// context may also be an x slab of a larger grid with ghost planes
// (single-shot domain decomposition).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <memory>
#include <sstream>
#include <string>
#include <tuple>
#include <vector>

#include "fdw_host.h"
#include "fdw_internal.h"
#include "fdw_tb.h"
#include "fdwave.h"

namespace fdw {

// ---------------------------------------------------------------- errors

struct Error {
  fdw_status st;
  std::string msg;
};

[[noreturn]] static void fail(fdw_status st, const std::string& msg) { throw Error{st, msg}; }

static void cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return;
  cudaGetLastError();
  if (e == cudaErrorMemoryAllocation) fail(FDW_ERR_OOM, std::string(what) + ": out of device memory");
  fail(FDW_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define CK(call) cuda_check((call), #call)

static bool env_flag(const char* name) {
  const char* v = std::getenv(name);
  return v && *v && std::strcmp(v, "0") != 0;
}

// Test hook: while the environment variable FDW_TEST_FAIL_ALLOC is set (and
// not "0"), every device allocation of the library fails as an exhausted
// device would, without calling the allocator, so that the tests can check
// that a failed allocation reports FDW_ERR_OOM and leaves the context usable.
template <class T>
static T* dalloc(size_t count) {
  void* p = nullptr;
  if (count == 0) count = 1;
  if (env_flag("FDW_TEST_FAIL_ALLOC")) fail(FDW_ERR_OOM, "cudaMalloc: out of device memory (test hook)");
  cuda_check(cudaMalloc(&p, count * sizeof(T)), "cudaMalloc");
  return static_cast<T*>(p);
}

static void dfree(void* p) {
  if (p) cudaFree(p);
}

// ---------------------------------------------------------------- TMA maps

// Pitched field(s) [slots][nx][ny][nzp] of element type dt; rank 3 when slots == 0.
static void make_map(CUtensorMap* map, CUtensorMapDataType dt, int esize, const void* base,
                     int nx, int ny, int nz, int nzp, int slots, long long slot_elems, int box_z,
                     int box_y) {
  const CUresult r = encode_field_map(map, dt, esize, base, nx, ny, nz, nzp, slots, slot_elems,
                                      box_z, box_y);
  if (r != CUDA_SUCCESS) {
    std::ostringstream os;
    os << "cuTensorMapEncodeTiled failed (" << (int)r << ") dims " << nz << "x" << ny << "x" << nx
       << " box " << box_z << "x" << box_y;
    fail(FDW_ERR_CUDA, os.str());
  }
}

// ---------------------------------------------------------------- kernels

static int device_sms(int dev) {
  int v = 0;
  CK(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
  return v;
}

static int device_smem_optin(int dev) {
  int v = 0;
  CK(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  return v;
}

}  // namespace fdw

using namespace fdw;

// ---------------------------------------------------------------- points

struct PointSet {
  int n = 0;
  std::vector<double> xyz;   // [n][ndim]
  std::vector<int> base;     // [n][3] computational base node (internal x, y, z)
  std::vector<float> w;      // [n][8]
  int* d_base = nullptr;
  float* d_w = nullptr;
  void release() {
    dfree(d_base);
    dfree(d_w);
    d_base = nullptr;
    d_w = nullptr;
  }
};

struct Plan;

struct fdw_ctx {
  int device = 0;
  int ndim = 3;
  int64_t phys[3] = {1, 1, 1};  // internal (x, y, z); y = 1 in 2D
  int nx = 1, ny = 1, nz = 1, nzp = 32;
  double h[3] = {1, 1, 1};      // internal (x, y, z)
  int order = 2, r = 1, nbl = 0;
  double dt = 1.0;
  int nt = 1;
  double vmax = 1.0;
  long long slot = 0;           // floats per pitched field

  float* u = nullptr;           // uslots slots (4 with two steps per pass)
  int uslots = 2;
  // forward passes of two time steps (fdw_set_time_blocking) and their tiling
  int tblock = 1;
  int tb_variant = -1, tb_lx = 0, tb_stages = 0;
  void* m = nullptr;
  int mtype = kF32;
  bool model_set = false;
  float* eta = nullptr;         // eta*dt/2 profiles [nx + ny + nz]
  std::vector<float> eta_host;  // the same profiles on the host
  float* etaf = nullptr;        // eta*dt/2 field (pitched)
  bool use_etaf = false;
  PointSet src, rec;
  int points_version = 0;

  // checkpoint store
  int ckpt_k = 0, snap_type = -1, nsnap = 0;
  int ckpt_budget = 0;          // most checkpoint pairs to store (0: one per k steps)
  // x slab of a larger grid (fdw_create_slab): local plane i is plane i + gx0
  // of the full computational grid of nx_full planes; the planes
  // [own0, own1) are updated here, the r planes on either side are ghosts
  bool slab = false;
  int gx0 = 0, nx_full = 0, own0 = 0, own1 = 0;
  bool revolve = false;         // checkpoints follow a binomial schedule
  void* snaps = nullptr;
  unsigned int* amax = nullptr;
  float* seg = nullptr;         // k+1 slots
  int seg_slots = 0;
  float* lam = nullptr;         // 2 slots
  float* acc = nullptr;         // 1 slot
  float* qsave = nullptr;
  bool have_ckpt = false;
  bool fwd_done = false, adj_done = false;
  int buffers_version = 0;

  // tiling override
  int tile = -1, xchunk = 0, stages = 0;
  // plain forward passes run as one persistent launch over all time steps
  // (slabs step one launch at a time)
  bool persist = true;

  // staging buffers for host arrays
  std::map<int, std::pair<void*, size_t>> staging;

  std::unique_ptr<Plan> plan;
  std::string err;
  ~fdw_ctx();
};

enum Role { kRoleFwd = 0, kRoleAdj = 1, kRoleRec = 2, kNumRoles = 3 };

struct RoleLists {
  std::vector<int> inj_ptr, smp_ptr, smp_pts, node_shot;
  std::vector<InjNode> nodes;
  std::vector<InjTerm> terms;
  int* d_inj_ptr = nullptr;
  int* d_smp_ptr = nullptr;
  int* d_smp_pts = nullptr;
  int* d_node_shot = nullptr;  // shot of each injection node (separate injection launches)
  InjNode* d_nodes = nullptr;
  InjTerm* d_terms = nullptr;
  void release() {
    dfree(d_inj_ptr); dfree(d_smp_ptr); dfree(d_smp_pts); dfree(d_nodes); dfree(d_terms);
    dfree(d_node_shot);
    d_node_shot = nullptr;
    d_inj_ptr = d_smp_ptr = d_smp_pts = nullptr;
    d_nodes = nullptr;
    d_terms = nullptr;
  }
};

struct Plan {
  std::vector<fdw_ctx*> shots;
  int device = 0;
  int r = 1;
  int tile = 0, lx = 16, stages = 8;
  int tile_req = -1, lx_req = 0, stages_req = 0;
  std::vector<Unit> units;
  Unit* d_units = nullptr;
  // rows of units (one x chunk of one shot with all its column tiles): the
  // rows a row's units read, units per row, finished units per row
  int nrows = 0;
  int2* d_row_deps = nullptr;
  int* d_row_units = nullptr;
  int* d_row_done = nullptr;
  RoleLists lists[kNumRoles];
  std::vector<ShotDesc> hdesc[kNumRoles];
  ShotDesc* d_desc[kNumRoles] = {nullptr, nullptr, nullptr};
  int* d_err = nullptr;
  cudaStream_t cap = nullptr;
  std::map<std::string, cudaGraphExec_t> graphs;
  // aux descriptors for snapshots: [nsnap][nshots] pack and unpack
  AuxShot* d_pack = nullptr;
  AuxShot* d_unpack = nullptr;
  // binomial schedule: actions, and snapshot descriptors [variant][slot][shot]
  // (variant 0/1: the forward wavefield pair with u^{t} in slot 0/1, variant
  // 2/3: the segment-buffer pair with the newer field in slot 0/1)
  std::vector<CkptAction> rv_actions;
  int rv_nseg = -1, rv_slots = -1;
  AuxShot* d_rv = nullptr;
  int aux_version = -1;
  std::vector<int> built_versions;   // points/buffers versions the lists and maps were built for
  struct LaunchInfo {
    const void* fn;
    int grid, threads, stages, cstages, cstage_bytes;
    size_t smem;
    int stage_bytes, off_p, off_m, off_f, off_a, off_e, off_c;
    int resident;  // CTAs that fit on the device at once
  };
  std::map<std::tuple<int, int, int, int, int, int>, LaunchInfo> launch_cache;
  std::vector<double> weights;       // unscaled second-derivative weights c_0..c_r
  bool built = false;
  int max_rec = 0, max_src = 0;
  bool test_stall = false;  // FDW_TEST_STALL: make every step's waits run out (tests only)
  long long max_points = 0;
  long long max_slot = 0;            // floats per pitched field, largest shot
  int grad_stages = 0, grad_stages_tile = -1;  // pipeline depth of the gradient step
  // two-step forward passes: their own units (output tiles of TY x 56 points),
  // injection and sampling lists, shot descriptors and launch shape
  struct Tb {
    bool built = false;
    int variant = 0, lx = 0, stages = 0;
    std::vector<Unit> units;
    std::vector<TbShot> hshots;
    Unit* d_units = nullptr;
    TbShot* d_shots = nullptr;
    int* d_inj_ptr = nullptr;
    int* d_ext_ptr = nullptr;
    int* d_smp_ptr = nullptr;
    int* d_smp_pts = nullptr;
    InjNode* d_inj_nodes = nullptr;
    InjNode* d_ext_nodes = nullptr;
    InjTerm* d_inj_terms = nullptr;
    InjTerm* d_ext_terms = nullptr;
    const void* fn = nullptr;
    int grid = 0, threads = 0, stage_bytes = 0, off_p = 0, off_s = 0;
    size_t smem = 0;
    void release() {
      dfree(d_units); dfree(d_shots); dfree(d_inj_ptr); dfree(d_ext_ptr); dfree(d_smp_ptr);
      dfree(d_smp_pts); dfree(d_inj_nodes); dfree(d_ext_nodes); dfree(d_inj_terms);
      dfree(d_ext_terms);
      d_units = nullptr; d_shots = nullptr;
      d_inj_ptr = d_ext_ptr = d_smp_ptr = d_smp_pts = nullptr;
      d_inj_nodes = d_ext_nodes = nullptr;
      d_inj_terms = d_ext_terms = nullptr;
      units.clear();
      hshots.clear();
      built = false;
    }
  } tb;
  // one unit-ticket counter per step launch of a pass, zeroed at the pass start
  int* d_tickets = nullptr;
  int ticket_cap = 0, ticket_next = 0;

  void clear_graphs() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    graphs.clear();
  }
  void release_lists() {
    for (auto& l : lists) l.release();
    dfree(d_units);
    dfree(d_row_deps);
    dfree(d_row_units);
    dfree(d_row_done);
    d_units = nullptr;
    d_row_deps = nullptr;
    d_row_units = nullptr;
    d_row_done = nullptr;
    nrows = 0;
  }
  ~Plan() {
    clear_graphs();
    release_lists();
    for (auto& d : d_desc) dfree(d);
    dfree(d_err);
    dfree(d_tickets);
    dfree(d_pack);
    dfree(d_unpack);
    dfree(d_rv);
    tb.release();
    if (cap) cudaStreamDestroy(cap);
  }
};

fdw_ctx::~fdw_ctx() {
  plan.reset();
  dfree(u); dfree(m); dfree(eta); dfree(etaf);
  src.release(); rec.release();
  dfree(snaps); dfree(amax); dfree(seg); dfree(lam); dfree(acc); dfree(qsave);
  for (auto& kv : staging) dfree(kv.second.first);
}

struct fdw_batch {
  std::vector<fdw_ctx*> shots;
  std::unique_ptr<Plan> plan;
  std::string err;
};

// ---------------------------------------------------------------- helpers

static int msize(int t) { return t == kF32 ? 4 : 2; }

static void* staging_buf(fdw_ctx* c, int key, size_t bytes) {
  auto it = c->staging.find(key);
  if (it != c->staging.end() && it->second.second >= bytes) return it->second.first;
  if (it != c->staging.end()) {  // dropped first: a failed allocation leaves no stale entry
    dfree(it->second.first);
    c->staging.erase(it);
  }
  void* p = dalloc<unsigned char>(bytes);
  c->staging[key] = {p, bytes};
  return p;
}

// Device view of a caller input array (copied when it lives on the host).
static const float* device_in(fdw_ctx* c, int key, const float* p, size_t count, cudaStream_t s) {
  if (!p || count == 0) return p;
  if (is_device_ptr(p)) return p;
  float* d = static_cast<float*>(staging_buf(c, key, count * sizeof(float)));
  CK(cudaMemcpyAsync(d, p, count * sizeof(float), cudaMemcpyHostToDevice, s));
  return d;
}

// Device buffer for a caller output array; copy_back() is needed when host.
static float* device_out(fdw_ctx* c, int key, float* p, size_t count, bool* host) {
  *host = false;
  if (!p || count == 0) return p;
  if (is_device_ptr(p)) return p;
  *host = true;
  return static_cast<float*>(staging_buf(c, key, count * sizeof(float)));
}

static void set_device(int dev) { CK(cudaSetDevice(dev)); }

// ---------------------------------------------------------------- points

static GridGeom ctx_geom(const fdw_ctx* c) {
  GridGeom g;
  g.ndim = c->ndim;
  g.nbl = c->nbl;
  for (int a = 0; a < 3; ++a) {
    g.phys[a] = c->phys[a];
    g.h[a] = c->h[a];
  }
  return g;
}

// samples: the set is sampled (receivers of the forward step) rather than
// injected; it decides which points a slab keeps.
static void compute_points(fdw_ctx* c, PointSet& ps, int n, const double* xyz, bool samples) {
  if (n < 0 || (n > 0 && !xyz)) fail(FDW_ERR_ARG, "bad point array");
  PointSet out;
  out.n = n;
  out.xyz.assign(xyz, xyz + (size_t)n * c->ndim);
  out.base.resize((size_t)n * 3);
  out.w.resize((size_t)n * 8);
  // internal axes: 3D (x, y, z); 2D (x, -, z) with user axes (x, z)
  const GridGeom g = ctx_geom(c);
  for (int j = 0; j < n; ++j) {
    int b[3];
    double f[3];
    const int bad = locate_point(g, xyz + (size_t)j * c->ndim, b, f);
    if (bad >= 0) {
      const int ia = (c->ndim == 2 && bad == 1) ? 2 : bad;
      std::ostringstream os;
      os << "point " << j << " coordinate " << bad << " = " << xyz[(size_t)j * c->ndim + bad]
         << " outside [0, " << (double)(c->phys[ia] - 1) * c->h[ia] << "]";
      fail(FDW_ERR_OUT_OF_DOMAIN, os.str());
    }
    // a slab keeps local x indices: a source keeps the corners in its planes,
    // a receiver is kept whole by the slab that owns its base plane (its
    // other corners are read from the ghost planes); everything else gets zero
    // weights and a base inside the slab, so it is never touched
    bool keep_point = true;
    if (c->slab) {
      b[0] -= c->gx0;
      if (samples && (b[0] < c->own0 || b[0] >= c->own1)) {
        keep_point = false;
        b[0] = c->own0;
      }
    }
    for (int a = 0; a < 3; ++a) out.base[(size_t)j * 3 + a] = (c->ndim == 2 && a == 1) ? 0 : b[a];
    for (int cc = 0; cc < 8; ++cc) {
      const int bx = (cc >> 2) & 1;
      float w = corner_weight(g, f, cc);
      if (!keep_point) w = 0.f;
      if (c->slab && !samples && (b[0] + bx < c->own0 || b[0] + bx >= c->own1)) w = 0.f;
      out.w[(size_t)j * 8 + cc] = w;
    }
    if (c->slab && !samples) {  // a base outside the slab: keep it inside (weights are zero)
      const int bxl = out.base[(size_t)j * 3];
      if (bxl + 1 < c->own0 || bxl >= c->own1) out.base[(size_t)j * 3] = c->own0;
    }
  }
  if (n > 0) {
    try {  // the context keeps its previous points if this fails
      out.d_base = dalloc<int>((size_t)n * 3);
      out.d_w = dalloc<float>((size_t)n * 8);
      CK(cudaMemcpy(out.d_base, out.base.data(), sizeof(int) * n * 3, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(out.d_w, out.w.data(), sizeof(float) * n * 8, cudaMemcpyHostToDevice));
    } catch (...) {
      out.release();
      throw;
    }
  }
  ps.release();
  ps = std::move(out);
  c->points_version++;
}

// ---------------------------------------------------------------- plan

static int plan_mtype(const Plan& pl) { return pl.shots[0]->mtype; }
static bool plan_etaf(const Plan& pl) {
  for (auto* c : pl.shots)
    if (c->use_etaf) return true;
  return false;
}

static void configure_kernel(const void* fn, size_t smem) { CK(raise_smem_limit(fn, smem)); }

// Resident CTAs per SM of a step launch.  For tiles whose x queue lives in
// tensor memory the runtime's occupancy query reports one CTA per SM (it
// treats any kernel that allocates tensor memory that way), while the SM
// holds as many as its registers, shared memory and threads allow (measured
// on the GB300): count those directly.
static int occupancy(const Plan& pl, int tile, const void* fn, int threads, size_t smem) {
  int nb = 0;
  if (!kTiles[tile].tq) {
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem));
    return nb;
  }
  cudaFuncAttributes a;
  CK(cudaFuncGetAttributes(&a, fn));
  int regs_sm = 0, smem_sm = 0, reserved = 0, threads_sm = 0, blocks_sm = 0;
  CK(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, pl.device));
  CK(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, pl.device));
  CK(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, pl.device));
  CK(cudaDeviceGetAttribute(&threads_sm, cudaDevAttrMaxThreadsPerMultiProcessor, pl.device));
  CK(cudaDeviceGetAttribute(&blocks_sm, cudaDevAttrMaxBlocksPerMultiprocessor, pl.device));
  const int warps = (threads + 31) / 32;
  const int regs_warp = ((a.numRegs + 7) / 8) * 8 * 32;   // allocated in units of 256 per warp
  const int by_regs = regs_sm / (regs_warp * warps);
  const int by_smem = (int)((size_t)smem_sm / (smem + a.sharedSizeBytes + (size_t)reserved));
  const int by_threads = threads_sm / (warps * 32);
  nb = std::min(std::min(by_regs, by_smem), std::min(by_threads, blocks_sm));
  return std::min(nb, 512 / tq_columns(pl.r));
}

// Dynamic shared memory of a step launch: the stage rings, and for a tile
// whose x queue lives in tensor memory, more if needed so that no more than
// 512 / tq_columns(r) CTAs fit on an SM: each CTA allocates that many of the
// SM's 512 columns, and a CTA that found too few free would wait in its
// allocation until another CTA on the SM finished.
static size_t launch_smem(const Plan& pl, int tile, const StageLayout& L, int stages,
                          const void* fn, int threads) {
  size_t smem = smem_bytes(L, stages);
  configure_kernel(fn, smem);
  if (!kTiles[tile].tq) return smem;
  const int maxc = 512 / tq_columns(pl.r);
  int smem_sm = 0, reserved = 0;
  CK(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, pl.device));
  CK(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, pl.device));
  cudaFuncAttributes a;
  CK(cudaFuncGetAttributes(&a, fn));
  // the shared memory alone must keep a (maxc + 1)-th CTA out
  const size_t need = (size_t)smem_sm / (maxc + 1) + 1 - a.sharedSizeBytes - reserved;
  if (smem < need) smem = (need + 127) & ~size_t(127);
  if (smem > (size_t)device_smem_optin(pl.device))
    fail(FDW_ERR_ARG, "tensor-memory tile: cannot limit the CTAs per SM");
  configure_kernel(fn, smem);
  return smem;
}

// Occupancy-limited number of resident CTAs of a launch.
static int resident_ctas(const Plan& pl, int tile, int stages, bool grad) {
  const StageLayout L = stage_layout(pl.r, tile, msize(plan_mtype(pl)), grad, plan_etaf(pl));
  const void* fn = step_fn(pl.r, tile, grad);
  const int threads = (kTiles[tile].warps + 1) * 32;
  const size_t smem = launch_smem(pl, tile, L, stages, fn, threads);
  const int nb = occupancy(pl, tile, fn, threads, smem);
  return std::max(nb, 1) * device_sms(pl.device);
}

static int max_stages(const Plan& pl, int tile) {
  const StageLayout L = stage_layout(pl.r, tile, 4, false, true);
  const int cap = device_smem_optin(pl.device) - 1024;  // static shared memory and slack
  int s = 2 * pl.r + 8;
  while (s > min_stages(pl.r, tile) && (int)smem_bytes(L, s) > cap) --s;
  return s;
}

static void choose_default_tiling(Plan& pl) {
  bool all2d = true;
  for (auto* c : pl.shots)
    if (c->ny > 1) all2d = false;
  // tile 9 (16 x 32 points, four consumer warps, the x queue in tensor
  // memory, one plane's reads per stage) measured fastest on the 3D cases
  // tried at space orders 4 to 16 and faster than the previous default
  // (tile 4) at order 2; four stages up to radius 4, five above
  pl.tile = pl.tile_req >= 0 ? pl.tile_req : (all2d ? 3 : 9);
  const int ms = max_stages(pl, pl.tile);
  const int st_def = kTiles[pl.tile].ca ? (pl.r > 4 ? 5 : 4) : pl.r + 4;
  pl.stages = pl.stages_req > 0 ? std::min(pl.stages_req, ms) : std::min(st_def, ms);
  if (pl.stages < min_stages(pl.r, pl.tile))
    fail(FDW_ERR_ARG, "pipeline too shallow for this order");
  if (pl.lx_req > 0) {
    pl.lx = pl.lx_req;
    return;
  }
  // x chunks of 32 planes (the 2r warm-up planes of a chunk stay a minor
  // share), halved while the grid gives fewer than two units per resident
  // CTA; with tile 9, chunks of 128 planes, halved while there are fewer
  // units than resident CTAs (its stages are short, and longer chunks
  // measured faster)
  const int slots = resident_ctas(pl, pl.tile, pl.stages, false);
  const bool ca = kTiles[pl.tile].ca;
  const int TY = tile_rows(kTiles[pl.tile]);
  long long cols = 0;
  int nxmax = 1;
  for (auto* c : pl.shots) {
    cols += (long long)((c->ny + TY - 1) / TY) * ((c->nz + kTZ - 1) / kTZ);
    nxmax = std::max(nxmax, c->nx);
  }
  int lx = std::min(ca ? 128 : 32, nxmax);
  while (lx > 8 && cols * ((nxmax + lx - 1) / lx) < (ca ? 1LL : 2LL) * slots) lx /= 2;
  pl.lx = std::max(1, lx);
}

static void upload_vec(void** dptr, const void* src, size_t bytes) {
  dfree(*dptr);
  *dptr = nullptr;
  *dptr = dalloc<unsigned char>(bytes);
  if (bytes) CK(cudaMemcpy(*dptr, src, bytes, cudaMemcpyHostToDevice));
}

// True when the built-in damping is zero at every grid point of the unit (the
// step kernel then skips the damping terms there).
static bool undamped(const fdw_ctx* c, const Unit& u, int TY) {
  if (c->use_etaf) return false;
  const std::vector<float>& e = c->eta_host;
  for (int x = u.x0; x < u.x1; ++x)
    if (e[x] != 0.f) return false;
  for (int y = u.y0; y < std::min(u.y0 + TY, c->ny); ++y)
    if (e[c->nx + y] != 0.f) return false;
  for (int z = u.z0; z < std::min(u.z0 + kTZ, c->nz); ++z)
    if (e[c->nx + c->ny + z] != 0.f) return false;
  return true;
}

// Units and the per-unit injection / sampling lists of each role.
static void build_lists(Plan& pl) {
  pl.release_lists();
  pl.clear_graphs();
  const int TY = tile_rows(kTiles[pl.tile]);
  pl.units.clear();
  // Rows of units: an x range of one shot times all its (y, z) column tiles,
  // in x order, shot after shot.  CTAs take units in this order, so the last
  // round of units is cut short: rows from the end of the table are split
  // into quarters (at least 8 planes) until one resident CTA's worth of units
  // is small, which shortens the idle tail when the tickets run out.
  struct Row {
    int shot, x0, x1, base;
    bool split;
  };
  std::vector<Row> rows;
  std::vector<std::array<int, 2>> cols(pl.shots.size());
  for (size_t s = 0; s < pl.shots.size(); ++s) {
    const fdw_ctx* c = pl.shots[s];
    column_tiles(c->ny, c->nz, TY, &cols[s][0], &cols[s][1]);
    for (int x0 = c->own0; x0 < c->own1; x0 += pl.lx)  // a slab's ghost planes are not updated
      rows.push_back(Row{(int)s, x0, std::min(c->own1, x0 + pl.lx), 0, false});
  }
  {
    const long long tail = resident_ctas(pl, pl.tile, pl.stages, false);
    long long covered = 0;
    for (size_t i = rows.size(); i-- > 0 && covered < tail;) {
      covered += (long long)cols[rows[i].shot][0] * cols[rows[i].shot][1];
      rows[i].split = true;
    }
  }
  std::vector<Row> fine;
  for (const Row& r : rows) {
    const int len = r.x1 - r.x0;
    const int piece = std::max(8, (len + 3) / 4);
    if (!r.split || len <= piece) {
      fine.push_back(r);
      continue;
    }
    for (int x0 = r.x0; x0 < r.x1; x0 += piece)
      fine.push_back(Row{r.shot, x0, std::min(r.x1, x0 + piece), 0, true});
  }
  std::vector<std::vector<int>> xrow(pl.shots.size());
  for (size_t s = 0; s < pl.shots.size(); ++s) xrow[s].assign(pl.shots[s]->nx, -1);
  for (size_t ri = 0; ri < fine.size(); ++ri)
    for (int x = fine[ri].x0; x < fine[ri].x1; ++x) xrow[fine[ri].shot][x] = (int)ri;
  // Within a row, units that carry sparse work at their tail (receiver and
  // source nodes: sampling in the forward step, injection of the residual in
  // the adjoint step) come first, so that the last units of a row, and of
  // the launch, are the light ones.
  std::vector<std::vector<int>> weight(fine.size());
  for (size_t ri = 0; ri < fine.size(); ++ri)
    weight[ri].assign((size_t)cols[fine[ri].shot][0] * cols[fine[ri].shot][1], 0);
  for (size_t si = 0; si < pl.shots.size(); ++si) {
    const fdw_ctx* c = pl.shots[si];
    for (const PointSet* ps : {&c->rec, &c->src})
      for (int j = 0; j < ps->n; ++j)
        for (int cc = 0; cc < 8; ++cc) {
          if (ps->w[(size_t)j * 8 + cc] == 0.f) continue;
          const int x = ps->base[(size_t)j * 3] + ((cc >> 2) & 1);
          const int y = ps->base[(size_t)j * 3 + 1] + ((cc >> 1) & 1);
          const int z = ps->base[(size_t)j * 3 + 2] + (cc & 1);
          if (xrow[si][x] < 0) continue;  // a slab's ghost plane (a receiver corner)
          weight[xrow[si][x]][(size_t)(y / TY) * cols[si][1] + z / kTZ]++;
        }
  }
  std::vector<std::vector<int>> pos(fine.size());  // local tile index -> place in its row
  for (size_t ri = 0; ri < fine.size(); ++ri) {
    Row& r = fine[ri];
    r.base = (int)pl.units.size();
    const int ck = cols[r.shot][1];
    const std::vector<int>& w = weight[ri];
    std::vector<int> order(w.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return w[a] > w[b]; });
    pos[ri].assign(order.size(), 0);
    for (size_t q = 0; q < order.size(); ++q) {
      const int li = order[q];
      pos[ri][li] = (int)q;
      Unit un = make_unit(r.shot, r.x0, r.x1, li, ck, TY);
      if (undamped(pl.shots[r.shot], un, TY)) un.flags |= kUnitUndamped;
      un.row = (int)ri;
      pl.units.push_back(un);
    }
  }
  {
    // a row's units read the planes x0 - r .. x1 + r - 1 of their shot: the
    // rows holding them are consecutive in the table
    std::vector<int2> deps(fine.size());
    std::vector<int> nu(fine.size());
    for (size_t ri = 0; ri < fine.size(); ++ri) {
      const Row& r = fine[ri];
      const fdw_ctx* c = pl.shots[r.shot];
      const int xa = std::max(r.x0 - pl.r, c->own0), xb = std::min(r.x1 + pl.r, c->own1) - 1;
      deps[ri] = make_int2(xrow[r.shot][xa], xrow[r.shot][xb]);
      nu[ri] = cols[r.shot][0] * cols[r.shot][1];
    }
    pl.nrows = (int)fine.size();
    upload_vec((void**)&pl.d_row_deps, deps.data(), deps.size() * sizeof(int2));
    upload_vec((void**)&pl.d_row_units, nu.data(), nu.size() * sizeof(int));
    pl.d_row_done = dalloc<int>(fine.size());
  }
  const int U = (int)pl.units.size();
  // unit of a node, -1 for a plane no unit updates (a slab's ghost planes)
  auto unit_of = [&](int s, int x, int y, int z) {
    if (x < 0 || x >= (int)xrow[s].size() || xrow[s][x] < 0) return -1;
    const int ri = xrow[s][x];
    return fine[ri].base + pos[ri][(y / TY) * cols[s][1] + z / kTZ];
  };
  pl.max_rec = pl.max_src = 0;
  pl.max_points = 0;
  pl.max_slot = 0;
  for (auto* c : pl.shots) {
    pl.max_rec = std::max(pl.max_rec, c->rec.n);
    pl.max_src = std::max(pl.max_src, c->src.n);
    pl.max_points = std::max(pl.max_points, (long long)c->nx * c->ny * c->nz);
    pl.max_slot = std::max(pl.max_slot, c->slot);
  }
  for (int role = 0; role < kNumRoles; ++role) {
    RoleLists& L = pl.lists[role];
    L = RoleLists();
    // injection: terms (j, w) grouped by node (unit, x, y, z), deterministic order
    std::vector<Corner> corners;
    // sampling: the sampled points of all shots, each with the unit that
    // records it (-1: none), numbered per shot
    std::vector<int> smp_unit, smp_j;
    for (size_t s = 0; s < pl.shots.size(); ++s) {
      const fdw_ctx* c = pl.shots[s];
      const PointSet& ip = (role == kRoleAdj) ? c->rec : c->src;
      for (int j = 0; j < ip.n; ++j)
        for (int cc = 0; cc < 8; ++cc) {
          const float w = ip.w[(size_t)j * 8 + cc];
          if (w == 0.f) continue;
          const int x = ip.base[(size_t)j * 3] + ((cc >> 2) & 1);
          const int y = ip.base[(size_t)j * 3 + 1] + ((cc >> 1) & 1);
          const int z = ip.base[(size_t)j * 3 + 2] + (cc & 1);
          // only a slab's adjoint lists meet ghost planes here, and a slab
          // has no adjoint step
          const int un = unit_of((int)s, x, y, z);
          if (un < 0) continue;
          corners.push_back(Corner{un, x, y, z, j, w});
        }
      if (role != kRoleRec) {
        const PointSet& sp = (role == kRoleAdj) ? c->src : c->rec;
        for (int j = 0; j < sp.n; ++j) {
          const int* b = &sp.base[(size_t)j * 3];
          smp_unit.push_back(unit_of((int)s, b[0], b[1], b[2]));
          smp_j.push_back(j);
        }
      }
    }
    L.nodes.resize(corners.size());
    L.terms.resize(corners.size());
    L.inj_ptr.assign(U + 1, 0);
    const int nn = group_corners(corners.data(), (int)corners.size(), U, L.nodes.data(),
                                 L.terms.data(), L.inj_ptr.data());
    L.nodes.resize(nn);
    for (int u = 0; u < U; ++u)
      for (int i = L.inj_ptr[u]; i < L.inj_ptr[u + 1]; ++i) L.node_shot.push_back(pl.units[u].shot);
    // units belong to one shot each, so a unit's list holds one shot's points
    L.smp_ptr.assign(U + 1, 0);
    L.smp_pts.resize(smp_unit.size());
    const int ns = bucket_points(smp_unit.data(), (int)smp_unit.size(), U, L.smp_ptr.data(),
                                 L.smp_pts.data());
    L.smp_pts.resize(ns);
    for (int& k : L.smp_pts) k = smp_j[k];
    upload_vec((void**)&L.d_inj_ptr, L.inj_ptr.data(), L.inj_ptr.size() * sizeof(int));
    upload_vec((void**)&L.d_smp_ptr, L.smp_ptr.data(), L.smp_ptr.size() * sizeof(int));
    upload_vec((void**)&L.d_smp_pts, L.smp_pts.data(), L.smp_pts.size() * sizeof(int));
    upload_vec((void**)&L.d_nodes, L.nodes.data(), L.nodes.size() * sizeof(InjNode));
    upload_vec((void**)&L.d_terms, L.terms.data(), L.terms.size() * sizeof(InjTerm));
    upload_vec((void**)&L.d_node_shot, L.node_shot.data(), L.node_shot.size() * sizeof(int));
  }
  upload_vec((void**)&pl.d_units, pl.units.data(), pl.units.size() * sizeof(Unit));
}

// Descriptor of one shot for one role; data pointers are filled per call.
static ShotDesc make_desc(const Plan& pl, fdw_ctx* c, int role) {
  ShotDesc d;
  std::memset(&d, 0, sizeof(d));
  const int TY = tile_rows(kTiles[pl.tile]);
  const int R4 = (pl.r + 3) & ~3;
  float* ubuf = nullptr;
  int uslots = 2;
  if (role == kRoleFwd) {
    ubuf = c->u;
    uslots = c->uslots;
  } else if (role == kRoleAdj) ubuf = c->lam;
  else { ubuf = c->seg; uslots = c->seg_slots; }
  d.nx = c->nx; d.ny = c->ny; d.nz = c->nz; d.nzp = c->nzp;
  d.mtype = c->mtype;
  d.u = ubuf;
  d.uslot = c->slot;
  if (ubuf) {
    make_map(&d.tm_uh, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ubuf, c->nx, c->ny, c->nz, c->nzp, uslots,
             c->slot, kTZ + 2 * R4, TY + 2 * pl.r);
    make_map(&d.tm_uc, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ubuf, c->nx, c->ny, c->nz, c->nzp, uslots,
             c->slot, kTZ, TY);
  }
  const CUtensorMapDataType mdt = c->mtype == kF16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                  : c->mtype == kBF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                      : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  make_map(&d.tm_m, mdt, msize(c->mtype), c->m, c->nx, c->ny, c->nz, c->nzp, 0, c->slot, kTZ, TY);
  if (role == kRoleAdj && c->seg) {
    make_map(&d.tm_f, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, c->seg, c->nx, c->ny, c->nz, c->nzp,
             c->seg_slots, c->slot, kTZ, TY);
    d.fwd = c->seg;
    d.fslot = c->slot;
    d.acc = c->acc;
    make_map(&d.tm_a, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, c->acc, c->nx, c->ny, c->nz, c->nzp, 0,
             c->slot, kTZ, TY);
  }
  if (c->use_etaf) {
    make_map(&d.tm_e, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, c->etaf, c->nx, c->ny, c->nz, c->nzp, 0,
             c->slot, kTZ, TY);
    d.etaf = c->etaf;
  }
  d.m = c->m;
  d.eta = c->eta;
  if (role == kRoleFwd) d.amax = c->amax;
  const PointSet& sp = (role == kRoleAdj) ? c->src : c->rec;
  if (role != kRoleRec) {
    d.pt_base = sp.d_base;
    d.pt_w = sp.d_w;
    d.smp_n = sp.n;
    d.smp_ld = sp.n;
  }
  d.inj_ld = (role == kRoleAdj) ? c->rec.n : c->src.n;
  return d;
}

static std::vector<int> current_versions(const Plan& pl) {
  std::vector<int> v;
  for (auto* c : pl.shots) {
    v.push_back(c->points_version);
    v.push_back(c->buffers_version);
    v.push_back(c->mtype);
    v.push_back(c->use_etaf ? 1 : 0);
    v.push_back(c->tblock);
    v.push_back(c->tb_variant);
    v.push_back(c->tb_lx);
    v.push_back(c->tb_stages);
  }
  return v;
}

// At least `cap` unit-ticket counters; a larger array invalidates the graphs
// that hold the old one.
static void ensure_tickets(Plan& pl, long long cap) {
  if (pl.ticket_cap >= cap) return;
  if (cap > (1LL << 30)) fail(FDW_ERR_ARG, "too many step launches in one pass");
  pl.clear_graphs();
  dfree(pl.d_tickets);
  pl.d_tickets = nullptr;
  pl.ticket_cap = 0;
  pl.d_tickets = dalloc<int>((size_t)cap);
  CK(cudaMemset(pl.d_tickets, 0, sizeof(int) * (size_t)cap));
  pl.ticket_cap = (int)cap;
}

// (Re)build units, lists and descriptors when points, buffers or tiling changed.
static void ensure_plan(Plan& pl) {
  set_device(pl.device);
  if (!pl.cap) CK(cudaStreamCreateWithFlags(&pl.cap, cudaStreamNonBlocking));
  if (!pl.d_err) {
    pl.d_err = dalloc<int>(1);
    CK(cudaMemset(pl.d_err, 0, sizeof(int)));
  }
  int nt_max = 1;
  for (auto* c : pl.shots) nt_max = std::max(nt_max, c->nt);
  ensure_tickets(pl, 2 * nt_max + 256);  // a gradient pass launches about 2 nt steps
  const std::vector<int> v = current_versions(pl);
  if (pl.built && v == pl.built_versions) return;
  if (!pl.built) choose_default_tiling(pl);
  // a rebuild that fails part-way (an allocation) leaves the plan marked
  // unbuilt, so the next call rebuilds it from scratch
  pl.built = false;
  build_lists(pl);
  pl.tb.release();
  for (int role = 0; role < kNumRoles; ++role) {
    pl.hdesc[role].clear();
    for (auto* c : pl.shots) pl.hdesc[role].push_back(make_desc(pl, c, role));
    dfree(pl.d_desc[role]);
    pl.d_desc[role] = nullptr;
    pl.d_desc[role] = dalloc<ShotDesc>(pl.shots.size());
    CK(cudaMemcpy(pl.d_desc[role], pl.hdesc[role].data(), sizeof(ShotDesc) * pl.shots.size(),
                  cudaMemcpyHostToDevice));
  }
  pl.aux_version = -1;
  pl.built_versions = v;
  pl.built = true;
}

static void upload_desc(Plan& pl, int role, cudaStream_t s) {
  CK(cudaMemcpyAsync(pl.d_desc[role], pl.hdesc[role].data(), sizeof(ShotDesc) * pl.shots.size(),
                     cudaMemcpyHostToDevice, s));
}

// ---------------------------------------------------------------- launches

// Pipeline depth of the gradient step, whose stages carry two more tiles than
// the forward step's: the deepest pipeline among those with the most resident
// CTAs per SM (more consumer warps hide more latency than a deeper prefetch).
static int grad_stages(Plan& pl) {
  if (pl.grad_stages_tile == pl.tile) return pl.grad_stages;
  const StageLayout L = stage_layout(pl.r, pl.tile, msize(plan_mtype(pl)), true, plan_etaf(pl));
  const void* fn = step_fn(pl.r, pl.tile, true);
  const int threads = (kTiles[pl.tile].warps + 1) * 32;
  const int cap = device_smem_optin(pl.device) - 1024;
  const int lo = min_stages(pl.r, pl.tile);
  int best = lo, best_nb = -1;
  for (int st = lo; st <= 2 * pl.r + 8 && (int)smem_bytes(L, st) <= cap; ++st) {
    const size_t smem = launch_smem(pl, pl.tile, L, st, fn, threads);
    const int nb = occupancy(pl, pl.tile, fn, threads, smem);
    if (nb >= best_nb) {
      best_nb = nb;
      best = st;
    }
  }
  pl.grad_stages = best;
  pl.grad_stages_tile = pl.tile;
  return best;
}

struct StepArgs {
  int role;
  int cur, prev, out, fslot;
  int inj_row, smp_row;
  int flags;
  bool grad;
  int amax_slot = 0;
  int step0 = 0, step_end = 1;  // kPersist: the steps of the launch
};

static const Plan::LaunchInfo& launch_info(Plan& pl, bool grad) {
  const bool etaf = plan_etaf(pl);
  const int mt = plan_mtype(pl);
  const int nunits = (int)pl.units.size();
  const int stages = grad ? grad_stages(pl) : pl.stages;
  auto key = std::make_tuple(pl.tile, stages, (int)grad, (int)etaf, mt, nunits);
  auto it = pl.launch_cache.find(key);
  if (it != pl.launch_cache.end()) return it->second;
  const StageLayout L = stage_layout(pl.r, pl.tile, msize(mt), grad, etaf);
  Plan::LaunchInfo li;
  li.stages = stages;
  li.cstages = second_ring_stages(L, stages);
  li.cstage_bytes = L.cbytes;
  li.fn = step_fn(pl.r, pl.tile, grad);
  li.threads = (kTiles[pl.tile].warps + 1) * 32;
  li.smem = launch_smem(pl, pl.tile, L, stages, li.fn, li.threads);
  const int nb = occupancy(pl, pl.tile, li.fn, li.threads, li.smem);
  li.resident = std::max(nb, 1) * device_sms(pl.device);
  li.grid = std::max(1, std::min(nunits, std::max(nb, 1) * device_sms(pl.device)));
  li.stage_bytes = L.bytes;
  li.off_p = L.off_p;
  li.off_m = L.off_m;
  li.off_f = L.off_f;
  li.off_a = L.off_a;
  li.off_e = L.off_e;
  li.off_c = L.off_c;
  return pl.launch_cache.emplace(key, li).first->second;
}

// Zero the unit tickets of the launches that follow on stream s.
static void reset_tickets(Plan& pl, cudaStream_t s) {
  CK(cudaMemsetAsync(pl.d_tickets, 0, sizeof(int) * pl.ticket_cap, s));
  pl.ticket_next = 0;
}

static void launch_step(Plan& pl, const StepArgs& a, cudaStream_t s);

// An adjoint step whose injection (the receiver data: thousands of nodes in a
// few units) runs as a launch of its own over all SMs after the step, instead
// of at the tails of the units that hold the nodes.
static void launch_adjoint_step(Plan& pl, StepArgs a, cudaStream_t s) {
  const bool inject = (a.flags & kInject) != 0;
  a.flags &= ~kInject;
  launch_step(pl, a, s);
  if (!inject) return;
  const RoleLists& L = pl.lists[kRoleAdj];
  const double dt = pl.shots[0]->dt;
  CK(launch_inject(pl.d_desc[kRoleAdj], L.d_nodes, L.d_node_shot, L.d_terms, (int)L.nodes.size(),
                   a.inj_row, a.out, a.fslot, (float)(dt * dt), (a.flags & kInjectDiff) != 0,
                   a.grad, plan_etaf(pl), s));
}

// dt^2 c_k / h_a^2 per axis (k = 1..r; an inactive axis of a 2D grid gets
// zeros), the sum of the centre weights over the axes, and dt^2.
static void stencil_weights(Plan& pl, float w[3][kMaxR + 1], float* csum, float* dt2) {
  const fdw_ctx* c0 = pl.shots[0];
  if (pl.weights.empty()) {
    pl.weights.assign(c0->r + 1, 0.0);
    fd_weights(c0->order, pl.weights.data());
  }
  const double dt = c0->dt;
  *dt2 = (float)(dt * dt);
  const std::vector<double>& cw = pl.weights;
  double cs = 0.0;
  for (int ax = 0; ax < 3; ++ax) {
    const bool active = !(c0->ny == 1 && c0->ndim == 2 && ax == 1);
    const double sc = active ? dt * dt / (c0->h[ax] * c0->h[ax]) : 0.0;
    for (int k = 0; k <= kMaxR; ++k) w[ax][k] = (k <= pl.r) ? (float)(cw[k] * sc) : 0.f;
    cs += cw[0] * sc;
  }
  *csum = (float)cs;
}

static void launch_step(Plan& pl, const StepArgs& a, cudaStream_t s) {
  const bool etaf = plan_etaf(pl);
  const Plan::LaunchInfo& li = launch_info(pl, a.grad);
  const int nunits = (int)pl.units.size();

  StepParams P;
  std::memset(&P, 0, sizeof(P));
  const RoleLists& Ls = pl.lists[a.role];
  P.shots = pl.d_desc[a.role];
  P.units = pl.d_units;
  P.nunits = nunits;
  if (pl.ticket_next >= pl.ticket_cap) fail(FDW_ERR_ARG, "too many step launches in one pass");
  P.ticket = pl.d_tickets + pl.ticket_next++;
  P.flags = a.flags | (etaf ? kEtaField : 0) | (pl.test_stall ? kTestStall : 0);
  P.inj_ptr = Ls.d_inj_ptr;
  P.inj_nodes = Ls.d_nodes;
  P.inj_terms = Ls.d_terms;
  P.smp_ptr = Ls.d_smp_ptr;
  P.smp_pts = Ls.d_smp_pts;
  P.inj_row = a.inj_row;
  P.smp_row = a.smp_row;
  P.cur = a.cur;
  P.prev = a.prev;
  P.out = a.out;
  P.fslot = a.fslot;
  P.amax_slot = a.amax_slot;
  P.stages = li.stages;
  P.stage_bytes = li.stage_bytes;
  P.cstages = li.cstages;
  P.cstage_bytes = li.cstage_bytes;
  P.off_p = li.off_p;
  P.off_m = li.off_m;
  P.off_f = li.off_f;
  P.off_a = li.off_a;
  P.off_e = li.off_e;
  P.off_c = li.off_c;
  stencil_weights(pl, P.w, &P.csum, &P.dt2);
  P.err = pl.d_err;
  const bool persist = (a.flags & kPersist) != 0;
  P.step0 = a.step0;
  P.step_end = a.step_end;
  P.row_done = pl.d_row_done;
  P.row_deps = pl.d_row_deps;
  P.row_units = pl.d_row_units;

  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  // a persistent launch has (step_end - step0) x nunits tickets: every CTA
  // that fits takes part
  cfg.gridDim = dim3(persist ? (unsigned)li.resident : (unsigned)li.grid);
  cfg.blockDim = dim3(li.threads);
  cfg.dynamicSmemBytes = li.smem;
  cfg.stream = s;
  void* args[] = {&P};
  CK(cudaLaunchKernelExC(&cfg, li.fn, args));
}

// Run `body` on stream s, through a cached CUDA graph unless FDW_NO_GRAPH is set.
template <class F>
static void run_graph(Plan& pl, const std::string& key, cudaStream_t s, F&& body) {
  if (env_flag("FDW_NO_GRAPH")) {
    body(s);
    return;
  }
  auto it = pl.graphs.find(key);
  if (it == pl.graphs.end()) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(pl.cap, cudaStreamCaptureModeThreadLocal));
    try {
      body(pl.cap);
    } catch (...) {
      cudaStreamEndCapture(pl.cap, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    CK(cudaStreamEndCapture(pl.cap, &g));
    cudaGraphExec_t ge = nullptr;
    cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    cuda_check(e, "cudaGraphInstantiate");
    it = pl.graphs.emplace(key, ge).first;
  }
  CK(cudaGraphLaunch(it->second, s));
}

// ---------------------------------------------------------------- passes

// Plain forward passes of a plan run as one persistent launch when every
// shot asks for it (fdw_set_persistent) and none is a slab.
static bool plan_persistent(const Plan& pl) {
  for (auto* c : pl.shots)
    if (!c->persist || c->slab) return false;
  return true;
}

// Forward time loop over all shots of a plan; snapshots every k steps if k > 0.
static void forward_body(Plan& pl, int k, int stype, cudaStream_t s) {
  const int nt = pl.shots[0]->nt;
  reset_tickets(pl, s);
  for (auto* c : pl.shots) CK(cudaMemsetAsync(c->u, 0, sizeof(float) * 2 * c->slot, s));
  int flags_base = 0;
  if (pl.max_src > 0) flags_base |= kInject;
  if (pl.max_rec > 0) flags_base |= kSample;
  const bool rv = k > 0 && pl.shots[0]->revolve;
  const int nsnap = k > 0 ? pl.shots[0]->nsnap : 0;
  const size_t ns = pl.shots.size();
  if (nsnap > 0)
    for (auto* c : pl.shots) CK(cudaMemsetAsync(c->amax, 0, sizeof(unsigned) * nsnap, s));
  // 16-bit snapshots need max |u| of the pair: with k >= 2 the two steps that
  // produce u^{jk-1} and u^{jk} fold it into amax[j-1] as they go; k = 1 (each
  // field in two pairs) and the binomial schedule take a separate pass
  const bool scaled = stype != kF32;
  const bool fused_max = scaled && k >= 2 && !rv;
  // binomial schedule: this sweep stores the checkpoints that the schedule
  // takes before its first reversal, and leaves the state at the start of
  // the last segment in the segment buffer (slot 1: u^{a}, slot 0: u^{a-1})
  std::map<int, int> take;  // segment -> slot
  int last_start = -1;
  if (rv) {
    int cur = 0;
    for (const CkptAction& act : pl.rv_actions) {
      if (act.op == kCkptReverse) break;
      if (act.op == kCkptAdvance) cur = act.arg;
      else if (act.op == kCkptTakeshot) take[cur] = act.arg;
    }
    last_start = (pl.rv_nseg - 1) * k;
    if (last_start == 0)
      for (auto* c : pl.shots) CK(cudaMemsetAsync(c->seg, 0, sizeof(float) * 2 * c->slot, s));
  }
  if (k == 0 && plan_persistent(pl)) {
    // plain forward: every step in one launch, units of step n + 1 starting
    // as soon as the rows they read have finished step n
    CK(cudaMemsetAsync(pl.d_row_done, 0, sizeof(int) * pl.nrows, s));
    if (nt > 1) {
      StepArgs a{kRoleFwd, 0, 1, 1, 0, 0, 0, flags_base | kPersist, false};
      a.step0 = 0;
      a.step_end = nt - 1;
      launch_step(pl, a, s);
    }
    if (pl.max_rec > 0)
      CK(launch_sample(pl.d_desc[kRoleFwd], (int)pl.shots.size(), pl.max_rec, (nt - 1) & 1, nt - 1,
                       s));
    return;
  }
  if (k > 0 && !rv && plan_persistent(pl)) {
    // checkpointed forward: one persistent launch per segment of k steps,
    // each ending where snapshot pair j = (u^{jk}, u^{jk-1}) is complete and
    // the pair is stored; with the fused maximum, the segment's last two
    // steps (those that make u^{jk-1} and u^{jk}) fold it into amax[j-1]
    for (int n0 = 0; n0 + 1 < nt;) {
      const int j = n0 / k + 1;
      const int n1 = std::min(j * k, nt - 1);  // steps n0 .. n1-1
      const bool pair = n1 == j * k && j <= nsnap;
      CK(cudaMemsetAsync(pl.d_row_done, 0, sizeof(int) * pl.nrows, s));
      StepArgs a{kRoleFwd, 0, 1, 1, 0, n0, 0, flags_base | kPersist, false};
      if (pair && fused_max) {
        a.flags |= kAbsMax;
        a.amax_slot = j - 1;
      }
      a.step0 = 0;
      a.step_end = n1 - n0;
      launch_step(pl, a, s);
      if (pair) {
        if (scaled && !fused_max)
          CK(launch_absmax(pl.d_pack + (size_t)(j - 1) * ns, (int)ns, pl.max_slot, s));
        CK(launch_pack(pl.d_pack + (size_t)(j - 1) * ns, (int)ns, pl.max_slot, stype, s));
      }
      n0 = n1;
    }
    if (pl.max_rec > 0)
      CK(launch_sample(pl.d_desc[kRoleFwd], (int)pl.shots.size(), pl.max_rec, (nt - 1) & 1, nt - 1,
                       s));
    return;
  }
  for (int n = 0; n + 1 < nt; ++n) {
    StepArgs a{kRoleFwd, n & 1, (n + 1) & 1, (n + 1) & 1, 0, n, n, flags_base, false};
    if (fused_max) {
      const int j = (n + 2) / k;  // u^{n+1} is the first or second field of pair j
      if (((n + 1) % k == 0 || (n + 2) % k == 0) && j >= 1 && j <= nsnap) {
        a.flags |= kAbsMax;
        a.amax_slot = j - 1;
      }
    }
    launch_step(pl, a, s);
    const int t = n + 1;  // u^t was just made; it lives in wavefield slot t & 1
    if (rv) {
      auto it = t % k == 0 ? take.find(t / k) : take.end();
      if (it != take.end()) {
        const AuxShot* d = pl.d_rv + ((size_t)(t & 1) * nsnap + it->second) * ns;
        if (scaled) CK(launch_absmax(d, (int)ns, pl.max_slot, s));
        CK(launch_pack(d, (int)ns, pl.max_slot, stype, s));
      }
      if (t == last_start)
        for (auto* c : pl.shots) {
          CK(cudaMemcpyAsync(c->seg + c->slot, c->u + (size_t)(t & 1) * c->slot,
                             sizeof(float) * c->slot, cudaMemcpyDeviceToDevice, s));
          CK(cudaMemcpyAsync(c->seg, c->u + (size_t)((t - 1) & 1) * c->slot,
                             sizeof(float) * c->slot, cudaMemcpyDeviceToDevice, s));
        }
    } else if (k > 0 && (n + 1) % k == 0 && (n + 1) / k <= nsnap) {
      const int j = (n + 1) / k;  // snapshot j holds (u^{jk}, u^{jk-1})
      if (scaled && !fused_max)
        CK(launch_absmax(pl.d_pack + (size_t)(j - 1) * ns, (int)ns, pl.max_slot, s));
      CK(launch_pack(pl.d_pack + (size_t)(j - 1) * ns, (int)ns, pl.max_slot, stype, s));
    }
  }
  if (pl.max_rec > 0)
    CK(launch_sample(pl.d_desc[kRoleFwd], (int)pl.shots.size(), pl.max_rec, (nt - 1) & 1, nt - 1, s));
}

// ---------------------------------------------------------------- two steps per pass

// A plan runs its plain forward passes two steps per launch when every shot
// asks for it (fdw_set_time_blocking) and takes its damping from the profiles.
static bool plan_uses_tb(const Plan& pl) {
  for (auto* c : pl.shots)
    if (c->tblock != 2 || c->use_etaf) return false;
  return true;
}

struct TbLayout {
  int bytes, off_p, off_s;
  size_t smem;
};

// Stage of the two-step kernel: the halo box of u^n, then the region-E tiles
// of u^{n-1} and s; after the stages, 2r + 2 region-E planes of u^{n+1}.
static TbLayout tb_layout(int r, int variant, int mtype, int stages) {
  const int EY = tb_ey(r, variant), HY = EY + 2 * r;
  TbLayout L;
  L.off_p = round128(HY * kTbHZ * 4);
  L.off_s = L.off_p + round128(EY * kTbEZ * 4);
  L.bytes = L.off_s + round128(mtype == kF32 ? EY * kTbEZ * 4 : EY * kTbHZ * 2);
  L.smem = (size_t)stages * L.bytes + (size_t)(2 * r + 2) * EY * kTbEZ * 4 +
           (size_t)(2 * stages) * 8 + 128;
  return L;
}

// Units, lists, descriptors and launch shape of the two-step kernel.
static void build_tb(Plan& pl) {
  Plan::Tb& T = pl.tb;
  T.release();
  const int r = pl.r;
  const fdw_ctx* c0 = pl.shots[0];
  T.variant = c0->tb_variant >= 0 ? c0->tb_variant : 0;
  const int EY = tb_ey(r, T.variant), TY = tb_ty(r, T.variant);
  const int mt = plan_mtype(pl);
  T.fn = tb_kernel_fn(r, T.variant);
  if (!T.fn) fail(FDW_ERR_ORDER, "no two-step kernel for this space order");
  // by default the deepest pipeline that keeps the CTAs per SM the registers
  // allow (two of variant 0, one of variant 1): the 2r + 1 planes held (a
  // plane's stage serves the first step at x and the second step r planes
  // later) and as many in flight as fit
  int smem_sm = 0;
  CK(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, pl.device));
  const size_t cap = (size_t)device_smem_optin(pl.device) - 1024;
  const size_t cap_cta = std::min(cap, (size_t)smem_sm / (T.variant == 0 ? 2 : 1) - 2048);
  int st = std::min(c0->tb_stages > 0 ? c0->tb_stages : kMaxStages, kMaxStages);
  while (st > 2 * r + 1 &&
         tb_layout(r, T.variant, mt, st).smem > (c0->tb_stages > 0 ? cap : cap_cta))
    --st;
  const TbLayout L = tb_layout(r, T.variant, mt, st);
  if (L.smem > cap) fail(FDW_ERR_ARG, "two-step pipeline does not fit in shared memory");
  T.stages = st;
  T.smem = L.smem;
  T.stage_bytes = L.bytes;
  T.off_p = L.off_p;
  T.off_s = L.off_s;
  T.threads = EY * 16 + 32;
  configure_kernel(T.fn, T.smem);
  int nb = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, T.fn, T.threads, T.smem));
  const long long slots = (long long)std::max(nb, 1) * device_sms(pl.device);

  // rows of units (an x chunk of one shot times its column tiles), the last
  // resident round cut into quarters as for the one-step kernel
  const size_t ns = pl.shots.size();
  std::vector<std::array<int, 2>> cols(ns);
  long long ncols = 0;
  int nxmax = 1;
  for (size_t s = 0; s < ns; ++s) {
    const fdw_ctx* c = pl.shots[s];
    cols[s] = {(c->ny + TY - 1) / TY, (c->nz + kTbTZ - 1) / kTbTZ};
    ncols += (long long)cols[s][0] * cols[s][1];
    nxmax = std::max(nxmax, c->nx);
  }
  int lx = c0->tb_lx;
  if (lx <= 0) {  // the longest chunk (nx / 2^k) that gives two units per resident CTA
    lx = nxmax;
    while (lx > 8 * r && ncols * ((nxmax + lx - 1) / lx) < 2 * slots) lx = (lx + 1) / 2;
  }
  T.lx = lx;
  struct Row {
    int shot, x0, x1;
    bool split;
  };
  std::vector<Row> rows;
  for (size_t s = 0; s < ns; ++s)
    for (int x0 = 0; x0 < pl.shots[s]->nx; x0 += lx)
      rows.push_back(Row{(int)s, x0, std::min(pl.shots[s]->nx, x0 + lx), false});
  {
    long long covered = 0;
    for (size_t i = rows.size(); i-- > 0 && covered < slots;) {
      covered += (long long)cols[rows[i].shot][0] * cols[rows[i].shot][1];
      rows[i].split = true;
    }
  }
  std::vector<Row> fine;
  for (const Row& rw : rows) {
    const int len = rw.x1 - rw.x0, piece = std::max(8, (len + 3) / 4);
    if (!rw.split || len <= piece) {
      fine.push_back(rw);
      continue;
    }
    for (int x0 = rw.x0; x0 < rw.x1; x0 += piece)
      fine.push_back(Row{rw.shot, x0, std::min(rw.x1, x0 + piece), true});
  }
  std::vector<int> rbase(fine.size());
  std::vector<std::vector<int>> xrow(ns);
  for (size_t s = 0; s < ns; ++s) xrow[s].assign(pl.shots[s]->nx, -1);
  for (size_t ri = 0; ri < fine.size(); ++ri) {
    const Row& rw = fine[ri];
    rbase[ri] = (int)T.units.size();
    for (int x = rw.x0; x < rw.x1; ++x) xrow[rw.shot][x] = (int)ri;
    for (int jy = 0; jy < cols[rw.shot][0]; ++jy)
      for (int jz = 0; jz < cols[rw.shot][1]; ++jz) {
        Unit un{};
        un.shot = rw.shot;
        un.x0 = rw.x0;
        un.x1 = rw.x1;
        un.y0 = jy * TY;
        un.z0 = jz * kTbTZ;
        T.units.push_back(un);
      }
  }
  const int U = (int)T.units.size();
  auto unit_at = [&](int ri, int jy, int jz) {
    return rbase[ri] + jy * cols[fine[ri].shot][1] + jz;
  };

  // source nodes: owned (unit of the node) and seen (units whose region E
  // over their first-step planes holds the node); std::map keeps each unit's
  // nodes in (x, y, z) order
  std::map<std::tuple<int, int, int, int>, std::vector<InjTerm>> own, ext;
  std::vector<std::vector<int>> smp(U);
  for (size_t s = 0; s < ns; ++s) {
    const fdw_ctx* c = pl.shots[s];
    for (int j = 0; j < c->src.n; ++j)
      for (int cc = 0; cc < 8; ++cc) {
        const float w = c->src.w[(size_t)j * 8 + cc];
        if (w == 0.f) continue;
        const int x = c->src.base[(size_t)j * 3] + ((cc >> 2) & 1);
        const int y = c->src.base[(size_t)j * 3 + 1] + ((cc >> 1) & 1);
        const int z = c->src.base[(size_t)j * 3 + 2] + (cc & 1);
        own[std::make_tuple(unit_at(xrow[s][x], y / TY, z / kTbTZ), x, y, z)].push_back(
            InjTerm{j, w});
        int last_ri = -1;
        for (int xx = std::max(0, x - r); xx <= std::min(c->nx - 1, x + r); ++xx) {
          const int ri = xrow[s][xx];
          if (ri == last_ri) continue;
          last_ri = ri;
          const Row& rw = fine[ri];
          if (x < rw.x0 - r || x >= rw.x1 + r) continue;
          for (int jy = 0; jy < cols[s][0]; ++jy) {
            if (y < jy * TY - r || y >= jy * TY + TY + r) continue;
            for (int jz = 0; jz < cols[s][1]; ++jz) {
              if (z < jz * kTbTZ - 4 || z >= jz * kTbTZ + kTbTZ + 4) continue;
              ext[std::make_tuple(unit_at(ri, jy, jz), x, y, z)].push_back(InjTerm{j, w});
            }
          }
        }
      }
    for (int j = 0; j < c->rec.n; ++j) {
      const int* b = &c->rec.base[(size_t)j * 3];
      smp[unit_at(xrow[s][b[0]], b[1] / TY, b[2] / kTbTZ)].push_back(j);
    }
  }
  auto flatten = [&](const std::map<std::tuple<int, int, int, int>, std::vector<InjTerm>>& m,
                     std::vector<int>& ptr, std::vector<InjNode>& nodes,
                     std::vector<InjTerm>& terms) {
    ptr.assign(U + 1, 0);
    for (auto& kv : m) {
      InjNode nd{};
      nd.x = std::get<1>(kv.first);
      nd.y = std::get<2>(kv.first);
      nd.z = std::get<3>(kv.first);
      nd.tbeg = (int)terms.size();
      for (const InjTerm& t : kv.second) terms.push_back(t);
      nd.tend = (int)terms.size();
      nd.j0 = kv.second.front().j;
      nd.w0 = kv.second.front().w;
      nodes.push_back(nd);
      ptr[std::get<0>(kv.first) + 1]++;
    }
    for (int u = 0; u < U; ++u) ptr[u + 1] += ptr[u];
  };
  std::vector<int> inj_ptr, ext_ptr, smp_ptr(U + 1, 0), smp_pts;
  std::vector<InjNode> inj_nodes, ext_nodes;
  std::vector<InjTerm> inj_terms, ext_terms;
  flatten(own, inj_ptr, inj_nodes, inj_terms);
  flatten(ext, ext_ptr, ext_nodes, ext_terms);
  for (int u = 0; u < U; ++u) {
    smp_ptr[u + 1] = smp_ptr[u] + (int)smp[u].size();
    for (int j : smp[u]) smp_pts.push_back(j);
  }
  upload_vec((void**)&T.d_units, T.units.data(), T.units.size() * sizeof(Unit));
  upload_vec((void**)&T.d_inj_ptr, inj_ptr.data(), inj_ptr.size() * sizeof(int));
  upload_vec((void**)&T.d_ext_ptr, ext_ptr.data(), ext_ptr.size() * sizeof(int));
  upload_vec((void**)&T.d_smp_ptr, smp_ptr.data(), smp_ptr.size() * sizeof(int));
  upload_vec((void**)&T.d_smp_pts, smp_pts.data(), smp_pts.size() * sizeof(int));
  upload_vec((void**)&T.d_inj_nodes, inj_nodes.data(), inj_nodes.size() * sizeof(InjNode));
  upload_vec((void**)&T.d_ext_nodes, ext_nodes.data(), ext_nodes.size() * sizeof(InjNode));
  upload_vec((void**)&T.d_inj_terms, inj_terms.data(), inj_terms.size() * sizeof(InjTerm));
  upload_vec((void**)&T.d_ext_terms, ext_terms.data(), ext_terms.size() * sizeof(InjTerm));

  const CUtensorMapDataType mdt = mt == kF16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                  : mt == kBF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  for (auto* c : pl.shots) {
    TbShot d;
    std::memset(&d, 0, sizeof(d));
    make_map(&d.tm_uh, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, c->u, c->nx, c->ny, c->nz, c->nzp, 4,
             c->slot, kTbHZ, EY + 2 * r);
    make_map(&d.tm_ue, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, c->u, c->nx, c->ny, c->nz, c->nzp, 4,
             c->slot, kTbEZ, EY);
    make_map(&d.tm_s, mdt, msize(mt), c->m, c->nx, c->ny, c->nz, c->nzp, 0, c->slot,
             mt == kF32 ? kTbEZ : kTbHZ, EY);
    d.u = c->u;
    d.uslot = c->slot;
    d.m = c->m;
    d.eta = c->eta;
    d.nx = c->nx;
    d.ny = c->ny;
    d.nz = c->nz;
    d.nzp = c->nzp;
    d.mtype = mt;
    d.q_ld = c->src.n;
    d.rec_ld = c->rec.n;
    d.pt_base = c->rec.d_base;
    d.pt_w = c->rec.d_w;
    T.hshots.push_back(d);
  }
  T.d_shots = dalloc<TbShot>(ns);
  T.grid = (int)std::max(1LL, std::min<long long>(U, slots));
  T.built = true;
}

// One two-step launch: u^{n+1}, u^{n+2} from u^{n-1}, u^n (u^t in slot t mod
// 4), wavelet rows n and n + 1 injected, trace rows srow_prev (-1: none) and
// n sampled from u^{n-1} and u^n.
static void launch_tb(Plan& pl, int n, int srow_prev, int flags, cudaStream_t s) {
  const Plan::Tb& T = pl.tb;
  TbParams P;
  std::memset(&P, 0, sizeof(P));
  P.shots = T.d_shots;
  P.units = T.d_units;
  P.nunits = (int)T.units.size();
  if (pl.ticket_next >= pl.ticket_cap) fail(FDW_ERR_ARG, "too many step launches in one pass");
  P.ticket = pl.d_tickets + pl.ticket_next++;
  P.flags = flags;
  P.inj_ptr = T.d_inj_ptr;
  P.inj_nodes = T.d_inj_nodes;
  P.inj_terms = T.d_inj_terms;
  P.ext_ptr = T.d_ext_ptr;
  P.ext_nodes = T.d_ext_nodes;
  P.ext_terms = T.d_ext_terms;
  P.smp_ptr = T.d_smp_ptr;
  P.smp_pts = T.d_smp_pts;
  P.row1 = n;
  P.row2 = n + 1;
  P.srow_prev = srow_prev;
  P.srow_cur = n;
  P.prev = (n + 3) & 3;
  P.cur = n & 3;
  P.out1 = (n + 1) & 3;
  P.out2 = (n + 2) & 3;
  P.stages = T.stages;
  P.stage_bytes = T.stage_bytes;
  P.off_p = T.off_p;
  P.off_s = T.off_s;
  stencil_weights(pl, P.w, &P.csum, &P.dt2);
  P.err = pl.d_err;
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(T.grid);
  cfg.blockDim = dim3(T.threads);
  cfg.dynamicSmemBytes = T.smem;
  cfg.stream = s;
  void* args[] = {&P};
  CK(cudaLaunchKernelExC(&cfg, T.fn, args));
}

// Plain forward loop, two steps per launch.  An odd number of steps starts
// with one one-step launch; the last two time levels are sampled by the
// sampling kernel and copied to the slots the one-step loop leaves them in
// (u^t in slot t & 1).
static void tb_forward_body(Plan& pl, cudaStream_t s) {
  const int nt = pl.shots[0]->nt;
  reset_tickets(pl, s);
  for (auto* c : pl.shots) CK(cudaMemsetAsync(c->u, 0, sizeof(float) * 4 * c->slot, s));
  int flags = 0;
  if (pl.max_src > 0) flags |= kInject;
  if (pl.max_rec > 0) flags |= kSample;
  int n = 0, next_row = 0;  // next_row: first trace row not yet recorded
  if ((nt - 1) % 2 == 1) {
    StepArgs a{kRoleFwd, 0, 3, 1, 0, 0, 0, flags, false};
    launch_step(pl, a, s);
    n = 1;
    next_row = 1;
  }
  for (; n + 2 < nt; n += 2) {
    launch_tb(pl, n, n - 1 >= next_row ? n - 1 : -1, flags, s);
    next_row = n + 1;
  }
  if (pl.max_rec > 0)
    for (int row = next_row; row < nt; ++row)
      CK(launch_sample(pl.d_desc[kRoleFwd], (int)pl.shots.size(), pl.max_rec, row & 3, row, s));
  for (int t = std::max(0, nt - 2); t < nt; ++t)
    if ((t & 3) != (t & 1))
      for (auto* c : pl.shots)
        CK(cudaMemcpyAsync(c->u + (size_t)(t & 1) * c->slot, c->u + (size_t)(t & 3) * c->slot,
                           sizeof(float) * c->slot, cudaMemcpyDeviceToDevice, s));
}

static void adjoint_body(Plan& pl, cudaStream_t s) {
  const int nt = pl.shots[0]->nt;
  reset_tickets(pl, s);
  for (auto* c : pl.shots) CK(cudaMemsetAsync(c->lam, 0, sizeof(float) * 2 * c->slot, s));
  int flags = 0;
  if (pl.max_rec > 0) flags |= kInject;
  if (pl.max_src > 0) flags |= kSample;
  if (plan_persistent(pl)) {
    // every adjoint step in one launch, time running backwards; the receiver
    // data are injected at the unit tails (spread over the units of every row)
    CK(cudaMemsetAsync(pl.d_row_done, 0, sizeof(int) * pl.nrows, s));
    if (nt > 1) {
      StepArgs a{kRoleAdj, 0, 1, 1, 0, nt - 1, nt - 1, flags | kPersist | kReverse, false};
      a.step0 = 0;
      a.step_end = nt - 1;
      launch_step(pl, a, s);
    }
  } else {
    for (int k = nt - 1; k >= 1; --k) {
      StepArgs a{kRoleAdj, (k + 1) & 1, k & 1, k & 1, 0, k, k, flags, false};
      launch_adjoint_step(pl, a, s);
    }
  }
  if (pl.max_src > 0)
    CK(launch_sample(pl.d_desc[kRoleAdj], (int)pl.shots.size(), pl.max_src, 1, 0, s));
}

static void gradient_body(Plan& pl, int k, int stype, bool diff, cudaStream_t s) {
  const int nt = pl.shots[0]->nt;
  reset_tickets(pl, s);
  const size_t ns = pl.shots.size();
  for (auto* c : pl.shots) {
    CK(cudaMemsetAsync(c->lam, 0, sizeof(float) * 2 * c->slot, s));
    CK(cudaMemsetAsync(c->acc, 0, sizeof(float) * c->slot, s));
  }
  const int adj_flags = (pl.max_rec > 0 ? kInject : 0) | (diff ? kInjectDiff : 0);
  const int rec_flags = pl.max_src > 0 ? kInject : 0;
  const int nseg = (nt + k - 1) / k;
  const bool persist = plan_persistent(pl);
  for (int j = nseg - 1; j >= 0; --j) {
    const int a0 = j * k, b0 = std::min((j + 1) * k, nt);
    if (j == 0) {
      for (auto* c : pl.shots) CK(cudaMemsetAsync(c->seg, 0, sizeof(float) * 2 * c->slot, s));
    } else {
      CK(launch_unpack(pl.d_unpack + (size_t)(j - 1) * ns, (int)ns, pl.max_slot, stype, s));
    }
    // recompute u^{a0+1} .. u^{b0-1}; slot i holds u^{a0-1+i}
    const int lo = std::max(a0, 1);
    if (persist) {
      // the segment's recompute steps as one persistent launch
      if (b0 - 1 > a0) {
        CK(cudaMemsetAsync(pl.d_row_done, 0, sizeof(int) * pl.nrows, s));
        StepArgs a{kRoleRec, 1, 0, 2, 0, a0, 0, rec_flags | kPersist | kLinear, false};
        a.step0 = 0;
        a.step_end = b0 - 1 - a0;
        launch_step(pl, a, s);
      }
    } else {
      for (int n = a0; n <= b0 - 2; ++n) {
        StepArgs a{kRoleRec, n - a0 + 1, n - a0, n - a0 + 2, 0, n, 0, rec_flags, false};
        launch_step(pl, a, s);
      }
    }
    // adjoint steps with the imaging condition, one launch each: the
    // residuals of thousands of receivers are injected by a launch of their
    // own over all SMs (at the unit tails of a persistent launch the few
    // units that hold them gate their rows' next steps: measured slower with
    // four shots per batch)
    for (int kk = b0 - 1; kk >= lo; --kk) {
      StepArgs a{kRoleAdj, (kk + 1) & 1, kk & 1, kk & 1, kk - a0 + 1, kk, 0, adj_flags, true};
      launch_adjoint_step(pl, a, s);
    }
  }
}

// Gradient pass under the binomial schedule: executes the schedule from its
// first reversal on.  The current forward state lives in segment-buffer slots
// 0 and 1 (the newer field in slot p); advancing steps it in place.
static void revolve_gradient_body(Plan& pl, int k, int stype, bool diff, cudaStream_t s) {
  const int nt = pl.shots[0]->nt;
  const size_t ns = pl.shots.size();
  const int nsnap = pl.shots[0]->nsnap;
  reset_tickets(pl, s);
  for (auto* c : pl.shots) {
    CK(cudaMemsetAsync(c->lam, 0, sizeof(float) * 2 * c->slot, s));
    CK(cudaMemsetAsync(c->acc, 0, sizeof(float) * c->slot, s));
  }
  const int adj_flags = (pl.max_rec > 0 ? kInject : 0) | (diff ? kInjectDiff : 0);
  const int rec_flags = pl.max_src > 0 ? kInject : 0;
  int p = 1;                   // segment-buffer slot of the newer field of the current state
  int cur = 0;                 // segment whose start state is current
  std::vector<int> slot_seg(std::max(nsnap, 1), -1);  // segment held by each slot
  bool started = false;
  for (const CkptAction& act : pl.rv_actions) {
    if (!started && act.op != kCkptReverse) {
      // done by the forward sweep, which leaves the last segment's start current
      if (act.op == kCkptAdvance) cur = act.arg;
      else if (act.op == kCkptTakeshot) slot_seg[act.arg] = cur;
      continue;
    }
    if (!started && cur != pl.rv_nseg - 1) fail(FDW_ERR_STATE, "checkpoint schedule out of step");
    started = true;
    if (act.op == kCkptAdvance) {
      for (int n = cur * k; n < act.arg * k; ++n) {
        StepArgs a{kRoleRec, p, 1 - p, 1 - p, 0, n, 0, rec_flags, false};
        launch_step(pl, a, s);
        p = 1 - p;
      }
      cur = act.arg;
    } else if (act.op == kCkptTakeshot) {
      const AuxShot* d = pl.d_rv + ((size_t)(2 + p) * nsnap + act.arg) * ns;
      if (stype != kF32) {
        for (auto* c : pl.shots) CK(cudaMemsetAsync(c->amax + act.arg, 0, sizeof(unsigned), s));
        CK(launch_absmax(d, (int)ns, pl.max_slot, s));
      }
      CK(launch_pack(d, (int)ns, pl.max_slot, stype, s));
      slot_seg[act.arg] = cur;
    } else if (act.op == kCkptRestore) {
      if (act.arg < 0) {
        for (auto* c : pl.shots) CK(cudaMemsetAsync(c->seg, 0, sizeof(float) * 2 * c->slot, s));
        cur = 0;
      } else {
        CK(launch_unpack(pl.d_rv + ((size_t)3 * nsnap + act.arg) * ns, (int)ns, pl.max_slot, stype, s));
        cur = slot_seg[act.arg];
      }
      p = 1;
    } else if (act.op == kCkptReverse) {
      const int j = act.arg;
      if (cur != j) fail(FDW_ERR_STATE, "checkpoint schedule out of step");
      const int a0 = j * k, b0 = std::min((j + 1) * k, nt);
      auto slot_of = [&](int t) { return t == a0 - 1 ? 1 - p : (t == a0 ? p : t - a0 + 1); };
      for (int n = a0; n <= b0 - 2; ++n) {
        StepArgs a{kRoleRec, slot_of(n), slot_of(n - 1), slot_of(n + 1), 0, n, 0, rec_flags, false};
        launch_step(pl, a, s);
      }
      for (int kk = b0 - 1; kk >= std::max(a0, 1); --kk) {
        StepArgs a{kRoleAdj, (kk + 1) & 1, kk & 1, kk & 1, slot_of(kk), kk, 0, adj_flags, true};
        launch_adjoint_step(pl, a, s);
      }
      cur = j;
    }
  }
}

// Checkpoint buffers of a context for k and snapshot type.
static void ensure_ckpt(fdw_ctx* c, int k, int stype) {
  // pairs (u^{jk}, u^{jk-1}) for j = 1 .. (nt-1)/k cover every segment start;
  // a smaller budget switches to the binomial schedule with that many slots
  const int nfull = (c->nt - 1) / k;
  const bool rv = c->ckpt_budget > 0 && c->ckpt_budget < nfull;
  const int nsnap = rv ? c->ckpt_budget : nfull;
  if (c->ckpt_k != k || c->snap_type != stype || !c->seg || c->revolve != rv || c->nsnap != nsnap) {
    dfree(c->snaps); dfree(c->amax); dfree(c->seg);
    c->snaps = nullptr; c->amax = nullptr; c->seg = nullptr;
    c->have_ckpt = false;
    const size_t per = (size_t)c->slot * 2 * msize(stype);  // pitched pair
    c->snaps = dalloc<unsigned char>(std::max<size_t>(1, per * (size_t)nsnap));
    c->amax = dalloc<unsigned int>(std::max(1, nsnap));
    c->seg_slots = k + 1;
    c->seg = dalloc<float>((size_t)c->slot * c->seg_slots);
    c->ckpt_k = k;
    c->snap_type = stype;
    c->nsnap = nsnap;
    c->revolve = rv;
    c->buffers_version++;
  }
  if (!c->lam) {
    c->lam = dalloc<float>((size_t)c->slot * 2);
    c->buffers_version++;
  }
  if (!c->acc) {
    c->acc = dalloc<float>((size_t)c->slot);
    c->buffers_version++;
  }
  if (!c->qsave) {
    c->qsave = dalloc<float>(std::max<size_t>(1, (size_t)c->nt * std::max(1, c->src.n)));
  }
}

static void ensure_aux(Plan& pl) {
  const int k = pl.shots[0]->ckpt_k;
  const int nsnap = pl.shots[0]->nsnap;
  const int ver = pl.shots[0]->buffers_version * 131 + k;
  if (pl.aux_version == ver && (pl.d_pack || pl.d_rv)) return;
  if (pl.shots[0]->revolve) {
    const fdw_ctx* c0 = pl.shots[0];
    const int nseg = (c0->nt + k - 1) / k;
    pl.rv_actions = revolve_schedule(nseg, nsnap);
    pl.rv_nseg = nseg;
    pl.rv_slots = nsnap;
    // step launches of the gradient pass: advances, recomputes and adjoint steps
    long long launches = 0, cur = 0;
    std::vector<long long> held(std::max(nsnap, 1), 0);
    for (const CkptAction& a : pl.rv_actions) {
      if (a.op == kCkptAdvance) {
        launches += (long long)(a.arg - cur) * k;
        cur = a.arg;
      } else if (a.op == kCkptTakeshot) {
        held[a.arg] = cur;
      } else if (a.op == kCkptRestore) {
        cur = a.arg < 0 ? 0 : held[a.arg];
      } else {
        launches += 2LL * k;
      }
    }
    ensure_tickets(pl, launches + 256);
    const size_t ns = pl.shots.size();
    std::vector<AuxShot> d((size_t)4 * nsnap * ns);
    for (int v = 0; v < 4; ++v)
      for (int j = 0; j < nsnap; ++j)
        for (size_t si = 0; si < ns; ++si) {
          fdw_ctx* c = pl.shots[si];
          AuxShot a;
          a.n = c->slot;
          a.snap = static_cast<unsigned char*>(c->snaps) + (size_t)c->slot * 2 * msize(c->snap_type) * j;
          a.amax = c->amax + j;
          float* base = v < 2 ? c->u : c->seg;
          const int newer = v & 1;
          a.a = base + (size_t)newer * c->slot;
          a.b = base + (size_t)(1 - newer) * c->slot;
          d[((size_t)v * nsnap + j) * ns + si] = a;
        }
    upload_vec((void**)&pl.d_rv, d.data(), d.size() * sizeof(AuxShot));
    pl.aux_version = ver;
    return;
  }
  const size_t ns = pl.shots.size();
  std::vector<AuxShot> pack((size_t)std::max(nsnap, 1) * ns), unpack(pack.size());
  for (int j = 1; j <= nsnap; ++j)
    for (size_t s = 0; s < ns; ++s) {
      fdw_ctx* c = pl.shots[s];
      const size_t per = (size_t)c->slot * 2 * msize(c->snap_type);
      AuxShot a;
      a.n = c->slot;
      a.snap = static_cast<unsigned char*>(c->snaps) + per * (size_t)(j - 1);
      a.amax = c->amax + (j - 1);
      a.a = c->u + (size_t)((j * k) & 1) * c->slot;       // u^{jk}
      a.b = c->u + (size_t)((j * k - 1) & 1) * c->slot;   // u^{jk-1}
      pack[(size_t)(j - 1) * ns + s] = a;
      a.a = c->seg + c->slot;   // slot 1: u^{a0}
      a.b = c->seg;             // slot 0: u^{a0-1}
      unpack[(size_t)(j - 1) * ns + s] = a;
    }
  upload_vec((void**)&pl.d_pack, pack.data(), pack.size() * sizeof(AuxShot));
  upload_vec((void**)&pl.d_unpack, unpack.data(), unpack.size() * sizeof(AuxShot));
  pl.aux_version = ver;
}

// ---------------------------------------------------------------- call helpers

template <class F>
static fdw_status guard(std::string* err, F&& f) {
  try {
    f();
    if (err) err->clear();
    return FDW_OK;
  } catch (const Error& e) {
    if (err) *err = e.msg;
    return e.st;
  } catch (const std::bad_alloc&) {
    if (err) *err = "host out of memory";
    return FDW_ERR_OOM;
  } catch (...) {
    if (err) *err = "unknown error";
    return FDW_ERR_CUDA;
  }
}

static Plan& ctx_plan(fdw_ctx* c) {
  if (!c->plan) {
    c->plan.reset(new Plan());
    c->plan->shots = {c};
    c->plan->device = c->device;
    c->plan->r = c->r;
    c->plan->tile_req = c->tile;
    c->plan->lx_req = c->xchunk;
    c->plan->stages_req = c->stages;
  }
  ensure_plan(*c->plan);
  return *c->plan;
}

static void require_model(const fdw_ctx* c) {
  if (!c->model_set) fail(FDW_ERR_STATE, "model not set (fdw_set_model)");
}

// Whole time loops need every plane of the grid: a slab steps with fdw_step.
static void require_whole(const fdw_ctx* c) {
  if (c->slab) fail(FDW_ERR_STATE, "a slab context steps with fdw_step and exchanges ghost planes");
}

static void check_compatible(const std::vector<fdw_ctx*>& v) {
  const fdw_ctx* a = v[0];
  for (auto* c : v) {
    if (c->order != a->order || c->nt != a->nt || c->dt != a->dt || c->mtype != a->mtype ||
        c->device != a->device || c->ndim != a->ndim)
      fail(FDW_ERR_ARG, "batched contexts must share order, dt, nt, ndim, device and model type");
    for (int ax = 0; ax < 3; ++ax)
      if (c->h[ax] != a->h[ax]) fail(FDW_ERR_ARG, "batched contexts must share the grid spacing");
    require_model(c);
  }
}

// Forward over a plan's shots with per-shot q / rec (host or device).
static void plan_forward(Plan& pl, const float* const* q, float* const* rec, int k, int stype,
                         cudaStream_t s) {
  const size_t ns = pl.shots.size();
  pl.test_stall = env_flag("FDW_TEST_STALL") && env_flag("FDW_NO_GRAPH");
  const bool tb = k == 0 && plan_uses_tb(pl);
  if (tb && !pl.tb.built) build_tb(pl);
  std::vector<std::pair<float*, float*>> copies;  // (host dst, staging src)
  std::vector<size_t> sizes;
  for (size_t i = 0; i < ns; ++i) {
    fdw_ctx* c = pl.shots[i];
    const size_t nq = (size_t)c->nt * c->src.n, nr = (size_t)c->nt * c->rec.n;
    if (c->src.n > 0 && !q[i]) fail(FDW_ERR_ARG, "source wavelet array is null");
    if (c->rec.n > 0 && !rec[i]) fail(FDW_ERR_ARG, "receiver output array is null");
    const float* qd = device_in(c, 1, q[i], nq, s);
    bool host = false;
    float* rd = device_out(c, 2, rec[i], nr, &host);
    if (host) {
      copies.push_back({rec[i], rd});
      sizes.push_back(nr);
    }
    pl.hdesc[kRoleFwd][i].inj_a = qd;
    pl.hdesc[kRoleFwd][i].inj_b = nullptr;
    pl.hdesc[kRoleFwd][i].smp_out = rd;
    if (tb) {
      pl.tb.hshots[i].q = qd;
      pl.tb.hshots[i].rec = rd;
    }
    if (k > 0 && nq > 0) CK(cudaMemcpyAsync(c->qsave, qd, nq * sizeof(float), cudaMemcpyDeviceToDevice, s));
  }
  upload_desc(pl, kRoleFwd, s);
  if (tb)
    CK(cudaMemcpyAsync(pl.tb.d_shots, pl.tb.hshots.data(), sizeof(TbShot) * ns,
                       cudaMemcpyHostToDevice, s));
  if (k > 0) {
    ensure_aux(pl);
    for (size_t i = 0; i < ns; ++i) pl.hdesc[kRoleRec][i].inj_a = pl.shots[i]->qsave;
    upload_desc(pl, kRoleRec, s);
  }
  std::ostringstream key;
  key << "fwd k" << k << " t" << stype << " rv" << (k > 0 && pl.shots[0]->revolve ? pl.shots[0]->nsnap : 0);
  if (tb) key << " tb";
  if (!tb && plan_persistent(pl)) key << " ps";
  run_graph(pl, key.str(), s, [&](cudaStream_t st) {
    if (tb) tb_forward_body(pl, st);
    else forward_body(pl, k, stype, st);
  });
  for (size_t i = 0; i < copies.size(); ++i)
    CK(cudaMemcpyAsync(copies[i].first, copies[i].second, sizes[i] * sizeof(float),
                       cudaMemcpyDeviceToHost, s));
  for (auto* c : pl.shots) {
    c->fwd_done = true;
    if (k > 0) c->have_ckpt = true;
  }
}

static void plan_gradient(Plan& pl, const float* const* resid, const float* const* sub,
                          float* const* grad, int layout, cudaStream_t s) {
  const size_t ns = pl.shots.size();
  bool diff = false;
  for (size_t i = 0; i < ns; ++i) {
    fdw_ctx* c = pl.shots[i];
    if (!c->have_ckpt) fail(FDW_ERR_STATE, "no checkpointed forward to differentiate");
    if (!grad[i]) fail(FDW_ERR_ARG, "gradient output is null");
    if (c->rec.n > 0 && !resid[i]) fail(FDW_ERR_ARG, "residual array is null");
    if (sub && sub[i]) diff = true;
  }
  for (size_t i = 0; i < ns; ++i) {
    fdw_ctx* c = pl.shots[i];
    const size_t nr = (size_t)c->nt * c->rec.n;
    pl.hdesc[kRoleAdj][i].inj_a = device_in(c, 3, resid[i], nr, s);
    const float* b = (sub && sub[i]) ? device_in(c, 4, sub[i], nr, s) : nullptr;
    if (diff && !b) {  // keep one flag for the whole launch: subtract zeros
      float* z = static_cast<float*>(staging_buf(c, 5, std::max<size_t>(nr, 1) * sizeof(float)));
      CK(cudaMemsetAsync(z, 0, std::max<size_t>(nr, 1) * sizeof(float), s));
      b = z;
    }
    pl.hdesc[kRoleAdj][i].inj_b = b;
    pl.hdesc[kRoleAdj][i].smp_out = nullptr;
  }
  upload_desc(pl, kRoleAdj, s);
  ensure_aux(pl);
  const int k = pl.shots[0]->ckpt_k, stype = pl.shots[0]->snap_type;
  const bool rv = pl.shots[0]->revolve;
  std::ostringstream key;
  key << "grad k" << k << " t" << stype << " d" << diff << " rv" << (rv ? pl.shots[0]->nsnap : 0);
  if (plan_persistent(pl)) key << " ps";
  run_graph(pl, key.str(), s, [&](cudaStream_t st) {
    if (rv) revolve_gradient_body(pl, k, stype, diff, st);
    else gradient_body(pl, k, stype, diff, st);
  });
  // the binomial schedule reuses the checkpoint slots and the current state
  // as it reverses: a next gradient needs a new checkpointed forward
  if (rv)
    for (auto* c : pl.shots) c->have_ckpt = false;
  for (size_t i = 0; i < ns; ++i) {
    fdw_ctx* c = pl.shots[i];
    const size_t nout = layout == FDW_LAYOUT_COMPUTATIONAL ? (size_t)c->nx * c->ny * c->nz
                                                           : (size_t)c->phys[0] * c->phys[1] * c->phys[2];
    bool host = false;
    float* gd = device_out(c, 6, grad[i], nout, &host);
    const double dt = c->dt;
    CK(launch_grad_out(c->acc, Geom{c->nx, c->ny, c->nz, c->nzp}, (float)(-1.0 / (dt * dt)), gd,
                       layout == FDW_LAYOUT_COMPUTATIONAL ? 1 : 0, c->nbl, c->ndim, (int)c->phys[0],
                       (int)c->phys[1], (int)c->phys[2], s));
    if (host) CK(cudaMemcpyAsync(grad[i], gd, nout * sizeof(float), cudaMemcpyDeviceToHost, s));
  }
}

static void plan_sync(Plan& pl) {
  set_device(pl.device);
  CK(cudaDeviceSynchronize());
  int e = 0;
  if (pl.d_err) {
    CK(cudaMemcpy(&e, pl.d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
      CK(cudaMemset(pl.d_err, 0, sizeof(int)));
      const fdw_status st = device_error_status(e);
      std::ostringstream os;
      os << (st == FDW_ERR_TIMEOUT ? "device-side wait timed out" : "device-side fault")
         << " (code " << e << ")";
      fail(st, os.str());
    }
  }
}

// ---------------------------------------------------------------- autotune

static std::string tune_key(const Plan& pl) {
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, pl.device));
  std::ostringstream os;
  os << prop.name << "|r" << pl.r << "|m" << plan_mtype(pl) << "|p" << plan_persistent(pl) << "|";
  for (auto* c : pl.shots) os << c->nx << "x" << c->ny << "x" << c->nz << ";";
  return os.str();
}

static bool tune_cache_lookup(const std::string& key, int* t, int* lx, int* st) {
  const char* path = std::getenv("FDW_AUTOTUNE_CACHE");
  if (!path || !*path) return false;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    const size_t p = line.rfind('\t');
    if (p == std::string::npos || line.substr(0, p) != key) continue;
    return std::sscanf(line.c_str() + p + 1, "%d %d %d", t, lx, st) == 3;
  }
  return false;
}

static void tune_cache_store(const std::string& key, int t, int lx, int st) {
  const char* path = std::getenv("FDW_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  std::ofstream f(path, std::ios::app);
  f << key << "\t" << t << " " << lx << " " << st << "\n";
}

static void plan_autotune(Plan& pl, int steps) {
  ensure_plan(pl);
  steps = std::min(steps, pl.ticket_cap - 2);
  const std::string key = tune_key(pl);
  int bt = -1, blx = 0, bst = 0;
  if (!tune_cache_lookup(key, &bt, &blx, &bst)) {
    bool all2d = true;
    int nxmax = 1;
    for (auto* c : pl.shots) {
      if (c->ny > 1) all2d = false;
      nxmax = std::max(nxmax, c->nx);
    }
    std::vector<int> tiles =
        all2d ? std::vector<int>{3} : std::vector<int>{0, 1, 2, 4, 5, 6, 7, 8, 9};
    // (half and whole columns as well: with one persistent launch over the
    // steps, the high orders measured fastest with one or two chunks per
    // column, which halve the 2r warm-up planes per update)
    std::vector<int> lxs = {16, 32, 48, 64, 80, 96, 128, 160, 192, 256, (nxmax + 1) / 2, nxmax};
    std::sort(lxs.begin(), lxs.end());
    lxs.erase(std::unique(lxs.begin(), lxs.end()), lxs.end());
    cudaStream_t s = pl.cap;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    // the timed steps inject (zeros) and sample like a real forward step, into
    // scratch wavelet and trace rows of their own
    const int rows = 2 * steps + 2;
    struct Scratch {  // freed on every exit
      std::vector<float*> v;
      float* add(size_t n) {
        v.push_back(nullptr);
        v.back() = dalloc<float>(n);
        return v.back();
      }
      ~Scratch() {
        for (float* p : v) dfree(p);
      }
    } scratch;
    std::vector<float*> tq, trec;
    for (auto* c : pl.shots) {
      tq.push_back(scratch.add((size_t)rows * std::max(1, c->src.n)));
      CK(cudaMemsetAsync(tq.back(), 0, sizeof(float) * rows * std::max(1, c->src.n), s));
      trec.push_back(scratch.add((size_t)rows * std::max(1, c->rec.n)));
    }
    int flags = 0;
    if (pl.max_src > 0) flags |= kInject;
    if (pl.max_rec > 0) flags |= kSample;
    // time `n` forward steps of one tiling (after two untimed ones), ms
    const bool persistent = plan_persistent(pl);
    auto time_config = [&](int t, int lx, int st, int n) {
      pl.tile = t;
      pl.lx = lx;
      pl.stages = st;
      build_lists(pl);
      for (size_t i = 0; i < pl.shots.size(); ++i) {
        pl.hdesc[kRoleFwd][i] = make_desc(pl, pl.shots[i], kRoleFwd);
        pl.hdesc[kRoleFwd][i].inj_a = tq[i];
        pl.hdesc[kRoleFwd][i].inj_b = nullptr;
        pl.hdesc[kRoleFwd][i].smp_out = trec[i];
      }
      upload_desc(pl, kRoleFwd, s);
      StepArgs a{kRoleFwd, 0, 1, 1, 0, 0, 0, flags, false};
      reset_tickets(pl, s);
      if (persistent) {
        // as the plain forward runs: one persistent launch over the steps
        a.flags |= kPersist;
        a.step0 = 0;
        a.step_end = 2;
        CK(cudaMemsetAsync(pl.d_row_done, 0, sizeof(int) * pl.nrows, s));
        launch_step(pl, a, s);
        CK(cudaMemsetAsync(pl.d_row_done, 0, sizeof(int) * pl.nrows, s));
        a.step_end = n;
        CK(cudaEventRecord(e0, s));
        launch_step(pl, a, s);
      } else {
        for (int w = 0; w < 2; ++w) launch_step(pl, a, s);
        CK(cudaEventRecord(e0, s));
        for (int i = 0; i < n; ++i) {
          a.cur = i & 1; a.prev = a.out = (i + 1) & 1;
          a.inj_row = a.smp_row = i + 2;
          launch_step(pl, a, s);
        }
      }
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      float ms_ = 0.f;
      CK(cudaEventElapsedTime(&ms_, e0, e1));
      return ms_;
    };
    // sweep every candidate once, then re-time the four fastest twice more,
    // interleaved, and keep the best time of each: short timings of single
    // configurations are noisy at the level that separates the leaders
    std::vector<std::tuple<float, int, int, int>> cand;
    for (int t : tiles) {
      const int ms = max_stages(pl, t);
      // r + 2 .. r + 4 stages; a tile whose stages hold one plane's reads
      // (ca) pipelines from two: 3, 4 and 5 stages (4, 5, 6 above radius 4,
      // where three of its CTAs fit on an SM with up to six)
      std::vector<int> sts;
      for (int extra : {1, 2, 3})
        sts.push_back(std::min(kTiles[t].ca ? (pl.r > 4 ? 3 + extra : 2 + extra)
                                            : pl.r + 1 + extra, ms));
      sts.erase(std::unique(sts.begin(), sts.end()), sts.end());
      for (int st : sts) {
        for (int lx : lxs) {
          if (lx > nxmax && lx != nxmax) continue;
          cand.emplace_back(time_config(t, lx, st, steps), t, lx, st);
        }
      }
    }
    std::sort(cand.begin(), cand.end());
    cand.resize(std::min<size_t>(cand.size(), 4));
    const int n2 = std::min(2 * steps, pl.ticket_cap - 2);
    for (int rep = 0; rep < 3; ++rep)
      for (auto& c : cand) {
        const float ms_ = time_config(std::get<1>(c), std::get<2>(c), std::get<3>(c), n2) *
                          (float)steps / (float)n2;
        std::get<0>(c) = std::min(std::get<0>(c), ms_);
      }
    std::sort(cand.begin(), cand.end());
    bt = std::get<1>(cand[0]);
    blx = std::get<2>(cand[0]);
    bst = std::get<3>(cand[0]);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    plan_sync(pl);
    tune_cache_store(key, bt, blx, bst);
  }
  pl.tile = bt;
  pl.lx = blx;
  pl.stages = bst;
  pl.tile_req = bt;
  pl.lx_req = blx;
  pl.stages_req = bst;
  pl.built = false;
  ensure_plan(pl);
}

// ================================================================= C ABI

extern "C" {

int fdw_version(void) { return 100; }

const char* fdw_status_string(fdw_status st) {
  switch (st) {
    case FDW_OK: return "ok";
    case FDW_ERR_ARG: return "invalid argument";
    case FDW_ERR_SHAPE: return "invalid shape";
    case FDW_ERR_ORDER: return "invalid space order";
    case FDW_ERR_CFL: return "time step above the stability limit";
    case FDW_ERR_OUT_OF_DOMAIN: return "point outside the domain";
    case FDW_ERR_OOM: return "out of memory";
    case FDW_ERR_CUDA: return "CUDA error";
    case FDW_ERR_TIMEOUT: return "device-side wait timed out";
    case FDW_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

fdw_status fdw_fd_weights(int space_order, double* c) {
  if (!valid_order(space_order)) return FDW_ERR_ORDER;
  if (!c) return FDW_ERR_ARG;
  fd_weights(space_order, c);
  return FDW_OK;
}

double fdw_dt_max(int ndim, const double* spacing, int space_order, double vmax) {
  if ((ndim != 2 && ndim != 3) || !spacing || !valid_order(space_order) || !(vmax > 0)) return -1.0;
  for (int a = 0; a < ndim; ++a)
    if (!(spacing[a] > 0)) return -1.0;
  return dt_limit(ndim, spacing, space_order, vmax);
}

// A whole grid (x_end < 0) or the x slab [x_begin, x_end) of its computational
// planes with r ghost planes on either side.
static fdw_status create_ctx(fdw_ctx** out, int ndim, const int64_t* shape, const double* spacing,
                             int space_order, int nbl, double dt, int nt, double vmax, int device,
                             int64_t x_begin, int64_t x_end) {
  if (!out) return FDW_ERR_ARG;
  *out = nullptr;
  if (ndim != 2 && ndim != 3) return FDW_ERR_SHAPE;
  if (!shape || !spacing) return FDW_ERR_ARG;
  if (!valid_order(space_order)) return FDW_ERR_ORDER;
  if (nbl < 0 || nt < 1 || !(dt > 0) || !(vmax > 0)) return FDW_ERR_ARG;
  for (int a = 0; a < ndim; ++a) {
    if (shape[a] < 2 || shape[a] + 2LL * nbl > (1LL << 20)) return FDW_ERR_SHAPE;
    if (!(spacing[a] > 0)) return FDW_ERR_ARG;
  }
  if (dt > dt_limit(ndim, spacing, space_order, vmax)) return FDW_ERR_CFL;
  std::unique_ptr<fdw_ctx> c(new fdw_ctx());
  fdw_status st = guard(nullptr, [&] {
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) fail(FDW_ERR_CUDA, "no such CUDA device");
    set_device(device);
    c->device = device;
    c->ndim = ndim;
    if (ndim == 3) {
      for (int a = 0; a < 3; ++a) { c->phys[a] = shape[a]; c->h[a] = spacing[a]; }
    } else {
      c->phys[0] = shape[0]; c->phys[1] = 1; c->phys[2] = shape[1];
      c->h[0] = spacing[0]; c->h[1] = 1.0; c->h[2] = spacing[1];
    }
    c->order = space_order;
    c->r = space_order / 2;
    c->nbl = nbl;
    c->dt = dt;
    c->nt = nt;
    c->vmax = vmax;
    c->nx = (int)(c->phys[0] + 2 * nbl);
    c->nx_full = c->nx;
    c->own0 = 0;
    c->own1 = c->nx;
    if (x_end >= 0) {
      if (x_begin < 0 || x_end > c->nx_full || x_end - x_begin < c->r)
        fail(FDW_ERR_SHAPE, "slab planes outside the grid or fewer than r = order/2");
      c->slab = true;
      c->gx0 = (int)x_begin - c->r;
      c->own0 = c->r;
      c->own1 = c->r + (int)(x_end - x_begin);
      c->nx = c->own1 + c->r;
    }
    c->ny = ndim == 3 ? (int)(c->phys[1] + 2 * nbl) : 1;
    c->nz = (int)(c->phys[2] + 2 * nbl);
    c->nzp = (c->nz + 31) & ~31;
    c->slot = (long long)c->nx * c->ny * c->nzp;
    c->u = dalloc<float>((size_t)c->slot * 2);
    c->m = dalloc<float>((size_t)c->slot);
    CK(cudaMemset(c->u, 0, sizeof(float) * 2 * c->slot));
    CK(cudaMemset(c->m, 0, sizeof(float) * c->slot));
    // built-in damping profiles, eta * dt / 2
    std::vector<float> prof((size_t)c->nx + c->ny + c->nz, 0.f);
    const int n3[3] = {c->nx, c->ny, c->nz};
    const GridGeom g = ctx_geom(c.get());
    size_t off = 0;
    for (int a = 0; a < 3; ++a) {
      for (int il = 0; il < n3[a]; ++il) {
        const long long i = a == 0 ? il + c->gx0 : il;  // index in the full grid
        prof[off + il] = damping_half_dt(g, a, i, vmax, dt);
      }
      off += n3[a];
    }
    c->eta = dalloc<float>(prof.size());
    CK(cudaMemcpy(c->eta, prof.data(), prof.size() * sizeof(float), cudaMemcpyHostToDevice));
    c->eta_host = prof;
  });
  if (st != FDW_OK) return st;
  *out = c.release();
  return FDW_OK;
}

fdw_status fdw_create(fdw_ctx** out, int ndim, const int64_t* shape, const double* spacing,
                      int space_order, int nbl, double dt, int nt, double vmax, int device) {
  return create_ctx(out, ndim, shape, spacing, space_order, nbl, dt, nt, vmax, device, 0, -1);
}

fdw_status fdw_create_slab(fdw_ctx** out, int ndim, const int64_t* shape, const double* spacing,
                           int space_order, int nbl, double dt, int nt, double vmax, int device,
                           int64_t x_begin, int64_t x_end) {
  if (x_end < 0) return FDW_ERR_SHAPE;
  return create_ctx(out, ndim, shape, spacing, space_order, nbl, dt, nt, vmax, device, x_begin,
                    x_end);
}

void fdw_destroy(fdw_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  delete ctx;
}

const char* fdw_last_error(const fdw_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

fdw_status fdw_set_model(fdw_ctx* c, const float* m, int layout, int m_dtype, void* stream) {
  if (!c) return FDW_ERR_ARG;
  return guard(&c->err, [&] {
    if (!m) fail(FDW_ERR_ARG, "model is null");
    if (layout != FDW_LAYOUT_PHYSICAL && layout != FDW_LAYOUT_COMPUTATIONAL) fail(FDW_ERR_ARG, "bad layout");
    if (m_dtype != kF32 && m_dtype != kF16 && m_dtype != kBF16) fail(FDW_ERR_ARG, "bad model type");
    set_device(c->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t n = layout == FDW_LAYOUT_PHYSICAL
                         ? (size_t)c->phys[0] * c->phys[1] * c->phys[2]
                         : (size_t)c->nx_full * c->ny * c->nz;
    const float* md = device_in(c, 7, m, n, s);
    if (m_dtype != c->mtype || !c->m) {  // no buffer: an earlier reallocation failed
      c->model_set = false;  // until the new buffer holds a model
      dfree(c->m);
      c->m = nullptr;
      c->m = dalloc<unsigned char>((size_t)c->slot * msize(m_dtype));
      CK(cudaMemsetAsync(c->m, 0, (size_t)c->slot * msize(m_dtype), s));
      c->mtype = m_dtype;
      c->buffers_version++;
    }
    CK(launch_model(md, layout == FDW_LAYOUT_PHYSICAL ? 0 : 1, (int)c->phys[0], (int)c->phys[1],
                    (int)c->phys[2], c->nbl, c->ndim, c->m, c->mtype,
                    Geom{c->nx, c->ny, c->nz, c->nzp}, s, c->gx0, c->nx_full));
    c->model_set = true;
  });
}

fdw_status fdw_set_damping(fdw_ctx* c, const float* eta, void* stream) {
  if (!c) return FDW_ERR_ARG;
  return guard(&c->err, [&] {
    set_device(c->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!eta) {
      if (c->use_etaf) {
        c->use_etaf = false;
        c->buffers_version++;
      }
      return;
    }
    if (!c->etaf) {
      c->etaf = dalloc<float>((size_t)c->slot);
      CK(cudaMemsetAsync(c->etaf, 0, sizeof(float) * c->slot, s));
    }
    const float* ed = device_in(c, 8, eta, (size_t)c->nx_full * c->ny * c->nz, s);
    CK(launch_eta_field(ed, (float)(0.5 * c->dt), c->etaf, Geom{c->nx, c->ny, c->nz, c->nzp}, s,
                        c->gx0, c->nx_full));
    if (!c->use_etaf) {
      c->use_etaf = true;
      c->buffers_version++;
    }
  });
}

fdw_status fdw_set_sources(fdw_ctx* c, int nsrc, const double* xyz) {
  if (!c) return FDW_ERR_ARG;
  return guard(&c->err, [&] {
    set_device(c->device);
    compute_points(c, c->src, nsrc, xyz, false);
    dfree(c->qsave);
    c->qsave = nullptr;
    c->have_ckpt = false;
  });
}

fdw_status fdw_set_receivers(fdw_ctx* c, int nrec, const double* xyz) {
  if (!c) return FDW_ERR_ARG;
  return guard(&c->err, [&] {
    set_device(c->device);
    compute_points(c, c->rec, nrec, xyz, true);
  });
}

fdw_status fdw_forward(fdw_ctx* c, const float* q, float* rec, void* stream) {
  if (!c) return FDW_ERR_ARG;
  return guard(&c->err, [&] {
    require_model(c);
    require_whole(c);
    set_device(c->device);
    Plan& pl = ctx_plan(c);
    plan_forward(pl, &q, &rec, 0, 0, static_cast<cudaStream_t>(stream));
  });
}

fdw_status fdw_forward_ckpt(fdw_ctx* c, const float* q, float* rec, int k, int stype, void* stream) {
  if (!c) return FDW_ERR_ARG;
  return guard(&c->err, [&] {
    require_model(c);
    require_whole(c);
    if (k < 1) fail(FDW_ERR_ARG, "ckpt_every must be >= 1");
    if (stype != kF32 && stype != kF16 && stype != kBF16) fail(FDW_ERR_ARG, "bad snapshot type");
    set_device(c->device);
    ensure_ckpt(c, k, stype);
    Plan& pl = ctx_plan(c);
    plan_forward(pl, &q, &rec, k, stype, static_cast<cudaStream_t>(stream));
  });
}

fdw_status fdw_adjoint(fdw_ctx* c, const float* d, float* qadj, void* stream) {
  if (!c) return FDW_ERR_ARG;
  return guard(&c->err, [&] {
    require_model(c);
    require_whole(c);
    set_device(c->device);
    if (!c->lam) {
      c->lam = dalloc<float>((size_t)c->slot * 2);
      c->buffers_version++;
    }
    Plan& pl = ctx_plan(c);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t nd = (size_t)c->nt * c->rec.n, nq = (size_t)c->nt * c->src.n;
    if (c->rec.n > 0 && !d) fail(FDW_ERR_ARG, "data array is null");
    if (c->src.n > 0 && !qadj) fail(FDW_ERR_ARG, "output array is null");
    bool host = false;
    pl.hdesc[kRoleAdj][0].inj_a = device_in(c, 3, d, nd, s);
    pl.hdesc[kRoleAdj][0].inj_b = nullptr;
    float* qo = device_out(c, 9, qadj, nq, &host);
    pl.hdesc[kRoleAdj][0].smp_out = qo;
    upload_desc(pl, kRoleAdj, s);
    run_graph(pl, plan_persistent(pl) ? "adj ps" : "adj", s,
              [&](cudaStream_t st) { adjoint_body(pl, st); });
    if (host) CK(cudaMemcpyAsync(qadj, qo, nq * sizeof(float), cudaMemcpyDeviceToHost, s));
    c->adj_done = true;
  });
}

fdw_status fdw_gradient(fdw_ctx* c, const float* resid, const float* resid_sub, float* grad,
                        int layout, void* stream) {
  if (!c) return FDW_ERR_ARG;
  return guard(&c->err, [&] {
    require_model(c);
    require_whole(c);
    if (layout != FDW_LAYOUT_PHYSICAL && layout != FDW_LAYOUT_COMPUTATIONAL) fail(FDW_ERR_ARG, "bad layout");
    set_device(c->device);
    Plan& pl = ctx_plan(c);
    plan_gradient(pl, &resid, &resid_sub, &grad, layout, static_cast<cudaStream_t>(stream));
  });
}

fdw_status fdw_step(fdw_ctx* c, int n, const float* q, float* rec, void* stream) {
  if (!c) return FDW_ERR_ARG;
  return guard(&c->err, [&] {
    require_model(c);
    if (n < 0 || n > c->nt - 1) fail(FDW_ERR_ARG, "step index outside 0 .. nt-1");
    if (c->src.n > 0 && !(q && is_device_ptr(q))) fail(FDW_ERR_ARG, "q must be a device array");
    if (c->rec.n > 0 && !(rec && is_device_ptr(rec)))
      fail(FDW_ERR_ARG, "rec must be a device array");
    set_device(c->device);
    Plan& pl = ctx_plan(c);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n == 0) CK(cudaMemsetAsync(c->u, 0, sizeof(float) * 2 * c->slot, s));
    ShotDesc& hd = pl.hdesc[kRoleFwd][0];
    if (n == 0 || hd.inj_a != q || hd.inj_b != nullptr || hd.smp_out != rec) {
      hd.inj_a = q;
      hd.inj_b = nullptr;
      hd.smp_out = rec;
      upload_desc(pl, kRoleFwd, s);
    }
    if (n == c->nt - 1) {  // the last time level: samples only
      if (c->rec.n > 0) CK(launch_sample(pl.d_desc[kRoleFwd], 1, c->rec.n, n & 1, n, s));
      c->fwd_done = true;
      return;
    }
    // one step launch: only its own ticket needs clearing
    CK(cudaMemsetAsync(pl.d_tickets, 0, sizeof(int), s));
    pl.ticket_next = 0;
    int flags = 0;
    if (c->src.n > 0) flags |= kInject;
    if (c->rec.n > 0) flags |= kSample;
    StepArgs a{kRoleFwd, n & 1, (n + 1) & 1, (n + 1) & 1, 0, n, n, flags, false};
    launch_step(pl, a, s);
  });
}

fdw_status fdw_halo_planes(fdw_ctx* c, int n, float** send_lo, float** send_hi, float** recv_lo,
                           float** recv_hi, int64_t* count) {
  if (!c) return FDW_ERR_ARG;
  return guard(&c->err, [&] {
    if (!c->slab) fail(FDW_ERR_ARG, "not a slab context");
    if (n < 0 || n > c->nt - 2) fail(FDW_ERR_ARG, "step index outside 0 .. nt-2");
    if (!send_lo || !send_hi || !recv_lo || !recv_hi || !count) fail(FDW_ERR_ARG, "null output");
    float* base = c->u + (size_t)((n + 1) & 1) * c->slot;  // u^{n+1}
    const size_t plane = (size_t)c->ny * c->nzp;
    *send_lo = base + (size_t)c->own0 * plane;
    *send_hi = base + (size_t)(c->own1 - c->r) * plane;
    *recv_lo = base + (size_t)(c->own0 - c->r) * plane;
    *recv_hi = base + (size_t)c->own1 * plane;
    *count = (int64_t)(c->r * plane);
  });
}

fdw_status fdw_exchange_ghosts(fdw_ctx* lower, fdw_ctx* upper, int n, void* stream) {
  if (!lower || !upper || lower == upper) return FDW_ERR_ARG;
  return guard(&upper->err, [&] {
    if (!lower->slab || !upper->slab) fail(FDW_ERR_ARG, "not slab contexts");
    if (lower->gx0 + lower->own1 != upper->gx0 + upper->own0 || lower->ny != upper->ny ||
        lower->nzp != upper->nzp || lower->r != upper->r)
      fail(FDW_ERR_ARG, "the slabs are not neighbours of one grid");
    float *sl0, *sh0, *rl0, *rh0, *sl1, *sh1, *rl1, *rh1;
    int64_t cnt = 0;
    if (fdw_halo_planes(lower, n, &sl0, &sh0, &rl0, &rh0, &cnt) != FDW_OK ||
        fdw_halo_planes(upper, n, &sl1, &sh1, &rl1, &rh1, &cnt) != FDW_OK)
      fail(FDW_ERR_ARG, "step index outside 0 .. nt-2");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = sizeof(float) * (size_t)cnt;
    set_device(upper->device);
    CK(cudaMemcpyPeerAsync(rl1, upper->device, sh0, lower->device, bytes, s));
    CK(cudaMemcpyPeerAsync(rh0, lower->device, sl1, upper->device, bytes, s));
  });
}

fdw_status fdw_halo_copy(fdw_ctx* c, int n, int dir, float* lo, float* hi, void* stream) {
  if (!c) return FDW_ERR_ARG;
  return guard(&c->err, [&] {
    if (dir != 0 && dir != 1) fail(FDW_ERR_ARG, "dir must be 0 (get) or 1 (put)");
    float *sl, *sh, *rl, *rh;
    int64_t cnt = 0;
    if (fdw_halo_planes(c, n, &sl, &sh, &rl, &rh, &cnt) != FDW_OK)
      fail(FDW_ERR_ARG, "not a slab context or step index outside 0 .. nt-2");
    set_device(c->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = sizeof(float) * (size_t)cnt;
    if (dir == 0) {
      if (lo) CK(cudaMemcpyAsync(lo, sl, bytes, cudaMemcpyDefault, s));
      if (hi) CK(cudaMemcpyAsync(hi, sh, bytes, cudaMemcpyDefault, s));
    } else {
      if (lo) CK(cudaMemcpyAsync(rl, lo, bytes, cudaMemcpyDefault, s));
      if (hi) CK(cudaMemcpyAsync(rh, hi, bytes, cudaMemcpyDefault, s));
    }
  });
}

fdw_status fdw_get_wavefield(fdw_ctx* c, int which, float* out, void* stream) {
  if (!c) return FDW_ERR_ARG;
  return guard(&c->err, [&] {
    if (!out) fail(FDW_ERR_ARG, "output is null");
    set_device(c->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const float* src = nullptr;
    if (which == 0) {
      if (!c->fwd_done) fail(FDW_ERR_STATE, "no forward run yet");
      src = c->u + (size_t)((c->nt - 1) & 1) * c->slot;
    } else if (which == 1) {
      if (!c->adj_done) fail(FDW_ERR_STATE, "no adjoint run yet");
      src = c->lam + c->slot;
    } else {
      fail(FDW_ERR_ARG, "which must be 0 or 1");
    }
    const size_t n = (size_t)c->nx * c->ny * c->nz;
    bool host = false;
    float* od = device_out(c, 10, out, n, &host);
    CK(launch_copy_out(src, Geom{c->nx, c->ny, c->nz, c->nzp}, od, s));
    if (host) CK(cudaMemcpyAsync(out, od, n * sizeof(float), cudaMemcpyDeviceToHost, s));
  });
}

fdw_status fdw_sync(fdw_ctx* c) {
  if (!c) return FDW_ERR_ARG;
  return guard(&c->err, [&] {
    if (c->plan) plan_sync(*c->plan);
    else {
      set_device(c->device);
      CK(cudaDeviceSynchronize());
    }
  });
}

fdw_status fdw_autotune(fdw_ctx* c, int steps) {
  if (!c) return FDW_ERR_ARG;
  return guard(&c->err, [&] {
    require_model(c);
    set_device(c->device);
    Plan& pl = ctx_plan(c);
    plan_autotune(pl, std::max(1, steps));
    c->fwd_done = false;
  });
}

fdw_status fdw_set_checkpoint_budget(fdw_ctx* c, int max_pairs) {
  if (!c) return FDW_ERR_ARG;
  return guard(&c->err, [&] {
    if (max_pairs < 0) fail(FDW_ERR_ARG, "checkpoint budget must be >= 0");
    if (max_pairs != c->ckpt_budget) {
      c->ckpt_budget = max_pairs;
      c->have_ckpt = false;  // the stored checkpoints follow the old schedule
    }
  });
}

fdw_status fdw_set_tiling(fdw_ctx* c, int tile, int xchunk, int stages) {
  if (!c) return FDW_ERR_ARG;
  return guard(&c->err, [&] {
    if (tile < -1 || tile >= kNumTiles) fail(FDW_ERR_ARG, "tile index out of range");
    if (xchunk < 0 || stages < 0) fail(FDW_ERR_ARG, "negative tiling value");
    if (stages > 0 && stages < min_stages(c->r, tile < 0 ? 0 : tile))
      fail(FDW_ERR_ARG, "stages must be >= r + 2 (>= 2 for tile 9)");
    c->tile = tile;
    c->xchunk = xchunk;
    c->stages = stages;
    c->plan.reset();
  });
}

fdw_status fdw_set_persistent(fdw_ctx* c, int on) {
  if (!c) return FDW_ERR_ARG;
  return guard(&c->err, [&] {
    if (on != 0 && on != 1) fail(FDW_ERR_ARG, "on must be 0 or 1");
    if (on && c->slab) fail(FDW_ERR_STATE, "a slab context steps one step at a time (fdw_step)");
    c->persist = on != 0;
  });
}

fdw_status fdw_get_tiling(fdw_ctx* c, int* out5) {
  if (!c || !out5) return FDW_ERR_ARG;
  return guard(&c->err, [&] {
    Plan& pl = ctx_plan(c);
    out5[0] = pl.tile;
    out5[1] = pl.lx;
    out5[2] = pl.stages;
    out5[3] = std::min((int)pl.units.size(), resident_ctas(pl, pl.tile, pl.stages, false));
    out5[4] = (int)pl.units.size();
  });
}

fdw_status fdw_set_time_blocking(fdw_ctx* c, int steps, int variant, int xchunk, int stages) {
  if (!c) return FDW_ERR_ARG;
  return guard(&c->err, [&] {
    if (steps != 1 && steps != 2) fail(FDW_ERR_ARG, "steps per pass must be 1 or 2");
    if (variant < -1 || variant >= kTbVariants || xchunk < 0 || stages < 0)
      fail(FDW_ERR_ARG, "bad two-step tiling");
    if (steps == 2) {
      if (c->ndim != 3) fail(FDW_ERR_ARG, "two steps per pass need a 3D grid");
      if (c->r > kTbMaxR) fail(FDW_ERR_ORDER, "two steps per pass exist for space orders 2 and 4");
      if (c->slab) fail(FDW_ERR_STATE, "a slab context steps one step at a time (fdw_step)");
      if (stages > 0 && stages < 2 * c->r + 1) fail(FDW_ERR_ARG, "stages must be >= 2r + 1");
      if (c->uslots < 4) {  // u^t lives in slot t mod 4 during a two-step pass
        set_device(c->device);
        CK(cudaDeviceSynchronize());
        float* nu = dalloc<float>((size_t)c->slot * 4);
        CK(cudaMemset(nu, 0, sizeof(float) * 4 * c->slot));
        dfree(c->u);
        c->u = nu;
        c->uslots = 4;
        c->fwd_done = false;
        c->buffers_version++;
      }
    }
    c->tblock = steps;
    c->tb_variant = variant;
    c->tb_lx = xchunk;
    c->tb_stages = stages;
    if (c->plan) {
      c->plan->tb.release();
      c->plan->clear_graphs();
    }
  });
}

fdw_status fdw_get_time_blocking(fdw_ctx* c, int* out5) {
  if (!c || !out5) return FDW_ERR_ARG;
  return guard(&c->err, [&] {
    for (int i = 0; i < 5; ++i) out5[i] = 0;
    out5[0] = c->tblock;
    if (c->tblock != 2) return;
    require_model(c);
    set_device(c->device);
    Plan& pl = ctx_plan(c);
    if (!pl.tb.built) build_tb(pl);
    out5[1] = pl.tb.variant;
    out5[2] = pl.tb.lx;
    out5[3] = pl.tb.stages;
    out5[4] = (int)pl.tb.units.size();
  });
}

fdw_status fdw_batch_create(fdw_batch** out, int nshots, fdw_ctx* const* ctxs) {
  if (!out || nshots < 1 || !ctxs) return FDW_ERR_ARG;
  *out = nullptr;
  std::unique_ptr<fdw_batch> b(new fdw_batch());
  fdw_status st = guard(&b->err, [&] {
    for (int i = 0; i < nshots; ++i) {
      if (!ctxs[i]) fail(FDW_ERR_ARG, "null context in batch");
      if (ctxs[i]->slab) fail(FDW_ERR_ARG, "slab contexts cannot be batched");
      b->shots.push_back(ctxs[i]);
    }
    check_compatible(b->shots);
    b->plan.reset(new Plan());
    b->plan->shots = b->shots;
    b->plan->device = b->shots[0]->device;
    b->plan->r = b->shots[0]->r;
  });
  if (st != FDW_OK) return st;
  *out = b.release();
  return FDW_OK;
}

void fdw_batch_destroy(fdw_batch* b) {
  if (!b) return;
  if (!b->shots.empty()) {
    cudaSetDevice(b->shots[0]->device);
    cudaDeviceSynchronize();
  }
  delete b;
}

const char* fdw_batch_last_error(const fdw_batch* b) { return b ? b->err.c_str() : "null batch"; }

fdw_status fdw_batch_forward(fdw_batch* b, const float* const* q, float* const* rec, void* stream) {
  if (!b || !q || !rec) return FDW_ERR_ARG;
  return guard(&b->err, [&] {
    check_compatible(b->shots);
    ensure_plan(*b->plan);
    plan_forward(*b->plan, q, rec, 0, 0, static_cast<cudaStream_t>(stream));
  });
}

fdw_status fdw_batch_forward_ckpt(fdw_batch* b, const float* const* q, float* const* rec, int k,
                                  int stype, void* stream) {
  if (!b || !q || !rec) return FDW_ERR_ARG;
  return guard(&b->err, [&] {
    if (k < 1) fail(FDW_ERR_ARG, "ckpt_every must be >= 1");
    if (stype != kF32 && stype != kF16 && stype != kBF16) fail(FDW_ERR_ARG, "bad snapshot type");
    check_compatible(b->shots);
    for (auto* c : b->shots)
      if (c->ckpt_budget != b->shots[0]->ckpt_budget)
        fail(FDW_ERR_ARG, "shots of a batch need the same checkpoint budget");
    set_device(b->plan->device);
    for (auto* c : b->shots) ensure_ckpt(c, k, stype);
    ensure_plan(*b->plan);
    plan_forward(*b->plan, q, rec, k, stype, static_cast<cudaStream_t>(stream));
  });
}

fdw_status fdw_batch_gradient(fdw_batch* b, const float* const* resid, const float* const* sub,
                              float* const* grad, int layout, void* stream) {
  if (!b || !resid || !grad) return FDW_ERR_ARG;
  return guard(&b->err, [&] {
    if (layout != FDW_LAYOUT_PHYSICAL && layout != FDW_LAYOUT_COMPUTATIONAL) fail(FDW_ERR_ARG, "bad layout");
    check_compatible(b->shots);
    ensure_plan(*b->plan);
    plan_gradient(*b->plan, resid, sub, grad, layout, static_cast<cudaStream_t>(stream));
  });
}

fdw_status fdw_batch_autotune(fdw_batch* b, int steps) {
  if (!b) return FDW_ERR_ARG;
  return guard(&b->err, [&] {
    check_compatible(b->shots);
    plan_autotune(*b->plan, std::max(1, steps));
  });
}

fdw_status fdw_batch_get_tiling(fdw_batch* b, int* out5) {
  if (!b || !out5) return FDW_ERR_ARG;
  return guard(&b->err, [&] {
    Plan& pl = *b->plan;
    ensure_plan(pl);
    out5[0] = pl.tile;
    out5[1] = pl.lx;
    out5[2] = pl.stages;
    out5[3] = std::min((int)pl.units.size(), resident_ctas(pl, pl.tile, pl.stages, false));
    out5[4] = (int)pl.units.size();
  });
}

}  // extern "C"
