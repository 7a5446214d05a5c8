// Internal declarations of libfdwave shared by the runtime and the kernel files.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "fdw_types.h"

namespace fdw {

// Tile shapes of the step kernel: BY consumer warps; each quarter-warp covers
// NY consecutive rows and each lane four z points, so a tile is (4 * BY * NY) x 32
// points in (y, z).  Tiles 0 and 2 unroll the x loop so the register queue
// rotates; the others shift it (smaller code).  Tile 3 is meant for 2D grids.
// Tile 6 is tile 4 with the per-plane tiles in a second ring: less shared
// memory per CTA, which lets the high orders (r >= 6) hold three CTAs per SM.
// Tiles 7 and 8 are tiles 4 and 6 with the x queue in tensor memory instead
// of registers (no per-plane queue moves; the CTA allocates tq_columns).
// Tile 9 is tile 7 with stages that hold exactly what one plane's update
// reads: the halo plane x, the tiles of plane x and the centre tile of plane
// x + r (the values that join the x queue), so every stage is freed after one
// plane instead of staying r + 1 planes, and a few stages pipeline; it also
// forms the neighbour pair sums two at a time (fewer registers), so at the
// high orders more CTAs fit on an SM.  Its gradient step stages the forward
// field and accumulator tiles of plane x in the same stage.
struct TileShape {
  int ny_pts;
  int warps;
  bool split;  // the forward and adjoint steps also keep the per-plane tiles
               // in a second ring (gradient steps always do)
  bool tq;     // x queue in tensor memory
  bool ca;     // centre tile of plane x + r staged with plane x (forward, adjoint)
};
constexpr int kNumTiles = 10;
constexpr TileShape kTiles[kNumTiles] = {
    {1, 4, false, false, false}, {2, 4, false, false, false}, {1, 8, false, false, false},
    {1, 1, false, false, false}, {1, 4, false, false, false}, {2, 2, false, false, false},
    {1, 4, true, false, false},  {1, 4, false, true, false},  {1, 4, true, true, false},
    {1, 4, false, true, true}};
// Tensor-memory columns a CTA of a tq tile allocates at radius r: the ring of
// 2r+1 planes of four values plus the second copies that a window of 2r
// planes starting at any slot reads past the ring's end (slots 0 .. 2r-2),
// 16 r columns, rounded up to a power of two of at least 32; an SM has 512.
__host__ __device__ constexpr int tq_columns(int r) {
  return 16 * r <= 32 ? 32 : (16 * r <= 64 ? 64 : 128);
}
constexpr int tile_rows(const TileShape& t) { return 4 * t.ny_pts * t.warps; }

// Kernel registry: one translation unit per stencil radius.
const void* step_kernel_r1(int tile, bool grad);
const void* step_kernel_r2(int tile, bool grad);
const void* step_kernel_r3(int tile, bool grad);
const void* step_kernel_r4(int tile, bool grad);
const void* step_kernel_r5(int tile, bool grad);
const void* step_kernel_r6(int tile, bool grad);
const void* step_kernel_r7(int tile, bool grad);
const void* step_kernel_r8(int tile, bool grad);
// Two-step (temporally blocked) forward kernel of radius r = 1 .. kTbMaxR and
// row variant 0 / 1 (fdw_tb.cu); null for other radii.
const void* tb_kernel_fn(int r, int variant);

// Geometry of one pitched field for the auxiliary kernels.
struct Geom {
  int nx, ny, nz, nzp;
};

// Per-shot descriptor of the auxiliary (per-call, not per-step) kernels.
struct AuxShot {
  long long n;          // floats per pitched field (a multiple of 32)
  float* a;             // first field (slot base)
  float* b;             // second field
  void* snap;           // snapshot pair base: two pitched fields of n elements
  unsigned int* amax;   // absolute maximum of the pair, float bits
};

cudaError_t launch_sample(const ShotDesc* shots, int nshots, int maxpts, int slot, int row,
                          cudaStream_t s);
// xoff, nxg: the field is an x slab, local plane x = plane x + xoff of a full
// computational grid of nxg planes (nxg = 0: the field is the whole grid)
cudaError_t launch_model(const float* in, int layout, int phys_x, int phys_y, int phys_z,
                         int nbl, int ndim, void* out, int mtype, Geom g, cudaStream_t s,
                         int xoff = 0, int nxg = 0);
cudaError_t launch_eta_field(const float* in, float scale, float* out, Geom g, cudaStream_t s,
                             int xoff = 0, int nxg = 0);
// maxn: the largest field (floats per pitched slot) of the shots
cudaError_t launch_absmax(const AuxShot* shots, int nshots, long long maxn, cudaStream_t s);
cudaError_t launch_pack(const AuxShot* shots, int nshots, long long maxn, int stype,
                        cudaStream_t s);
cudaError_t launch_unpack(const AuxShot* shots, int nshots, long long maxn, int stype,
                          cudaStream_t s);
cudaError_t launch_grad_out(const float* acc, Geom g, float scale, float* out, int layout,
                            int nbl, int ndim, int phys_x, int phys_y, int phys_z,
                            cudaStream_t s);
cudaError_t launch_copy_out(const float* field, Geom g, float* out, cudaStream_t s);
// One step's injection as its own launch (see fdw_aux.cu): node_shot[i] is
// the shot of nodes[i]; out / fslot the wavefield and forward-field slots.
cudaError_t launch_inject(const ShotDesc* shots, const InjNode* nodes, const int* node_shot,
                          const InjTerm* terms, int nnodes, int row, int out, int fslot, float dt2,
                          bool diff, bool grad, bool etaf, cudaStream_t s);

// Binomial checkpoint schedules over the segments of the gradient pass
// (fdw_revolve.cu).
enum CkptOp : int { kCkptAdvance = 1, kCkptTakeshot = 2, kCkptRestore = 3, kCkptReverse = 4 };
struct CkptAction {
  int op;
  int arg;  // segment (advance, reverse) or slot (takeshot, restore; -1 = zero state)
};
// Fewest segment advances that reverse l segments from a held start state
// with c free slots.
long long revolve_cost(long long l, int c);
std::vector<CkptAction> revolve_schedule(int nseg, int nslots);

}  // namespace fdw
