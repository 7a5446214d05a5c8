// Types of the two-step (temporally blocked) forward pass, shared by the host
// runtime and its kernel.
//
// One launch advances u^{n-1}, u^n to u^{n+1}, u^{n+2}: the explicit scheme of
// Sec. 5 (Eq. 3, centred time differences) applied twice per pass over
// memory.  A work unit is an output tile of TY x 56 points (y, z) streamed
// along a chunk [x0, x1) of x.  The first step of the pass is computed on the
// tile grown by r rows in y and 4 points in z on either side (region E, EY =
// TY + 2r rows of 64 points, one four-point quad per consumer thread) and for
// r planes beyond the chunk in x, so the second step finds every neighbour of
// its points in shared memory; neighbouring units recompute the overlap.
// Four wavefield slots (u^t in slot t mod 4) keep the fields read in a pass
// apart from the fields written.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "fdw_types.h"

namespace fdw {

constexpr int kTbQ = 14;             // quads of the output tile along z
constexpr int kTbTZ = 4 * kTbQ;      // 56 output points along z
constexpr int kTbEZ = kTbTZ + 8;     // 64: region E along z, z0-4 .. z0+59
constexpr int kTbHZ = kTbTZ + 16;    // 72: halo box along z, z0-8 .. z0+63
constexpr int kTbMaxR = 2;           // largest radius with a two-step kernel
// Rows of region E: EY = 18 at radius 1 and 16 at radius 2 (variant 0: 9 or
// 8 consumer warps and a producer warp, two CTAs per SM) or 34 / 32 (variant
// 1: 17 or 16 consumer warps, one CTA per SM); the output tile has TY = EY - 2r
// rows.  The first step gives each consumer thread one quad of region E, the
// second step one quad of the output tile (16 threads per output row, the
// last two idle, so that a row's shared-memory reads are free of bank
// conflicts).
constexpr int kTbVariants = 2;

constexpr int tb_ey(int r, int variant) {
  return variant == 0 ? (r == 1 ? 18 : 16) : (r == 1 ? 34 : 32);
}
constexpr int tb_ty(int r, int variant) { return tb_ey(r, variant) - 2 * r; }

struct alignas(128) TbShot {
  CUtensorMap tm_uh;  // wavefield slots, halo box (72, EY + 2r, 1, 1) at (z0 - 8, y0 - 2r)
  CUtensorMap tm_ue;  // wavefield slots, region-E box (64, EY, 1, 1) at (z0 - 4, y0 - r)
  CUtensorMap tm_s;   // model s = 1/m: (64, EY) at z0 - 4 for f32, (72, EY) at z0 - 8 for 16 bits
  float* u;           // base of the four wavefield slots
  long long uslot;    // floats per slot
  const void* m;      // s = 1/m, pitched, type mtype
  const float* eta;   // eta*dt/2 profiles, [nx] then [ny] then [nz]
  int nx, ny, nz, nzp;
  int mtype;
  const float* q;     // source wavelets [nt][q_ld]
  int q_ld;
  float* rec;         // traces [nt][rec_ld]
  int rec_ld;
  const int* pt_base; // receivers: base node (x, y, z)
  const float* pt_w;  // receivers: eight corner weights
};

struct TbParams {
  const TbShot* shots;
  const Unit* units;
  int nunits;
  int* ticket;         // unit counter of this launch (zero before it)
  int flags;           // kInject, kSample
  // source nodes each unit owns (added into u^{n+1} and u^{n+2} in global
  // memory at the unit's tail), and the source nodes inside each unit's
  // region E over its first-step planes, sorted by x (added into the shared
  // copy of u^{n+1} before the second step reads it)
  const int* inj_ptr;
  const InjNode* inj_nodes;
  const InjTerm* inj_terms;
  const int* ext_ptr;
  const InjNode* ext_nodes;
  const InjTerm* ext_terms;
  // receivers whose base node a unit owns
  const int* smp_ptr;
  const int* smp_pts;
  int row1, row2;      // wavelet rows injected into u^{n+1} and u^{n+2}
  int srow_prev;       // trace row sampled from slot prev (-1: none)
  int srow_cur;        // trace row sampled from slot cur (-1: none)
  int prev, cur, out1, out2;  // slots of u^{n-1}, u^n, u^{n+1}, u^{n+2}
  int stages;          // pipeline depth (planes of u^n in flight or held, >= 2r + 1)
  int stage_bytes;
  int off_p, off_s;    // region-E tiles of u^{n-1} and s inside a stage
  float dt2;
  float csum;
  float w[3][kMaxR + 1];
  int* err;
};

}  // namespace fdw
