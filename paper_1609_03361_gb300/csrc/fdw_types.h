// Types shared by the host runtime and the CUDA kernels of libfdwave.
//
// One "shot" is one independent wave-propagation problem (its own grid, model,
// wavefields and sparse points).  The time-step kernel walks a table of work
// units; each unit is a column of TY x TZ grid points (y, z) streamed along a
// chunk [x0, x1) of the slowest axis x.  Several shots of different sizes share
// one launch by sharing one unit table.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace fdw {

// Tile width along z (the contiguous axis): one warp lane per z.
constexpr int kTZ = 32;
// Largest stencil radius r = p/2 (space order 16).
constexpr int kMaxR = 8;
// Deepest pipeline of the step kernel.
constexpr int kMaxStages = 2 * kMaxR + 8;

enum MType : int { kF32 = 0, kF16 = 1, kBF16 = 2 };

// Flags of one step launch.
enum StepFlags : int {
  kInject = 1,       // add the injection list of each unit into the new field
  kSample = 2,       // record the sampling list of each unit from the current field
  kEtaField = 4,     // damping read from a full field instead of 1-D profiles
  kInjectDiff = 8,   // inject (a - b) instead of a
  kTestStall = 16,   // test hook: the producer issues no loads, so every consumer
                     // wait runs out of its clock budget and reports an error
  kAbsMax = 32,      // fold max |u^{n+1}| of every unit into amax[amax_slot] of its shot
  kPersist = 64,     // forward, recompute and adjoint roles: one launch runs the steps
                     // [step0, step_end); tickets run over (step, unit), step by
                     // step, and a unit of step n + 1 starts once the rows of units
                     // it reads have finished step n (row_done counts finished
                     // units per row)
  kReverse = 128,    // with kPersist: step n of the launch is the adjoint step at
                     // time t = inj_row - n (time runs backwards)
  kLinear = 256,     // with kPersist: step n reads slots n + 1 (u^t) and n (u^{t-1})
                     // and writes slot n + 2, t = inj_row + n (recompute buffers)
};

// Per-shot description; lives in device memory, 128-byte aligned (tensor maps).
struct alignas(128) ShotDesc {
  CUtensorMap tm_uh;   // wavefield slots [slots][nx][ny][nzp] f32, halo box (TZ+2R4, TY+2R, 1, 1)
  CUtensorMap tm_uc;   // the same slots, centre box (TZ, TY, 1, 1)
  CUtensorMap tm_m;    // model s = 1/m [nx][ny][nzp] (f32 / f16 / bf16), centre box (TZ, TY, 1)
  CUtensorMap tm_f;    // forward-wavefield slots (gradient), centre box (TZ, TY, 1, 1)
  CUtensorMap tm_e;    // damping field (eta*dt/2) [nx][ny][nzp] f32, centre box (optional)
  CUtensorMap tm_a;    // gradient accumulator [nx][ny][nzp] f32, centre box (gradient)
  float* u;            // base of the wavefield slots
  long long uslot;     // floats per slot
  const float* fwd;    // forward-wavefield slots (adjoint + gradient)
  long long fslot;
  float* acc;          // gradient accumulator, one slot (pitched)
  const void* m;       // model as s = 1/m, pitched, type mtype
  const float* eta;    // eta*dt/2 profiles, [nx] then [ny] then [nz]
  const float* etaf;   // eta*dt/2 field, pitched (when kEtaField)
  unsigned int* amax;  // per-snapshot absolute maxima (float bits), forward role
  int nx, ny, nz, nzp;
  int mtype;
  int smp_n;           // number of sampled points of the current role
  // sparse data of the current call
  const float* inj_a;  // [nt][inj_ld]
  const float* inj_b;  // [nt][inj_ld] or null; injected value is a - b
  float* smp_out;      // [nt][smp_ld]
  int inj_ld, smp_ld;
  const int* pt_base;  // sampling points: [npts][3] base node (x, y, z)
  const float* pt_w;   // sampling points: [npts][8] corner weights (x bit 2, y bit 1, z bit 0)
};

struct Unit {
  int shot;
  int x0, x1;
  int y0, z0;
  int flags;           // kUnitUndamped: eta = 0 at every grid point of the unit
  int row;             // the unit's row: one x chunk of one shot, all its column tiles
  int pad;
};

enum UnitFlags : int { kUnitUndamped = 1 };

// One grid node that receives an injected value, and the range of its terms.
struct InjNode {
  int x, y, z;
  int tbeg, tend;      // terms [tbeg, tend) in the term array
  int j0;              // the first term (terms[tbeg]) again, so that a sum
  float w0;            // needs no term load before its first data load
  int pad;
};

struct InjTerm {
  int j;               // point index (column of the data array)
  float w;             // multilinear weight of this node for that point
};

struct StepParams {
  const ShotDesc* shots;
  const Unit* units;
  int nunits;
  // Work distribution: with a ticket counter (zero before the launch) each CTA
  // takes the next unit in table order when it is ready for one; without, CTA
  // b takes units b, b + gridDim.x, ...
  int* ticket;
  int flags;
  // injection: unit u owns nodes [inj_ptr[u], inj_ptr[u+1])
  const int* inj_ptr;
  const InjNode* inj_nodes;
  const InjTerm* inj_terms;
  // sampling: unit u records points smp_pts[smp_ptr[u] .. smp_ptr[u+1])
  const int* smp_ptr;
  const int* smp_pts;
  int inj_row;         // time row of the injected data
  int smp_row;         // time row of the recorded samples
  int cur, prev, out;  // wavefield slots: u^n, u^{n-1}, u^{n+1} (out may equal prev)
  int fslot;           // forward-wavefield slot (gradient)
  int stages;          // pipeline depth (halo planes of u^n)
  int stage_bytes;     // bytes of one pipeline stage
  // Gradient steps keep the per-plane tiles (u^{n-1}, model, forward field,
  // accumulator, damping) in a ring of their own, loaded with the halo plane
  // R planes ahead and freed as soon as the plane is updated: cstages stages
  // of cstage_bytes, the offsets below relative to a stage of that ring.
  // Otherwise cstages = 0 and the tiles share the halo plane's stage.
  int cstages;
  int cstage_bytes;
  int off_p, off_m, off_f, off_e;  // byte offsets of the per-plane tiles
  int off_a;           // byte offset of the gradient-accumulator tile (gradient)
  int off_c;           // byte offset of the centre tile of u^n, R planes ahead
                       // of the stage's own plane (tiles that stage it)
  int amax_slot;       // snapshot index of kAbsMax
  float dt2;           // dt^2
  float csum;          // sum of the centre weights over the axes
  float w[3][kMaxR + 1];  // dt^2 c_k / h_a^2, k = 0..r (k = 0 unused; see csum)
  int* err;            // error word (0 = fine)
  // kPersist: steps of the launch, finished units per row (zero before the
  // launch), the rows [lo, hi] whose planes a row's units read, units per row
  int step0, step_end;
  int* row_done;
  const int2* row_deps;
  const int* row_units;
};

// Bits of the device error word: a consumer (full) or producer (empty) wait gave up.
enum ErrBits : int { kErrTimeoutFull = 1, kErrTimeoutEmpty = 2 };

}  // namespace fdw
