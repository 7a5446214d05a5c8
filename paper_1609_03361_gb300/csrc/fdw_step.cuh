// One explicit time step of the damped acoustic wave equation
//     m u_tt + eta u_t - lap(u) = q                      (paper Sec. 5, Eq. 3)
// in the three-level form
//     u^{n+1} = [ 2 m u^n - (m - eta dt/2) u^{n-1} + dt^2 L u^n ] / (m + eta dt/2)
// (centred u_tt as in the `dt2` expansion of Sec. 3.1, centred u_t for the
// damping term, order-p Laplacian L with a zero halo), fused with the sparse
// point-to-grid injection and grid-to-point sampling of Sec. 5.2.  The same
// kernel performs the adjoint step of Sec. 5.1 (Listing 7): that recursion has
// exactly this algebra with the roles of the time levels read backwards, so
// only the wavefield slots and the point lists change.  With GRAD it also
// accumulates the FWI imaging term u^k (lambda^k - 2 lambda^{k+1} + lambda^{k+2}).
//
// Layout: every field is [x][y][zp] (z contiguous, rows padded to zp), x the
// slowest axis.  The model is stored as s = 1/m, so the update reads
//     u^{n+1} = [ 2 u^n - (1 - e s) u^{n-1} + s dt^2 L u^n ] / (1 + e s),  e = eta dt/2,
// which needs no division where e = 0.  A CTA owns a column tile of TY x TZ
// points (y, z) and streams along a chunk [x0, x1) of x:
//  - a producer warp issues TMA loads, one pipeline stage per x plane: the
//    u^n plane with its (r, R4) halo in y and z (zero-filled outside the grid,
//    which is the zero halo of the scheme), and for computed planes the
//    u^{n-1}, m (and forward-wavefield / damping) tiles;
//  - consumer warps keep the 2r+1 values of u^n along x of their points in
//    registers (a queue), take y and z neighbours from shared memory with
//    16-byte loads (each lane owns four z-neighbouring points, each
//    quarter-warp NY rows), write u^{n+1} with 16-byte coalesced stores and
//    release the stage;
//  - after the chunk, the consumers add the injected values into the nodes the
//    unit owns (deterministic order, no atomics: no other CTA reads u^{n+1}
//    during this step) and record the sampled points of u^n.
// With TQ the x queue lives in tensor memory instead of registers: each
// thread owns one TMEM lane, where a ring of 2r+1 planes (four values each) is
// stored with a second copy of slots 0 .. 2r-2 after its end, so that the 2r
// planes x-r .. x+r-1 around the plane being updated are always 8r
// consecutive columns (16 r columns in all), read with one load per plane.
// A plane is written once (two 16-byte stores) when it arrives, and nothing
// shifts: the register queue costs 2r moves per point and plane, and 2r+1
// live registers per point.
// With CA each stage holds exactly what one update reads: the halo plane x,
// the tiles of plane x and a separate centre tile of plane x + r (the values
// that join the queue), after 2r stages of centre tiles that fill the queue;
// a stage is freed as soon as its plane is updated, so two stages already
// pipeline (otherwise the stages of planes x .. x + r stay staged while
// plane x is updated).  CA also forms the neighbour pair sums of two points
// per instruction (correctly rounded, the scalar sums), to save registers.
#pragma once

#include <cstdio>

#include "fdw_device.cuh"
#include "fdw_internal.h"

namespace fdw {

template <int R>
struct Halo {
  static constexpr int R4 = (R + 3) & ~3;  // z halo rounded up to 16 bytes (TMA x alignment)
  static constexpr int ZW = kTZ + 2 * R4;  // staged row length
};

struct Cursor {
  int stage;
  uint32_t phase;
  __device__ __forceinline__ void next(int S) {
    if (++stage == S) { stage = 0; phase ^= 1u; }
  }
  __device__ __forceinline__ void skip(int k, int S) {  // k < S
    stage += k;
    if (stage >= S) { stage -= S; phase ^= 1u; }
  }
};

// Hand a pipeline stage back to the producer.  The consumer reads the stage
// through the generic proxy while the producer refills it through the async
// proxy (TMA); the mbarrier release/acquire chain alone does not order the two
// proxies, so each lane fences its own reads before the warp arrives.  Without
// the fence a read still in flight could observe the next plane's data.
__device__ __forceinline__ void release_stage(uint32_t empty_bar, int lane) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
  if (lane == 0) mbar_arrive(empty_bar);
}

// The same for one stage of each ring.
__device__ __forceinline__ void release_stages(uint32_t empty_a, uint32_t empty_b, int lane) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
  if (lane == 0) {
    mbar_arrive(empty_a);
    mbar_arrive(empty_b);
  }
}

__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity, volatile int* abort) {
  if (mbar_try_wait(bar, parity)) return true;
  long long t0 = clock64();
#pragma unroll 1
  while (true) {
    // parked in hardware (up to 20 us per try) rather than spinning
    if (mbar_try_wait_suspend(bar, parity, 20000u)) return true;
    if (*abort) return false;
    if (clock64() - t0 > kWaitBudget) return false;
  }
}


// Consumer waits of a warp that uses tensor memory: the warp-collective
// tcgen05 instructions need every lane to take the same path, so a wait that
// gave up in any lane counts as given up in all.
template <bool UNIFORM>
__device__ __forceinline__ bool cwait(uint32_t bar, uint32_t parity, volatile int* abort) {
  const bool ok = wait_or_abort(bar, parity, abort);
  if constexpr (UNIFORM) return __all_sync(0xffffffffu, ok);
  return ok;
}

// Model values are stored as s = 1/m (squared velocity) in one of three types.
template <typename MT>
__device__ __forceinline__ float4 load_quad(const unsigned char* base, int i);
template <>
__device__ __forceinline__ float4 load_quad<float>(const unsigned char* base, int i) {
  return *reinterpret_cast<const float4*>(base + 4 * i);
}
template <>
__device__ __forceinline__ float4 load_quad<__half>(const unsigned char* base, int i) {
  const uint2 raw = *reinterpret_cast<const uint2*>(base + 2 * i);
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&raw.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&raw.y));
  return make_float4(a.x, a.y, b.x, b.y);
}
template <>
__device__ __forceinline__ float4 load_quad<__nv_bfloat16>(const unsigned char* base, int i) {
  const uint2 raw = *reinterpret_cast<const uint2*>(base + 2 * i);
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw.y));
  return make_float4(a.x, a.y, b.x, b.y);
}

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float pick(const float4& a, int v) {
  return v == 0 ? a.x : (v == 1 ? a.y : (v == 2 ? a.z : a.w));
}

// Thread layout of a consumer warp: four quarter-warps of 8 lanes, each on NY
// consecutive rows (y) of the tile; every lane owns four neighbouring points
// along z, so a quarter-warp covers one 32-point row with 16-byte accesses.
constexpr int kVZ = 4;
struct Lanes {
  int r0;  // first local row of the thread
  int zl;  // local z of the thread's first point (multiple of 4)
};

// Wavefield slots, time rows and snapshot-maximum flag of the step a unit
// belongs to.  One step per launch: the launch's.  kPersist: the unit's own
// step n of the launch, at time t = inj_row + n with u^t in slot t & 1 and
// u^{t+1} written over u^{t-1} in slot (t + 1) & 1, the snapshot maximum
// (kAbsMax) folded on the launch's last two steps; with kReverse the adjoint
// step at time t = inj_row - n (lambda^{t+1} in slot (t + 1) & 1, lambda^t
// written over lambda^{t+2} in slot t & 1); with kLinear slots n + 1, n and
// n + 2 (the recompute buffer).
struct StepCtx {
  int cur, prev, out;
  int inj_row, smp_row;
  bool amx;
};

__device__ __forceinline__ StepCtx step_ctx(const StepParams& P, int n) {
  if (P.flags & kPersist) {
    if (P.flags & kReverse) {
      const int t = P.inj_row - n;
      return StepCtx{(t + 1) & 1, t & 1, t & 1, t, t, false};
    }
    const int t = P.inj_row + n;
    const bool amx = (P.flags & kAbsMax) != 0 && n >= P.step_end - 2;
    if (P.flags & kLinear) return StepCtx{n + 1, n, n + 2, t, P.smp_row, amx};
    return StepCtx{t & 1, (t + 1) & 1, (t + 1) & 1, t, t, amx};
  }
  return StepCtx{P.cur, P.prev, P.out, P.inj_row, P.smp_row, (P.flags & kAbsMax) != 0};
}

// kPersist: wait (bounded) until every unit of the rows that a unit of `row`
// reads has finished the launch's step k - 1, then order those units'
// global writes before this thread's tensor loads.  The counters are read
// together first; a fence turns the reads that saw the counts into acquires.
__device__ __forceinline__ bool wait_rows(const StepParams& P, int row, int k,
                                          volatile int* abort) {
  const int2 dr = P.row_deps[row];
  long long t0 = 0;
  bool first = true;
#pragma unroll 1
  while (true) {
    bool ready = true;
#pragma unroll 1
    for (int r = dr.x; r <= dr.y; ++r)
      if (ld_relaxed_gpu(P.row_done + r) < k * P.row_units[r]) ready = false;
    if (ready) break;
    if (first) {
      t0 = clock64();
      first = false;
    }
    if (*abort || clock64() - t0 > kWaitBudget) return false;
    __nanosleep(128);
  }
  fence_acq_rel_gpu();
  fence_proxy_async_global();
  return true;
}

#ifdef FDW_DEBUG_VERIFY
// Debug builds only: compare a staged value with the global field it came from.
__device__ int g_dbg_count;
__device__ __forceinline__ void dbg_check(const char* what, float got, const float* base,
                                          long long slot, int x, int y, int z, int nx, int ny,
                                          int nz, int nzp, int u) {
  float want = 0.f;
  if (x >= 0 && x < nx && y >= 0 && y < ny && z >= 0 && z < nz)
    want = base[slot + ((long long)x * ny + y) * nzp + z];
  if (got != want) {
    const int k = atomicAdd(&g_dbg_count, 1);
    if (k < 24)
      printf("DBG %s unit %d x %d y %d z %d got %g want %g blk %d\n", what, u, x, y, z, got, want,
             blockIdx.x);
  }
}
#endif

// Streams one work unit through the pipeline: warm-up of the x queue, then
// one update per plane of [x0, x1).  XU: the x loop is unrolled by the queue
// length 2R+1 so that the queue slots rotate; otherwise the queue shifts by one
// slot per plane (smaller code).  SPLIT: the per-plane tiles come from the
// second ring (cursor cc).  CA: the stage of plane x also carries the centre
// tile of plane x + R, so the unit takes 2R warm-up stages (centre tiles of
// planes x0-R .. x0+R-1) and then exactly one stage per updated plane, each
// released as soon as that plane is done (cursor ca alone).  Returns false if
// a wait gave up.
template <int R, int NY, int BY, bool GRAD, bool XU, bool SPLIT, bool TQ, bool CA, typename MT,
          bool DAMP = true>
__device__ __forceinline__ bool run_unit(const StepParams& P, const Unit& un, const ShotDesc* d,
                                         int u, const unsigned char* smem, uint32_t full0,
                                         uint32_t empty0, Cursor& ca, Cursor& cb,
                                         const unsigned char* csmem, uint32_t cfull0,
                                         uint32_t cempty0, Cursor& cc,
                                         volatile int* abort_flag, int lane, const Lanes L,
                                         float& tmax, uint32_t tq, const StepCtx sc) {
  static_assert(!TQ || (NY == 1 && !XU), "the tensor-memory queue holds one row per thread");
  static_assert(!CA || (TQ && !SPLIT), "centre tiles are staged for the tensor-memory queue");
  constexpr int TZ = kTZ;
  constexpr int R4 = Halo<R>::R4;
  constexpr int ZW = Halo<R>::ZW;
  constexpr int Q = 2 * R + 1;     // x queue length
  constexpr int XS = XU ? Q : 1;   // planes per iteration of the x loop
  constexpr int NW = 4 + 2 * R4;   // z window of a row: z-R4 .. z+3+R4
  const int S = P.stages;
  const int ny = d->ny, nz = d->nz, nzp = d->nzp;
  const bool etaf = (P.flags & kEtaField) != 0;
  const bool amx = sc.amx;
  const int r0 = L.r0, zl = L.zl;
  const int z = un.z0 + zl;
  const bool zin = z < nz;

  // damping: y and z parts of the separable profile, per point
  float eyz[NY][kVZ];
  int rowoff[NY];
  bool rowok[NY];
#pragma unroll
  for (int j = 0; j < NY; ++j) {
    const int y = un.y0 + r0 + j;
    const float ey = (!etaf && y < ny) ? d->eta[d->nx + y] : 0.f;
#pragma unroll
    for (int v = 0; v < kVZ; ++v) {
      const int zz = z + v;
      eyz[j][v] = ey + ((!etaf && zz < nz) ? d->eta[d->nx + ny + zz] : 0.f);
    }
    rowok[j] = zin && y < ny;
    rowoff[j] = y * nzp + z;
  }
  const long long plane = (long long)ny * nzp;

  // x queue of centre values: slot (p - x0 + R) mod Q holds plane p (XU), or
  // slot i holds plane x - R + i (shift)
  // (with TQ: the ring slot of plane p is (p - x0 + R) mod Q, columns
  // 4 slot and, for slots 0 .. 2R-2, 4 (slot + Q) of the thread's lane from tq)
  float qv[NY][kVZ][TQ ? 1 : Q];
  if constexpr (TQ) tmem_wait_st();  // the previous unit's last stores are done
  bool ok = true;
#pragma unroll
  for (int i = 0; i < 2 * R; ++i) {
    if (ok) ok = cwait<TQ>(full0 + 8 * ca.stage, ca.phase, abort_flag);
    const float* U = reinterpret_cast<const float*>(smem + ca.stage * P.stage_bytes +
                                                    (CA ? P.off_c : 0));
#pragma unroll
    for (int j = 0; j < NY; ++j) {
      const int ci = CA ? (r0 + j) * TZ + zl : (r0 + j + R) * ZW + R4 + zl;
      const float4 cv = ok ? lds4(U + ci) : make_float4(0.f, 0.f, 0.f, 0.f);
      if constexpr (TQ) {
        tmem_st4(tq + 4 * i, cv);
        if (i <= 2 * R - 2) tmem_st4(tq + 4 * (i + Q), cv);  // read past the ring's end
      } else {
#pragma unroll
        for (int v = 0; v < kVZ; ++v) qv[j][v][i] = pick(cv, v);
      }
#ifdef FDW_DEBUG_VERIFY
      dbg_check("warm", cv.x, d->u, (long long)sc.cur * d->uslot, un.x0 - R + i, un.y0 + r0 + j,
                z, d->nx, ny, nz, nzp, u);
#endif
    }
    const int p = un.x0 - R + i;
    if (CA || p < un.x0 || p >= un.x1) release_stage(empty0 + 8 * ca.stage, lane);
    ca.next(S);
  }
  if (!ok) return false;
  if constexpr (!CA) cb.skip(R, S);

  float* uo = d->u + (long long)sc.out * d->uslot;
  float* acc = d->acc;
  const float* eta_x = d->eta;
  float ex_next = etaf ? 0.f : eta_x[un.x0];  // x part of the damping, one plane ahead
  int tq_sl = 0;  // ring slot of plane x - R (TQ)
  (void)tq_sl;
#pragma unroll 1
  for (int xb = un.x0; xb < un.x1; xb += XS) {
#pragma unroll
    for (int t0 = 0; t0 < XS; ++t0) {
      const int t = XU ? t0 : 0;
      const int x = xb + t0;
      if (x >= un.x1) break;
      // TQ: planes x-R .. x+R-1 come from the tensor-memory ring; the window
      // starts at the slot of plane x-R, and its load is in flight while the
      // warp waits for the halo planes and reads them
      TmemWindow<TQ ? R : 1> win;
      (void)win;
      if constexpr (TQ) {
        tmem_wait_st();  // the previous plane's ring stores are done
        win.issue(tq + 4 * tq_sl);
      }
      // centre values of plane x+R join the queue
      if (!cwait<TQ>(full0 + 8 * ca.stage, ca.phase, abort_flag)) {
        if constexpr (TQ) win.wait();
        return false;
      }
      float4 ahead[NY];
      (void)ahead;
      {
        const float* Ua = reinterpret_cast<const float*>(smem + ca.stage * P.stage_bytes +
                                                         (CA ? P.off_c : 0));
#pragma unroll
        for (int j = 0; j < NY; ++j) {
          const float4 cv = lds4(Ua + (CA ? (r0 + j) * TZ + zl : (r0 + j + R) * ZW + R4 + zl));
          if constexpr (TQ) {
            ahead[j] = cv;
          } else {
#pragma unroll
            for (int v = 0; v < kVZ; ++v) qv[j][v][(t + 2 * R) % Q] = pick(cv, v);
          }
#ifdef FDW_DEBUG_VERIFY
          dbg_check("ahead", cv.x, d->u, (long long)sc.cur * d->uslot, x + R, un.y0 + r0 + j, z,
                    d->nx, ny, nz, nzp, u);
#endif
        }
      }
      if constexpr (TQ) {
        // plane x+R takes the slot of plane x-R-1, outside the window in flight
        const int sa = tq_sl == 0 ? Q - 1 : tq_sl - 1;
        tmem_st4(tq + 4 * sa, ahead[0]);
        // the second copy for slots 0 .. 2R-2; the other slots write their
        // one copy again (no branch around the warp-wide store)
        tmem_st4(tq + 4 * (sa <= 2 * R - 2 ? sa + Q : sa), ahead[0]);
        tq_sl = tq_sl + 1 == Q ? 0 : tq_sl + 1;
      }
      // a look-ahead plane past the chunk is only needed for its centre
      // values; it is handed back after the update below has consumed them
      const int ahead_stage = ca.stage;
      ca.next(S);

      // neighbours in y and z of plane x from the staged halo plane (CA: the
      // stage just read, which holds plane x itself)
      const unsigned char* sb = smem + (CA ? ahead_stage : cb.stage) * P.stage_bytes;
      const float* U = reinterpret_cast<const float*>(sb);
      const unsigned char* tb = sb;  // the plane's own tiles
      if (SPLIT) {
        if (!cwait<TQ>(cfull0 + 8 * cc.stage, cc.phase, abort_flag)) {
          if constexpr (TQ) win.wait();
          return false;
        }
        tb = csmem + cc.stage * P.cstage_bytes;
      }
      const float ex = ex_next;
      if (DAMP && !etaf && x + 1 < un.x1) ex_next = eta_x[x + 1];
      const float* Pp = reinterpret_cast<const float*>(tb + P.off_p);
      const long long xoff = (long long)x * plane;
      // y neighbours of the thread's rows: local rows r0-R .. r0+NY-1+R
      float4 yr[NY + 2 * R];
      float val[NY][kVZ];
      float d2t[NY][kVZ];
      float4 fw[NY];
      float4 aw[NY];
      (void)d2t;
      (void)fw;
      (void)aw;
#pragma unroll
      for (int i = 0; i < R; ++i) {
        yr[i] = lds4(U + (r0 + i) * ZW + R4 + zl);
        yr[NY + R + i] = lds4(U + (r0 + NY + R + i) * ZW + R4 + zl);
      }
      // with several rows per thread, each row's centre is a y neighbour of
      // the others: load all of them before any row is updated
      if (NY > 1) {
#pragma unroll
        for (int j = 0; j < NY; ++j) yr[R + j] = lds4(U + (r0 + j + R) * ZW + R4 + zl);
      }
      if constexpr (TQ && !CA) win.wait();
#pragma unroll
      for (int j = 0; j < NY; ++j) {
        float wz[NW];
#pragma unroll
        for (int i = 0; i < NW / 4; ++i) {
          const float4 w4 = lds4(U + (r0 + j + R) * ZW + zl + 4 * i);
          wz[4 * i] = w4.x;
          wz[4 * i + 1] = w4.y;
          wz[4 * i + 2] = w4.z;
          wz[4 * i + 3] = w4.w;
        }
        const int li = (r0 + j) * TZ + zl;
        const float4 pv = lds4(Pp + li);
        const float4 sv = load_quad<MT>(tb + P.off_m, li);
        float4 ev;
        if (etaf) ev = lds4(reinterpret_cast<const float*>(tb + P.off_e) + li);
        else ev = make_float4(ex + eyz[j][0], ex + eyz[j][1], ex + eyz[j][2], ex + eyz[j][3]);
        // the update of point v from its three axis sums
        auto finish = [&](int v, float lx, float ly, float lz) {
          const float c = wz[R4 + v];
          const float lap = fmaf(P.csum, c, lx + ly + lz);
          const float sm = pick(sv, v), prev = pick(pv, v);
          if constexpr (DAMP) {
            const float es = pick(ev, v) * sm;
            // [2u - (1 - e s) u- + s dt^2 L u] / (1 + e s): the three-level update divided by m
            const float num = fmaf(es, prev, fmaf(sm, lap, 2.f * c) - prev);
            val[j][v] = __fdividef(num, 1.f + es);
          } else {  // e = 0 at every point of the unit: 2u - u- + s dt^2 L u
            val[j][v] = fmaf(sm, lap, 2.f * c) - prev;
          }
          if (GRAD) d2t[j][v] = val[j][v] - 2.f * c + prev;  // second time difference of lambda
        };
        if constexpr (CA) {
          // the neighbour pair sums of two points at a time (fadd2: two
          // correctly rounded adds, the scalar results), then one FMA per
          // point and k in the scalar order; the y and z sums first, while
          // the tensor-memory window is still in flight
          float ly[kVZ] = {0.f, 0.f, 0.f, 0.f}, lz[kVZ] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int k = 1; k <= R; ++k) {
            const float4 ym = yr[R + j - k], yp = yr[R + j + k];
            const float2 ya = __fadd2_rn(make_float2(ym.x, ym.y), make_float2(yp.x, yp.y));
            const float2 yb = __fadd2_rn(make_float2(ym.z, ym.w), make_float2(yp.z, yp.w));
            ly[0] = fmaf(P.w[1][k], ya.x, ly[0]);
            ly[1] = fmaf(P.w[1][k], ya.y, ly[1]);
            ly[2] = fmaf(P.w[1][k], yb.x, ly[2]);
            ly[3] = fmaf(P.w[1][k], yb.y, ly[3]);
            if ((k & 1) == 0) {
              // R4 -+ k even: the pairs (e, e+1) of both sides are aligned
              const int m = R4 - k, q = R4 + k;
              const float2 za = __fadd2_rn(make_float2(wz[m], wz[m + 1]), make_float2(wz[q], wz[q + 1]));
              const float2 zb = __fadd2_rn(make_float2(wz[m + 2], wz[m + 3]),
                                           make_float2(wz[q + 2], wz[q + 3]));
              lz[0] = fmaf(P.w[2][k], za.x, lz[0]);
              lz[1] = fmaf(P.w[2][k], za.y, lz[1]);
              lz[2] = fmaf(P.w[2][k], zb.x, lz[2]);
              lz[3] = fmaf(P.w[2][k], zb.y, lz[3]);
            } else {
#pragma unroll
              for (int v = 0; v < kVZ; ++v)
                lz[v] = fmaf(P.w[2][k], wz[R4 + v - k] + wz[R4 + v + k], lz[v]);
            }
          }
          win.wait();
          float lx[kVZ] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int k = 1; k <= R; ++k) {
            const int i0 = 4 * (R - k), i1 = 4 * (R + k);
            const float2 ma = make_float2(win.v(i0), win.v(i0 + 1));
            const float2 mb = make_float2(win.v(i0 + 2), win.v(i0 + 3));
            const float2 pa = k < R ? make_float2(win.v(i1), win.v(i1 + 1))
                                    : make_float2(ahead[j].x, ahead[j].y);
            const float2 pb = k < R ? make_float2(win.v(i1 + 2), win.v(i1 + 3))
                                    : make_float2(ahead[j].z, ahead[j].w);
            const float2 xa = __fadd2_rn(ma, pa), xb = __fadd2_rn(mb, pb);
            lx[0] = fmaf(P.w[0][k], xa.x, lx[0]);
            lx[1] = fmaf(P.w[0][k], xa.y, lx[1]);
            lx[2] = fmaf(P.w[0][k], xb.x, lx[2]);
            lx[3] = fmaf(P.w[0][k], xb.y, lx[3]);
          }
#pragma unroll
          for (int v = 0; v < kVZ; ++v) finish(v, lx[v], ly[v], lz[v]);
        } else {
#pragma unroll
          for (int v = 0; v < kVZ; ++v) {
            float lx = 0.f, ly = 0.f, lz = 0.f;
#pragma unroll
            for (int k = 1; k <= R; ++k) {
              if constexpr (TQ) {
                const float xb = k < R ? win.v(4 * (R + k) + v) : pick(ahead[j], v);
                lx = fmaf(P.w[0][k], win.v(4 * (R - k) + v) + xb, lx);
              } else {
                lx = fmaf(P.w[0][k], qv[j][v][(t + R - k) % Q] + qv[j][v][(t + R + k) % Q], lx);
              }
              ly = fmaf(P.w[1][k], pick(yr[R + j - k], v) + pick(yr[R + j + k], v), ly);
              lz = fmaf(P.w[2][k], wz[R4 + v - k] + wz[R4 + v + k], lz);
            }
            finish(v, lx, ly, lz);
          }
        }
        if (GRAD) {
          fw[j] = lds4(reinterpret_cast<const float*>(tb + P.off_f) + li);
          aw[j] = lds4(reinterpret_cast<const float*>(tb + P.off_a) + li);
        }
      }
      // every read of the staged planes is done: hand them back before the
      // global stores, which only read registers
      if constexpr (CA) {
        release_stage(empty0 + 8 * ahead_stage, lane);
      } else {
        if (SPLIT) {
          release_stages(empty0 + 8 * cb.stage, cempty0 + 8 * cc.stage, lane);
          cc.next(P.cstages);
        } else {
          release_stage(empty0 + 8 * cb.stage, lane);
        }
        if (x + R >= un.x1) release_stage(empty0 + 8 * ahead_stage, lane);
        cb.next(S);
      }
      if (amx) {  // points past the grid compute to zero and do not move the maximum
#pragma unroll
        for (int j = 0; j < NY; ++j)
#pragma unroll
          for (int v = 0; v < kVZ; ++v) tmax = fmaxf(tmax, fabsf(val[j][v]));
      }
#pragma unroll
      for (int j = 0; j < NY; ++j) {
        if (rowok[j]) {
          const long long off = xoff + rowoff[j];
          *reinterpret_cast<float4*>(uo + off) =
              make_float4(val[j][0], val[j][1], val[j][2], val[j][3]);
          if (GRAD) {
            float4 a = aw[j];  // the accumulator tile was staged with the plane
            a.x = fmaf(fw[j].x, d2t[j][0], a.x);
            a.y = fmaf(fw[j].y, d2t[j][1], a.y);
            a.z = fmaf(fw[j].z, d2t[j][2], a.z);
            a.w = fmaf(fw[j].w, d2t[j][3], a.w);
            *reinterpret_cast<float4*>(acc + off) = a;
          }
        }
      }
      if (!XU && !TQ) {
#pragma unroll
        for (int j = 0; j < NY; ++j)
#pragma unroll
          for (int v = 0; v < kVZ; ++v)
#pragma unroll
            for (int i = 0; i < 2 * R; ++i) qv[j][v][i] = qv[j][v][i + 1];
      }
    }
  }
  if constexpr (!CA) cb.skip(R, S);
  return true;
}

// The forward step with a second ring at radius 7 and 8 asks for three
// resident CTAs per SM (136 registers a thread), which its smaller shared
// memory allows; every other instance leaves the register count to the
// compiler (a minimum of 0 blocks states no constraint).
template <int R, int NY, int BY, bool GRAD, bool XU, bool SPLIT = GRAD, bool TQ = false,
          bool CA = false>
__global__ void __launch_bounds__((BY + 1) * 32, (SPLIT && !GRAD && R >= 7 && !TQ) ? 3 : 0)
step_kernel(const __grid_constant__ StepParams P) {
  static_assert(!TQ || BY == 4, "the tensor-memory queue maps the four consumer warps to the four lane quarters");
  static_assert(!CA || (TQ && !SPLIT), "centre tiles are staged for the tensor-memory queue");
  constexpr int TZ = kTZ;
  constexpr int TY = 4 * BY * NY;
  constexpr int R4 = Halo<R>::R4;
  constexpr int ZW = Halo<R>::ZW;
  constexpr int YW = TY + 2 * R;
  constexpr int NCONS = BY * 32;

  extern __shared__ unsigned char smem_raw[];
  __shared__ int s_abort;
  __shared__ int s_issued;
  // the unit that starts at each stage (index -1: no more units), written by
  // the producer before the stage's first arrival, read by the consumers
  __shared__ Unit s_unit[kMaxStages];
  __shared__ int s_uidx[kMaxStages];
  __shared__ int s_step[kMaxStages];  // the step of that unit (kPersist)
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const int S = P.stages;
  const int SC = SPLIT ? P.cstages : 0;
  const unsigned char* csmem = smem + S * P.stage_bytes;  // second ring (SPLIT)
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * P.stage_bytes + SC * P.cstage_bytes);
  const uint32_t full0 = smem_u32(bars);
  const uint32_t empty0 = smem_u32(bars + S);
  const uint32_t cfull0 = smem_u32(bars + 2 * S);
  const uint32_t cempty0 = smem_u32(bars + 2 * S + SC);
  const uint32_t tail = smem_u32(bars + 2 * S + 2 * SC);  // consumer-only barrier at the end of a unit
  volatile int* abort_flag = &s_abort;
  __shared__ int s_issued_c;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  // tensor-memory ring of the x queue (TQ): allocated by warp 0, freed by it
  // at the end; each consumer warp w uses lanes 32 w .. 32 w + 31
  __shared__ uint32_t s_tmem;
  if constexpr (TQ) {
    if (warp == 0) {
      tmem_alloc(smem_u32(&s_tmem), (uint32_t)tq_columns(R));
      tmem_fence_before_sync();
    }
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, BY);
    }
    for (int s = 0; s < SC; ++s) {
      mbar_init(cfull0 + 8 * s, 1);
      mbar_init(cempty0 + 8 * s, BY);
    }
    mbar_init(tail, NCONS);
    s_abort = 0;
    s_issued = 0;
    s_issued_c = 0;
    fence_barrier_init();
  }
  __syncthreads();
  uint32_t tq = 0;
  if constexpr (TQ) {
    tmem_fence_after_sync();
    tq = s_tmem + ((uint32_t)(32 * (warp & 3)) << 16);
  }

  if (warp == BY) {
    // ------------------------------ producer ------------------------------
    if (lane == 0) {
      Cursor c{0, 0u};
      Cursor c2{0, 0u};  // second ring (SPLIT)
      int issued = 0, issued_c = 0;
      const uint32_t bytes_u = YW * ZW * 4;
      const bool stall = (P.flags & kTestStall) != 0;
      // tickets: units of the launch's step, or (kPersist) (step, unit) pairs
      // in step order, ticket t = k nunits + u for step step0 + k
      const bool persist = (P.flags & kPersist) != 0;
      const int total = persist ? (P.step_end - P.step0) * P.nunits : P.nunits;
      auto grab = [&](int after) { return P.ticket ? atomicAdd(P.ticket, 1) : after + (int)gridDim.x; };
      int t = stall ? total : (P.ticket ? atomicAdd(P.ticket, 1) : (int)blockIdx.x);
      bool failed = false;
      while (t < total && !failed) {
        const int k = persist ? t / P.nunits : 0;
        const int u = t - k * P.nunits;
        const StepCtx sc = step_ctx(P, P.step0 + k);
        const Unit un = P.units[u];
        const ShotDesc* d = P.shots + un.shot;
        const uint32_t bytes_in = TY * TZ * 4 + TY * TZ * (d->mtype == kF32 ? 4 : 2) +
                                  (GRAD ? 2 * TY * TZ * 4 : 0) +
                                  ((P.flags & kEtaField) ? TY * TZ * 4 : 0);
        // the planes this unit reads were written by the previous step
        if (persist && k > 0 && !wait_rows(P, un.row, k, abort_flag)) {
          atomicOr(P.err, kErrTimeoutEmpty);
          *abort_flag = 1;
          failed = true;
          break;
        }
        int next = total;
        if constexpr (CA) {
          // 2R warm-up stages with the centre tiles of planes x0-R .. x0+R-1,
          // then per plane x of the chunk: the centre tile of plane x + R, the
          // halo plane x and the tiles of x
          const uint32_t bytes_c = TY * TZ * 4;
          const int nst = 2 * R + (un.x1 - un.x0);
          for (int i = 0; i < nst; ++i) {
            const uint32_t full = full0 + 8 * c.stage, empty = empty0 + 8 * c.stage;
            if (issued >= S && !wait_or_abort(empty, c.phase ^ 1u, abort_flag)) {
              atomicOr(P.err, kErrTimeoutEmpty);
              *abort_flag = 1;
              failed = true;
              break;
            }
            if (i == 0) {
              s_unit[c.stage] = un;
              s_uidx[c.stage] = u;
              s_step[c.stage] = P.step0 + k;
            }
            if (i == nst - 1) next = grab(t);
            const bool warm = i < 2 * R;
            const int x = un.x0 + i - 2 * R;               // plane updated (after warm-up)
            const int pc = warm ? un.x0 - R + i : x + R;   // plane of the centre tile
            mbar_arrive_expect_tx(full, bytes_c + (warm ? 0u : bytes_u + bytes_in));
            const uint32_t sb = smem_u32(smem + c.stage * P.stage_bytes);
            tma_load_4d(sb + P.off_c, &d->tm_uc, un.z0, un.y0, pc, sc.cur, full);
            if (!warm) {
              tma_load_4d(sb, &d->tm_uh, un.z0 - R4, un.y0 - R, x, sc.cur, full);
              tma_load_4d(sb + P.off_p, &d->tm_uc, un.z0, un.y0, x, sc.prev, full);
              tma_load_3d(sb + P.off_m, &d->tm_m, un.z0, un.y0, x, full);
              if (GRAD) {
                tma_load_4d(sb + P.off_f, &d->tm_f, un.z0, un.y0, x, P.fslot, full);
                tma_load_3d(sb + P.off_a, &d->tm_a, un.z0, un.y0, x, full);
              }
              if (P.flags & kEtaField) tma_load_3d(sb + P.off_e, &d->tm_e, un.z0, un.y0, x, full);
            }
            ++issued;
            c.next(S);
          }
        } else {
          for (int p = un.x0 - R; p < un.x1 + R; ++p) {
            const uint32_t full = full0 + 8 * c.stage, empty = empty0 + 8 * c.stage;
            if (issued >= S && !wait_or_abort(empty, c.phase ^ 1u, abort_flag)) {
              atomicOr(P.err, kErrTimeoutEmpty);
              *abort_flag = 1;
              failed = true;
              break;
            }
            if (p == un.x0 - R) {
              s_unit[c.stage] = un;
              s_uidx[c.stage] = u;
              s_step[c.stage] = P.step0 + k;
            }
            // the next unit is claimed while the last plane of this one is in
            // flight: late enough to leave it to a CTA that is free earlier,
            // early enough to hide the atomic behind the stages still queued
            if (p == un.x1 + R - 1) next = grab(t);
            // the per-plane tiles of plane q: with the halo plane q itself, or
            // (SPLIT) in the second ring together with the halo plane q + R
            const int q = SPLIT ? p - R : p;
            const bool inner = q >= un.x0 && q < un.x1;
            mbar_arrive_expect_tx(full, bytes_u + (!SPLIT && inner ? bytes_in : 0u));
            const uint32_t sb = smem_u32(smem + c.stage * P.stage_bytes);
            tma_load_4d(sb, &d->tm_uh, un.z0 - R4, un.y0 - R, p, sc.cur, full);
            ++issued;
            c.next(S);
            if (inner) {
              uint32_t tb = sb, tfull = full;
              if (SPLIT) {
                tfull = cfull0 + 8 * c2.stage;
                if (issued_c >= SC && !wait_or_abort(cempty0 + 8 * c2.stage, c2.phase ^ 1u, abort_flag)) {
                  atomicOr(P.err, kErrTimeoutEmpty);
                  *abort_flag = 1;
                  failed = true;
                  break;
                }
                mbar_arrive_expect_tx(tfull, bytes_in);
                tb = smem_u32(csmem + c2.stage * P.cstage_bytes);
              }
              tma_load_4d(tb + P.off_p, &d->tm_uc, un.z0, un.y0, q, sc.prev, tfull);
              tma_load_3d(tb + P.off_m, &d->tm_m, un.z0, un.y0, q, tfull);
              if (GRAD) {
                tma_load_4d(tb + P.off_f, &d->tm_f, un.z0, un.y0, q, P.fslot, tfull);
                tma_load_3d(tb + P.off_a, &d->tm_a, un.z0, un.y0, q, tfull);
              }
              if (P.flags & kEtaField) tma_load_3d(tb + P.off_e, &d->tm_e, un.z0, un.y0, q, tfull);
              if (SPLIT) {
                ++issued_c;
                c2.next(SC);
              }
            }
          }
        }
        t = next;
      }
      // end marker: a stage that carries no data and unit index -1
      if (!failed && !stall) {
        if (issued >= S && !wait_or_abort(empty0 + 8 * c.stage, c.phase ^ 1u, abort_flag)) {
          atomicOr(P.err, kErrTimeoutEmpty);
          *abort_flag = 1;
        } else {
          s_uidx[c.stage] = -1;
          mbar_arrive(full0 + 8 * c.stage);
          ++issued;
        }
      }
      s_issued = issued;
      s_issued_c = issued_c;
    }
  } else {
    // ------------------------------ consumers -----------------------------
    Lanes L;
    L.r0 = warp * 4 * NY + (lane >> 3) * NY;
    L.zl = kVZ * (lane & 7);
    Cursor ca{0, 0u};   // read-ahead cursor: every plane in order (centre values)
    Cursor cb{0, 0u};   // compute cursor: the plane being updated
    Cursor cc{0, 0u};   // second-ring cursor (SPLIT): the plane being updated
    uint32_t tail_phase = 0u;
    const int tid = threadIdx.x;
    float tmax = 0.f;  // max |u^{n+1}| of the thread's points in the current unit (kAbsMax)
    bool ok = true;
    while (true) {
      // the stage of the next unit's first plane names the unit
      if (!cwait<TQ>(full0 + 8 * ca.stage, ca.phase, abort_flag)) {
        ok = false;
        break;
      }
      const int u = s_uidx[ca.stage];
      if (u < 0) break;
      const Unit un = s_unit[ca.stage];
      const StepCtx sc = step_ctx(P, s_step[ca.stage]);
      const ShotDesc* d = P.shots + un.shot;
      const int mtype = d->mtype;
      // the maximum covers this unit alone (a persistent launch mixes units
      // of steps that fold it with units of steps that do not)
      tmax = 0.f;
      if (mtype == kF16)
        ok = run_unit<R, NY, BY, GRAD, XU, SPLIT, TQ, CA, __half>(P, un, d, u, smem, full0, empty0, ca, cb, csmem, cfull0, cempty0, cc,
                                               abort_flag, lane, L, tmax, tq, sc);
      else if (mtype == kBF16)
        ok = run_unit<R, NY, BY, GRAD, XU, SPLIT, TQ, CA, __nv_bfloat16>(P, un, d, u, smem, full0, empty0, ca, cb, csmem, cfull0, cempty0, cc,
                                                      abort_flag, lane, L, tmax, tq, sc);
      else if (!XU && (un.flags & kUnitUndamped))  // every point of the unit undamped
        ok = run_unit<R, NY, BY, GRAD, XU, SPLIT, TQ, CA, float, false>(P, un, d, u, smem, full0, empty0, ca, cb, csmem, cfull0, cempty0, cc,
                                                     abort_flag, lane, L, tmax, tq, sc);
      else
        ok = run_unit<R, NY, BY, GRAD, XU, SPLIT, TQ, CA, float>(P, un, d, u, smem, full0, empty0, ca, cb, csmem, cfull0, cempty0, cc,
                                              abort_flag, lane, L, tmax, tq, sc);
      if (!ok) break;

      // ---- unit tail: injection into u^{n+1} and sampling of u^n ----
      mbar_arrive(tail);
      if (!cwait<TQ>(tail, tail_phase, abort_flag)) { ok = false; break; }
      tail_phase ^= 1u;
      const int nx = d->nx, ny = d->ny, nzp = d->nzp;
      const bool etaf = (P.flags & kEtaField) != 0;
      if (P.flags & kInject) {
        const int ib = P.inj_ptr[u], ie = P.inj_ptr[u + 1];
        const float* A = d->inj_a + (long long)sc.inj_row * d->inj_ld;
        const float* B = (P.flags & kInjectDiff) ? d->inj_b + (long long)sc.inj_row * d->inj_ld
                                                 : nullptr;
        float* uo = d->u + (long long)sc.out * d->uslot;
        const InjNode* nodes = P.inj_nodes;
        const InjTerm* terms = P.inj_terms;
        const void* mp = d->m;
        const float* eta = d->eta;
        const float* etafp = d->etaf;
        float* accp = d->acc;
        const float* fwdp = GRAD ? d->fwd + (long long)P.fslot * d->fslot : nullptr;
        // the terms in order, the first one from the node record itself
        auto node_sum = [&](const InjNode& nd) {
          float sum = 0.f;
          if (nd.tend > nd.tbeg) {
            sum = fmaf(nd.w0, B ? A[nd.j0] - B[nd.j0] : A[nd.j0], sum);
            for (int t = nd.tbeg + 1; t < nd.tend; ++t) {
              const InjTerm tm = terms[t];
              const float v = B ? A[tm.j] - B[tm.j] : A[tm.j];
              sum = fmaf(tm.w, v, sum);
            }
          }
          return sum;
        };
        // dt^2 q / (m + eta dt/2) with s = 1/m, at node nd
        auto node_delta = [&](const InjNode& nd, long long off, float sum) {
          const float s = load_m(mp, mtype, off);
          const float e = etaf ? etafp[off] : eta[nd.x] + eta[nx + nd.y] + eta[nx + ny + nd.z];
          return P.dt2 * sum * s / (1.f + e * s);
        };
        // two nodes per pass: their independent loads overlap (receiver
        // residuals in the adjoint step put about a thousand nodes in a unit)
        for (int i = ib + tid; i < ie; i += 2 * NCONS) {
          const int i2 = i + NCONS;
          const bool two = i2 < ie;
          const InjNode n1 = nodes[i];
          const InjNode n2 = nodes[two ? i2 : i];
          const long long off1 = ((long long)n1.x * ny + n1.y) * nzp + n1.z;
          const long long off2 = ((long long)n2.x * ny + n2.y) * nzp + n2.z;
          const float d1 = node_delta(n1, off1, node_sum(n1));
          const float d2 = node_delta(n2, off2, node_sum(n2));
          const float u1 = uo[off1], u2 = uo[off2];
          float f1 = 0.f, f2 = 0.f, a1 = 0.f, a2 = 0.f;
          if (GRAD) {
            f1 = fwdp[off1];
            f2 = fwdp[off2];
            a1 = accp[off1];
            a2 = accp[off2];
          }
          uo[off1] = u1 + d1;
          tmax = fmaxf(tmax, fabsf(u1 + d1));
          if (GRAD) accp[off1] = fmaf(f1, d1, a1);
          if (two) {
            uo[off2] = u2 + d2;
            tmax = fmaxf(tmax, fabsf(u2 + d2));
            if (GRAD) accp[off2] = fmaf(f2, d2, a2);
          }
        }
      }
      if (sc.amx) {
        // the unit's maximum after injection (an injected node also counted
        // its value before injection: an upper bound, which is all the
        // snapshot scale needs)
        float m = tmax;
#pragma unroll
        for (int k = 16; k > 0; k >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, k));
        if (lane == 0 && m > 0.f) atomicMax(d->amax + P.amax_slot, __float_as_uint(m));
        tmax = 0.f;
      }
      if (P.flags & kSample) {
        const int sbg = P.smp_ptr[u], se = P.smp_ptr[u + 1];
        const float* uc = d->u + (long long)sc.cur * d->uslot;
        float* out = d->smp_out + (long long)sc.smp_row * d->smp_ld;
        for (int i = sbg + tid; i < se; i += NCONS) {
          const int j = P.smp_pts[i];
          const int bx = d->pt_base[3 * j], by = d->pt_base[3 * j + 1], bz = d->pt_base[3 * j + 2];
          const float* w = d->pt_w + 8 * j;
          float acc = 0.f;
#pragma unroll
          for (int cc = 0; cc < 8; ++cc) {
            const float wc = w[cc];
            if (wc != 0.f) {
              const long long off =
                  ((long long)(bx + ((cc >> 2) & 1)) * ny + (by + ((cc >> 1) & 1))) * nzp + bz + (cc & 1);
              // at the L2 (kPersist: the field was written by other CTAs
              // within this launch, after this SM may have cached an older
              // step's values of the same slot)
              acc = fmaf(wc, __ldcg(uc + off), acc);
            }
          }
          out[j] = acc;
        }
      }
      if (P.flags & kPersist) {
        // every consumer's writes of this unit (updated planes, injected
        // nodes, samples) come before the unit counts as finished
        mbar_arrive(tail);
        if (!cwait<TQ>(tail, tail_phase, abort_flag)) {
          ok = false;
          break;
        }
        tail_phase ^= 1u;
        if (tid == 0) red_release_add_gpu(P.row_done + un.row, 1);
      }
    }
    if (!ok) {
      atomicOr(P.err, kErrTimeoutFull);
      *abort_flag = 1;
    }
    if constexpr (TQ) {  // the warp's last ring stores are done before the ring is freed
      tmem_wait_st();
      tmem_fence_before_sync();
    }
  }
  __syncthreads();
  // On an aborted launch, wait (bounded) for the loads still in flight before
  // the CTA's shared memory is released.
  if (*abort_flag && threadIdx.x == BY * 32) {
    const int issued = s_issued;
    for (int k = (issued > S ? issued - S : 0); k < issued; ++k) {
      const int st = k % S;
      const uint32_t ph = (uint32_t)((k / S) & 1);
      long long t0 = clock64();
      while (!mbar_try_wait(full0 + 8 * st, ph) && clock64() - t0 < kWaitBudget) {
      }
    }
    if constexpr (SPLIT) {
      const int issued_c = s_issued_c;
      for (int k = (issued_c > SC ? issued_c - SC : 0); k < issued_c; ++k) {
        const int st = k % SC;
        const uint32_t ph = (uint32_t)((k / SC) & 1);
        long long t0 = clock64();
        while (!mbar_try_wait(cfull0 + 8 * st, ph) && clock64() - t0 < kWaitBudget) {
        }
      }
    }
  }
  if constexpr (TQ) {
    if (warp == 0) {
      tmem_fence_after_sync();
      tmem_dealloc(s_tmem, (uint32_t)tq_columns(R));
    }
  }
}

}  // namespace fdw
