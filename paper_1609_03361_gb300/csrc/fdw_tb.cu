// Two time steps of the damped acoustic wave equation per pass over memory:
// temporal blocking of the explicit scheme of Sec. 5 (Eq. 3),
//     u^{t+1} = [ 2 u^t - (1 - e s) u^{t-1} + s dt^2 L u^t ] / (1 + e s),
// s = 1/m, e = eta dt/2, order-p Laplacian L with a zero halo, applied for
// t = n and t = n + 1 in one launch, with the point-source injection of
// Sec. 5.2 into both new levels and the receiver sampling of both old ones.
//
// A CTA owns an output tile of TY x 56 points (y, z) and streams a chunk
// [x0, x1) of x planes:
//  - a producer warp issues TMA loads into a ring of stages, one per x plane
//    q of u^n: the halo box of the plane (region E grown by r rows and 4
//    points, zero-filled outside the grid) and, for the planes of the first
//    step, the region-E tiles of u^{n-1} and s;
//  - first step: consumer thread (ry, qz) owns one four-point quad of region
//    E; at plane p it computes u^{n+1} there (x neighbours from a register
//    queue of u^n, y and z neighbours from the halo box) and writes it into a
//    ring of 2r + 2 region-E planes in shared memory;
//  - second step, r planes behind: thread (ty, tq) owns one quad of the
//    output tile and computes u^{n+2} at plane x = p - r with every neighbour
//    from that ring; u^n and s at x come from plane x's stage, which stays
//    held until then (the pipeline keeps at least 2r + 1 stages);
//  - the first step's points outside the grid are set to zero, which is the
//    scheme's zero halo for the second step;
//  - sources inside region E are added into the shared u^{n+1} plane before
//    the second step reads it; the nodes the unit owns get both levels'
//    injections in global memory at the unit's tail, where the receivers are
//    also sampled from u^{n-1} and u^n (neither is written during the pass).
// Consumer warps meet at a named barrier after each plane; every mbarrier
// wait is bounded, and a wait that gives up is reported at the next barrier.
#include "fdw_internal.h"
#include "fdw_step.cuh"
#include "fdw_tb.h"

namespace fdw {

// The three-level update divided by m; `l` is dt^2 L u without its centre term.
__device__ __forceinline__ float tb_update(float c, float l, float prev, float s, float e,
                                           float csum) {
  const float lap = fmaf(csum, c, l);
  const float es = e * s;
  const float num = fmaf(es, prev, fmaf(s, lap, 2.f * c) - prev);
  return __fdividef(num, 1.f + es);
}

// dt^2 q / (m + eta dt/2) at node nd for the wavelet row `row` (s = 1/m).
__device__ __forceinline__ float tb_delta(const TbShot* d, const InjNode& nd,
                                          const InjTerm* terms, int row, float dt2) {
  const float* A = d->q + (long long)row * d->q_ld;
  float sum = 0.f;
  for (int t = nd.tbeg; t < nd.tend; ++t) {
    const InjTerm tm = terms[t];
    sum = fmaf(tm.w, A[tm.j], sum);
  }
  const long long off = ((long long)nd.x * d->ny + nd.y) * d->nzp + nd.z;
  const float s = load_m(d->m, d->mtype, off);
  const float e = d->eta[nd.x] + d->eta[d->nx + nd.y] + d->eta[d->nx + d->ny + nd.z];
  return dt2 * sum * s / (1.f + e * s);
}

// Barrier of the NCT consumer threads (named barrier 1; the producer warp
// never takes part) that also ORs a failure flag over them, so that after a
// wait that gave up every consumer leaves at the same barrier.  Like bar.sync
// it orders the threads' shared-memory accesses across the barrier.
template <int NCT>
__device__ __forceinline__ bool tb_sync_any(bool fail) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)fail), "n"(NCT)
      : "memory");
  return r != 0;
}

template <int R, int EY, typename MT>
__device__ __forceinline__ bool tb_unit(const TbParams& P, const Unit& un, const TbShot* d, int u,
                                        const unsigned char* smem, float* u1, uint32_t full0,
                                        uint32_t empty0, Cursor& ca, Cursor& cb,
                                        volatile int* abort_flag, int lane, int tid) {
  constexpr int TY = EY - 2 * R;
  constexpr int U1 = 2 * R + 2;      // planes of u^{n+1} kept in shared memory
  constexpr int Q = 2 * R + 1;       // x queue length
  constexpr int EPL = EY * kTbEZ;    // floats of one region-E plane
  constexpr int NCT = EY * 16;       // consumer threads
  // second-step threads: one output quad each, 16 threads per output row (the
  // last 16 - kTbQ of them idle), so that the eight threads of a 16-byte
  // shared-memory access phase read eight consecutive quads of one row: no
  // bank conflicts whatever the row pitch (with rows of kTbQ threads back to
  // back, a phase straddled two rows whose pitches map to the same banks)
  constexpr int NT2 = TY * 16;
  static_assert(NT2 <= NCT, "second-step threads");
  constexpr bool F32 = sizeof(MT) == 4;
  const int S = P.stages;
  const int nx = d->nx, ny = d->ny, nz = d->nz, nzp = d->nzp;
  const float* eta = d->eta;
  const long long plane = (long long)ny * nzp;

  // first step: the thread's quad of region E
  const int ry = tid >> 4, qz = tid & 15;
  const int y = un.y0 - R + ry;
  const int zq = un.z0 - 4 + 4 * qz;
  const bool yin = y >= 0 && y < ny;
  const bool own = ry >= R && ry < R + TY && qz >= 1 && qz <= kTbQ && yin && zq < nz;
  bool zin[4];
  float eyz[4];
  {
    const float ey = yin ? eta[nx + y] : 0.f;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int zz = zq + v;
      zin[v] = zz >= 0 && zz < nz;
      eyz[v] = ey + (zin[v] ? eta[nx + ny + zz] : 0.f);
    }
  }
  const long long rowoff = own ? (long long)y * nzp + zq : 0;
  const int hoff = (ry + R) * kTbHZ + 4 + 4 * qz;  // the quad in the halo box
  const int eoff = ry * kTbEZ + 4 * qz;            // the quad in a region-E plane
  const int soff = F32 ? eoff : ry * kTbHZ + 4 + 4 * qz;

  // second step: output quad (ty, tq) of the tile, threads below NT2
  const int ty = tid >> 4, tq = tid & 15;
  const bool two = tid < NT2 && tq < kTbQ;
  const int y2 = un.y0 + ty, z2 = un.z0 + 4 * tq;
  const bool own2 = two && y2 < ny && z2 < nz;
  bool zin2[4];
  float eyz2[4];
  {
    const float ey = own2 ? eta[nx + y2] : 0.f;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      zin2[v] = z2 + v < nz;
      eyz2[v] = ey + ((own2 && zin2[v]) ? eta[nx + ny + z2 + v] : 0.f);
    }
  }
  const long long rowoff2 = own2 ? (long long)y2 * nzp + z2 : 0;
  const int eoff2 = (ty + R) * kTbEZ + 4 + 4 * tq;   // the output quad in a region-E plane
  const int hoff2 = (ty + 2 * R) * kTbHZ + 8 + 4 * tq;  // ... in the halo box
  const int soff2 = F32 ? eoff2 : (ty + R) * kTbHZ + 8 + 4 * tq;
  float* C = d->u + (long long)P.out1 * d->uslot;
  float* D = d->u + (long long)P.out2 * d->uslot;

  float qn[4][Q];   // u^n at planes p - r .. p + r of the first-step quad
  float qe[R + 1];  // x part of the damping at planes p - r .. p
#pragma unroll
  for (int i = 0; i <= R; ++i) qe[i] = 0.f;

  // warm-up: planes x0 - 2r .. x0 - 1 enter the queue; the first r of them
  // are needed for nothing else.  A wait that gives up marks the thread bad;
  // it carries on (reading stale but in-bounds shared memory) to the next
  // consumer barrier, where all consumers leave together.
  bool bad = false;
#pragma unroll
  for (int i = 0; i < 2 * R; ++i) {
    if (!bad) bad = !wait_or_abort(full0 + 8 * ca.stage, ca.phase, abort_flag);
    const float* H = reinterpret_cast<const float*>(smem + ca.stage * P.stage_bytes);
    const float4 cv = lds4(H + hoff);
#pragma unroll
    for (int v = 0; v < 4; ++v) qn[v][i] = pick(cv, v);
    if (i < R) release_stage(empty0 + 8 * ca.stage, lane);
    ca.next(S);
  }
  cb.skip(R, S);
  // the second step's plane x: its stage is held from the first step at x
  // until the second step at x has read u^n and s there
  Cursor cc = cb;
  cc.skip(R, S);

  float ex_next = (un.x0 - R >= 0 && un.x0 - R < nx) ? eta[un.x0 - R] : 0.f;
  int ei = P.ext_ptr[u];
  const int ee = P.ext_ptr[u + 1];
  const bool inj = (P.flags & kInject) != 0;
  int wslot = 0;  // ring slot of the first step's plane p (plane x0 - r in slot 0)
#pragma unroll 1
  for (int p = un.x0 - R; p < un.x1 + R; ++p, wslot = (wslot + 1 == U1 ? 0 : wslot + 1)) {
    const int x = p - R;  // plane of the second step
    const bool step2 = x >= un.x0;
    // centre values of plane p + r join the queue
    if (!bad) bad = !wait_or_abort(full0 + 8 * ca.stage, ca.phase, abort_flag);
    {
      const float* H = reinterpret_cast<const float*>(smem + ca.stage * P.stage_bytes);
      const float4 cv = lds4(H + hoff);
#pragma unroll
      for (int v = 0; v < 4; ++v) qn[v][2 * R] = pick(cv, v);
    }
    const int ahead_stage = ca.stage;
    ca.next(S);

    // ---- first step: u^{n+1} at plane p on region E ----
    float v1[4];
    {
      const unsigned char* sb = smem + cb.stage * P.stage_bytes;
      const float* H = reinterpret_cast<const float*>(sb);
      float4 ym[R], yp[R];
#pragma unroll
      for (int k = 1; k <= R; ++k) {
        ym[k - 1] = lds4(H + hoff - k * kTbHZ);
        yp[k - 1] = lds4(H + hoff + k * kTbHZ);
      }
      float wz[12];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float4 w4 = lds4(H + hoff - 4 + 4 * i);
        wz[4 * i] = w4.x;
        wz[4 * i + 1] = w4.y;
        wz[4 * i + 2] = w4.z;
        wz[4 * i + 3] = w4.w;
      }
      const float4 pv = lds4(reinterpret_cast<const float*>(sb + P.off_p) + eoff);
      const float4 sv = load_quad<MT>(sb + P.off_s, soff);
      const bool pin = p >= 0 && p < nx;
      const float ex = ex_next;
      ex_next = (p + 1 >= 0 && p + 1 < nx) ? eta[p + 1] : 0.f;
      qe[R] = ex;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const float c = qn[v][R];
        float lx = 0.f, ly = 0.f, lz = 0.f;
#pragma unroll
        for (int k = 1; k <= R; ++k) {
          lx = fmaf(P.w[0][k], qn[v][R - k] + qn[v][R + k], lx);
          ly = fmaf(P.w[1][k], pick(ym[k - 1], v) + pick(yp[k - 1], v), ly);
          lz = fmaf(P.w[2][k], wz[4 + v - k] + wz[4 + v + k], lz);
        }
        const float val = tb_update(c, lx + ly + lz, pick(pv, v), pick(sv, v), ex + eyz[v],
                                    P.csum);
        v1[v] = (pin && yin && zin[v]) ? val : 0.f;
      }
    }
    // plane p's stage is done unless the second step comes back to it; so is
    // a look-ahead plane past the chunk, whose centre values are in the queue
    if (p < un.x0 || p >= un.x1) release_stage(empty0 + 8 * cb.stage, lane);
    if (p >= un.x1) release_stage(empty0 + 8 * ahead_stage, lane);
    cb.next(S);
    float* W = u1 + wslot * EPL;
    *reinterpret_cast<float4*>(W + eoff) = make_float4(v1[0], v1[1], v1[2], v1[3]);
    if (own && p >= un.x0 && p < un.x1)
      *reinterpret_cast<float4*>(C + (long long)p * plane + rowoff) =
          make_float4(v1[0], v1[1], v1[2], v1[3]);
    if (tb_sync_any<NCT>(bad)) return false;

    // sources inside region E at plane p: into the shared plane of u^{n+1}
    if (inj && ei < ee && P.ext_nodes[ei].x == p) {
      int ej = ei;
      while (ej < ee && P.ext_nodes[ej].x == p) ++ej;
      for (int i = ei + tid; i < ej; i += NCT) {
        const InjNode nd = P.ext_nodes[i];
        W[(nd.y - (un.y0 - R)) * kTbEZ + nd.z - (un.z0 - 4)] +=
            tb_delta(d, nd, P.ext_terms, P.row1, P.dt2);
      }
      ei = ej;
      if (tb_sync_any<NCT>(false)) return false;
    }

    // ---- second step: u^{n+2} at plane x = p - r on the output tile ----
    if (step2 && two) {
      // ring slots of planes x - r .. x + r (x + r = p)
      int sl[2 * R + 1];
#pragma unroll
      for (int k = 0; k <= 2 * R; ++k) {
        const int t = wslot - 2 * R + k;
        sl[k] = t < 0 ? t + U1 : t;
      }
      const float* V = u1 + sl[R] * EPL;
      const unsigned char* sb = smem + cc.stage * P.stage_bytes;
      const float4 c2 = lds4(reinterpret_cast<const float*>(sb) + hoff2);  // u^n
      const float4 s2 = load_quad<MT>(sb + P.off_s, soff2);
      float4 xm[R], xp[R], ym[R], yp[R];
#pragma unroll
      for (int k = 1; k <= R; ++k) {
        xm[k - 1] = lds4(u1 + sl[R - k] * EPL + eoff2);
        xp[k - 1] = lds4(u1 + sl[R + k] * EPL + eoff2);
        ym[k - 1] = lds4(V + eoff2 - k * kTbEZ);
        yp[k - 1] = lds4(V + eoff2 + k * kTbEZ);
      }
      float wz[12];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float4 w4 = lds4(V + eoff2 - 4 + 4 * i);
        wz[4 * i] = w4.x;
        wz[4 * i + 1] = w4.y;
        wz[4 * i + 2] = w4.z;
        wz[4 * i + 3] = w4.w;
      }
      const float ex = qe[0];
      float v2[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const float c = wz[4 + v];
        float lx = 0.f, ly = 0.f, lz = 0.f;
#pragma unroll
        for (int k = 1; k <= R; ++k) {
          lx = fmaf(P.w[0][k], pick(xm[k - 1], v) + pick(xp[k - 1], v), lx);
          ly = fmaf(P.w[1][k], pick(ym[k - 1], v) + pick(yp[k - 1], v), ly);
          lz = fmaf(P.w[2][k], wz[4 + v - k] + wz[4 + v + k], lz);
        }
        const float val = tb_update(c, lx + ly + lz, pick(c2, v), pick(s2, v), ex + eyz2[v],
                                    P.csum);
        v2[v] = zin2[v] ? val : 0.f;
      }
      if (own2)
        *reinterpret_cast<float4*>(D + (long long)x * plane + rowoff2) =
            make_float4(v2[0], v2[1], v2[2], v2[3]);
    }
    if (step2) {  // every consumer warp hands plane x's stage back
      release_stage(empty0 + 8 * cc.stage, lane);
      cc.next(S);
    }

#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int i = 0; i < 2 * R; ++i) qn[v][i] = qn[v][i + 1];
#pragma unroll
    for (int i = 0; i < R; ++i) qe[i] = qe[i + 1];
  }
  cb.skip(R, S);
  return true;
}

template <int R, int EY>
__global__ void __launch_bounds__(EY * 16 + 32, EY <= 18 ? 2 : 1) tb_kernel(const __grid_constant__ TbParams P) {
  constexpr int NC = EY / 2;  // consumer warps, two rows of region E each
  constexpr int NCT = NC * 32;
  constexpr int HY = EY + 2 * R;
  constexpr int U1 = 2 * R + 2;
  constexpr int EPL = EY * kTbEZ;

  extern __shared__ unsigned char smem_raw[];
  __shared__ int s_abort;
  __shared__ int s_issued;
  __shared__ Unit s_unit[kMaxStages];
  __shared__ int s_uidx[kMaxStages];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const int S = P.stages;
  float* u1 = reinterpret_cast<float*>(smem + S * P.stage_bytes);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * P.stage_bytes + U1 * EPL * 4);
  const uint32_t full0 = smem_u32(bars);
  const uint32_t empty0 = smem_u32(bars + S);
  volatile int* abort_flag = &s_abort;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, NC);
    }
    s_abort = 0;
    s_issued = 0;
    fence_barrier_init();
  }
  __syncthreads();

  if (warp == NC) {
    // ------------------------------ producer ------------------------------
    if (lane == 0) {
      Cursor c{0, 0u};
      int issued = 0;
      const uint32_t bytes_h = HY * kTbHZ * 4;
      auto grab = [&](int after) {
        return P.ticket ? atomicAdd(P.ticket, 1) : after + (int)gridDim.x;
      };
      int u = P.ticket ? atomicAdd(P.ticket, 1) : (int)blockIdx.x;
      bool failed = false;
      while (u < P.nunits && !failed) {
        const Unit un = P.units[u];
        const TbShot* d = P.shots + un.shot;
        const bool f32 = d->mtype == kF32;
        const uint32_t bytes_e = EY * kTbEZ * 4 + (f32 ? EY * kTbEZ * 4 : EY * kTbHZ * 2);
        int next = P.nunits;
        for (int q = un.x0 - 2 * R; q < un.x1 + 2 * R; ++q) {
          const uint32_t full = full0 + 8 * c.stage, empty = empty0 + 8 * c.stage;
          if (issued >= S && !wait_or_abort(empty, c.phase ^ 1u, abort_flag)) {
            atomicOr(P.err, kErrTimeoutEmpty);
            *abort_flag = 1;
            failed = true;
            break;
          }
          if (q == un.x0 - 2 * R) {
            s_unit[c.stage] = un;
            s_uidx[c.stage] = u;
          }
          if (q == un.x1 + 2 * R - 1) next = grab(u);
          const bool first = q >= un.x0 - R && q < un.x1 + R;  // a first-step plane
          mbar_arrive_expect_tx(full, bytes_h + (first ? bytes_e : 0u));
          const uint32_t sb = smem_u32(smem + c.stage * P.stage_bytes);
          tma_load_4d(sb, &d->tm_uh, un.z0 - 8, un.y0 - 2 * R, q, P.cur, full);
          if (first) {
            tma_load_4d(sb + P.off_p, &d->tm_ue, un.z0 - 4, un.y0 - R, q, P.prev, full);
            tma_load_3d(sb + P.off_s, &d->tm_s, un.z0 - (f32 ? 4 : 8), un.y0 - R, q, full);
          }
          ++issued;
          c.next(S);
        }
        u = next;
      }
      if (!failed) {  // end marker: a stage with no data and unit index -1
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
    }
  } else {
    // ------------------------------ consumers -----------------------------
    const int tid = threadIdx.x;
    Cursor ca{0, 0u};  // read-ahead cursor: every plane of u^n in order
    Cursor cb{0, 0u};  // the first step's plane
    bool ok = true;
    while (true) {
      // the stage of the next unit's first plane names the unit
      const bool bad = !wait_or_abort(full0 + 8 * ca.stage, ca.phase, abort_flag);
      if (tb_sync_any<NCT>(bad)) {
        ok = false;
        break;
      }
      const int u = s_uidx[ca.stage];
      if (u < 0) break;
      const Unit un = s_unit[ca.stage];
      const TbShot* d = P.shots + un.shot;
      if (d->mtype == kF16)
        ok = tb_unit<R, EY, __half>(P, un, d, u, smem, u1, full0, empty0, ca, cb, abort_flag,
                                    lane, tid);
      else if (d->mtype == kBF16)
        ok = tb_unit<R, EY, __nv_bfloat16>(P, un, d, u, smem, u1, full0, empty0, ca, cb,
                                           abort_flag, lane, tid);
      else
        ok = tb_unit<R, EY, float>(P, un, d, u, smem, u1, full0, empty0, ca, cb, abort_flag,
                                   lane, tid);
      if (!ok) break;

      // ---- unit tail: every store of the unit is done ----
      if (tb_sync_any<NCT>(false)) {
        ok = false;
        break;
      }
      const int ny = d->ny, nzp = d->nzp;
      if (P.flags & kInject) {
        float* C = d->u + (long long)P.out1 * d->uslot;
        float* Dn = d->u + (long long)P.out2 * d->uslot;
        for (int i = P.inj_ptr[u] + tid; i < P.inj_ptr[u + 1]; i += NCT) {
          const InjNode nd = P.inj_nodes[i];
          const long long off = ((long long)nd.x * ny + nd.y) * nzp + nd.z;
          const float d1 = tb_delta(d, nd, P.inj_terms, P.row1, P.dt2);
          const float d2 = tb_delta(d, nd, P.inj_terms, P.row2, P.dt2);
          C[off] = C[off] + d1;
          Dn[off] = Dn[off] + d2;
        }
      }
      if (P.flags & kSample) {
        for (int i = P.smp_ptr[u] + tid; i < P.smp_ptr[u + 1]; i += NCT) {
          const int j = P.smp_pts[i];
          const int bx = d->pt_base[3 * j], by = d->pt_base[3 * j + 1], bz = d->pt_base[3 * j + 2];
          const float* w = d->pt_w + 8 * j;
#pragma unroll
          for (int lev = 0; lev < 2; ++lev) {
            const int row = lev == 0 ? P.srow_prev : P.srow_cur;
            if (row < 0) continue;
            const float* uc = d->u + (long long)(lev == 0 ? P.prev : P.cur) * d->uslot;
            float acc = 0.f;
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) {
              const float wc = w[cc];
              if (wc != 0.f) {
                const long long off = ((long long)(bx + ((cc >> 2) & 1)) * ny +
                                       (by + ((cc >> 1) & 1))) * nzp + bz + (cc & 1);
                acc = fmaf(wc, uc[off], acc);
              }
            }
            d->rec[(long long)row * d->rec_ld + j] = acc;
          }
        }
      }
    }
    if (!ok) {
      atomicOr(P.err, kErrTimeoutFull);
      *abort_flag = 1;
    }
  }
  __syncthreads();
  // On an aborted launch, wait (bounded) for the loads still in flight before
  // the CTA's shared memory is released.
  if (*abort_flag && threadIdx.x == NCT) {
    const int issued = s_issued;
    for (int k = (issued > S ? issued - S : 0); k < issued; ++k) {
      const int st = k % S;
      const uint32_t ph = (uint32_t)((k / S) & 1);
      long long t0 = clock64();
      while (!mbar_try_wait(full0 + 8 * st, ph) && clock64() - t0 < kWaitBudget) {
      }
    }
  }
}

const void* tb_kernel_fn(int r, int variant) {
  switch (r * 2 + variant) {
    case 2: return (const void*)&tb_kernel<1, tb_ey(1, 0)>;
    case 3: return (const void*)&tb_kernel<1, tb_ey(1, 1)>;
    case 4: return (const void*)&tb_kernel<2, tb_ey(2, 0)>;
    case 5: return (const void*)&tb_kernel<2, tb_ey(2, 1)>;
    default: return nullptr;
  }
}

}  // namespace fdw
