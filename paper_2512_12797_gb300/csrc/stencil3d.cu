// stencil3d.cu -- 3D time-step kernels (forward recursion; adjoint recursion
// with the imaging condition), same algebra as the 2D kernels in stencil.cu:
//     p^{n+1} = p^n + b (p^n - p^{n-1}) + cc (L p^n + s^n),  L = sum_a sum_k a_k/h_a^2 [(p_{+k} + p_{-k}) - 2p]
//     q^k     = q^{k+1} + b (q^{k+1} - q^{k+2}) + cc (L q^{k+1} + R^T rhat^{k-1}),  G += q^k L p^{k-1}
// (cc = v^2 dt^2/(1 + gamma dt) comes from the expanded array, b = (1 - gamma dt)/(1 + gamma dt)
// from the per-axis gamma*dt table).
//
// 2.5D blocking: a CTA owns a 64 (x) x 16 (y) column of one wavefield and
// marches through z; each thread owns 4 consecutive x points of one y row (a
// warp covers two rows, one per half-warp) and keeps the 9 z-levels its
// z-derivative needs in a circular register queue (the level loop is unrolled
// by 9 so the queue never moves).  64 x 16 rather than 128 x 8: the padded x
// extents of the 3D grids (e.g. 296) leave less of a last x-tile idle, and the
// halo plane is 1.7 rather than 2.1 times the tile.  Ring
// sequence q carries the x-y halo plane (72 x 24) of level q-4 -- whose
// centre enters the queue at q and whose x-y neighbours serve level q-4 at
// q+4 -- and the plain planes (64 x 16) of level q-8: p^{n-1}, cc and, in the
// adjoint, the imaging accumulator; the adjoint also streams halo planes of
// the snapshot p^{k-1} with its own register queue for L p^{k-1}.  Level
// z = q - 8 is computed once sequence q has landed.  Every warp releases the
// slot of sequence q-4 after computing level q-8 (per-warp "empty" mbarrier
// arrivals).  The CTA is warp-specialised: warps 0-7 compute (two y rows each),
// and lane 0 of warp 8 (a producer warpgroup that setmaxnreg shrinks) refills
// the ring in sequence order, waiting on each slot's "empty" barrier, so that
// no consumer warp carries the refill work.
//
// Pair tiles (PAIR): a CTA runs two wavefields of one sample (supergathers
// 2i and 2i+1) over a 64 x 8 column each: warps 0-3 the first, warps 4-7 the
// second, two rows per warp as above.  The cc plane is loaded once for both,
// and in the adjoint the two supergathers' imaging terms meet in shared
// memory (the second wavefield's warp hands its q L p to the first's, through
// a two-buffer exchange guarded by mbarriers) and go into one accumulator per
// pair: G += q_a L p_a + q_b L p_b.  The forward's arithmetic per point is
// the same in both tile forms, so the autotuner may pick either; the
// adjoint's accumulator sums in another order than the per-wavefield form, so
// the pair adjoint is never chosen by timing: it runs only when a forced
// variant selects it.
#include "fwi_internal.cuh"

namespace fwi {

constexpr int NCW3 = TY3 / 2;        // consumer warps (two y rows each)
constexpr int NTHREADS3 = 32 * NCW3 + 128;  // + producer warpgroup
constexpr int REG3_LAUNCH = 168, REG3_PRODUCER = 72, REG3_CONSUMER = 216;
constexpr int WDONE3 = 8;            // column-completion counters (ring), multi-step launches
static_assert(128 * REG3_PRODUCER + 32 * NCW3 * REG3_CONSUMER <= NTHREADS3 * REG3_LAUNCH,
              "register split exceeds the launch allocation");

// One ring stage: per wavefield the halo plane of the stepped level (and of
// the snapshot), per wavefield the plain plane of the older level, then the
// shared cc plane and (adjoint) the accumulator plane.  Every part starts on
// a 128-byte boundary.
template <bool ADJ, bool PAIR>
struct Smem3D {
  static constexpr int NWF = PAIR ? 2 : 1;    // wavefields per CTA
  static constexpr int TYW = TY3 / NWF;       // rows of a wavefield's tile (16 or 8)
  static constexpr int HYW = TYW + 2 * HALO;
  static constexpr int PLANE = HYW * HX3;     // floats in one wavefield's halo plane
  static constexpr int PPLANE = TYW * TX3;    // floats in one wavefield's plain plane
  static constexpr int NST = ADJ ? 8 : 10;    // ring slots
  static constexpr int OFF_SNAP = NWF * PLANE;
  static constexpr int OFF_PREV = NWF * PLANE * (ADJ ? 2 : 1);
  static constexpr int OFF_CC = OFF_PREV + NWF * PPLANE;
  static constexpr int OFF_G = OFF_CC + PPLANE;
  static constexpr int STAGE = OFF_G + (ADJ ? PPLANE : 0);
  static constexpr int OFF_X = NST * STAGE;   // pair exchange of the adjoint: 2 buffers of one plane
  static constexpr int OFF_GZ = OFF_X + (ADJ && PAIR ? 2 * PPLANE : 0);  // gamma*dt of every z level
  static constexpr int NXB = ADJ && PAIR ? 16 : 0;  // exchange barriers: full[4][2], empty[4][2]
  static size_t bytes(int nzp) {
    // + abort word, dependency counter, column-completion counters
    return ((size_t)OFF_GZ + ((nzp + 31) / 32) * 32) * 4 + (2 * NST + NXB) * 8 + (2 + WDONE3) * 4 + 8;
  }
  static_assert((PLANE * 4) % 128 == 0 && (PPLANE * 4) % 128 == 0 && (STAGE * 4) % 128 == 0,
                "stage parts must stay 128-byte aligned");
};

__device__ __forceinline__ float4 ld4s(const float* p) { return *reinterpret_cast<const float4*>(p); }

__device__ __forceinline__ float comp(const float4& v, int j) {
  return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 half2of(const float4& v, int j) { return j == 0 ? f2(v.x, v.y) : f2(v.z, v.w); }

// Laplacian of the thread's 4 points: x and y neighbours from the halo plane H
// (row ly+4, columns lx..lx+11, row stride HX3), z neighbours from the circular register queue
// Q of NQ levels (Q[(C+k) % NQ] holds level z+k, k = -4..4, C the index of the centre).
// Adjacent columns are computed as pairs with the packed FP32 instructions;
// each point sees the operations of the scalar form in the same order
// (x - y as fma(y, -1, x), exact).  ISO (hx == hy == hz): the axes share
// coefficients and each k costs one bracket
//   [(x_{+k} + x_{-k}) + (y_{+k} + y_{-k}) - 4p] + [(z_{+k} + z_{-k}) - 2p],
// which is still exactly zero on a constant field, so the chain of
// coefficient FMAs is 4 long instead of 12.
template <int C, bool ISO, int NQ>
__device__ __forceinline__ void lap3(const float* __restrict__ H, const float4 (&Q)[NQ], int ly, int lx,
                                     const Coef& K, float (&lap)[4]) {
  const float* row = H + (ly + HALO) * HX3;
  const float4 xl = ld4s(row + lx), xr = ld4s(row + lx + 8);
  const float4 ce = Q[C % NQ];
  const float w[12] = {xl.x, xl.y, xl.z, xl.w, ce.x, ce.y, ce.z, ce.w, xr.x, xr.y, xr.z, xr.w};
  float4 yn[8];
#pragma unroll
  for (int k = 1; k <= 4; k++) {
    yn[k - 1] = ld4s(H + (ly + HALO - k) * HX3 + lx + 4);
    yn[k + 3] = ld4s(H + (ly + HALO + k) * HX3 + lx + 4);
  }
  const float2 m1 = f2(-1.f, -1.f);
#pragma unroll
  for (int j = 0; j < 4; j += 2) {
    const float2 p = f2(w[4 + j], w[5 + j]);
    const float2 p2 = __fadd2_rn(p, p);
    // odd k straddles the float4 quads: two scalar adds whose results land in a pair
    auto xs = [&](int k) {
      return (k & 1) ? f2(w[4 + j + k] + w[4 + j - k], w[5 + j + k] + w[5 + j - k])
                     : __fadd2_rn(f2(w[4 + j + k], w[5 + j + k]), f2(w[4 + j - k], w[5 + j - k]));
    };
    auto ys = [&](int k) { return __fadd2_rn(half2of(yn[k + 3], j), half2of(yn[k - 1], j)); };
    auto zs = [&](int k) { return __fadd2_rn(half2of(Q[(C + k) % NQ], j), half2of(Q[(C + NQ - k) % NQ], j)); };
    if (ISO) {
      const float2 m4 = f2(-4.f, -4.f);
      auto br = [&](int k) {
        return __fadd2_rn(__ffma2_rn(m4, p, __fadd2_rn(xs(k), ys(k))), __ffma2_rn(p2, m1, zs(k)));
      };
      float2 a = __fmul2_rn(f2(K.cx[4], K.cx[4]), br(4));
      a = __ffma2_rn(f2(K.cx[3], K.cx[3]), br(3), a);
      a = __ffma2_rn(f2(K.cx[2], K.cx[2]), br(2), a);
      a = __ffma2_rn(f2(K.cx[1], K.cx[1]), br(1), a);
      lap[j] = a.x;
      lap[j + 1] = a.y;
      continue;
    }
    float2 a = __fmul2_rn(f2(K.cx[4], K.cx[4]), __ffma2_rn(p2, m1, xs(4)));
    a = __ffma2_rn(f2(K.cx[3], K.cx[3]), __ffma2_rn(p2, m1, xs(3)), a);
    a = __ffma2_rn(f2(K.cx[2], K.cx[2]), __ffma2_rn(p2, m1, xs(2)), a);
    a = __ffma2_rn(f2(K.cx[1], K.cx[1]), __ffma2_rn(p2, m1, xs(1)), a);
    a = __ffma2_rn(f2(K.cy[4], K.cy[4]), __ffma2_rn(p2, m1, ys(4)), a);
    a = __ffma2_rn(f2(K.cy[3], K.cy[3]), __ffma2_rn(p2, m1, ys(3)), a);
    a = __ffma2_rn(f2(K.cy[2], K.cy[2]), __ffma2_rn(p2, m1, ys(2)), a);
    a = __ffma2_rn(f2(K.cy[1], K.cy[1]), __ffma2_rn(p2, m1, ys(1)), a);
    a = __ffma2_rn(f2(K.cz[4], K.cz[4]), __ffma2_rn(p2, m1, zs(4)), a);
    a = __ffma2_rn(f2(K.cz[3], K.cz[3]), __ffma2_rn(p2, m1, zs(3)), a);
    a = __ffma2_rn(f2(K.cz[2], K.cz[2]), __ffma2_rn(p2, m1, zs(2)), a);
    a = __ffma2_rn(f2(K.cz[1], K.cz[1]), __ffma2_rn(p2, m1, zs(1)), a);
    lap[j] = a.x;
    lap[j + 1] = a.y;
  }
}

// Column `it` of a launch -> (unit, tile) in the CTA order P.order3 picks:
// tile-major order runs all tiles of a unit back to back; wavefield-fastest
// order runs the tile of every unit side by side.
__device__ __forceinline__ void column_of(const StepParams& P, int it, int nunits, int& u, int& tile) {
  u = P.order3 ? it % nunits : it / P.ntiles;
  tile = P.order3 ? it / nunits : it % P.ntiles;
}

// Multi-step launches: bounded poll of the progress flags of the 3 x 3 tile
// neighbourhood of column (u, tile) until each has completed `need` steps,
// then acquire-orders the neighbours' stores before the TMA loads that
// follow.  Gives up on timeout, on the CTA's abort word, or when another CTA
// has recorded an error.
// (The fields of the launch's StepParams come by value: a reference to the
// kernel parameter would give every thread a local copy of it.)
__device__ __noinline__ bool wait_columns3(const int* done, int ntx, int ntiles, int* status, int u, int tile,
                                           int need, volatile int* abort_flag) {
  const int tx = tile % ntx, ty = tile / ntx, nty = ntiles / ntx;
  const int* base = done + (long long)u * ntiles;
  const int y_lo = max(ty - 1, 0), y_hi = min(ty + 1, nty - 1);
  const int x_lo = max(tx - 1, 0), x_hi = min(tx + 1, ntx - 1);
  const long long t0 = clock64();
  for (;;) {
    int lo = need;
    for (int y = y_lo; y <= y_hi; y++)
      for (int x = x_lo; x <= x_hi; x++) lo = min(lo, ld_relaxed_gpu(base + y * ntx + x));
    if (lo >= need) break;
    if (*abort_flag || ld_relaxed_gpu(status) != 0) {
      *abort_flag = 1;
      return false;
    }
    if (clock64() - t0 > WAIT_CYCLES) {
      atomicCAS(status, 0, (int)FWI_ERR_TIMEOUT);
      *abort_flag = 1;
      return false;
    }
    __nanosleep(128);
  }
  fence_acq_rel_gpu();
  fence_proxy_async_global();
  return true;
}

// Bounded wait until the shared counter *c exceeds v (acquire at CTA scope).
__device__ __forceinline__ bool wait_counter(const int* c, int v, int* status, volatile int* abort_flag) {
  const long long t0 = clock64();
  while (ld_acquire_cta_shared(c) <= v) {
    if (*abort_flag) return false;
    if (clock64() - t0 > WAIT_CYCLES) {
      atomicCAS(status, 0, (int)FWI_ERR_TIMEOUT);
      *abort_flag = 1;
      return false;
    }
    __nanosleep(32);
  }
  return true;
}

// The Laplacian of the snapshot for the imaging condition, in the plain form
// c0 p + sum_a sum_k c_{a,k} (p_{+k} + p_{-k}): it enters the gradient, not
// the recursion, so it needs neither the bracket form's exact zero on a
// constant field nor its 2p subtractions (the 2D adjoint does the same).
// Operand loads as lap3.
template <int C, int NQ>
__device__ __forceinline__ void lap3_img(const float* __restrict__ H, const float4 (&Q)[NQ], int ly, int lx,
                                         const Coef& K, float (&lap)[4]) {
  const float* row = H + (ly + HALO) * HX3;
  const float4 xl = ld4s(row + lx), xr = ld4s(row + lx + 8);
  const float4 ce = Q[C % NQ];
  const float w[12] = {xl.x, xl.y, xl.z, xl.w, ce.x, ce.y, ce.z, ce.w, xr.x, xr.y, xr.z, xr.w};
  float4 yn[8];
#pragma unroll
  for (int k = 1; k <= 4; k++) {
    yn[k - 1] = ld4s(H + (ly + HALO - k) * HX3 + lx + 4);
    yn[k + 3] = ld4s(H + (ly + HALO + k) * HX3 + lx + 4);
  }
#pragma unroll
  for (int j = 0; j < 4; j += 2) {
    const float2 p = f2(w[4 + j], w[5 + j]);
    auto xs = [&](int k) {
      return (k & 1) ? f2(w[4 + j + k] + w[4 + j - k], w[5 + j + k] + w[5 + j - k])
                     : __fadd2_rn(f2(w[4 + j + k], w[5 + j + k]), f2(w[4 + j - k], w[5 + j - k]));
    };
    auto ys = [&](int k) { return __fadd2_rn(half2of(yn[k + 3], j), half2of(yn[k - 1], j)); };
    auto zs = [&](int k) { return __fadd2_rn(half2of(Q[(C + k) % NQ], j), half2of(Q[(C + NQ - k) % NQ], j)); };
    float2 a = __fmul2_rn(f2(K.c0_3d, K.c0_3d), p);
#pragma unroll
    for (int k = 4; k >= 1; k--) {
      a = __ffma2_rn(f2(K.cx[k], K.cx[k]), xs(k), a);
      a = __ffma2_rn(f2(K.cy[k], K.cy[k]), ys(k), a);
      a = __ffma2_rn(f2(K.cz[k], K.cz[k]), zs(k), a);
    }
    lap[j] = a.x;
    lap[j + 1] = a.y;
  }
}

template <bool ADJ, bool ISO, int NQ, bool PAIR>
struct March3D {
  using S = Smem3D<ADJ, PAIR>;
  static constexpr int NST = S::NST;
  static constexpr int PLANE = S::PLANE, PPLANE = S::PPLANE;
  const Layout& L;
  const Coef& K;
  const StepParams& P;
  const CUtensorMap* th;
  const CUtensorMap* tp;
  const CUtensorMap* tcc;
  const CUtensorMap* tg;
  float* sm;
  uint64_t* full;
  uint64_t* empty;
  uint64_t* xfull;       // pair exchange (adjoint): [pair of warps][buffer]
  uint64_t* xempty;
  volatile int* abort_flag;
  int lane, ly, lx, x0, y0, gx, gy, b, s, tile, last_q;
  int zc;                // levels computed by this CTA's warps over all its columns (pair exchange buffers)
  bool carry;            // after the first column: the previous column's last 4 slots are still held
  int b0, k;             // first wavefield of the CTA, this warp's wavefield index in it
  int s_cur, s_prev, s_out, s_snap, t;  // slots and record time of the current step
  int xpair;             // pair tiles: index of this warp within its wavefield's group (0-3)
  int acc;               // imaging accumulator of this warp's wavefield (per wavefield or per pair)
  bool colv;
  float gyv, gxv[4];
  const float* gz;       // shared gamma*dt per z level
  int pq, pst;           // producer: next sequence, its slot
  int cslot;             // consumer, landing side: slot of the next sequence to land (running)
  uint32_t cphase;       // consumer: its phase, (q / NST) & 1
  int lslot, hslot;      // consumer, level side: slots of sequences q and q - 4 (running, no division)
  uint32_t pround;
  int ie_cur, ie_end, se_cur, se_end;  // point-list cursors (entries sorted by z)
  int inj_z, smp_z;                    // z of the entries under the cursors (INT_MAX: none left)
  float4 Q[NQ], QS[NQ];
  float4 gpend;          // pair tiles, first wavefield's warps: G + q_a L p_a of the previous level

  // Slots and record time of step n of the launch: from the step table of a
  // multi-step launch, else from P (one step).
  __device__ __forceinline__ void set_step(int n) {
    if (P.steps) {
      const int4 d = __ldg(reinterpret_cast<const int4*>(P.steps + n));
      s_cur = d.x;
      s_prev = d.y;
      s_out = d.z;
      s_snap = d.w;
      t = __ldg(&P.steps[n].t);
    } else {
      s_cur = P.s_cur;
      s_prev = P.s_prev;
      s_out = P.s_out;
      s_snap = P.s_snap;
      t = P.t;
    }
  }

  // Column `it` of the launch (tiles x units).  In wavefield-fastest order
  // the supergathers of a sample read the same cc plane within microseconds
  // of each other (one DRAM read, the others L2 hits).  A unit is one
  // wavefield, or two (pair tiles).
  __device__ __forceinline__ void set_column(int it, int nunits) {
    int u;
    column_of(P, it, nunits, u, tile);
    b0 = u * S::NWF;
    b = b0 + k;
    acc = PAIR ? b0 / 2 : b;
    x0 = (tile % P.ntx) * TX3;
    y0 = (tile / P.ntx) * S::TYW;
    s = b0 / P.nsg;
    gx = x0 + lx;
    gy = y0 + ly;
    colv = gx < L.nxp && gy < L.nyp;
  }

  // Imaging accumulator row of level z (this thread's 4 points).
  __device__ __forceinline__ void store_g(int z, const float4& g) {
    if (!colv) return;
    float* gp = P.grad + (long long)acc * L.field + L.off(z, gy, gx);
    if (gx + 3 < L.nxp) {
      *reinterpret_cast<float4*>(gp) = g;
    } else {
      const float gv[4] = {g.x, g.y, g.z, g.w};
      for (int j = 0; j < 4; j++)
        if (gx + j < L.nxp) gp[j] = gv[j];
    }
  }

  // Pair tiles, first wavefield's warps: adds the second wavefield's q L p of
  // level zp (the CTA's zcp-th computed level: buffer zcp & 1) to gpend and
  // stores the pair's accumulator.
  __device__ __forceinline__ bool pair_finish(int zp, int zcp) {
    const int xb = zcp & 1, use = zcp >> 1, pr = xpair;
    if (!mbar_wait_abortable(&xfull[pr * 2 + xb], (uint32_t)(use & 1), P.status, abort_flag)) return false;
    const float4 cb = ld4s(sm + S::OFF_X + xb * PPLANE + ly * TX3 + lx);
    __syncwarp();
    if (lane == 0) mbar_arrive(&xempty[pr * 2 + xb]);
    const float2 g01 = __fadd2_rn(f2(gpend.x, gpend.y), f2(cb.x, cb.y));
    const float2 g23 = __fadd2_rn(f2(gpend.z, gpend.w), f2(cb.z, cb.w));
    store_g(zp, make_float4(g01.x, g01.y, g23.x, g23.y));
    return true;
  }

  __device__ __forceinline__ void issue() {
    const int zh = pq - HALO, zp = pq - 2 * HALO;
    const bool plain = zp >= 0 && zp < L.nzp;
    float* base = sm + pst * S::STAGE;
    const uint32_t bytes = S::NWF * PLANE * 4 * (ADJ ? 2 : 1) +
                           (plain ? (S::NWF * PPLANE + PPLANE * (ADJ ? 2 : 1)) * 4 : 0);
    mbar_arrive_expect_tx(&full[pst], bytes);
#pragma unroll
    for (int w = 0; w < S::NWF; w++) {
      tma_load_5d(base + w * PLANE, th, x0, y0, zh + HALO, b0 + w, s_cur, &full[pst]);
      if (ADJ) tma_load_5d(base + S::OFF_SNAP + w * PLANE, th, x0, y0, zh + HALO, b0 + w, s_snap, &full[pst]);
    }
    if (plain) {
#pragma unroll
      for (int w = 0; w < S::NWF; w++)
        tma_load_5d(base + S::OFF_PREV + w * PPLANE, tp, x0 + HALO, y0 + HALO, zp + HALO, b0 + w, s_prev,
                    &full[pst]);
      tma_load_4d(base + S::OFF_CC, tcc, x0 + HALO, y0 + HALO, zp + HALO, s, &full[pst]);
      if (ADJ) tma_load_4d(base + S::OFF_G, tg, x0 + HALO, y0 + HALO, zp + HALO, PAIR ? b0 / 2 : b0, &full[pst]);
    }
    pq++;
    if (++pst == NST) { pst = 0; pround ^= 1; }
  }


  // Landing of the next sequence q: waits for its slot and moves the centre
  // of its halo plane (level q - 4) into queue index CI = (q - 4 + 4) % NQ.
  template <int CI>
  __device__ __forceinline__ bool land() {
    if (!mbar_wait_abortable(&full[cslot], cphase, P.status, abort_flag)) return false;
    const float* stage = sm + cslot * S::STAGE + k * PLANE;
    Q[CI] = ld4s(stage + (ly + HALO) * HX3 + lx + HALO);
    if (ADJ) QS[CI] = ld4s(stage + S::OFF_SNAP + (ly + HALO) * HX3 + lx + HALO);
    if (++cslot == NST) {
      cslot = 0;
      cphase ^= 1u;
    }
    return true;
  }

  // p^{n+1} (forward) or q^k (adjoint) at the thread's 4 points of level z,
  // from the halo plane hpl of level z (queue centre at index C) and the
  // plain planes of stage: cc * L p + (p + b (p - pm)).  No side effects.
  template <int C>
  __device__ __forceinline__ void advance(int z, const float* hpl, const float* stage, float (&nv)[4]) const {
    float lap[4];
    lap3<C, ISO, NQ>(hpl, Q, ly, lx, K, lap);
    const float4 pm = ld4s(stage + S::OFF_PREV + k * PPLANE + ly * TX3 + lx);
    const float4 cv = ld4s(stage + S::OFF_CC + ly * TX3 + lx);
    const float gzy = gz[z] + gyv;
#pragma unroll
    for (int j = 0; j < 4; j += 2) {  // in pairs
      const float2 bb = f2(sponge_b(gzy + gxv[j]), sponge_b(gzy + gxv[j + 1]));
      const float2 p = half2of(Q[C % NQ], j);
      const float2 d = __ffma2_rn(half2of(pm, j), f2(-1.f, -1.f), p);
      const float2 n2 = __ffma2_rn(half2of(cv, j), f2(lap[j], lap[j + 1]), __ffma2_rn(bb, d, p));
      nv[j] = n2.x;
      nv[j + 1] = n2.y;
    }
  }

  // Injection / sampling at level z: staged in this warp's two rows of the
  // p^{n-1} plane of stage (already consumed); entry .x is the point's index
  // in that plane, and its row / 2 names the warp that owns it.
  __device__ __forceinline__ void inject(int z, float* stage, float (&nv)[4]) {
    if (inj_z != z && smp_z != z) return;
    float* pl = stage + S::OFF_PREV + k * PPLANE;
    const int wrow = ly >> 1;
    __syncwarp();
    *reinterpret_cast<float4*>(pl + ly * TX3 + lx) = make_float4(nv[0], nv[1], nv[2], nv[3]);
    __syncwarp();
    // The entries of level z are the next ones under each cursor (lists are
    // sorted by z); the warp reads them 32 at a time, and a ballot counts
    // those at level z (a prefix of the 32).  Lane n of the last read holds
    // the next entry, whose level becomes the cursor's.
    while (inj_z == z) {
      const int e = ie_cur + lane;
      int4 en = make_int4(0, 0, 0, 0x7fffffff);
      if (e < ie_end) en = P.inj[e];
      const bool here = en.w == z;
      const int n = __popc(__ballot_sync(0xffffffffu, here));
      // Entries of one list never share a point (fwi_create rejects duplicate
      // receivers, and each wavefield's coincident sources are merged into
      // one entry), so the lanes add to distinct words.
      if (here && (en.x / TX3) >> 1 == wrow) {
        const float ccp = __ldg(P.c + (long long)s * L.field + L.off(z, y0 + en.x / TX3, x0 + en.x % TX3));
        pl[en.x] += ccp * (__int_as_float(en.z) *
                           P.series[(long long)b * P.series_bstride + (long long)t * P.series_ld + en.y]);
      }
      __syncwarp();
      ie_cur += n;
      inj_z = n < 32 ? __shfl_sync(0xffffffffu, en.w, n & 31) : z;
    }
    const float4 v = ld4s(pl + ly * TX3 + lx);
    nv[0] = v.x; nv[1] = v.y; nv[2] = v.z; nv[3] = v.w;
    while (smp_z == z) {
      const int e = se_cur + lane;
      int4 en = make_int4(0, 0, 0x7fffffff, 0);
      if (e < se_end) en = P.smp4[e];
      const bool here = en.z == z;
      const int n = __popc(__ballot_sync(0xffffffffu, here));
      if (here && (en.x / TX3) >> 1 == wrow)
        P.smp_out[(long long)b * P.smp_bstride_out + (long long)t * P.smp_ld + en.y] = pl[en.x];
      se_cur += n;
      smp_z = n < 32 ? __shfl_sync(0xffffffffu, en.z, n & 31) : z;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }

  // The new wavefield's row of level z (this thread's 4 points).
  __device__ __forceinline__ void store_p(int z, const float (&nv)[4]) {
    if (!colv) return;
    float* o = P.pool + (long long)s_out * P.slot_elems + (long long)b * L.field + L.off(z, gy, gx);
    if (gx + 3 < L.nxp) {
      *reinterpret_cast<float4*>(o) = make_float4(nv[0], nv[1], nv[2], nv[3]);
    } else {
      for (int j = 0; j < 4; j++)
        if (gx + j < L.nxp) o[j] = nv[j];
    }
  }

  // Level z = q - 8 from landed sequences q (plain planes) and q - 4 (halo
  // plane), queue centre at compile-time index C = (q - 4) % NQ; then the
  // slot of sequence q - 4 is released.
  template <int C>
  __device__ __forceinline__ bool level(int q) {
    float* stage = sm + lslot * S::STAGE;
    const int z = q - 2 * HALO;
    if (z >= 0) {
      const float* hpl = sm + hslot * S::STAGE + k * PLANE;  // halo plane of level z (sequence q - 4)
      float nv[4];
      advance<C>(z, hpl, stage, nv);
      inject(z, stage, nv);
      if (ADJ) {
        float lps[4];
        lap3_img<C, NQ>(hpl + S::OFF_SNAP, QS, ly, lx, K, lps);
        float4 g = ld4s(stage + S::OFF_G + ly * TX3 + lx);
        if (PAIR) {
          // The second wavefield's warp hands q L p of level z to the first's
          // through buffer zc & 1 (zc counts the CTA's computed levels over
          // all its columns); the first takes it one level later (level z + 1,
          // or the flush after the column's last level), so that neither warp
          // waits for the other's current level: it keeps G + q_a L p_a of
          // level z in registers until then.
          const int pr = xpair;
          if (k == 1) {
            const int xb = zc & 1, use = zc >> 1;
            if (use > 0 && !mbar_wait_abortable(&xempty[pr * 2 + xb], (uint32_t)((use - 1) & 1), P.status,
                                                 abort_flag))
              return false;
            const float2 c01 = __fmul2_rn(f2(nv[0], nv[1]), f2(lps[0], lps[1]));
            const float2 c23 = __fmul2_rn(f2(nv[2], nv[3]), f2(lps[2], lps[3]));
            *reinterpret_cast<float4*>(sm + S::OFF_X + xb * PPLANE + ly * TX3 + lx) =
                make_float4(c01.x, c01.y, c23.x, c23.y);
            __syncwarp();
            if (lane == 0) mbar_arrive(&xfull[pr * 2 + xb]);
          } else {
            if (z > 0 && !pair_finish(z - 1, zc - 1)) return false;
            const float2 g01 = __ffma2_rn(f2(nv[0], nv[1]), f2(lps[0], lps[1]), f2(g.x, g.y));
            const float2 g23 = __ffma2_rn(f2(nv[2], nv[3]), f2(lps[2], lps[3]), f2(g.z, g.w));
            gpend = make_float4(g01.x, g01.y, g23.x, g23.y);
          }
        } else {
          const float2 g01 = __ffma2_rn(f2(nv[0], nv[1]), f2(lps[0], lps[1]), f2(g.x, g.y));
          const float2 g23 = __ffma2_rn(f2(nv[2], nv[3]), f2(lps[2], lps[3]), f2(g.z, g.w));
          store_g(z, make_float4(g01.x, g01.y, g23.x, g23.y));
        }
      }
      store_p(z, nv);
    }
    if (z >= 0) zc++;
    // release the slot of sequence q-4: its halo plane served level q-8 above
    // (on a later column, at q < 4: the previous column's last sequences)
    if (q >= HALO || carry) {
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[hslot]);
    }
    if (++lslot == NST) lslot = 0;
    if (++hslot == NST) hslot = 0;
    return true;
  }

};

template <bool ADJ, bool ISO, int NQ, bool PAIR>
__global__ void __launch_bounds__(NTHREADS3, 1)
step3d_kernel(const __grid_constant__ CUtensorMap tm_halo, const __grid_constant__ CUtensorMap tm_plain,
              const __grid_constant__ CUtensorMap tm_cc, const __grid_constant__ CUtensorMap tm_g, const Layout L,
              const Coef K, const StepParams P) {
  using S = Smem3D<ADJ, PAIR>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  float* gz = sm + S::OFF_GZ;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + (((size_t)S::OFF_GZ + ((L.nzp + 31) / 32) * 32) * 4));
  uint64_t* empty = full + S::NST;
  uint64_t* xfull = empty + S::NST;
  uint64_t* xempty = xfull + S::NXB / 2;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + S::NST + S::NXB);
  int* deps_ok = const_cast<int*>(abort_flag) + 1;  // multi-step: columns whose neighbourhood is ready
  int* wdone = deps_ok + 1;                          // multi-step: consumer warps done with column ic

  const int tid = threadIdx.x, warp = tid >> 5;
  March3D<ADJ, ISO, NQ, PAIR> M{L, K, P, &tm_halo, &tm_plain, &tm_cc, &tm_g, sm, full, empty, xfull, xempty,
                                abort_flag};
  M.lane = tid & 31;
  // warp -> (wavefield of the CTA, rows): one wavefield over 16 rows, or
  // (pair tiles) warps 0-3 and 4-7 over 8 rows of the first and second
  constexpr int WPG = NCW3 / S::NWF;  // consumer warps per wavefield
  M.k = warp < NCW3 ? warp / WPG : 0;
  M.xpair = warp % WPG;
  M.ly = 2 * (warp % WPG) + (tid >> 4 & 1);
  // The launch's columns (tiles x units) are dealt to the CTAs in turn: CTA
  // c runs columns c, c + gridDim.x, ... back to back (a persistent grid of
  // one CTA per SM), so the TMA ring runs on from one column into the next
  // instead of draining and refilling at every column.
  //
  // A multi-step launch (P.steps set; persistent grids only, launched
  // cooperatively) runs P.nsteps time steps this way, chained column by
  // column instead of by kernel boundaries: the loads of column (step n,
  // unit u, tile) wait until the 3 x 3 tile neighbourhood of u has finished
  // step n - 1 (progress flags P.done[u][tile], zero at launch).  A level's
  // slot is next written one or two steps after it was read as the stepped
  // level, so the same condition covers the write-after-read hazards of the
  // slots.  Roles in the producer warpgroup: warp 8 lane 0 the TMA ring,
  // warp 9 lane 0 polls the flags of upcoming columns, warp 10 lane 0
  // publishes a column's flag once every consumer warp has stored it.
  const int nunits = P.nunits3;
  const int ncols = P.ntiles * nunits;
  const bool multi = P.steps != nullptr;
  const int nsteps = multi ? P.nsteps : 1;
  const int G = (int)gridDim.x;
  const int my_cols = (int)blockIdx.x < ncols ? (ncols - 1 - (int)blockIdx.x) / G + 1 : 0;
  M.lx = 4 * (M.lane & 15);
  M.last_q = L.nzp + 7;
  M.gz = gz;
  M.pq = 0;
  M.pst = 0;
  M.pround = 0;
  M.cslot = 0;
  M.lslot = 0;
  M.hslot = S::NST - HALO;  // (0 - 4) mod NST: first used at q = 4
  M.cphase = 0;
  M.zc = 0;
  M.carry = false;

  if (tid == 0) {
    tma_prefetch_desc(&tm_halo);
    tma_prefetch_desc(&tm_plain);
    tma_prefetch_desc(&tm_cc);
    if (ADJ) tma_prefetch_desc(&tm_g);
    for (int i = 0; i < S::NST; i++) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], NCW3);
    }
    for (int i = 0; i < S::NXB; i++) mbar_init(&xfull[i], 1);  // xfull and xempty: one arrival each
    *abort_flag = 0;
    *deps_ok = my_cols;  // step 0 depends on nothing in the launch
    for (int i = 0; i < WDONE3; i++) wdone[i] = 0;
    fence_mbar_init();
  }
  for (int i = tid; i < L.nzp; i += NTHREADS3) gz[i] = P.gtab[i];
  __syncthreads();

  if (warp >= NCW3) {  // -------------------------------------------- producer warpgroup
    setmaxnreg_dec<REG3_PRODUCER>();
    if (warp == NCW3 && M.lane == 0) {
      // sequence g (counted over all columns) into slot g % NST once every
      // consumer warp has released sequence g - NST (whose halo plane served
      // the level 4 below it, or, at a column's end, landed last)
      int gq = 0, ic = 0;
      bool ok = true;
      for (int n = 0; n < nsteps && ok; n++) {
        M.set_step(n);
        for (int it = blockIdx.x; it < ncols && ok; it += G, ic++) {
          M.set_column(it, nunits);
          if (n > 0) {  // the column's neighbourhood has finished step n - 1 (counted by warp 9)
            if (!wait_counter(deps_ok, ic, P.status, abort_flag)) {
              ok = false;
              break;
            }
            fence_proxy_async_global();
          }
          for (M.pq = 0; M.pq <= M.last_q; gq++) {
            if (gq >= S::NST &&
                !mbar_wait_abortable(&empty[M.pst], (uint32_t)((gq / S::NST - 1) & 1), P.status, abort_flag)) {
              ok = false;
              break;
            }
            M.issue();
          }
        }
      }
      if (!ok) {  // gave up: bounded wait for the copies in flight
        for (int i = gq - S::NST > 0 ? gq - S::NST : 0; i < gq; i++) {
          const long long t0 = clock64();
          while (!mbar_try_wait(&full[i % S::NST], (uint32_t)((i / S::NST) & 1)) && clock64() - t0 < (1LL << 24)) {
          }
        }
      }
    } else if (multi && warp == NCW3 + 1 && M.lane == 0) {
      // columns of steps 1.. in the producer's order: neighbourhood ready
      for (int n = 1, ic = my_cols; n < nsteps; n++)
        for (int kk = 0; kk < my_cols; kk++, ic++) {
          int u, tile;
          column_of(P, (int)blockIdx.x + kk * G, nunits, u, tile);
          if (!wait_columns3(P.done, P.ntx, P.ntiles, P.status, u, tile, n, abort_flag)) return;
          asm volatile("st.release.cta.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(deps_ok)), "r"(ic + 1) : "memory");
        }
    } else if (multi && warp == NCW3 + 2 && M.lane == 0) {
      // column ic of this CTA (step ic / my_cols) is complete when every
      // consumer warp has counted it in wdone[ic % WDONE3]; its flag (steps
      // done) is then published at GPU scope.  The last step's flags are
      // read by nobody.
      const int nic = my_cols * (nsteps - 1);
      for (int ic = 0; ic < nic; ic++) {
        const int n = ic / my_cols, kk = ic - n * my_cols;
        if (!wait_counter(&wdone[ic % WDONE3], NCW3 * (ic / WDONE3 + 1) - 1, P.status, abort_flag)) return;
        fence_acq_rel_gpu();
        int u, tile;
        column_of(P, (int)blockIdx.x + kk * G, nunits, u, tile);
        st_relaxed_gpu(P.done + (long long)u * P.ntiles + tile, n + 1);
      }
    }
    return;
  }
  setmaxnreg_inc<REG3_CONSUMER>();

  // Sequence q lands at queue index q % NQ (the centre of level q - 4) and
  // level q - 8 has its centre at (q - 4) % NQ.  NQ = 9: one sequence, one
  // level at a time.  NQ = 10: two sequences land, then their two levels are
  // computed together (two independent chains per thread), the queue holding
  // levels z - 4 .. z + 5.
#define FWI_ONE(k)                                          \
  if (!M.template land<(k) % NQ>()) return;                 \
  if (!M.template level<((k) + NQ - 4) % NQ>(q + (k))) return;
#define FWI_TWO(k)                                          \
  if (!M.template land<(k)>()) return;                      \
  if (!M.template land<(k) + 1>()) return;                  \
  if (!M.template level<((k) + 6) % 10>(q + (k))) return;   \
  if (!M.template level<((k) + 7) % 10>(q + (k) + 1)) return;
  int icc = 0;
  for (int n = 0; n < nsteps; n++) {
  M.set_step(n);
  for (int it = blockIdx.x; it < ncols; it += G, icc++) {
    M.set_column(it, nunits);
    M.gyv = M.gy < L.nyp ? __ldg(P.gtab + L.nzp + M.gy) : 0.f;
#pragma unroll
    for (int j = 0; j < 4; j++) M.gxv[j] = M.gx + j < L.nxp ? __ldg(P.gtab + L.nzp + L.nyp + M.gx + j) : 0.f;
    M.ie_cur = P.inj_off[M.b * P.inj_bstride + M.tile];
    M.ie_end = P.inj_off[M.b * P.inj_bstride + M.tile + 1];
    M.se_cur = P.smp4 ? P.smp_off[M.b * P.smp_bstride + M.tile] : 0;
    M.se_end = P.smp4 ? P.smp_off[M.b * P.smp_bstride + M.tile + 1] : 0;
    M.inj_z = M.ie_cur < M.ie_end ? P.inj[M.ie_cur].w : 0x7fffffff;
    M.smp_z = M.se_cur < M.se_end ? P.smp4[M.se_cur].z : 0x7fffffff;
#pragma unroll
    for (int i = 0; i < NQ; i++) {
      M.Q[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      M.QS[i] = M.Q[i];
    }
    int q = 0;
    if constexpr (NQ == 9) {
      for (; q + 9 <= M.last_q + 1; q += 9) {
        FWI_ONE(0) FWI_ONE(1) FWI_ONE(2) FWI_ONE(3) FWI_ONE(4) FWI_ONE(5) FWI_ONE(6) FWI_ONE(7) FWI_ONE(8)
      }
      const int rem = M.last_q + 1 - q;
      if (rem > 0) { FWI_ONE(0) }
      if (rem > 1) { FWI_ONE(1) }
      if (rem > 2) { FWI_ONE(2) }
      if (rem > 3) { FWI_ONE(3) }
      if (rem > 4) { FWI_ONE(4) }
      if (rem > 5) { FWI_ONE(5) }
      if (rem > 6) { FWI_ONE(6) }
      if (rem > 7) { FWI_ONE(7) }
    } else {
      for (; q + 10 <= M.last_q + 1; q += 10) {
        FWI_TWO(0) FWI_TWO(2) FWI_TWO(4) FWI_TWO(6) FWI_TWO(8)
      }
      const int rem = M.last_q + 1 - q;
      if (rem >= 2) { FWI_TWO(0) } else if (rem == 1) { FWI_ONE(0) }
      if (rem >= 4) { FWI_TWO(2) } else if (rem == 3) { FWI_ONE(2) }
      if (rem >= 6) { FWI_TWO(4) } else if (rem == 5) { FWI_ONE(4) }
      if (rem >= 8) { FWI_TWO(6) } else if (rem == 7) { FWI_ONE(6) }
      if (rem == 9) { FWI_ONE(8) }
    }
    // pair tiles: the first wavefield's warps still hold the column's last level
    if (ADJ && PAIR && M.k == 0 && !M.pair_finish(L.nzp - 1, M.zc - 1)) return;
    M.carry = true;
    if (multi) {  // this warp's stores of the column are done: count it for the publisher
      __syncwarp();
      if (M.lane == 0) red_release_cta_shared(&wdone[icc % WDONE3], 1);
    }
  }
  }
#undef FWI_ONE
#undef FWI_TWO
}

template <bool ADJ, bool ISO, bool PAIR>
static cudaError_t launch3(const CUtensorMap& tm_halo, const CUtensorMap& tm_plain, const CUtensorMap& tm_cc,
                           const CUtensorMap& tm_g, const Layout& L, const Coef& K, const StepParams& P, dim3 grid,
                           cudaStream_t st) {
  const size_t bytes = Smem3D<ADJ, PAIR>::bytes(L.nzp);
  auto kern = P.zpair3 ? step3d_kernel<ADJ, ISO, 10, PAIR> : step3d_kernel<ADJ, ISO, 9, PAIR>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  if (!P.steps) {
    kern<<<grid, NTHREADS3, bytes, st>>>(tm_halo, tm_plain, tm_cc, tm_g, L, K, P);
    return cudaGetLastError();
  }
  // multi-step: CTAs wait on one another's progress flags, so all of them
  // must be resident at once (a cooperative launch refuses a grid that is not)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(NTHREADS3);
  cfg.dynamicSmemBytes = bytes;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, tm_halo, tm_plain, tm_cc, tm_g, L, K, P);
}

cudaError_t launch_step3d(bool adj, const CUtensorMap& tm_halo, const CUtensorMap& tm_plain, const CUtensorMap& tm_cc,
                          const CUtensorMap& tm_g, const Layout& L, const Coef& K, const StepParams& P, int B,
                          cudaStream_t st) {
  // columns: tiles x units (one wavefield, or a pair of supergathers of one
  // sample), dealt in turn to a persistent grid of at most one CTA per SM
  if (P.pair3 && (B % 2 || P.nsg % 2)) return cudaErrorInvalidValue;
  // a multi-step launch needs the persistent grid, its step table and flags
  if (P.steps && (P.ctas_per_sm3 != 1 || P.nsteps < 1 || !P.done)) return cudaErrorInvalidValue;
  StepParams Q = P;
  Q.nunits3 = P.pair3 ? B / 2 : B;
  const long long ncols = (long long)P.ntiles * Q.nunits3;
  static int nsm = 0;
  if (nsm <= 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || nsm <= 0)
      nsm = 1;
  }
  const long long cap = (long long)nsm * P.ctas_per_sm3;
  dim3 grid((unsigned)(P.ctas_per_sm3 > 0 && ncols > cap ? cap : ncols));
  // On isotropic grids both recursions use the one-bracket Laplacian (the
  // adjoint's imaging term has its own plain form, lap3_img).
  bool iso = true;
  for (int k = 1; k <= 4; k++) iso = iso && K.cx[k] == K.cy[k] && K.cx[k] == K.cz[k];
  if (adj) {
    if (P.pair3)
      return iso ? launch3<true, true, true>(tm_halo, tm_plain, tm_cc, tm_g, L, K, Q, grid, st)
                 : launch3<true, false, true>(tm_halo, tm_plain, tm_cc, tm_g, L, K, Q, grid, st);
    return iso ? launch3<true, true, false>(tm_halo, tm_plain, tm_cc, tm_g, L, K, Q, grid, st)
               : launch3<true, false, false>(tm_halo, tm_plain, tm_cc, tm_g, L, K, Q, grid, st);
  }
  if (P.pair3)
    return iso ? launch3<false, true, true>(tm_halo, tm_plain, tm_cc, tm_g, L, K, Q, grid, st)
               : launch3<false, false, true>(tm_halo, tm_plain, tm_cc, tm_g, L, K, Q, grid, st);
  return iso ? launch3<false, true, false>(tm_halo, tm_plain, tm_cc, tm_g, L, K, Q, grid, st)
             : launch3<false, false, false>(tm_halo, tm_plain, tm_cc, tm_g, L, K, Q, grid, st);
}

}  // namespace fwi
