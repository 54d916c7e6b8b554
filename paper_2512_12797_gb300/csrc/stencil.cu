// stencil.cu -- multi-step kernels of the damped 8th-order acoustic recursion
// (2D) and of its exact discrete adjoint with the imaging condition.
//
// Forward step:
//     p^{n+1} = p^n + b (p^n - p^{n-1}) + cc (L p^n + s^n)
// with b = (1 - gamma dt)/(1 + gamma dt), cc = v^2 dt^2/(1 + gamma dt).  This is
// the damped leapfrog p^{n+1} = [2p^n - (1-gamma dt)p^{n-1} + c(Lp^n + s^n)]/(1+gamma dt)
// rewritten with 2/(1+gamma dt) = 1 + b, which keeps the FP32 recursion free of
// the spurious growth that rounding 2/(1+gamma dt) and b separately introduces
// in the sponge.  L is evaluated as sum_k a_k/h^2 [(p_{+k} + p_{-k}) - 2p], which
// equals the textbook 8th-order form because a_0 = -2 sum_k a_k; the bracket is
// exactly zero for a constant field in FP32, so the rounded coefficients add no
// spurious mass term to the recursion.
//
// Adjoint step: with q = cc * lambda the transpose of the recursion above is the
// same recursion, driven by cc * R^T dJ/dd at the receivers:
//     q^k = q^{k+1} + b (q^{k+1} - q^{k+2}) + cc (L q^{k+1} + R^T rhat^{k-1}),
// and the imaging condition dJ/dc = (1/c) sum_n q^{n+1} (L p^n + s^n) is
// accumulated here as G += q^k * L p^{k-1} (the source term is added from
// source-point samples after the time loop).
//
// One cooperative launch runs many time steps.  Work items are 128 x 32 (x, z)
// tiles of one posterior sample; CTA c owns items c, c + G, c + 2G, ... in
// every step and processes each for all of the sample's supergathers in a row.
// Steps are chained tile by tile instead of by kernel boundaries: an item's
// loads for step n wait until the 3 x 3 tile neighbourhood has finished step
// n-1 (per-item progress flags in global memory).  Because a level's slot is
// reused at the earliest three steps later, that single condition also covers
// the write-after-read hazards of the slot ring.
//
// Each CTA is warp-specialised: two consumer warpgroups (8 warps, 4 rows x 4
// columns per thread) compute, and a producer warpgroup runs
//   warp 8  -- the TMA ring: halo tile of the stepped level (and of the
//              snapshot in the adjoint), plain tile of the older level, the cc
//              tile once per item; waits for the progress flags first;
//   warp 9  -- the point lists of each iteration (injection entries with their
//              scaled series values, sampling entries), copied into the stage
//              so that no consumer waits on a dependent global load;
//   warp 10 -- publishes an item's progress flag once all consumer warps have
//              stored its outputs;
//   warp 11 -- polls the progress flags of upcoming items ahead of warp 8 and
//              counts the items whose neighbourhood is ready.
// setmaxnreg moves registers from the producer to the consumer warpgroups.
#include "fwi_internal.cuh"

namespace fwi {

constexpr int NCW2D = 8;                     // consumer warps; R rows per thread, tiles of 8R rows
__host__ __device__ constexpr int tile_rows2(int R) { return NCW2D * R; }
constexpr int NTHREADS2D = 32 * NCW2D + 128;  // + producer warpgroup
constexpr int PCAP = 128;                    // point-list entries staged per stage and list
constexpr int WDONE = 8;                     // item-completion counters (ring)
constexpr int REG_LAUNCH = 168, REG_PRODUCER = 72, REG_CONSUMER = 216;
static_assert(128 * REG_PRODUCER + 32 * NCW2D * REG_CONSUMER <= NTHREADS2D * REG_LAUNCH,
              "register split exceeds the launch allocation");
// L2 eviction priorities: the cc tiles and the imaging accumulator, re-read
// every step, are kept (evict-last); the older level and the output, which
// stream through once per step, go first; the halo tiles of the stepped level
// and of the snapshot keep the normal priority so that neighbouring tiles
// find their overlap in L2.
constexpr bool kL2Hints = true;
// One ring stage: halo tile of the stepped level, plain tile of the older
// level, [halo tile of the snapshot], and the iteration's point lists:
//   PTS[0..5]   = staged injection count, staged sampling count, global
//                 injection range [begin, end), global sampling range [begin, end)
//   PTS[32 ..]  = injection local index [PCAP], injection value [PCAP],
//                 sampling local index [PCAP], sampling record column [PCAP].
// Two cc tiles follow the stages.  Every part starts on 128 bytes.
template <bool ADJ, int NS, int R>
struct Smem2D {
  static constexpr int IN = (tile_rows2(R) + 2 * HALO) * HX;  // floats in one halo tile
  static constexpr int PV = tile_rows2(R) * TX;               // floats in one plain tile
  static constexpr int PTS = 32 + 4 * PCAP;
  static constexpr int OFF_SNAP = IN + PV;
  static constexpr int OFF_PTS = OFF_SNAP + (ADJ ? IN : 0);
  static constexpr int STAGE = OFF_PTS + PTS;
  static constexpr int OFF_C = NS * STAGE;
  static constexpr int nfloat = OFF_C + 2 * PV;
  static constexpr int nbar = 2 * NS + 4;  // full[NS], empty[NS], cfull[2], cempty[2]
  static constexpr int bytes = nfloat * 4 + nbar * 8 + (WDONE + 4) * 4;
  static_assert((STAGE * 4) % 128 == 0 && (PTS * 4) % 128 == 0, "stage parts must stay 128-byte aligned");
};

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// 8th-order Laplacian of the 4 x R block whose top-left element sits at
// shared row r0+4, column c0+4 of a halo tile T (row stride HX).  With
// ISO (hx == hz) the two axes share coefficients and each k costs one bracket
// [(x_{+k} + x_{-k}) + (z_{+k} + z_{-k}) - 4p], also exactly zero for a
// constant field.  Adjacent columns are computed as pairs with the packed
// FP32 instructions (two independent IEEE operations each, so every point
// sees exactly the operations of the scalar form); x - y is formed as
// fma(y, -1, x) and x - 4p as fma(-4, p, x), both exact rewrites.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

template <int R, bool ISO>
__device__ __forceinline__ void lap_block(const float* __restrict__ T, int r0, int c0, const Coef& K,
                                          float (&lap)[R][4], float (&ctr)[R][4]) {
  float4 zc[R + 8];
#pragma unroll
  for (int i = 0; i < R + 8; i++) zc[i] = lds4(T + (r0 + i) * HX + c0 + 4);
  const float* zp = reinterpret_cast<const float*>(&zc[0]);  // zc[i] component j is zp[4*i + j]
  const float2 m1 = f2(-1.f, -1.f), m4 = f2(-4.f, -4.f);
#pragma unroll
  for (int r = 0; r < R; r++) {
    const float4 xl = lds4(T + (r0 + r + 4) * HX + c0);
    const float4 xr = lds4(T + (r0 + r + 4) * HX + c0 + 8);
    const float4 ce = zc[r + 4];
    const float w[12] = {xl.x, xl.y, xl.z, xl.w, ce.x, ce.y, ce.z, ce.w, xr.x, xr.y, xr.z, xr.w};
#pragma unroll
    for (int j = 0; j < 4; j += 2) {
      const float2 p = f2(w[4 + j], w[5 + j]);
      // (x_{+k} + x_{-k}) and (z_{+k} + z_{-k}) of the pair
      // odd k straddles the float4 quads: two scalar adds whose results land in a pair
      auto xs = [&](int k) {
        return (k & 1) ? f2(w[4 + j + k] + w[4 + j - k], w[5 + j + k] + w[5 + j - k])
                       : __fadd2_rn(f2(w[4 + j + k], w[5 + j + k]), f2(w[4 + j - k], w[5 + j - k]));
      };
      auto zs = [&](int k) {
        return __fadd2_rn(f2(zp[4 * (r + 4 + k) + j], zp[4 * (r + 4 + k) + j + 1]),
                          f2(zp[4 * (r + 4 - k) + j], zp[4 * (r + 4 - k) + j + 1]));
      };
      float2 a;
      if (ISO) {
        auto br = [&](int k) { return __ffma2_rn(m4, p, __fadd2_rn(xs(k), zs(k))); };
        a = __fmul2_rn(f2(K.cx[4], K.cx[4]), br(4));
        a = __ffma2_rn(f2(K.cx[3], K.cx[3]), br(3), a);
        a = __ffma2_rn(f2(K.cx[2], K.cx[2]), br(2), a);
        a = __ffma2_rn(f2(K.cx[1], K.cx[1]), br(1), a);
      } else {
        const float2 p2 = __fadd2_rn(p, p);
        a = __fmul2_rn(f2(K.cx[4], K.cx[4]), __ffma2_rn(p2, m1, xs(4)));
        a = __ffma2_rn(f2(K.cx[3], K.cx[3]), __ffma2_rn(p2, m1, xs(3)), a);
        a = __ffma2_rn(f2(K.cx[2], K.cx[2]), __ffma2_rn(p2, m1, xs(2)), a);
        a = __ffma2_rn(f2(K.cx[1], K.cx[1]), __ffma2_rn(p2, m1, xs(1)), a);
        a = __ffma2_rn(f2(K.cz[4], K.cz[4]), __ffma2_rn(p2, m1, zs(4)), a);
        a = __ffma2_rn(f2(K.cz[3], K.cz[3]), __ffma2_rn(p2, m1, zs(3)), a);
        a = __ffma2_rn(f2(K.cz[2], K.cz[2]), __ffma2_rn(p2, m1, zs(2)), a);
        a = __ffma2_rn(f2(K.cz[1], K.cz[1]), __ffma2_rn(p2, m1, zs(1)), a);
      }
      lap[r][j] = a.x;
      lap[r][j + 1] = a.y;
      ctr[r][j] = p.x;
      ctr[r][j + 1] = p.y;
    }
  }
}

// The Laplacian of the snapshot for the imaging condition, in the plain form
// c0 p + sum_k c_k [(x_{+k} + x_{-k}) (+ (z_{+k} + z_{-k}))]: it only enters
// the gradient, not the recursion, so it does not need the bracket form's
// exact zero on constant fields, and saves the 4 subtractions of 4p (or 2p)
// per point.  Same pair arithmetic and operand loads as lap_block.
template <int R, bool ISO>
__device__ __forceinline__ void lap_img(const float* __restrict__ T, int r0, int c0, const Coef& K,
                                        float (&lap)[R][4]) {
  float4 zc[R + 8];
#pragma unroll
  for (int i = 0; i < R + 8; i++) zc[i] = lds4(T + (r0 + i) * HX + c0 + 4);
  const float* zp = reinterpret_cast<const float*>(&zc[0]);
#pragma unroll
  for (int r = 0; r < R; r++) {
    const float4 xl = lds4(T + (r0 + r + 4) * HX + c0);
    const float4 xr = lds4(T + (r0 + r + 4) * HX + c0 + 8);
    const float4 ce = zc[r + 4];
    const float w[12] = {xl.x, xl.y, xl.z, xl.w, ce.x, ce.y, ce.z, ce.w, xr.x, xr.y, xr.z, xr.w};
#pragma unroll
    for (int j = 0; j < 4; j += 2) {
      const float2 p = f2(w[4 + j], w[5 + j]);
      // odd k straddles the float4 quads: two scalar adds whose results land in a pair
      auto xs = [&](int k) {
        return (k & 1) ? f2(w[4 + j + k] + w[4 + j - k], w[5 + j + k] + w[5 + j - k])
                       : __fadd2_rn(f2(w[4 + j + k], w[5 + j + k]), f2(w[4 + j - k], w[5 + j - k]));
      };
      auto zs = [&](int k) {
        return __fadd2_rn(f2(zp[4 * (r + 4 + k) + j], zp[4 * (r + 4 + k) + j + 1]),
                          f2(zp[4 * (r + 4 - k) + j], zp[4 * (r + 4 - k) + j + 1]));
      };
      float2 a = __fmul2_rn(f2(K.c0_2d, K.c0_2d), p);
      if (ISO) {
#pragma unroll
        for (int k = 4; k >= 1; k--) a = __ffma2_rn(f2(K.cx[k], K.cx[k]), __fadd2_rn(xs(k), zs(k)), a);
      } else {
#pragma unroll
        for (int k = 4; k >= 1; k--) a = __ffma2_rn(f2(K.cx[k], K.cx[k]), xs(k), a);
#pragma unroll
        for (int k = 4; k >= 1; k--) a = __ffma2_rn(f2(K.cz[k], K.cz[k]), zs(k), a);
      }
      lap[r][j] = a.x;
      lap[r][j + 1] = a.y;
    }
  }
}

// Bounded poll of the progress flags of the 3 x 3 tile neighbourhood of item
// (s, tile) until each has completed `need` steps; then acquire-orders the
// neighbours' stores before the TMA loads that follow.  Gives up on timeout,
// on the CTA's abort word, or when another CTA has recorded an error.
__device__ __noinline__ bool wait_neighbours(const StepParams& P, int s, int tile, int need,
                                             volatile int* abort_flag) {
  const int tx = tile % P.ntx, tz = tile / P.ntx, ntz = P.ntiles / P.ntx;
  const int* base = P.done + (long long)s * P.ntiles;
  const int z_lo = max(tz - 1, 0), z_hi = min(tz + 1, ntz - 1);
  const int x_lo = max(tx - 1, 0), x_hi = min(tx + 1, P.ntx - 1);
  const long long t0 = clock64();
  for (;;) {
    int lo = need;
    for (int z = z_lo; z <= z_hi; z++)
      for (int x = x_lo; x <= x_hi; x++) lo = min(lo, ld_relaxed_gpu(base + z * P.ntx + x));
    if (lo >= need) break;
    if (*abort_flag || ld_relaxed_gpu(P.status) != 0) {
      *abort_flag = 1;
      return false;
    }
    if (clock64() - t0 > WAIT_CYCLES) {
      atomicCAS(P.status, 0, (int)FWI_ERR_TIMEOUT);
      *abort_flag = 1;
      return false;
    }
    __nanosleep(128);
  }
  fence_acq_rel_gpu();
  fence_proxy_async_global();
  return true;
}

// After an abort: bounded wait for the copies this thread issued into the
// last `n` stages (or cc buffers) so that none lands after the CTA exits.
__device__ __forceinline__ void drain(uint64_t* bars, int nbars, int issued, int n) {
  for (int i = max(issued - n, 0); i < issued; i++) {
    const long long t0 = clock64();
    while (!mbar_try_wait(&bars[i % nbars], (uint32_t)((i / nbars) & 1)))
      if (clock64() - t0 > (1LL << 24)) break;
  }
}

// Warp 8, lane 0: TMA ring.  Iteration m = ((step n, item k), supergather j)
// fills stage m % NS; the cc tile of (n, k) goes to buffer ic & 1.
template <bool ADJ, int NS, int R>
__device__ __forceinline__ void produce_tma(const CUtensorMap* tm_halo, const CUtensorMap* tm_plain,
                                            const CUtensorMap* tm_c, const StepParams& P, float* sm,
                                            uint64_t* full, uint64_t* empty, uint64_t* cfull, uint64_t* cempty,
                                            int* deps_ok, int my_items, volatile int* abort_flag) {
  using S = Smem2D<ADJ, NS, R>;
  constexpr uint32_t TX_BYTES = (S::IN + S::PV + (ADJ ? S::IN : 0)) * 4;
  const int G = gridDim.x, nsg = P.nsg;
  const uint64_t pol_first = l2_evict_first(), pol_last = l2_evict_last();
  int m = 0, ic = 0;
  for (int n = 0; n < P.nsteps; n++) {
    const int4 d = __ldg(reinterpret_cast<const int4*>(P.steps + n));  // cur, prev, out, snap
    for (int k = 0; k < my_items; k++, ic++) {
      const int item = (int)blockIdx.x + k * G;
      const int s = item / P.ntiles, tile = item - s * P.ntiles;
      const int x0 = (tile % P.ntx) * TX, z0 = (tile / P.ntx) * tile_rows2(R);
      if (n > 0) {  // neighbourhood of (n, k) ready: counted by warp 11
        const long long t0 = clock64();
        while (ld_acquire_cta_shared(deps_ok) <= ic) {
          if (*abort_flag) goto aborted;
          if (clock64() - t0 > WAIT_CYCLES) {
            atomicCAS(P.status, 0, (int)FWI_ERR_TIMEOUT);
            *abort_flag = 1;
            goto aborted;
          }
          __nanosleep(32);
        }
        fence_proxy_async_global();
      }
      {
        const int cs = ic & 1;
        if (ic >= 2 && !mbar_wait_abortable(&cempty[cs], (uint32_t)(((ic >> 1) - 1) & 1), P.status, abort_flag))
          goto aborted;
        mbar_arrive_expect_tx(&cfull[cs], S::PV * 4);
        if (kL2Hints)
          tma_load_3d_hint(sm + S::OFF_C + cs * S::PV, tm_c, x0 + HALO, z0 + HALO, s, &cfull[cs], pol_last);
        else
          tma_load_3d(sm + S::OFF_C + cs * S::PV, tm_c, x0 + HALO, z0 + HALO, s, &cfull[cs]);
      }
      for (int j = 0; j < nsg; j++, m++) {
        const int st = m % NS;
        if (m >= NS && !mbar_wait_abortable(&empty[st], (uint32_t)((m / NS - 1) & 1), P.status, abort_flag))
          goto aborted;
        const int b = s * nsg + j;
        float* base = sm + st * S::STAGE;
        mbar_arrive_expect_tx(&full[st], TX_BYTES);
        tma_load_4d(base, tm_halo, x0, z0, b, d.x, &full[st]);
        if (kL2Hints)
          tma_load_4d_hint(base + S::IN, tm_plain, x0 + HALO, z0 + HALO, b, d.y, &full[st], pol_first);
        else
          tma_load_4d(base + S::IN, tm_plain, x0 + HALO, z0 + HALO, b, d.y, &full[st]);
        if (ADJ) tma_load_4d(base + S::OFF_SNAP, tm_halo, x0, z0, b, d.w, &full[st]);
      }
    }
  }
  return;
aborted:
  drain(full, NS, m, NS);
  drain(cfull, 2, ic, 2);
}

// Warp 9: point lists.  For every iteration the warp copies the injection
// entries of (wavefield, tile) with their values cc * amp * series[t] and the
// sampling entries into the stage's PTS block (at most PCAP of each; the
// consumers take any rest from global memory), then arrives on the stage's
// full barrier.  Offsets of an item's supergathers are loaded one item ahead.
template <bool ADJ, int NS, int R>
__device__ __forceinline__ void produce_points(const Layout& L, const StepParams& P, float* sm, uint64_t* full,
                                               uint64_t* empty, int my_items, int lane,
                                               volatile int* abort_flag) {
  using S = Smem2D<ADJ, NS, R>;
  const int G = gridDim.x, nsg = P.nsg;
  const bool has_smp = P.smp != nullptr;
  // offsets of supergather j0 + lane of item k: inj [a0, a1), smp [b0, b1)
  auto load_offsets = [&](int k, int j0, int& a0, int& a1, int& b0, int& b1) {
    const int item = (int)blockIdx.x + k * G;
    const int s = item / P.ntiles, tile = item - s * P.ntiles;
    a0 = a1 = b0 = b1 = 0;
    if (j0 + lane < nsg) {
      const int b = s * nsg + j0 + lane;
      const int* io = P.inj_off + (long long)b * P.inj_bstride + tile;
      a0 = __ldg(io);
      a1 = __ldg(io + 1);
      if (has_smp) {
        const int* so = P.smp_off + (long long)b * P.smp_bstride + tile;
        b0 = __ldg(so);
        b1 = __ldg(so + 1);
      }
    }
  };
  int na0, na1, nb0, nb1;
  load_offsets(0, 0, na0, na1, nb0, nb1);
  int m = 0;
  for (int n = 0; n < P.nsteps; n++) {
    const int t = __ldg(&P.steps[n].t);
    for (int k = 0; k < my_items; k++) {
      const int item = (int)blockIdx.x + k * G;
      const int s = item / P.ntiles, tile = item - s * P.ntiles;
      const int x0 = (tile % P.ntx) * TX, z0 = (tile / P.ntx) * tile_rows2(R);
      const float* cs = P.c + (long long)s * L.field;
      for (int j0 = 0; j0 < nsg; j0 += 32) {
        int a0 = na0, a1 = na1, b0 = nb0, b1 = nb1;
        // prefetch the next chunk (or the next item's first chunk)
        if (j0 + 32 < nsg)
          load_offsets(k, j0 + 32, na0, na1, nb0, nb1);
        else
          load_offsets(k + 1 < my_items ? k + 1 : 0, 0, na0, na1, nb0, nb1);
        const int jn = min(32, nsg - j0);
        for (int jj = 0; jj < jn; jj++, m++) {
          const int io0 = __shfl_sync(0xffffffffu, a0, jj), io1 = __shfl_sync(0xffffffffu, a1, jj);
          const int so0 = __shfl_sync(0xffffffffu, b0, jj), so1 = __shfl_sync(0xffffffffu, b1, jj);
          const int st = m % NS;
          const int b = s * nsg + j0 + jj;
          const int ni = min(io1 - io0, PCAP), nsm = min(so1 - so0, PCAP);
          // all loads before the wait for the stage, so that their latency
          // overlaps the consumers' work on it
          constexpr int NCH = PCAP / 32;
          int4 ie[NCH];
          int2 se[NCH];
#pragma unroll
          for (int c = 0; c < NCH; c++) {
            const int e = c * 32 + lane;
            ie[c] = e < ni ? __ldg(P.inj + io0 + e) : make_int4(0, 0, 0, 0);
            se[c] = e < nsm ? __ldg(P.smp + so0 + e) : make_int2(0, 0);
          }
          float iv[NCH];
#pragma unroll
          for (int c = 0; c < NCH; c++) {
            iv[c] = 0.f;
            if (c * 32 + lane < ni) {
              const int rz = ie[c].x / TX;
              const float ccp = __ldg(cs + L.off(z0 + rz, 0, x0 + ie[c].x % TX));
              const float ser =
                  __ldg(P.series + (long long)b * P.series_bstride + (long long)t * P.series_ld + ie[c].y);
              iv[c] = ccp * (__int_as_float(ie[c].z) * ser);
            }
          }
          int ok = 1;
          if (m >= NS && lane == 0)
            ok = mbar_wait_abortable(&empty[st], (uint32_t)((m / NS - 1) & 1), P.status, abort_flag);
          if (!__shfl_sync(0xffffffffu, ok, 0)) return;
          int* pts = reinterpret_cast<int*>(sm + st * S::STAGE + S::OFF_PTS);
#pragma unroll
          for (int c = 0; c < NCH; c++) {
            const int e = c * 32 + lane;
            if (e < ni) {
              pts[32 + e] = ie[c].x;
              pts[32 + PCAP + e] = __float_as_int(iv[c]);
            }
            if (e < nsm) {
              pts[32 + 2 * PCAP + e] = se[c].x;
              pts[32 + 3 * PCAP + e] = se[c].y;
            }
          }
          if (lane == 0) {
            *reinterpret_cast<int4*>(pts) = make_int4(ni, nsm, io0, io1);
            *reinterpret_cast<int2*>(pts + 4) = make_int2(so0, so1);
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&full[st]);
        }
      }
    }
  }
}

// Warp 11, lane 0: items (n >= 1, k) in order; deps_ok = number of this CTA's
// items whose 3 x 3 neighbourhood has finished the previous step (the items of
// the first step need nothing and are counted from the start).
__device__ __forceinline__ void watch_deps(const StepParams& P, int* deps_ok, int my_items,
                                           volatile int* abort_flag) {
  const int G = gridDim.x;
  const int nic = my_items * P.nsteps;
  for (int ic = my_items; ic < nic; ic++) {
    const int n = ic / my_items, k = ic - n * my_items;
    const int item = (int)blockIdx.x + k * G;
    const int s = item / P.ntiles, tile = item - s * P.ntiles;
    if (!wait_neighbours(P, s, tile, n, abort_flag)) return;
    asm volatile("st.release.cta.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(deps_ok)), "r"(ic + 1) : "memory");
  }
}

// Warp 10, lane 0: progress flags.  Item ic of this CTA (step ic / my_items)
// is complete when all consumer warps have counted it in wdone[ic % WDONE];
// the flag (steps done) is then published with release semantics at GPU
// scope.  Steps whose flags nobody reads (the launch's last) are skipped.
__device__ __forceinline__ void publish(const StepParams& P, int* wdone, int my_items, volatile int* abort_flag) {
  const int G = gridDim.x;
  const int nic = my_items * (P.nsteps - 1);
  for (int ic = 0; ic < nic; ic++) {
    const int n = ic / my_items, k = ic - n * my_items;
    const int target = NCW2D * (ic / WDONE + 1);
    const long long t0 = clock64();
    while (ld_acquire_cta_shared(&wdone[ic % WDONE]) < target) {
      if (*abort_flag) return;
      if (clock64() - t0 > WAIT_CYCLES) {
        atomicCAS(P.status, 0, (int)FWI_ERR_TIMEOUT);
        *abort_flag = 1;
        return;
      }
      __nanosleep(64);
    }
    fence_acq_rel_gpu();
    st_relaxed_gpu(P.done + (int)blockIdx.x + k * G, n + 1);
  }
}

template <bool ADJ, int NS, bool ISO, int R>
__global__ void __launch_bounds__(NTHREADS2D, 1)
step2d_kernel(const __grid_constant__ CUtensorMap tm_halo, const __grid_constant__ CUtensorMap tm_plain,
              const __grid_constant__ CUtensorMap tm_c, const Layout L, const Coef K, const StepParams P,
              int nitems) {
  using S = Smem2D<ADJ, NS, R>;
  constexpr int NCW = NCW2D, TZR = tile_rows2(R);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + S::nfloat * 4);
  uint64_t* empty = full + NS;
  uint64_t* cfull = empty + NS;
  uint64_t* cempty = cfull + 2;
  int* wdone = reinterpret_cast<int*>(cempty + 2);
  volatile int* abort_flag = wdone + WDONE;
  int* deps_ok = wdone + WDONE + 1;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = gridDim.x;
  const int my_items = (int)blockIdx.x < nitems ? (nitems - 1 - (int)blockIdx.x) / G + 1 : 0;
  const int nsg = P.nsg;
  if (my_items == 0 || P.nsteps <= 0 || nsg <= 0) return;  // uniform over the CTA

  if (tid == 0) {
    tma_prefetch_desc(&tm_halo);
    tma_prefetch_desc(&tm_plain);
    tma_prefetch_desc(&tm_c);
    for (int i = 0; i < NS; i++) {
      mbar_init(&full[i], 2);      // TMA expect_tx arrival + point-list arrival
      mbar_init(&empty[i], NCW);
    }
    for (int i = 0; i < 2; i++) {
      mbar_init(&cfull[i], 1);
      mbar_init(&cempty[i], NCW);
    }
    for (int i = 0; i < WDONE; i++) wdone[i] = 0;
    *abort_flag = 0;
    *deps_ok = my_items;
    fence_mbar_init();
  }
  __syncthreads();

  if (warp >= NCW) {  // ------------------------------------------- producer warpgroup
    setmaxnreg_dec<REG_PRODUCER>();
    if (warp == NCW && lane == 0)
      produce_tma<ADJ, NS, R>(&tm_halo, &tm_plain, &tm_c, P, sm, full, empty, cfull, cempty, deps_ok, my_items,
                           abort_flag);
    else if (warp == NCW + 1)
      produce_points<ADJ, NS, R>(L, P, sm, full, empty, my_items, lane, abort_flag);
    else if (warp == NCW + 2 && lane == 0)
      publish(P, wdone, my_items, abort_flag);
    else if (warp == NCW + 3 && lane == 0)
      watch_deps(P, deps_ok, my_items, abort_flag);
    return;
  }
  setmaxnreg_inc<REG_CONSUMER>();

  // ------------------------------------------------------------------ consumers
  const int lx = 4 * lane, lz = R * warp;
  const uint64_t pol_first = l2_evict_first(), pol_last = l2_evict_last();
  const float* gzt = P.gtab;
  const float* gxt = P.gtab + L.nzp + L.nyp;
  // next item's imaging accumulator rows (adjoint) and sponge table entries
  float4 gpre[R];
  float gzpre[R], gxpre[4];
  auto prefetch_item = [&](int k_) {
    const int item_ = (int)blockIdx.x + k_ * G;
    const int s_ = item_ / P.ntiles, tile_ = item_ - s_ * P.ntiles;
    const int gx_ = (tile_ % P.ntx) * TX + lx, zb = (tile_ / P.ntx) * TZR + lz;
#pragma unroll
    for (int r = 0; r < R; r++) {
      const bool v = zb + r < L.nzp && gx_ < L.nxp;
      gzpre[r] = zb + r < L.nzp ? __ldg(gzt + zb + r) : 0.f;
      if (ADJ) {
        const float* gp = P.grad + (long long)s_ * L.field + L.off(zb + r, 0, gx_);
        gpre[r] = !v ? make_float4(0.f, 0.f, 0.f, 0.f)
                     : (kL2Hints ? ld4_hint(gp, pol_last) : *reinterpret_cast<const float4*>(gp));
      }
    }
#pragma unroll
    for (int q = 0; q < 4; q++) gxpre[q] = gx_ + q < L.nxp ? __ldg(gxt + gx_ + q) : 0.f;
  };
  // With one item per CTA the adjoint keeps the accumulator in registers
  // across steps (a prefetch would read the rows before this thread stores them).
  const bool carry = my_items == 1;
  prefetch_item(0);
  float gacc[R][4];

  int st = 0;
  uint32_t ph = 0;
  int ic = 0;
  for (int n = 0; n < P.nsteps; n++) {
    const int4 d = __ldg(reinterpret_cast<const int4*>(P.steps + n));
    const int t = __ldg(&P.steps[n].t);
    for (int k = 0; k < my_items; k++, ic++) {
      const int item = (int)blockIdx.x + k * G;
      const int s = item / P.ntiles, tile = item - s * P.ntiles;
      const int x0 = (tile % P.ntx) * TX, z0 = (tile / P.ntx) * TZR;
      const int gx = x0 + lx;
      const bool colv0 = gx < L.nxp, live = z0 + lz < L.nzp;
      const bool sponge =
          L.nb > 0 && (x0 < L.nb || x0 + TX > L.nb + L.nx || z0 < L.nb || z0 + TZR > L.nb + L.nz);
      bool rowv[R];
      float cc[R][4], bc[R][4];
#pragma unroll
      for (int r = 0; r < R; r++) {
        rowv[r] = z0 + lz + r < L.nzp;
#pragma unroll
        for (int q = 0; q < 4; q++) bc[r][q] = sponge ? sponge_b(gzpre[r] + gxpre[q]) : 1.f;
        if (ADJ && (!carry || ic == 0)) {
          gacc[r][0] = gpre[r].x; gacc[r][1] = gpre[r].y; gacc[r][2] = gpre[r].z; gacc[r][3] = gpre[r].w;
        }
      }
      const long long row0 = L.off(z0 + lz, 0, gx);
      float* obase = P.pool + (long long)d.z * P.slot_elems + (long long)s * nsg * L.field + row0;
      if (!carry) prefetch_item(k + 1 < my_items ? k + 1 : 0);

      for (int j = 0; j < nsg; j++) {
        const int b = s * nsg + j;
        if (!mbar_wait_abortable(&full[st], ph, P.status, abort_flag)) return;
        float* I = sm + st * S::STAGE;
        float* PV = I + S::IN;
        const int* pts = reinterpret_cast<const int*>(I + S::OFF_PTS);
        if (j == 0) {
          const int cs = ic & 1;
          if (!mbar_wait_abortable(&cfull[cs], (uint32_t)((ic >> 1) & 1), P.status, abort_flag)) return;
          const float* C = sm + S::OFF_C + cs * S::PV;
#pragma unroll
          for (int r = 0; r < R; r++) {
            const float4 c4 = lds4(C + (lz + r) * TX + lx);
            cc[r][0] = c4.x; cc[r][1] = c4.y; cc[r][2] = c4.z; cc[r][3] = c4.w;
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&cempty[cs]);
        }
        float nv[R][4];
        if (live) {
          float lap[R][4], ctr[R][4];
          lap_block<R, ISO>(I, lz, lx, K, lap, ctr);
#pragma unroll
          for (int r = 0; r < R; r++) {
            const float4 pm = lds4(PV + (lz + r) * TX + lx);
            const float pmv[4] = {pm.x, pm.y, pm.z, pm.w};
#pragma unroll
            for (int q = 0; q < 4; q += 2) {  // cc * lap + (ctr + bc * (ctr - pm)), in pairs
              const float2 c2 = f2(ctr[r][q], ctr[r][q + 1]);
              const float2 d2 = __ffma2_rn(f2(pmv[q], pmv[q + 1]), f2(-1.f, -1.f), c2);
              const float2 n2 = __ffma2_rn(f2(cc[r][q], cc[r][q + 1]), f2(lap[r][q], lap[r][q + 1]),
                                           __ffma2_rn(f2(bc[r][q], bc[r][q + 1]), d2, c2));
              nv[r][q] = n2.x;
              nv[r][q + 1] = n2.y;
            }
          }
          const int4 h = *reinterpret_cast<const int4*>(pts);        // staged counts, injection range
          const int2 h2 = *reinterpret_cast<const int2*>(pts + 4);   // sampling range
          if (h.z < h.w || h2.x < h2.y) {
            // Injection (sources in the forward, residual at receivers in the
            // adjoint) and sampling (receivers in the forward, sources in the
            // adjoint), staged in this warp's own rows of the consumed p^{n-1} tile.
            __syncwarp();
#pragma unroll
            for (int r = 0; r < R; r++)
              *reinterpret_cast<float4*>(PV + (lz + r) * TX + lx) =
                  make_float4(nv[r][0], nv[r][1], nv[r][2], nv[r][3]);
            __syncwarp();
            for (int e0 = 0; e0 < h.x; e0 += 32) {
              const int e = e0 + lane;
              int loc = -1 - lane;  // unique key for lanes without an entry of this warp
              float val = 0.f;
              if (e < h.x) {
                const int l = pts[32 + e];
                const int rz = l / TX;
                if (rz >= lz && rz < lz + R) {
                  loc = l;
                  val = __int_as_float(pts[32 + PCAP + e]);
                }
              }
              const unsigned peers = __match_any_sync(0xffffffffu, loc);
              if (__any_sync(0xffffffffu, loc >= 0 && peers != (1u << lane))) {
                // coincident points in this chunk: add them in entry order
                for (int i = 0; i < 32; i++) {
                  const int li = __shfl_sync(0xffffffffu, loc, i);
                  const float vi = __shfl_sync(0xffffffffu, val, i);
                  if (lane == 0 && li >= 0) PV[li] += vi;
                }
              } else if (loc >= 0) {
                PV[loc] += val;
              }
              __syncwarp();
            }
            if (h.w - h.z > PCAP && lane == 0) {  // entries beyond the staged ones, in order
              for (int e = h.z + PCAP; e < h.w; e++) {
                const int4 en = P.inj[e];
                const int rz = en.x / TX;
                if (rz < lz || rz >= lz + R) continue;
                const float ccp = __ldg(P.c + (long long)s * L.field + L.off(z0 + rz, 0, x0 + en.x % TX));
                const float ser =
                    P.series[(long long)b * P.series_bstride + (long long)t * P.series_ld + en.y];
                PV[en.x] += ccp * (__int_as_float(en.z) * ser);
              }
            }
            __syncwarp();
#pragma unroll
            for (int r = 0; r < R; r++) {
              const float4 v = lds4(PV + (lz + r) * TX + lx);
              nv[r][0] = v.x; nv[r][1] = v.y; nv[r][2] = v.z; nv[r][3] = v.w;
            }
            float* so = P.smp_out + (long long)b * P.smp_bstride_out + (long long)t * P.smp_ld;
            for (int e = lane; e < h.y; e += 32) {
              const int l = pts[32 + 2 * PCAP + e];
              const int rz = l / TX;
              if (rz >= lz && rz < lz + R) so[pts[32 + 3 * PCAP + e]] = PV[l];
            }
            for (int e = h2.x + PCAP + lane; e < h2.y; e += 32) {
              const int2 en = P.smp[e];
              const int rz = en.x / TX;
              if (rz >= lz && rz < lz + R) so[en.y] = PV[en.x];
            }
            // generic-proxy writes to the stage are ordered before the TMA that refills it
            fence_proxy_async_shared();
          }
          if (ADJ) {
            float lps[R][4];
            lap_img<R, ISO>(I + S::OFF_SNAP, lz, lx, K, lps);
#pragma unroll
            for (int r = 0; r < R; r++)
#pragma unroll
              for (int q = 0; q < 4; q += 2) {
                const float2 g2 = __ffma2_rn(f2(nv[r][q], nv[r][q + 1]), f2(lps[r][q], lps[r][q + 1]),
                                             f2(gacc[r][q], gacc[r][q + 1]));
                gacc[r][q] = g2.x;
                gacc[r][q + 1] = g2.y;
              }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
        if (live) {
          float* o = obase + (long long)j * L.field;
#pragma unroll
          for (int r = 0; r < R; r++) {
            if (!rowv[r] || !colv0) continue;
            if (gx + 3 < L.nxp) {
              const float4 v4 = make_float4(nv[r][0], nv[r][1], nv[r][2], nv[r][3]);
              if (kL2Hints)
                st4_hint(o + r * L.SX, v4, pol_first);
              else
                *reinterpret_cast<float4*>(o + r * L.SX) = v4;
            } else {
#pragma unroll
              for (int q = 0; q < 4; q++)
                if (gx + q < L.nxp) o[r * L.SX + q] = nv[r][q];
            }
          }
        }
        if (++st == NS) { st = 0; ph ^= 1; }
      }
      if (ADJ && live) {
        float* gb = P.grad + (long long)s * L.field + row0;
#pragma unroll
        for (int r = 0; r < R; r++) {
          if (!rowv[r] || !colv0) continue;
          if (gx + 3 < L.nxp) {
            const float4 v4 = make_float4(gacc[r][0], gacc[r][1], gacc[r][2], gacc[r][3]);
            if (kL2Hints)
              st4_hint(gb + r * L.SX, v4, pol_last);
            else
              *reinterpret_cast<float4*>(gb + r * L.SX) = v4;
          } else {
#pragma unroll
            for (int q = 0; q < 4; q++)
              if (gx + q < L.nxp) gb[r * L.SX + q] = gacc[r][q];
          }
        }
      }
      // this warp's stores of the item are done: count it for the publisher
      __syncwarp();
      if (lane == 0) red_release_cta_shared(&wdone[ic % WDONE], 1);
    }
  }
}

static int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// Compiled variants differ in the ring depth NS and the tile height (8R rows:
// 128 x 32 or 128 x 24); the arithmetic per grid point is the same in every
// variant, so their results are bit-identical and the autotuner in fwi_api.cu picks the fastest per call shape.  The launch is
// cooperative: CTAs wait on one another's progress flags, so all of them must
// be resident (one per SM).
template <bool ADJ, int NS, bool ISO, int R>
static cudaError_t launch_iso(const CUtensorMap& th, const CUtensorMap& tp, const CUtensorMap& tc, const Layout& L,
                              const Coef& K, const StepParams& P, int nsamp, cudaStream_t st) {
  using S = Smem2D<ADJ, NS, R>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(step2d_kernel<ADJ, NS, ISO, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         S::bytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int nitems = P.ntiles * nsamp;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nitems < num_sms() ? nitems : num_sms());
  cfg.blockDim = dim3(NTHREADS2D);
  cfg.dynamicSmemBytes = S::bytes;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, step2d_kernel<ADJ, NS, ISO, R>, th, tp, tc, L, K, P, nitems);
}

template <bool ADJ, int NS, int R>
static cudaError_t launch_variant(const CUtensorMap& th, const CUtensorMap& tp, const CUtensorMap& tc,
                                  const Layout& L, const Coef& K, const StepParams& P, int nsamp, cudaStream_t st) {
  if (K.cx[1] == K.cz[1] && K.cx[2] == K.cz[2] && K.cx[3] == K.cz[3] && K.cx[4] == K.cz[4])
    return launch_iso<ADJ, NS, true, R>(th, tp, tc, L, K, P, nsamp, st);
  return launch_iso<ADJ, NS, false, R>(th, tp, tc, L, K, P, nsamp, st);
}

struct Variant2D {
  const char* name;
  cudaError_t (*fn)(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const Layout&, const Coef&,
                    const StepParams&, int, cudaStream_t);
};

// Variant v: bit 0 the ring depth, bit 1 the tile shape (tile_shape2d).
static const Variant2D kFwd2D[] = {
    {"fwd2d 128x32 NS4 (8+4 warps)", launch_variant<false, 4, 4>},
    {"fwd2d 128x32 NS3 (8+4 warps)", launch_variant<false, 3, 4>},
    {"fwd2d 128x24 NS4 (8+4 warps)", launch_variant<false, 4, 3>},
    {"fwd2d 128x24 NS3 (8+4 warps)", launch_variant<false, 3, 3>},
};
static const Variant2D kAdj2D[] = {
    {"adj2d 128x32 NS3 (8+4 warps)", launch_variant<true, 3, 4>},
    {"adj2d 128x32 NS2 (8+4 warps)", launch_variant<true, 2, 4>},
    {"adj2d 128x24 NS3 (8+4 warps)", launch_variant<true, 3, 3>},
    {"adj2d 128x24 NS2 (8+4 warps)", launch_variant<true, 2, 3>},
};

int tile_rows2d(int sh) { return sh ? tile_rows2(3) : tile_rows2(4); }

int num_variants2d(bool adj) {
  return adj ? (int)(sizeof(kAdj2D) / sizeof(kAdj2D[0])) : (int)(sizeof(kFwd2D) / sizeof(kFwd2D[0]));
}

const char* variant2d_name(bool adj, int v) {
  if (v < 0 || v >= num_variants2d(adj)) return "invalid";
  return adj ? kAdj2D[v].name : kFwd2D[v].name;
}

cudaError_t launch_step2d(bool adj, int variant, const CUtensorMap& tm_halo, const CUtensorMap& tm_plain,
                          const CUtensorMap& tm_c, const Layout& L, const Coef& K, const StepParams& P, int nsamp,
                          cudaStream_t st) {
  if (variant < 0 || variant >= num_variants2d(adj)) variant = 0;
  return (adj ? kAdj2D[variant] : kFwd2D[variant]).fn(tm_halo, tm_plain, tm_c, L, K, P, nsamp, st);
}

}  // namespace fwi
