// stencil.cu -- time-step kernels of the damped 8th-order acoustic recursion
// and of its exact discrete adjoint with the imaging condition.
//
// Forward step (one launch per time step, all wavefields of the call):
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
// Tiling: work items are 128 x 32 (x, z) tiles of one posterior sample; a
// CTA processes an item for all of the sample's supergathers in a row, so the
// velocity coefficients and the imaging accumulator are loaded once per tile
// and reused across them.  Halo tiles (136 x 40) of p^n (and of the snapshot
// p^{k-1} in the adjoint) and the tile of p^{n-1} are fetched by TMA into a
// multi-stage shared-memory ring.  Each thread computes a 4 (x) x R (z) block:
// x-neighbours from two float4 shared loads per row, z-neighbours from an
// (R+8)-row float4 column window held in registers.
#include "fwi_internal.cuh"

namespace fwi {

template <bool ADJ, int NS>
struct Smem2D {
  static constexpr int IN = HZ * HX;   // floats in one halo tile
  static constexpr int PV = TZ * TX;   // floats in one plain tile
  static constexpr int STAGE = IN + PV + (ADJ ? IN : 0);
  static constexpr int nfloat = NS * STAGE;
  static constexpr int bytes = nfloat * 4 + 2 * NS * 8;  // + full and empty barriers
};

// Ring depth: the forward stage (38 KB) fits five times, the adjoint stage
// (59 KB, with the snapshot tile) three times, in one SM's shared memory.
constexpr int NS_FWD = 5;
constexpr int NS_ADJ = 3;
// Rows of the 4-wide block per consumer thread (8 consumer warps cover the
// 32-row tile with 16 points per thread).
constexpr int ROWS_PER_THREAD = 4;

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// 8th-order Laplacian of the 4 x R block whose top-left element sits at
// shared row r0+4, column c0+4 of a halo tile T (row stride HX).
template <int R>
__device__ __forceinline__ void lap_block(const float* __restrict__ T, int r0, int c0, const Coef& K,
                                          float (&lap)[R][4], float (&ctr)[R][4]) {
  float4 zc[R + 8];
#pragma unroll
  for (int i = 0; i < R + 8; i++) zc[i] = lds4(T + (r0 + i) * HX + c0 + 4);
  const float* zp = reinterpret_cast<const float*>(&zc[0]);  // zc[i] component j is zp[4*i + j]
#pragma unroll
  for (int r = 0; r < R; r++) {
    const float4 xl = lds4(T + (r0 + r + 4) * HX + c0);
    const float4 xr = lds4(T + (r0 + r + 4) * HX + c0 + 8);
    const float4 ce = zc[r + 4];
    const float w[12] = {xl.x, xl.y, xl.z, xl.w, ce.x, ce.y, ce.z, ce.w, xr.x, xr.y, xr.z, xr.w};
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const float p = w[4 + j], p2 = p + p;
      float sx = K.cx[4] * ((w[8 + j] + w[j]) - p2);
      sx = fmaf(K.cx[3], (w[7 + j] + w[1 + j]) - p2, sx);
      sx = fmaf(K.cx[2], (w[6 + j] + w[2 + j]) - p2, sx);
      sx = fmaf(K.cx[1], (w[5 + j] + w[3 + j]) - p2, sx);
      float sz = fmaf(K.cz[4], (zp[4 * (r + 8) + j] + zp[4 * r + j]) - p2, sx);
      sz = fmaf(K.cz[3], (zp[4 * (r + 7) + j] + zp[4 * (r + 1) + j]) - p2, sz);
      sz = fmaf(K.cz[2], (zp[4 * (r + 6) + j] + zp[4 * (r + 2) + j]) - p2, sz);
      sz = fmaf(K.cz[1], (zp[4 * (r + 5) + j] + zp[4 * (r + 3) + j]) - p2, sz);
      lap[r][j] = sz;
      ctr[r][j] = p;
    }
  }
}

// Sponge coefficients at padded (z, x): b = (1-g dt)/(1+g dt), inv = 1/(1+g dt).
__device__ __forceinline__ void sponge2d(const Layout& L, const Coef& K, int z, int x, float& b, float& inv) {
  const float dz = pad_depth(z, L.nz, L.nb) * K.inv_nb;
  const float dx = pad_depth(x, L.nx, L.nb) * K.inv_nb;
  const float gdt = K.gdt * (dz * dz + dx * dx);
  inv = __frcp_rn(1.0f + gdt);
  b = (1.0f - gdt) * inv;
}

// Persistent kernel with per-stage full/empty mbarriers.  One CTA per SM walks
// a flat sequence of iterations (work item k = tile of one sample, supergather
// j).  Every warp waits on the stage's "full" mbarrier (TMA transaction count),
// computes its rows, and releases the stage on its "empty" mbarrier (one
// arrival per warp).  Lane 0 of the last warp is the producer: at iteration it
// it waits until every warp has released iteration it-1 and refills that
// stage with iteration it-1+NS, so loads run NS-1 iterations ahead with no
// CTA-wide barrier in the loop (eight warps keep two per SM sub-partition,
// leaving each thread up to 255 registers).  Source injection and receiver
// sampling are staged by each warp in its own rows of the stage's p^{n-1}
// buffer, which it has already consumed.  The next item's velocity
// coefficients (and imaging accumulator) are prefetched into registers a
// whole item ahead.
template <bool ADJ, int NS, int R>
__global__ void __launch_bounds__(32 * (TZ / R), 1)
step2d_kernel(const __grid_constant__ CUtensorMap tm_halo, const __grid_constant__ CUtensorMap tm_plain,
              const Layout L, const Coef K, const StepParams P, int nitems) {
  using S = Smem2D<ADJ, NS>;
  constexpr int NCW = TZ / R;  // consumer warps
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + S::nfloat * 4);
  uint64_t* empty = full + NS;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = gridDim.x;
  const int my_items = (int)blockIdx.x < nitems ? (nitems - 1 - (int)blockIdx.x) / G + 1 : 0;
  const int n_it = my_items * P.nsg;
  if (n_it == 0) return;

  if (tid == 0) {
    tma_prefetch_desc(&tm_halo);
    tma_prefetch_desc(&tm_plain);
    for (int i = 0; i < NS; i++) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], NCW);
    }
    fence_mbar_init();
  }
  __syncthreads();
  (void)lane;

  // producer cursor (lane 0 of the last warp): (supergather, sample, tile) of the next load
  constexpr uint32_t TX_BYTES = (S::IN + S::PV + (ADJ ? S::IN : 0)) * 4;
  const bool producer = warp == NCW - 1 && lane == 0;
  int pj = 0, ps = 0, ptile = blockIdx.x, pit = 0;
  while (ptile >= P.ntiles) { ptile -= P.ntiles; ps++; }
  auto issue_next = [&]() {
    const int st = pit % NS;
    const int b = ps * P.nsg + pj;
    const int x0_ = (ptile % P.ntx) * TX, z0_ = (ptile / P.ntx) * TZ;
    float* base = sm + st * S::STAGE;
    mbar_arrive_expect_tx(&full[st], TX_BYTES);
    tma_load_4d(base, &tm_halo, x0_, z0_, b, P.s_cur, &full[st]);
    tma_load_4d(base + S::IN, &tm_plain, x0_ + HALO, z0_ + HALO, b, P.s_prev, &full[st]);
    if (ADJ) tma_load_4d(base + S::IN + S::PV, &tm_halo, x0_, z0_, b, P.s_snap, &full[st]);
    pit++;
    if (++pj == P.nsg) {
      pj = 0;
      ptile += G;
      while (ptile >= P.ntiles) { ptile -= P.ntiles; ps++; }
    }
  };
  if (producer)
    while (pit < NS && pit < n_it) issue_next();

  // ------------------------------------------------------------------ consumers
  const int lx = 4 * lane, lz = R * warp;
  float4 cpre[R], gpre[R];
  auto prefetch_item = [&](int s_, int tile_) {
    const int gx_ = (tile_ % P.ntx) * TX + lx, zb = (tile_ / P.ntx) * TZ + lz;
    const float* cs_ = P.c + (long long)s_ * L.field;
#pragma unroll
    for (int r = 0; r < R; r++) {
      const bool v = zb + r < L.nzp && gx_ < L.nxp;
      cpre[r] = v ? __ldg(reinterpret_cast<const float4*>(cs_ + L.off(zb + r, 0, gx_))) : make_float4(0.f, 0.f, 0.f, 0.f);
      if (ADJ)
        gpre[r] = v ? *reinterpret_cast<const float4*>(P.grad + (long long)s_ * L.field + L.off(zb + r, 0, gx_))
                    : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  int s = 0, tile = blockIdx.x;
  while (tile >= P.ntiles) { tile -= P.ntiles; s++; }
  prefetch_item(s, tile);
  int ns_ = s, ntile_ = tile;  // the item after the current one

  int x0 = 0, z0 = 0, gx = 0;
  bool rowv[R], colv0 = false;
  float cc[R][4], bc[R][4], gacc[R][4];
  const float* cs = P.c;
  int j = 0;
  for (int it = 0; it < n_it; it++) {
    const int st = it % NS;
    if (j == 0) {  // new work item: take the prefetched rows, prefetch the next item
      s = ns_;
      tile = ntile_;
      x0 = (tile % P.ntx) * TX;
      z0 = (tile / P.ntx) * TZ;
      gx = x0 + lx;
      colv0 = gx < L.nxp;
      cs = P.c + (long long)s * L.field;
      const bool sponge = L.nb > 0 && (x0 < L.nb || x0 + TX > L.nb + L.nx || z0 < L.nb || z0 + TZ > L.nb + L.nz);
#pragma unroll
      for (int r = 0; r < R; r++) {
        const int z = z0 + lz + r;
        rowv[r] = z < L.nzp;
        const float cvv[4] = {cpre[r].x, cpre[r].y, cpre[r].z, cpre[r].w};
#pragma unroll
        for (int q = 0; q < 4; q++) {
          float b = 1.f, inv = 1.f;
          if (sponge) sponge2d(L, K, z, gx + q, b, inv);
          bc[r][q] = b;
          cc[r][q] = cvv[q] * inv;
        }
        if (ADJ) {
          gacc[r][0] = gpre[r].x; gacc[r][1] = gpre[r].y; gacc[r][2] = gpre[r].z; gacc[r][3] = gpre[r].w;
        }
      }
      ntile_ = tile + G;
      ns_ = s;
      while (ntile_ >= P.ntiles) { ntile_ -= P.ntiles; ns_++; }
      if (it + P.nsg < n_it) prefetch_item(ns_, ntile_);
    }
    const int b = s * P.nsg + j;
    if (producer && it >= 1 && pit < n_it) {
      // refill the stage released by iteration it-1 once every warp has released it
      if (!mbar_wait_bounded(&empty[(it - 1) % NS], ((it - 1) / NS) & 1, P.status)) return;
      issue_next();
    }
    if (!mbar_wait_bounded(&full[st], (it / NS) & 1, P.status)) return;

    float* I = sm + st * S::STAGE;
    float* PV = I + S::IN;
    float lap[R][4], ctr[R][4], nv[R][4];
    lap_block<R>(I, lz, lx, K, lap, ctr);
#pragma unroll
    for (int r = 0; r < R; r++) {
      const float4 pm = lds4(PV + (lz + r) * TX + lx);
      const float pmv[4] = {pm.x, pm.y, pm.z, pm.w};
#pragma unroll
      for (int q = 0; q < 4; q++)
        nv[r][q] = fmaf(cc[r][q], lap[r][q], fmaf(bc[r][q], ctr[r][q] - pmv[q], ctr[r][q]));
    }

    // Injection (sources in the forward, residual at receivers in the adjoint)
    // and sampling (receivers in the forward, sources in the adjoint), staged
    // in this warp's own rows of PV.
    const int ib = P.inj_off[b * P.inj_bstride + tile], ie = P.inj_off[b * P.inj_bstride + tile + 1];
    int sb = 0, se = 0;
    if (P.smp) {
      sb = P.smp_off[b * P.smp_bstride + tile];
      se = P.smp_off[b * P.smp_bstride + tile + 1];
    }
    if (ie > ib || se > sb) {
      __syncwarp();
#pragma unroll
      for (int r = 0; r < R; r++)
        *reinterpret_cast<float4*>(PV + (lz + r) * TX + lx) = make_float4(nv[r][0], nv[r][1], nv[r][2], nv[r][3]);
      __syncwarp();
      for (int e = ib + lane; e < ie; e += 32) {
        const int4 en = P.inj[e];
        const int rz = en.x / TX;
        if (rz < lz || rz >= lz + R) continue;
        const int zz = z0 + rz, xx = x0 + en.x % TX;
        float bb, inv;
        sponge2d(L, K, zz, xx, bb, inv);
        const float ccp = __ldg(cs + L.off(zz, 0, xx)) * inv;
        PV[en.x] += ccp * (__int_as_float(en.z) *
                           P.series[(long long)b * P.series_bstride + (long long)P.t * P.series_ld + en.y]);
      }
      __syncwarp();
#pragma unroll
      for (int r = 0; r < R; r++) {
        const float4 v = lds4(PV + (lz + r) * TX + lx);
        nv[r][0] = v.x; nv[r][1] = v.y; nv[r][2] = v.z; nv[r][3] = v.w;
      }
      for (int e = sb + lane; e < se; e += 32) {
        const int2 en = P.smp[e];
        const int rz = en.x / TX;
        if (rz < lz || rz >= lz + R) continue;
        P.smp_out[(long long)b * P.smp_bstride_out + (long long)P.t * P.smp_ld + en.y] = PV[en.x];
      }
      // generic-proxy writes to the stage must be ordered before the TMA that refills it
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }

    if (ADJ) {
      float lps[R][4], dummy[R][4];
      lap_block<R>(I + S::IN + S::PV, lz, lx, K, lps, dummy);
#pragma unroll
      for (int r = 0; r < R; r++)
#pragma unroll
        for (int q = 0; q < 4; q++) gacc[r][q] = fmaf(nv[r][q], lps[r][q], gacc[r][q]);
    }
    // all reads of the stage by this warp are done
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);

    float* outp = P.pool + (long long)P.s_out * P.slot_elems + (long long)b * L.field;
#pragma unroll
    for (int r = 0; r < R; r++) {
      if (!rowv[r] || !colv0) continue;
      float* o = outp + L.off(z0 + lz + r, 0, gx);
      if (gx + 3 < L.nxp) {
        *reinterpret_cast<float4*>(o) = make_float4(nv[r][0], nv[r][1], nv[r][2], nv[r][3]);
      } else {
#pragma unroll
        for (int q = 0; q < 4; q++)
          if (gx + q < L.nxp) o[q] = nv[r][q];
      }
    }
    if (++j == P.nsg) {
      j = 0;
      if (ADJ) {
        float* gs = P.grad + (long long)s * L.field;
#pragma unroll
        for (int r = 0; r < R; r++) {
          if (!rowv[r] || !colv0) continue;
          float* o = gs + L.off(z0 + lz + r, 0, gx);
          if (gx + 3 < L.nxp) {
            *reinterpret_cast<float4*>(o) = make_float4(gacc[r][0], gacc[r][1], gacc[r][2], gacc[r][3]);
          } else {
#pragma unroll
            for (int q = 0; q < 4; q++)
              if (gx + q < L.nxp) o[q] = gacc[r][q];
          }
        }
      }
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

cudaError_t launch_step2d(bool adj, const CUtensorMap& tm_halo, const CUtensorMap& tm_plain,
                          const Layout& L, const Coef& K, const StepParams& P, int nsamp, cudaStream_t st) {
  static bool attr_set[2] = {false, false};
  const int nitems = P.ntiles * nsamp;
  const int grid = nitems < num_sms() ? nitems : num_sms();
  constexpr int R = ROWS_PER_THREAD;
  constexpr int NT = 32 * (TZ / R);
  if (adj) {
    using S = Smem2D<true, NS_ADJ>;
    if (!attr_set[1]) {
      cudaFuncSetAttribute(step2d_kernel<true, NS_ADJ, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::bytes);
      attr_set[1] = true;
    }
    step2d_kernel<true, NS_ADJ, R><<<grid, NT, S::bytes, st>>>(tm_halo, tm_plain, L, K, P, nitems);
  } else {
    using S = Smem2D<false, NS_FWD>;
    if (!attr_set[0]) {
      cudaFuncSetAttribute(step2d_kernel<false, NS_FWD, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::bytes);
      attr_set[0] = true;
    }
    step2d_kernel<false, NS_FWD, R><<<grid, NT, S::bytes, st>>>(tm_halo, tm_plain, L, K, P, nitems);
  }
  return cudaGetLastError();
}

}  // namespace fwi
