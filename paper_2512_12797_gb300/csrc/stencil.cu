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

// One ring stage: halo tile of the field being stepped, plain tile of the older
// level, [halo tile of the snapshot], plain tile of cc (filled for the first
// supergather of a work item), and the four point-list offsets of the
// iteration (inj begin/end, smp begin/end).  Every part starts on 128 bytes.
template <bool ADJ, int NS>
struct Smem2D {
  static constexpr int IN = HZ * HX;   // floats in one halo tile
  static constexpr int PV = TZ * TX;   // floats in one plain tile
  static constexpr int OFF_SNAP = IN + PV;
  static constexpr int OFF_C = OFF_SNAP + (ADJ ? IN : 0);
  static constexpr int OFF_IDX = OFF_C + PV;
  static constexpr int STAGE = OFF_IDX + 32;
  static constexpr int nfloat = NS * STAGE;
  static constexpr int bytes = nfloat * 4 + 2 * NS * 8;  // + full and empty barriers
};

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// 8th-order Laplacian of the 4 x R block whose top-left element sits at
// shared row r0+4, column c0+4 of a halo tile T (row stride HX).  With
// ISO (hx == hz) the two axes share coefficients and each k costs one bracket
// [(x_{+k} + x_{-k}) + (z_{+k} + z_{-k}) - 4p], also exactly zero for a
// constant field.
template <int R, bool ISO>
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
      const float p = w[4 + j];
      if (ISO) {
        const float p4 = 4.f * p;
        float a = K.cx[4] * (((w[8 + j] + w[j]) + (zp[4 * (r + 8) + j] + zp[4 * r + j])) - p4);
        a = fmaf(K.cx[3], ((w[7 + j] + w[1 + j]) + (zp[4 * (r + 7) + j] + zp[4 * (r + 1) + j])) - p4, a);
        a = fmaf(K.cx[2], ((w[6 + j] + w[2 + j]) + (zp[4 * (r + 6) + j] + zp[4 * (r + 2) + j])) - p4, a);
        a = fmaf(K.cx[1], ((w[5 + j] + w[3 + j]) + (zp[4 * (r + 5) + j] + zp[4 * (r + 3) + j])) - p4, a);
        lap[r][j] = a;
      } else {
        const float p2 = p + p;
        float sx = K.cx[4] * ((w[8 + j] + w[j]) - p2);
        sx = fmaf(K.cx[3], (w[7 + j] + w[1 + j]) - p2, sx);
        sx = fmaf(K.cx[2], (w[6 + j] + w[2 + j]) - p2, sx);
        sx = fmaf(K.cx[1], (w[5 + j] + w[3 + j]) - p2, sx);
        float sz = fmaf(K.cz[4], (zp[4 * (r + 8) + j] + zp[4 * r + j]) - p2, sx);
        sz = fmaf(K.cz[3], (zp[4 * (r + 7) + j] + zp[4 * (r + 1) + j]) - p2, sz);
        sz = fmaf(K.cz[2], (zp[4 * (r + 6) + j] + zp[4 * (r + 2) + j]) - p2, sz);
        sz = fmaf(K.cz[1], (zp[4 * (r + 5) + j] + zp[4 * (r + 3) + j]) - p2, sz);
        lap[r][j] = sz;
      }
      ctr[r][j] = p;
    }
  }
}

// Persistent kernel with per-stage full/empty mbarriers.  One CTA per SM walks
// its work items (item = tile of one sample) and, inside each, the sample's
// supergathers; iteration number it counts (item, supergather) pairs.  Every
// warp waits on the stage's "full" mbarrier (TMA transaction count plus one
// arrival from the cp.async copy of the iteration's point-list offsets),
// computes its rows and releases the stage on its "empty" mbarrier (one
// arrival per warp).  Lane 0 of the last warp is also the producer: it refills
// a stage as soon as every warp has released it, testing the empty barrier
// without blocking, and blocks only when the iteration its own warp needs next
// has not been issued yet, so loads run up to NS-1 iterations ahead with no
// CTA-wide barrier in the loop.  The cc tile of an item travels with the
// item's first supergather; sponge coefficients come from per-axis gamma*dt
// tables.  Source injection and receiver sampling are staged by each warp in
// its own rows of the stage's p^{n-1} buffer, which it has already consumed.
template <bool ADJ, int NS, int R, bool ISO>
__global__ void __launch_bounds__(32 * (TZ / R), 1)
step2d_kernel(const __grid_constant__ CUtensorMap tm_halo, const __grid_constant__ CUtensorMap tm_plain,
              const __grid_constant__ CUtensorMap tm_c, const Layout L, const Coef K, const StepParams P,
              int nitems) {
  using S = Smem2D<ADJ, NS>;
  constexpr int NCW = TZ / R;  // warps
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + S::nfloat * 4);
  uint64_t* empty = full + NS;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = gridDim.x;
  const int my_items = (int)blockIdx.x < nitems ? (nitems - 1 - (int)blockIdx.x) / G + 1 : 0;
  const int nsg = P.nsg;
  const int n_it = my_items * nsg;
  if (n_it == 0) return;

  if (tid == 0) {
    tma_prefetch_desc(&tm_halo);
    tma_prefetch_desc(&tm_plain);
    tma_prefetch_desc(&tm_c);
    for (int i = 0; i < NS; i++) {
      mbar_init(&full[i], 2);  // producer's expect_tx arrival + cp.async arrival
      mbar_init(&empty[i], NCW);
    }
    fence_mbar_init();
  }
  __syncthreads();

  // ---------------------------------------------------------------- producer
  constexpr uint32_t TX_BYTES = (S::IN + S::PV + (ADJ ? S::IN : 0)) * 4;
  const bool producer = warp == NCW - 1 && lane == 0;
  int pit = 0, pst = 0, pj = 0, ps = 0, ptile = blockIdx.x;
  uint32_t pround = 0;  // parity of the ring round of the next load
  while (ptile >= P.ntiles) { ptile -= P.ntiles; ps++; }
  auto issue_next = [&]() {
    const int b = ps * nsg + pj;
    const int x0_ = (ptile % P.ntx) * TX, z0_ = (ptile / P.ntx) * TZ;
    float* base = sm + pst * S::STAGE;
    int* idx = reinterpret_cast<int*>(base + S::OFF_IDX);
    const int* io = P.inj_off + b * P.inj_bstride + ptile;
    const int* so = P.smp_off + b * P.smp_bstride + ptile;
    cp_async4(idx + 0, io);
    cp_async4(idx + 1, io + 1);
    cp_async4(idx + 2, so);
    cp_async4(idx + 3, so + 1);
    cp_async_arrive(&full[pst]);
    mbar_arrive_expect_tx(&full[pst], TX_BYTES + (pj == 0 ? S::PV * 4 : 0));
    tma_load_4d(base, &tm_halo, x0_, z0_, b, P.s_cur, &full[pst]);
    tma_load_4d(base + S::IN, &tm_plain, x0_ + HALO, z0_ + HALO, b, P.s_prev, &full[pst]);
    if (ADJ) tma_load_4d(base + S::OFF_SNAP, &tm_halo, x0_, z0_, b, P.s_snap, &full[pst]);
    if (pj == 0) tma_load_3d(base + S::OFF_C, &tm_c, x0_ + HALO, z0_ + HALO, ps, &full[pst]);
    pit++;
    if (++pst == NS) { pst = 0; pround ^= 1; }
    if (++pj == nsg) {
      pj = 0;
      ptile += G;
      while (ptile >= P.ntiles) { ptile -= P.ntiles; ps++; }
    }
  };
  // Refill every stage whose previous occupant all warps have released; block
  // only for the load of iteration `need` (the one this warp waits on next).
  auto refill = [&](int need) -> bool {
    while (pit < n_it && pit < need + NS) {
      if (pit >= NS) {
        if (pit <= need) {
          if (!mbar_wait_bounded(&empty[pst], pround ^ 1, P.status)) return false;
        } else if (!mbar_try_wait(&empty[pst], pround ^ 1)) {
          break;
        }
      }
      issue_next();
    }
    return true;
  };

  // ------------------------------------------------------------------ consumers
  const int lx = 4 * lane, lz = R * warp;
  const float* gzt = P.gtab;
  const float* gxt = P.gtab + L.nzp + L.nyp;
  // next item's imaging accumulator rows (adjoint) and sponge table entries
  float4 gpre[R];
  float gzpre[R], gxpre[4];
  auto prefetch_item = [&](int s_, int tile_) {
    const int gx_ = (tile_ % P.ntx) * TX + lx, zb = (tile_ / P.ntx) * TZ + lz;
#pragma unroll
    for (int r = 0; r < R; r++) {
      const bool v = zb + r < L.nzp && gx_ < L.nxp;
      gzpre[r] = zb + r < L.nzp ? __ldg(gzt + zb + r) : 0.f;
      if (ADJ)
        gpre[r] = v ? *reinterpret_cast<const float4*>(P.grad + (long long)s_ * L.field + L.off(zb + r, 0, gx_))
                    : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < 4; q++) gxpre[q] = gx_ + q < L.nxp ? __ldg(gxt + gx_ + q) : 0.f;
  };
  int s = 0, tile = blockIdx.x;
  while (tile >= P.ntiles) { tile -= P.ntiles; s++; }
  prefetch_item(s, tile);

  int st = 0;
  uint32_t round = 0;
  int it = 0;
  for (int k = 0; k < my_items; k++) {
    // ---- new work item: sponge coefficients, output base, prefetch of the next item
    const int x0 = (tile % P.ntx) * TX, z0 = (tile / P.ntx) * TZ;
    const int gx = x0 + lx;
    const bool colv0 = gx < L.nxp, live = z0 + lz < L.nzp;
    const bool sponge = L.nb > 0 && (x0 < L.nb || x0 + TX > L.nb + L.nx || z0 < L.nb || z0 + TZ > L.nb + L.nz);
    bool rowv[R];
    float cc[R][4], bc[R][4], gacc[R][4];
#pragma unroll
    for (int r = 0; r < R; r++) {
      rowv[r] = z0 + lz + r < L.nzp;
#pragma unroll
      for (int q = 0; q < 4; q++) bc[r][q] = sponge ? sponge_b(gzpre[r] + gxpre[q]) : 1.f;
      if (ADJ) {
        gacc[r][0] = gpre[r].x; gacc[r][1] = gpre[r].y; gacc[r][2] = gpre[r].z; gacc[r][3] = gpre[r].w;
      }
    }
    const long long row0 = L.off(z0 + lz, 0, gx);
    float* obase = P.pool + (long long)P.s_out * P.slot_elems + (long long)s * nsg * L.field + row0;
    int ntile = tile + G, ns_ = s;
    while (ntile >= P.ntiles) { ntile -= P.ntiles; ns_++; }
    if (k + 1 < my_items) prefetch_item(ns_, ntile);

    for (int j = 0; j < nsg; j++, it++) {
      const int b = s * nsg + j;
      if (producer && !refill(it)) return;
      if (!mbar_wait_bounded(&full[st], round, P.status)) return;

      float* I = sm + st * S::STAGE;
      float* PV = I + S::IN;
      const int4 off = *reinterpret_cast<const int4*>(I + S::OFF_IDX);
      if (j == 0) {
#pragma unroll
        for (int r = 0; r < R; r++) {
          const float4 c4 = lds4(I + S::OFF_C + (lz + r) * TX + lx);
          cc[r][0] = c4.x; cc[r][1] = c4.y; cc[r][2] = c4.z; cc[r][3] = c4.w;
        }
      }
      if (live) {
        float lap[R][4], ctr[R][4], nv[R][4];
        lap_block<R, ISO>(I, lz, lx, K, lap, ctr);
#pragma unroll
        for (int r = 0; r < R; r++) {
          const float4 pm = lds4(PV + (lz + r) * TX + lx);
          const float pmv[4] = {pm.x, pm.y, pm.z, pm.w};
#pragma unroll
          for (int q = 0; q < 4; q++)
            nv[r][q] = fmaf(cc[r][q], lap[r][q], fmaf(bc[r][q], ctr[r][q] - pmv[q], ctr[r][q]));
        }
        // Injection (sources in the forward, residual at receivers in the
        // adjoint) and sampling (receivers in the forward, sources in the
        // adjoint), staged in this warp's own rows of PV.
        if (off.y > off.x || off.w > off.z) {
          __syncwarp();
#pragma unroll
          for (int r = 0; r < R; r++)
            *reinterpret_cast<float4*>(PV + (lz + r) * TX + lx) = make_float4(nv[r][0], nv[r][1], nv[r][2], nv[r][3]);
          __syncwarp();
          for (int e = off.x + lane; e < off.y; e += 32) {
            const int4 en = P.inj[e];
            const int rz = en.x / TX;
            if (rz < lz || rz >= lz + R) continue;
            const float ccp = __ldg(P.c + (long long)s * L.field + L.off(z0 + rz, 0, x0 + en.x % TX));
            PV[en.x] += ccp * (__int_as_float(en.z) *
                               P.series[(long long)b * P.series_bstride + (long long)P.t * P.series_ld + en.y]);
          }
          __syncwarp();
#pragma unroll
          for (int r = 0; r < R; r++) {
            const float4 v = lds4(PV + (lz + r) * TX + lx);
            nv[r][0] = v.x; nv[r][1] = v.y; nv[r][2] = v.z; nv[r][3] = v.w;
          }
          for (int e = off.z + lane; e < off.w; e += 32) {
            const int2 en = P.smp[e];
            const int rz = en.x / TX;
            if (rz < lz || rz >= lz + R) continue;
            P.smp_out[(long long)b * P.smp_bstride_out + (long long)P.t * P.smp_ld + en.y] = PV[en.x];
          }
          // generic-proxy writes to the stage are ordered before the TMA that refills it
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        if (ADJ) {
          float lps[R][4], dummy[R][4];
          lap_block<R, ISO>(I + S::OFF_SNAP, lz, lx, K, lps, dummy);
#pragma unroll
          for (int r = 0; r < R; r++)
#pragma unroll
            for (int q = 0; q < 4; q++) gacc[r][q] = fmaf(nv[r][q], lps[r][q], gacc[r][q]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
        float* o = obase + (long long)j * L.field;
#pragma unroll
        for (int r = 0; r < R; r++) {
          if (!rowv[r] || !colv0) continue;
          if (gx + 3 < L.nxp) {
            *reinterpret_cast<float4*>(o + r * L.SX) = make_float4(nv[r][0], nv[r][1], nv[r][2], nv[r][3]);
          } else {
#pragma unroll
            for (int q = 0; q < 4; q++)
              if (gx + q < L.nxp) o[r * L.SX + q] = nv[r][q];
          }
        }
      } else {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
      }
      if (++st == NS) { st = 0; round ^= 1; }
    }
    if (ADJ && live) {
      float* o = P.grad + (long long)s * L.field + row0;
#pragma unroll
      for (int r = 0; r < R; r++) {
        if (!rowv[r] || !colv0) continue;
        if (gx + 3 < L.nxp) {
          *reinterpret_cast<float4*>(o + r * L.SX) = make_float4(gacc[r][0], gacc[r][1], gacc[r][2], gacc[r][3]);
        } else {
#pragma unroll
          for (int q = 0; q < 4; q++)
            if (gx + q < L.nxp) o[r * L.SX + q] = gacc[r][q];
        }
      }
    }
    s = ns_;
    tile = ntile;
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

// Compiled variants (R rows per thread, i.e. 32*32/R threads; ring depth NS).  The
// arithmetic per grid point is the same in every variant, so their results
// are bit-identical; the autotuner in fwi_api.cu picks the fastest per call shape.
template <bool ADJ, int NS, int R, bool ISO>
static cudaError_t launch_iso(const CUtensorMap& th, const CUtensorMap& tp, const CUtensorMap& tc, const Layout& L,
                              const Coef& K, const StepParams& P, int nsamp, cudaStream_t st) {
  using S = Smem2D<ADJ, NS>;
  constexpr int NT = 32 * (TZ / R);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(step2d_kernel<ADJ, NS, R, ISO>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, S::bytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int nitems = P.ntiles * nsamp;
  const int grid = nitems < num_sms() ? nitems : num_sms();
  step2d_kernel<ADJ, NS, R, ISO><<<grid, NT, S::bytes, st>>>(th, tp, tc, L, K, P, nitems);
  return cudaGetLastError();
}

template <bool ADJ, int NS, int R>
static cudaError_t launch_variant(const CUtensorMap& th, const CUtensorMap& tp, const CUtensorMap& tc,
                                  const Layout& L, const Coef& K, const StepParams& P, int nsamp, cudaStream_t st) {
  if (K.cx[1] == K.cz[1] && K.cx[2] == K.cz[2] && K.cx[3] == K.cz[3] && K.cx[4] == K.cz[4])
    return launch_iso<ADJ, NS, R, true>(th, tp, tc, L, K, P, nsamp, st);
  return launch_iso<ADJ, NS, R, false>(th, tp, tc, L, K, P, nsamp, st);
}

struct Variant2D {
  const char* name;
  cudaError_t (*fn)(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const Layout&, const Coef&,
                    const StepParams&, int, cudaStream_t);
};

static const Variant2D kFwd2D[] = {
    {"fwd2d R4 NS4 (8 warps)", launch_variant<false, 4, 4>},
    {"fwd2d R4 NS3 (8 warps)", launch_variant<false, 3, 4>},
    {"fwd2d R2 NS4 (16 warps)", launch_variant<false, 4, 2>},
    {"fwd2d R2 NS3 (16 warps)", launch_variant<false, 3, 2>},
};
static const Variant2D kAdj2D[] = {
    {"adj2d R4 NS3 (8 warps)", launch_variant<true, 3, 4>},
    {"adj2d R4 NS2 (8 warps)", launch_variant<true, 2, 4>},
    {"adj2d R2 NS3 (16 warps)", launch_variant<true, 3, 2>},
    {"adj2d R2 NS2 (16 warps)", launch_variant<true, 2, 2>},
};

int num_variants2d(bool adj) { return adj ? (int)(sizeof(kAdj2D) / sizeof(kAdj2D[0])) : (int)(sizeof(kFwd2D) / sizeof(kFwd2D[0])); }

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
