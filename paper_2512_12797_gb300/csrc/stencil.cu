// stencil.cu -- time-step kernels of the damped 8th-order acoustic recursion
// and of its exact discrete adjoint with the imaging condition.
//
// Forward step (one launch per time step, all wavefields of the call):
//     p^{n+1} = p^n + b (p^n - p^{n-1}) + cc (L p^n + s^n)
// with b = (1 - gamma dt)/(1 + gamma dt), cc = v^2 dt^2/(1 + gamma dt).  This is
// the damped leapfrog p^{n+1} = [2p^n - (1-gamma dt)p^{n-1} + c(Lp^n + s^n)]/(1+gamma dt)
// rewritten with 2/(1+gamma dt) = 1 + b, which keeps the FP32 recursion free of
// the spurious growth that rounding 2/(1+gamma dt) and b separately introduces
// in the sponge.  L is evaluated as sum_k a_k/h^2 [(p_{+k} - p) + (p_{-k} - p)],
// which equals the textbook 8th-order form because a_0 = -2 sum_k a_k, and keeps
// L(constant) = 0 exactly in FP32.
//
// Adjoint step: with q = cc * lambda the transpose of the recursion above is the
// same recursion, driven by cc * R^T dJ/dd at the receivers:
//     q^k = q^{k+1} + b (q^{k+1} - q^{k+2}) + cc (L q^{k+1} + R^T rhat^{k-1}),
// and the imaging condition dJ/dc = (1/c) sum_n q^{n+1} (L p^n + s^n) is
// accumulated here as G += q^k * L p^{k-1} (the source term is added from
// source-point samples after the time loop).
//
// Tiling: a CTA owns a 128 x 32 (x, z) tile of one posterior sample and loops
// over the sample's supergathers, so the velocity coefficients and the
// imaging accumulator are loaded once per tile and reused across them.  Halo
// tiles (136 x 40) of p^n (and of the snapshot p^{k-1} in the adjoint) and
// the tile of p^{n-1} are fetched by TMA into a two-stage shared-memory ring,
// one stage ahead of the compute.  Each thread computes a 4 (x) x 4 (z) block:
// x-neighbours from two float4 shared loads per row, z-neighbours from a
// 12-row float4 column window held in registers.
#include "fwi_internal.cuh"

namespace fwi {

template <bool ADJ>
struct Smem2D {
  static constexpr int IN = HZ * HX;   // floats in one halo tile
  static constexpr int PV = TZ * TX;   // floats in one plain tile
  static constexpr int off_prev = 2 * IN;
  static constexpr int off_snap = off_prev + 2 * PV;
  static constexpr int nfloat = off_snap + (ADJ ? 2 * IN : 0);
  static constexpr int bytes = nfloat * 4 + 2 * 8;
};

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// 8th-order Laplacian of the 4x4 block whose top-left element sits at shared
// row r0+4, column c0+4 of a halo tile T (row stride HX).
__device__ __forceinline__ void lap_block(const float* __restrict__ T, int r0, int c0, const Coef& K,
                                          float (&lap)[RZ][4], float (&ctr)[RZ][4]) {
  float4 zc[RZ + 8];
#pragma unroll
  for (int i = 0; i < RZ + 8; i++) zc[i] = lds4(T + (r0 + i) * HX + c0 + 4);
#pragma unroll
  for (int r = 0; r < RZ; r++) {
    const float4 xl = lds4(T + (r0 + r + 4) * HX + c0);
    const float4 xr = lds4(T + (r0 + r + 4) * HX + c0 + 8);
    const float4 ce = zc[r + 4];
    const float w[12] = {xl.x, xl.y, xl.z, xl.w, ce.x, ce.y, ce.z, ce.w, xr.x, xr.y, xr.z, xr.w};
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const float p = w[4 + j];
      float sx = K.cx[4] * ((w[8 + j] - p) + (w[j] - p));
      sx = fmaf(K.cx[3], (w[7 + j] - p) + (w[1 + j] - p), sx);
      sx = fmaf(K.cx[2], (w[6 + j] - p) + (w[2 + j] - p), sx);
      sx = fmaf(K.cx[1], (w[5 + j] - p) + (w[3 + j] - p), sx);
      const float* zp = reinterpret_cast<const float*>(&zc[0]);
      // zc[i] component j is zp[4*i + j]
      float sz = K.cz[4] * ((zp[4 * (r + 8) + j] - p) + (zp[4 * r + j] - p));
      sz = fmaf(K.cz[3], (zp[4 * (r + 7) + j] - p) + (zp[4 * (r + 1) + j] - p), sz);
      sz = fmaf(K.cz[2], (zp[4 * (r + 6) + j] - p) + (zp[4 * (r + 2) + j] - p), sz);
      sz = fmaf(K.cz[1], (zp[4 * (r + 5) + j] - p) + (zp[4 * (r + 3) + j] - p), sz);
      lap[r][j] = sx + sz;
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

template <bool ADJ>
__global__ void __launch_bounds__(NTHREADS, 1)
step2d_kernel(const __grid_constant__ CUtensorMap tm_halo, const __grid_constant__ CUtensorMap tm_plain,
              const Layout L, const Coef K, const StepParams P) {
  using S = Smem2D<ADJ>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float* s_in = reinterpret_cast<float*>(smem_raw);
  float* s_prev = s_in + S::off_prev;
  float* s_snap = s_in + S::off_snap;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + S::nfloat * 4);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int x0 = blockIdx.x * TX, z0 = blockIdx.y * TZ, s = blockIdx.z;
  const int tile = blockIdx.y * P.ntx + blockIdx.x;
  const int lx = 4 * lane, lz = RZ * warp;
  const int gx = x0 + lx;

  if (tid == 0) {
    tma_prefetch_desc(&tm_halo);
    tma_prefetch_desc(&tm_plain);
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();

  constexpr uint32_t TX_BYTES = (S::IN + S::PV + (ADJ ? S::IN : 0)) * 4;
  auto issue = [&](int j) {
    const int st = j & 1, b = s * P.nsg + j;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(&bar[st], TX_BYTES);
    tma_load_4d(s_in + st * S::IN, &tm_halo, x0, z0, b, P.s_cur, &bar[st]);
    tma_load_4d(s_prev + st * S::PV, &tm_plain, x0 + HALO, z0 + HALO, b, P.s_prev, &bar[st]);
    if (ADJ) tma_load_4d(s_snap + st * S::IN, &tm_halo, x0, z0, b, P.s_snap, &bar[st]);
  };
  if (tid == 0) issue(0);

  // Per-point coefficients of this thread's 4x4 block (shared by all supergathers).
  bool rowv[RZ];
  const bool colv0 = gx < L.nxp;
  float cc[RZ][4], bc[RZ][4];
  const float* cs = P.c + (long long)s * L.field;
#pragma unroll
  for (int r = 0; r < RZ; r++) {
    const int z = z0 + lz + r;
    rowv[r] = z < L.nzp;
    float4 cv = make_float4(0.f, 0.f, 0.f, 0.f);
    if (rowv[r] && colv0) cv = __ldg(reinterpret_cast<const float4*>(cs + L.off(z, 0, gx)));
    const float cvv[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
    for (int j = 0; j < 4; j++) {
      float b, inv;
      sponge2d(L, K, z, gx + j, b, inv);
      bc[r][j] = b;
      cc[r][j] = cvv[j] * inv;
    }
  }
  float gacc[RZ][4];
  float* gs = ADJ ? P.grad + (long long)s * L.field : nullptr;
  if (ADJ) {
#pragma unroll
    for (int r = 0; r < RZ; r++) {
      float4 gv = make_float4(0.f, 0.f, 0.f, 0.f);
      if (rowv[r] && colv0) gv = *reinterpret_cast<const float4*>(gs + L.off(z0 + lz + r, 0, gx));
      gacc[r][0] = gv.x; gacc[r][1] = gv.y; gacc[r][2] = gv.z; gacc[r][3] = gv.w;
    }
  }

  for (int j = 0; j < P.nsg; j++) {
    const int st = j & 1, b = s * P.nsg + j;
    if (tid == 0 && j + 1 < P.nsg) issue(j + 1);
    const bool ok = mbar_wait_bounded(&bar[st], (j >> 1) & 1, P.status);
    if (__syncthreads_or(!ok)) return;

    const float* I = s_in + st * S::IN;
    float* PV = s_prev + st * S::PV;
    float lap[RZ][4], ctr[RZ][4], nv[RZ][4];
    lap_block(I, lz, lx, K, lap, ctr);
#pragma unroll
    for (int r = 0; r < RZ; r++) {
      const float4 pm = lds4(PV + (lz + r) * TX + lx);
      const float pmv[4] = {pm.x, pm.y, pm.z, pm.w};
#pragma unroll
      for (int q = 0; q < 4; q++)
        nv[r][q] = fmaf(cc[r][q], lap[r][q], fmaf(bc[r][q], ctr[r][q] - pmv[q], ctr[r][q]));
    }

    // Injection (sources in the forward, residual at receivers in the adjoint)
    // and sampling (receivers in the forward, sources in the adjoint).
    const int ib = P.inj_off[b * P.inj_bstride + tile], ie = P.inj_off[b * P.inj_bstride + tile + 1];
    int sb = 0, se = 0;
    if (P.smp) {
      sb = P.smp_off[b * P.smp_bstride + tile];
      se = P.smp_off[b * P.smp_bstride + tile + 1];
    }
    if (ie > ib || se > sb) {
      __syncthreads();  // all reads of PV done: reuse it as the output staging tile
#pragma unroll
      for (int r = 0; r < RZ; r++)
        *reinterpret_cast<float4*>(PV + (lz + r) * TX + lx) = make_float4(nv[r][0], nv[r][1], nv[r][2], nv[r][3]);
      __syncthreads();
      for (int e = ib + tid; e < ie; e += NTHREADS) {
        const int4 en = P.inj[e];
        const int zz = z0 + en.x / TX, xx = x0 + en.x % TX;
        float bb, inv;
        sponge2d(L, K, zz, xx, bb, inv);
        const float ccp = __ldg(cs + L.off(zz, 0, xx)) * inv;
        PV[en.x] += ccp * (__int_as_float(en.z) *
                           P.series[(long long)b * P.series_bstride + (long long)P.t * P.series_ld + en.y]);
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < RZ; r++) {
        const float4 v = lds4(PV + (lz + r) * TX + lx);
        nv[r][0] = v.x; nv[r][1] = v.y; nv[r][2] = v.z; nv[r][3] = v.w;
      }
      for (int e = sb + tid; e < se; e += NTHREADS) {
        const int2 en = P.smp[e];
        P.smp_out[(long long)b * P.smp_bstride_out + (long long)P.t * P.smp_ld + en.y] = PV[en.x];
      }
    }

    if (ADJ) {
      float lps[RZ][4], dummy[RZ][4];
      lap_block(s_snap + st * S::IN, lz, lx, K, lps, dummy);
#pragma unroll
      for (int r = 0; r < RZ; r++)
#pragma unroll
        for (int q = 0; q < 4; q++) gacc[r][q] = fmaf(nv[r][q], lps[r][q], gacc[r][q]);
    }

    float* outp = P.pool + (long long)P.s_out * P.slot_elems + (long long)b * L.field;
#pragma unroll
    for (int r = 0; r < RZ; r++) {
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
    __syncthreads();  // stage st is free for the load issued at iteration j+1
  }

  if (ADJ) {
#pragma unroll
    for (int r = 0; r < RZ; r++) {
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

cudaError_t launch_step2d(bool adj, const CUtensorMap& tm_halo, const CUtensorMap& tm_plain,
                          const Layout& L, const Coef& K, const StepParams& P, int nsamp, cudaStream_t st) {
  static bool attr_set[2] = {false, false};
  dim3 grid(P.ntx, P.ntiles / P.ntx, nsamp);
  if (adj) {
    if (!attr_set[1]) {
      cudaFuncSetAttribute(step2d_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem2D<true>::bytes);
      attr_set[1] = true;
    }
    step2d_kernel<true><<<grid, NTHREADS, Smem2D<true>::bytes, st>>>(tm_halo, tm_plain, L, K, P);
  } else {
    if (!attr_set[0]) {
      cudaFuncSetAttribute(step2d_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem2D<false>::bytes);
      attr_set[0] = true;
    }
    step2d_kernel<false><<<grid, NTHREADS, Smem2D<false>::bytes, st>>>(tm_halo, tm_plain, L, K, P);
  }
  return cudaGetLastError();
}

}  // namespace fwi
