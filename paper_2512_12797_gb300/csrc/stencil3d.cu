// stencil3d.cu -- 3D time-step kernels (forward recursion; adjoint recursion
// with the imaging condition), same algebra as the 2D kernels in stencil.cu:
//     p^{n+1} = p^n + b (p^n - p^{n-1}) + cc (L p^n + s^n),  L = sum_a sum_k a_k/h_a^2 [(p_{+k} + p_{-k}) - 2p]
// (cc = v^2 dt^2/(1 + gamma dt) is read from the expanded array; b = (1 - gamma dt)/(1 + gamma dt)
// from the per-axis gamma*dt table)
//     q^k     = q^{k+1} + b (q^{k+1} - q^{k+2}) + cc (L q^{k+1} + R^T rhat^{k-1}),  G += q^k L p^{k-1}.
//
// 2.5D blocking: a CTA owns a 128 (x) x 8 (y) column of one wavefield and
// marches through z.  Each thread owns 4 consecutive x points of one y row and
// keeps the 9 z-levels its z-derivative needs in a register queue.  x-y halo
// planes (136 x 16) of the field being stepped, and plain planes (128 x 8) of
// the older level, stream through an 8-slot shared-memory ring by TMA, three
// planes ahead of the compute; in the adjoint the snapshot p^{k-1} has its own
// halo-plane ring and register queue for L p^{k-1}.  Sequence number q of the
// ring carries the halo plane z = q - 4 and the plain plane z = q - 8; level
// z = q - 8 is computed once sequence q has landed.
#include "fwi_internal.cuh"

namespace fwi {

constexpr int HY3 = TY3 + 2 * HALO;  // 16
constexpr int PLANE = HY3 * HX;     // floats in a halo plane
constexpr int PPLANE = TY3 * TX;    // floats in a plain plane
constexpr int NST = 8;              // ring slots

template <bool ADJ>
struct Smem3D {
  static constexpr int off_prev = NST * PLANE;
  static constexpr int off_snap = off_prev + NST * PPLANE;
  static constexpr int off_stage = off_snap + (ADJ ? NST * PLANE : 0);
  static constexpr int nfloat = off_stage + PPLANE;
  static constexpr int bytes = nfloat * 4 + NST * 8;
};

__device__ __forceinline__ float4 ld4s(const float* p) { return *reinterpret_cast<const float4*>(p); }

__device__ __forceinline__ float comp(const float4& v, int j) {
  return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}

// Laplacian of the thread's 4 points: x and y neighbours from the halo plane H
// (row ly+4, columns lx..lx+11), z neighbours from the register queue Q[0..8]
// (Q[4] is the centre level).
__device__ __forceinline__ void lap3(const float* __restrict__ H, const float4 (&Q)[9], int ly, int lx,
                                     const Coef& K, float (&lap)[4]) {
  const float* row = H + (ly + HALO) * HX;
  const float4 xl = ld4s(row + lx), xr = ld4s(row + lx + 8);
  const float4 ce = Q[4];
  const float w[12] = {xl.x, xl.y, xl.z, xl.w, ce.x, ce.y, ce.z, ce.w, xr.x, xr.y, xr.z, xr.w};
  float4 yn[8];
#pragma unroll
  for (int k = 1; k <= 4; k++) {
    yn[k - 1] = ld4s(H + (ly + HALO - k) * HX + lx + 4);
    yn[k + 3] = ld4s(H + (ly + HALO + k) * HX + lx + 4);
  }
#pragma unroll
  for (int j = 0; j < 4; j++) {
    const float p = w[4 + j], p2 = p + p;
    float a = K.cx[4] * ((w[8 + j] + w[j]) - p2);
    a = fmaf(K.cx[3], (w[7 + j] + w[1 + j]) - p2, a);
    a = fmaf(K.cx[2], (w[6 + j] + w[2 + j]) - p2, a);
    a = fmaf(K.cx[1], (w[5 + j] + w[3 + j]) - p2, a);
    a = fmaf(K.cy[4], (comp(yn[7], j) + comp(yn[3], j)) - p2, a);
    a = fmaf(K.cy[3], (comp(yn[6], j) + comp(yn[2], j)) - p2, a);
    a = fmaf(K.cy[2], (comp(yn[5], j) + comp(yn[1], j)) - p2, a);
    a = fmaf(K.cy[1], (comp(yn[4], j) + comp(yn[0], j)) - p2, a);
    a = fmaf(K.cz[4], (comp(Q[8], j) + comp(Q[0], j)) - p2, a);
    a = fmaf(K.cz[3], (comp(Q[7], j) + comp(Q[1], j)) - p2, a);
    a = fmaf(K.cz[2], (comp(Q[6], j) + comp(Q[2], j)) - p2, a);
    a = fmaf(K.cz[1], (comp(Q[5], j) + comp(Q[3], j)) - p2, a);
    lap[j] = a;
  }
}

template <bool ADJ>
__global__ void __launch_bounds__(NTHREADS, 1)
step3d_kernel(const __grid_constant__ CUtensorMap tm_halo, const __grid_constant__ CUtensorMap tm_plain,
              const Layout L, const Coef K, const StepParams P) {
  using S = Smem3D<ADJ>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float* s_cur = reinterpret_cast<float*>(smem_raw);
  float* s_prev = s_cur + S::off_prev;
  float* s_snap = s_cur + S::off_snap;
  float* s_stage = s_cur + S::off_stage;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + S::nfloat * 4);

  const int tid = threadIdx.x, lane = tid & 31, ly = tid >> 5;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY3, b = blockIdx.z;
  const int s = b / P.nsg;
  const int tile = blockIdx.y * P.ntx + blockIdx.x;
  const int lx = 4 * lane;
  const int gx = x0 + lx, gy = y0 + ly;
  const bool colv = gx < L.nxp && gy < L.nyp;

  if (tid == 0) {
    tma_prefetch_desc(&tm_halo);
    tma_prefetch_desc(&tm_plain);
    for (int i = 0; i < NST; i++) mbar_init(&bar[i], 1);
    fence_mbar_init();
  }
  __syncthreads();

  const int last_q = L.nzp + 7;
  auto issue = [&](int q) {
    const int slot = q % NST;
    const int zh = q - HALO;       // halo plane level
    const int zp = q - 2 * HALO;   // plain plane level
    const bool with_prev = zp >= 0 && zp < L.nzp;
    uint32_t bytes = PLANE * 4 * (ADJ ? 2 : 1) + (with_prev ? PPLANE * 4 : 0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(&bar[slot], bytes);
    tma_load_5d(s_cur + slot * PLANE, &tm_halo, x0, y0, zh + HALO, b, P.s_cur, &bar[slot]);
    if (ADJ) tma_load_5d(s_snap + slot * PLANE, &tm_halo, x0, y0, zh + HALO, b, P.s_snap, &bar[slot]);
    if (with_prev)
      tma_load_5d(s_prev + slot * PPLANE, &tm_plain, x0 + HALO, y0 + HALO, zp + HALO, b, P.s_prev, &bar[slot]);
  };
  if (tid == 0)
    for (int q = 0; q < NST && q <= last_q; q++) issue(q);

  // per-call point lists of this tile (entries sorted by z)
  const int ib = P.inj_off[b * P.inj_bstride + tile], ie = P.inj_off[b * P.inj_bstride + tile + 1];
  int sb = 0, se = 0;
  if (P.smp4) {
    sb = P.smp_off[b * P.smp_bstride + tile];
    se = P.smp_off[b * P.smp_bstride + tile + 1];
  }
  const float* cs = P.c + (long long)s * L.field;
  float* outp = P.pool + (long long)P.s_out * P.slot_elems + (long long)b * L.field;
  float* gb = ADJ ? P.grad + (long long)b * L.field : nullptr;

  // sponge table entries of this thread's y row and x columns
  const float gyv = gy < L.nyp ? __ldg(P.gtab + L.nzp + gy) : 0.f;
  float gxv[4];
#pragma unroll
  for (int j = 0; j < 4; j++) gxv[j] = gx + j < L.nxp ? __ldg(P.gtab + L.nzp + L.nyp + gx + j) : 0.f;

  float4 Q[9], QS[9];
#pragma unroll
  for (int i = 0; i < 9; i++) {
    Q[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    QS[i] = Q[i];
  }

  for (int q = 0; q <= last_q; q++) {
    const int slot = q % NST;
    const bool ok = mbar_wait_bounded(&bar[slot], (q / NST) & 1, P.status);
    if (__syncthreads_or(!ok)) return;
    // shift the queues and append the centre of halo plane q-4 (level q-4)
#pragma unroll
    for (int i = 0; i < 8; i++) {
      Q[i] = Q[i + 1];
      if (ADJ) QS[i] = QS[i + 1];
    }
    Q[8] = ld4s(s_cur + slot * PLANE + (ly + HALO) * HX + lx + HALO);
    if (ADJ) QS[8] = ld4s(s_snap + slot * PLANE + (ly + HALO) * HX + lx + HALO);

    const int z = q - 2 * HALO;  // level computed at this sequence
    if (z >= 0) {
      const int hslot = (q - HALO) % NST;  // halo plane of level z
      float lap[4];
      lap3(s_cur + hslot * PLANE, Q, ly, lx, K, lap);
      const float4 pm = ld4s(s_prev + slot * PPLANE + ly * TX + lx);
      float4 cv = make_float4(0.f, 0.f, 0.f, 0.f);
      if (colv) cv = __ldg(reinterpret_cast<const float4*>(cs + L.off(z, gy, gx)));
      const float gzy = __ldg(P.gtab + z) + gyv;
      float nv[4];
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const float bb = sponge_b(gzy + gxv[j]);
        const float p = comp(Q[4], j);
        nv[j] = fmaf(comp(cv, j), lap[j], fmaf(bb, p - comp(pm, j), p));
      }
      // injection / sampling at this level (only tiles with points at level z)
      bool mine = false;
      for (int e = ib + tid; e < ie; e += NTHREADS) mine |= P.inj[e].w == z;
      for (int e = sb + tid; e < se; e += NTHREADS) mine |= P.smp4[e].z == z;
      if (__syncthreads_or(mine)) {
        *reinterpret_cast<float4*>(s_stage + ly * TX + lx) = make_float4(nv[0], nv[1], nv[2], nv[3]);
        __syncthreads();
        for (int e = ib + tid; e < ie; e += NTHREADS) {
          const int4 en = P.inj[e];
          if (en.w != z) continue;
          const int yy = y0 + en.x / TX, xx = x0 + en.x % TX;
          const float ccp = __ldg(cs + L.off(z, yy, xx));
          s_stage[en.x] += ccp * (__int_as_float(en.z) *
                                  P.series[(long long)b * P.series_bstride + (long long)P.t * P.series_ld + en.y]);
        }
        __syncthreads();
        const float4 v = ld4s(s_stage + ly * TX + lx);
        nv[0] = v.x; nv[1] = v.y; nv[2] = v.z; nv[3] = v.w;
        for (int e = sb + tid; e < se; e += NTHREADS) {
          const int4 en = P.smp4[e];
          if (en.z != z) continue;
          P.smp_out[(long long)b * P.smp_bstride_out + (long long)P.t * P.smp_ld + en.y] = s_stage[en.x];
        }
      }
      if (ADJ) {
        float lps[4];
        lap3(s_snap + hslot * PLANE, QS, ly, lx, K, lps);
        if (colv) {
          float4* gp = reinterpret_cast<float4*>(gb + L.off(z, gy, gx));
          float4 g = *gp;
          g.x = fmaf(nv[0], lps[0], g.x);
          g.y = fmaf(nv[1], lps[1], g.y);
          g.z = fmaf(nv[2], lps[2], g.z);
          g.w = fmaf(nv[3], lps[3], g.w);
          if (gx + 3 < L.nxp) {
            *gp = g;
          } else {
            float* gs = reinterpret_cast<float*>(gp);
            const float gv[4] = {g.x, g.y, g.z, g.w};
            for (int j = 0; j < 4; j++)
              if (gx + j < L.nxp) gs[j] = gv[j];
          }
        }
      }
      if (colv) {
        float* o = outp + L.off(z, gy, gx);
        if (gx + 3 < L.nxp) {
          *reinterpret_cast<float4*>(o) = make_float4(nv[0], nv[1], nv[2], nv[3]);
        } else {
          for (int j = 0; j < 4; j++)
            if (gx + j < L.nxp) o[j] = nv[j];
        }
      }
    }
    __syncthreads();  // slot of sequence q-4 (halo of level z) is free
    if (tid == 0 && q >= HALO && q + HALO <= last_q) issue(q + HALO);
  }
}

cudaError_t launch_step3d(bool adj, const CUtensorMap& tm_halo, const CUtensorMap& tm_plain, const Layout& L,
                          const Coef& K, const StepParams& P, int B, cudaStream_t st) {
  static bool attr_set[2] = {false, false};
  const int nty = (L.nyp + TY3 - 1) / TY3;
  dim3 grid(P.ntx, nty, B);
  if (adj) {
    if (!attr_set[1]) {
      cudaFuncSetAttribute(step3d_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem3D<true>::bytes);
      attr_set[1] = true;
    }
    step3d_kernel<true><<<grid, NTHREADS, Smem3D<true>::bytes, st>>>(tm_halo, tm_plain, L, K, P);
  } else {
    if (!attr_set[0]) {
      cudaFuncSetAttribute(step3d_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem3D<false>::bytes);
      attr_set[0] = true;
    }
    step3d_kernel<false><<<grid, NTHREADS, Smem3D<false>::bytes, st>>>(tm_halo, tm_plain, L, K, P);
  }
  return cudaGetLastError();
}

}  // namespace fwi
