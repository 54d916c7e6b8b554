// fwi_internal.cuh -- layout, kernel parameter blocks and sm_103a helpers
// shared by the translation units of libfwi.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fwi.h"

namespace fwi {

// Wavefield storage.  Every wavefield is a padded grid (physical grid plus nb
// sponge cells per side) surrounded by a 4-cell zero halo, so the 8th-order
// stencil reads neighbours without bounds tests.  Row stride SX is rounded to
// 32 floats (128 B): rows start on cache-line boundaries and every 4-column
// group is 16-byte aligned for float4 and TMA access.
//   element (z, y, x), padded coordinates, at ((z+4)*NY + y+4*(ndim==3))*SX + x+4
constexpr int HALO = 4;
constexpr int TX = 128;   // tile width (x): 32 lanes x float4
constexpr int TZ = 32;    // tile height (z): 8 warps x 4 rows
constexpr int RZ = 4;     // rows per thread
constexpr int NTHREADS = 256;
constexpr int HX = TX + 2 * HALO;   // 136
constexpr int HZ = TZ + 2 * HALO;   // 40
constexpr int TX3 = 64;             // 3D tile width (x): 16 lanes x float4
constexpr int TY3 = 16;             // 3D tile height (y): 8 warps x 2 rows
constexpr int HX3 = TX3 + 2 * HALO; // 72

struct Layout {
  int ndim;
  int nz, ny, nx, nb;       // physical grid, sponge width
  int nzp, nyp, nxp;        // padded grid (nyp = 1 in 2D)
  int NZ, NY, SX;           // stored extents including the zero halo (NY = 1 in 2D)
  long long field;          // floats per wavefield
  long long phys;           // physical points
  __host__ __device__ long long off(int z, int y, int x) const {
    return ((long long)(z + HALO) * NY + (ndim == 3 ? y + HALO : 0)) * SX + (x + HALO);
  }
};

// Stencil coefficients and sponge parameters in FP32 as the kernels use them.
struct Coef {
  float cz[5], cy[5], cx[5];  // a_k / h_a^2, k = 1..4 used (sum-zero form)
  float gdt;                  // gmax * dt
  float inv_nb;               // 1 / nb (0 when nb == 0)
  float c0_2d;                // a_0/hx^2 + a_0/hz^2: centre weight of the 2D Laplacian in plain form
  float c0_3d;                // a_0/hx^2 + a_0/hy^2 + a_0/hz^2: the same for the 3D Laplacian
};

// Slots and record time of one step of a multi-step launch.
struct StepDesc {
  int cur, prev, out, snap;  // pool slots of the stepped level, the older level, the output, the snapshot
  int t;                     // record time index of the step's injection and sampling
  int pad[3];
};

// One time step of the forward recursion (FWD) or of the adjoint recursion
// with the imaging condition (ADJ) over all wavefields of a call; the 2D
// kernels run nsteps such steps, described by steps[], in one launch.
struct StepParams {
  float* pool;              // slot pool base
  long long slot_elems;     // B * field floats per slot
  int s_cur, s_prev, s_out, s_snap;   // slot indices
  const float* c;           // [nsamp][field] cc = v^2 dt^2 / (1 + gamma dt) (padded)
  const float* gtab;        // gamma*dt per axis: z [nzp], then y [nyp], then x [nxp]
  float* grad;              // ADJ: [nsamp][field] imaging accumulator
  int nsg;                  // wavefields per sample (b = s * nsg + j)
  int t;                    // series / record time index
  int ntx, ntiles;
  // injection points per (wavefield, tile): CSR offsets inj_off[b * inj_bstride + tile]
  const int* inj_off; int inj_bstride;
  const int4* inj;          // {local = row * tile width + column, col, amp (float bits), unused}
  const float* series; long long series_bstride; int series_ld;  // amp * series[b*bs + t*ld + col]
  // sampling points, same CSR form; smp == nullptr disables sampling
  const int* smp_off; int smp_bstride;
  const int2* smp;          // {local, col}                      (2D)
  const int4* smp4;         // {local, col, z, 0}                (3D; inj .w holds z)
  float* smp_out; long long smp_bstride_out; int smp_ld;
  int* status;
  // multi-step launches (2D; 3D persistent variants): step descriptors and
  // per-item progress flags (item = tile of one sample in 2D, of one unit in
  // 3D; flag = steps completed; zero at launch).  3D: steps == nullptr for a
  // one-step launch that takes its slots and t from the fields above.
  const StepDesc* steps; int nsteps;
  int* done;
  int order3;               // 3D CTA order: 0 tile-major, 1 wavefield-fastest
  int zpair3;               // 3D march: 0 one level at a time, 1 two levels together
  int pair3;                // 3D tiles: 0 one wavefield over 64 x 16, 1 two supergathers over 64 x 8 each
  int nunits3;              // 3D: wavefield units of the launch (set by launch_step3d)
  int ctas_per_sm3;         // 3D: persistent grid of this many CTAs per SM (0: one per column)
};

// Host-side launchers (stencil.cu)
// Runs P.nsteps steps of all nsamp * P.nsg wavefields in one cooperative launch;
// P.done must hold nsamp * P.ntiles zeroed ints.
cudaError_t launch_step2d(bool adj, int variant, const CUtensorMap& tm_halo, const CUtensorMap& tm_plain,
                          const CUtensorMap& tm_c, const Layout& L, const Coef& K, const StepParams& P, int nsamp,
                          cudaStream_t st);
int num_variants2d(bool adj);
// Rows of a 2D tile for tile shape sh (variant bit 1): 128 x 32, or 128 x 24.
int tile_rows2d(int sh);
const char* variant2d_name(bool adj, int v);
cudaError_t launch_step3d(bool adj, const CUtensorMap& tm_halo, const CUtensorMap& tm_plain,
                          const CUtensorMap& tm_cc, const CUtensorMap& tm_g, const Layout& L, const Coef& K,
                          const StepParams& P, int B, cudaStream_t st);

// Auxiliary kernels (aux.cu)
cudaError_t launch_expand(const Layout& L, const float* vel, int nsamp, double dt, const float* gtab, float* c,
                          float vmax_cfl, int* status, cudaStream_t st);
cudaError_t launch_wavelet(int nt, double dt, double f0, double t0, float* wav, cudaStream_t st);
cudaError_t launch_residual(int B, int nt, int nr, const float* dpred, const float* dobs,
                            const int* shot_off, const int* shot_id, const float* shot_w,
                            double inv_sigma2, float* rhat, double* part, int nblk, cudaStream_t st);
cudaError_t launch_misfit(int nsamp, int nsg, const double* part, int nblk, double factor,
                          double* misfit, int* status, cudaStream_t st);
cudaError_t launch_source_imaging(int B, int nsg, int nt, int E, const float* qsrc,
                                  const float* wav, const int* src_cnt, const long long* src_pos,
                                  const float* src_amp, float* tmp, float* grad,
                                  long long field, int wf_per_acc, cudaStream_t st);
cudaError_t launch_finalize(const Layout& L, const float* vel, const float* G, int nsamp, int g_per_sample,
                            double scale, float* grad, cudaStream_t st);
cudaError_t launch_langevin(float* z, const float* g, long long n, double eta, double nu,
                            double vmin, double vmax, uint64_t seed, uint64_t counter,
                            cudaStream_t st);
cudaError_t launch_langevin_precond(float* z, const float* g, float* v, float* m, int nsamp, long long per,
                                    double alpha, double beta1, double eps, long long k, double eta, double nu,
                                    double vmin, double vmax, uint64_t seed, uint64_t counter, double* part,
                                    int nblk, cudaStream_t st);
cudaError_t launch_renoise(float* xp, const float* xt, const float* x0, long long n, double c0,
                           double ct, double sd, uint64_t seed, uint64_t counter, cudaStream_t st);
cudaError_t launch_prior(const Layout& L, const float* z, const float* zref, int nsamp,
                         double lam, double mu, double hz, double hy, double hx, float* grad,
                         cudaStream_t st);

// ------------------------------------------------------------ device helpers

#ifdef __CUDACC__
// Bounded waits: a wait gives up after ~2^31 SM cycles (about a second at
// GB300 clocks), records FWI_ERR_TIMEOUT in the status word and returns false.
constexpr long long WAIT_CYCLES = 1LL << 31;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* status) {
  if (mbar_try_wait(bar, parity)) return true;
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > WAIT_CYCLES) {
      atomicCAS(status, 0, (int)FWI_ERR_TIMEOUT);
      return false;
    }
  }
  return true;
}

// Shared-memory fetch-add with acquire-release semantics at CTA scope.
__device__ __forceinline__ int atom_add_acq_rel(int* p, int v) {
  int old;
  asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(smem_u32(p)), "r"(v)
               : "memory");
  return old;
}

// Wait with a suspend-time hint (ns) between hardware polls.
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t* bar, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}

// Bounded wait that also gives up when another warp of the CTA has set the
// shared abort word (after its own wait ran out).
__device__ __forceinline__ bool mbar_wait_abortable(uint64_t* bar, uint32_t parity, int* status,
                                                    volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait_hint(bar, parity, 1000000u)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > WAIT_CYCLES) {
      atomicCAS(status, 0, (int)FWI_ERR_TIMEOUT);
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}

// Memory-model helpers for the cross-CTA progress flags.
__device__ __forceinline__ int ld_relaxed_gpu(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_gpu(int* p, int v) {
  asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire_cta_shared(const int* p) {
  int v;
  asm volatile("ld.acquire.cta.shared::cta.b32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_cta_shared(int* p, int v) {
  asm volatile("red.release.cta.shared::cta.add.u32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Register reallocation between warpgroups (all warps of a warpgroup execute it).
template <int N>
__device__ __forceinline__ void setmaxnreg_inc() {
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(N));
}
template <int N>
__device__ __forceinline__ void setmaxnreg_dec() {
  asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(N));
}

// TMA tiled loads into shared memory, completion counted on an mbarrier.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2,
                                            int c3, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2,
                                            int c3, int c4, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
      "r"(smem_u32(bar))
      : "memory");
}

// L2 eviction-priority policies and the loads/stores that carry them.
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void tma_load_4d_hint(void* dst, const CUtensorMap* tm, int c0, int c1, int c2, int c3,
                                                 uint64_t* bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3, %4, %5}], [%6], %7;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}
__device__ __forceinline__ void tma_load_3d_hint(void* dst, const CUtensorMap* tm, int c0, int c1, int c2,
                                                 uint64_t* bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}
// (plain global accesses: no "memory" clobber, so the compiler keeps its freedom
// to schedule the surrounding shared-memory work; volatile keeps their order)
__device__ __forceinline__ void st4_hint(float* p, float4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y),
               "f"(v.z), "f"(v.w), "l"(pol));
}
__device__ __forceinline__ float4 ld4_hint(const float* p, uint64_t pol) {
  float4 v;
  asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p), "l"(pol));
  return v;
}

// 4-byte asynchronous global->shared copies whose completion is counted as
// one (non-incrementing) arrival on an mbarrier.
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Sponge coefficient b = (1 - g)/(1 + g) from g = gamma*dt (fast reciprocal).
__device__ __forceinline__ float sponge_b(float g) { return (1.0f - g) * __fdividef(1.0f, 1.0f + g); }

__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap* tm) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tm)) : "memory");
}

// Depth into the sponge of padded index i along an axis with n physical cells.
__device__ __forceinline__ int pad_depth(int i, int n, int nb) {
  return i < nb ? nb - i : (i >= nb + n ? i - (nb + n - 1) : 0);
}
#endif

}  // namespace fwi
