// prior.cu -- tensor-core kernels of the learned prior (the denoiser g_theta
// of Sec. 2.2): a BF16 GEMM on the 5th-generation tensor cores and the 3x3
// convolution built on it.
//
// D[M x N] = A[M x K] * B[N x K]^T (+ bias[N]), A and B BF16 and K-contiguous,
// accumulated in FP32 in tensor memory (TMEM).  One CTA computes a 128 x BN
// tile:
//   warp 0, lane 0 -- TMA producer: 128 x 64 tiles of A and BN x 64 tiles of B
//                     (128-byte swizzle) into a STAGES-deep shared-memory ring;
//   warp 1, lane 0 -- MMA issuer: four tcgen05.mma (K = 16 each) per stage,
//                     then tcgen05.commit to the stage's "empty" barrier so
//                     the producer reuses it once the tensor core has read it;
//                     after the last stage a commit to the accumulator barrier;
//   warps 0-3     -- epilogue: each warp reads its 32 TMEM lanes (rows) with
//                     tcgen05.ld and writes FP32 or BF16 rows (+ bias, + ReLU).
// Every wait is bounded; a timeout sets the status word and the CTA leaves
// (after a bounded wait for its own copies in flight).
//
// The convolution (conv3x3_bf16) is the same pipeline with A gathered by TMA
// from an NHWC activation tensor: for output rows y0.. and each tap (dy, dx)
// and 64-channel block, the A tile is the input box shifted by (dy-1, dx-1);
// coordinates outside the image read zeros, which is the padding.  The 3D
// convolution (conv3x3x3_bf16, NDHWC volumes) takes a 5D box shifted by
// (dz-1, dy-1, dx-1) for each of its 27 taps.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "prior.h"

namespace prior {

constexpr long long WAIT_CYCLES = 1LL << 31;
constexpr int BM = 128, BK = 64;

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t c) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(c) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t par) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(par)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t par, int* status, volatile int* abort_flag) {
  if (mbar_try(b, par)) return true;
  const long long t0 = clock64();
  while (!mbar_try(b, par)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > WAIT_CYCLES) {
      atomicCAS(status, 0, (int)PRIOR_ERR_TIMEOUT);
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma2d(void* dst, const CUtensorMap* m, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(c0), "r"(c1), "r"(saddr(bar))
      : "memory");
}
__device__ __forceinline__ void tma4d(void* dst, const CUtensorMap* m, int c0, int c1, int c2, int c3,
                                      uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(saddr(bar))
      : "memory");
}

__device__ __forceinline__ void tma5d(void* dst, const CUtensorMap* m, int c0, int c1, int c2, int c3, int c4,
                                      uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(saddr(bar))
      : "memory");
}

__device__ __forceinline__ void tma3d(void* dst, const CUtensorMap* m, int c0, int c1, int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(c0), "r"(c1), "r"(c2), "r"(saddr(bar))
      : "memory");
}

// Kernel modes: plain GEMM; 3x3 convolution (forward, and data gradient with
// flipped weights); weight gradient of the 3x3 (or 3x3x3) convolution: per tap
// a GEMM over pixels, dY^T [Cout x P] times the tap-shifted input [Cin x P]^T,
// split over pixel ranges and accumulated atomically in FP32; 3x3x3
// convolution of NDHWC volumes.
enum Mode { GEMM = 0, CONV = 1, WGRAD = 2, CONV3 = 3 };

// Shared-memory matrix descriptor of a K-major operand tile written by TMA with
// the 128-byte swizzle: rows of 64 BF16 (128 B), 8-row swizzle atoms 1024 B
// apart (stride byte offset), descriptor version 1, layout "128-byte swizzle".
__device__ __forceinline__ uint64_t sw128_desc(uint32_t smem_byte_addr) {
  uint64_t d = 0;
  d |= (uint64_t)((smem_byte_addr >> 4) & 0x3FFF);  // start address
  d |= (uint64_t)1 << 16;                           // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;                 // stride byte offset
  d |= (uint64_t)1 << 46;                           // descriptor version
  d |= (uint64_t)2 << 61;                           // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 accumulator,
// both operands K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4)                        // D format: F32
         | (1u << 7)                      // A format: BF16
         | (1u << 10)                     // B format: BF16
         | ((uint32_t)(n >> 3) << 17)     // N / 8
         | ((uint32_t)(BM >> 4) << 24);   // M / 16
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // a in the low half
  return *reinterpret_cast<const uint32_t*>(&h);
}

struct Args {
  int M, N, K;       // GEMM extents (convolution: M = images*H*W, N = Cout, K = 9*Cin)
  int ldd;           // row stride of D in elements
  void* D;
  int d_bf16;        // D in BF16 (else FP32)
  const float* bias; // [N] or null
  int relu;
  int H, W, Cin, TW, TH;  // convolution geometry (tile = TH rows x TW columns of one image)
  int Dd, TD;        // 3D convolution: depth, and planes per tile (tile = TD x TH x TW)
  int ntap;          // weight gradient: taps (9 or 27)
  int splits;        // weight gradient: pixel ranges per tap (grid z = ntap * splits)
  float* part;       // weight gradient: per-split slices [splits][M][ldd] (plain stores), or null (atomics into D)
  int* status;
};

template <int BN, int STAGES>
struct Smem {
  static constexpr int A_BYTES = BM * BK * 2;  // 16 KB
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int OFF_BAR = STAGES * STAGE;
  static constexpr int bytes = OFF_BAR + (2 * STAGES + 2) * 8 + 16 + 1024;  // + alignment slack
};

template <int BN, int STAGES, int MODE>
__global__ void __launch_bounds__(128, 2)
gemm_kernel(const __grid_constant__ CUtensorMap tma_a, const __grid_constant__ CUtensorMap tma_b, const Args g) {
  using S = Smem<BN, STAGES>;
  constexpr uint32_t TMEM_COLS = BN < 32 ? 32 : BN;
  extern __shared__ unsigned char smem_dyn[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + S::OFF_BAR);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;
  uint32_t* tbase_s = reinterpret_cast<uint32_t*>(accf + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tbase_s + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  // K blocks of this CTA: all of K, or (weight gradient) this split's 64-pixel chunks
  int kb0 = 0, nk = g.K / BK, tap = 0, split = 0;
  if (MODE == WGRAD) {
    tap = blockIdx.z % g.ntap;
    split = blockIdx.z / g.ntap;
    const int chunks = g.K / BK;
    kb0 = (int)((long long)chunks * split / g.splits);
    nk = (int)((long long)chunks * (split + 1) / g.splits) - kb0;
  }

  if (tid == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tma_a)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tma_b)) : "memory");
    for (int i = 0; i < STAGES; i++) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(&accf[0], 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {  // tensor-memory accumulator: TMEM_COLS FP32 columns x 128 lanes
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tbase_s)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = *tbase_s;

  // convolution tile: TH rows x TW columns of image img starting at (y0, x0)
  // (3D: TD x TH x TW starting at (z0, y0, x0))
  int img = 0, z0 = 0, y0 = 0, x0 = 0, ncb = 1;
  if (MODE == CONV) {
    const int hw = g.H * g.W;
    img = m0 / hw;
    const int rem = m0 - img * hw;
    y0 = rem / g.W;
    x0 = rem - y0 * g.W;
    ncb = g.Cin / BK;
  } else if (MODE == CONV3) {
    const int hw = g.H * g.W, dhw = g.Dd * hw;
    img = m0 / dhw;
    int rem = m0 - img * dhw;
    z0 = rem / hw;
    rem -= z0 * hw;
    y0 = rem / g.W;
    x0 = rem - y0 * g.W;
    ncb = g.Cin / BK;
  }

  if (warp == 0 && lane == 0) {  // ---------------------------------------------- TMA producer
    int kb = 0;
    for (; kb < nk; kb++) {
      const int s = kb % STAGES;
      if (kb >= STAGES && !mbar_wait(&empty[s], (uint32_t)((kb / STAGES - 1) & 1), g.status, abort_flag)) break;
      unsigned char* st = sm + s * S::STAGE;
      mbar_expect_tx(&full[s], S::STAGE);
      if (MODE == CONV) {
        const int t = kb / ncb, cb = kb - t * ncb;
        const int dy = t / 3 - 1, dx = t % 3 - 1;
        tma4d(st, &tma_a, cb * BK, x0 + dx, y0 + dy, img, &full[s]);
        tma2d(st + S::A_BYTES, &tma_b, kb * BK, n0, &full[s]);
      } else if (MODE == CONV3) {
        const int t = kb / ncb, cb = kb - t * ncb;  // tap t = dz*9 + dy*3 + dx
        const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
        tma5d(st, &tma_a, cb * BK, x0 + dx, y0 + dy, z0 + dz, img, &full[s]);
        tma2d(st + S::A_BYTES, &tma_b, kb * BK, n0, &full[s]);
      } else if (MODE == WGRAD) {
        // 64-pixel chunk p0: dY^T rows m0.. and the tap's shifted input rows n0..
        const int p0 = (kb0 + kb) * BK;
        tma2d(st, &tma_a, p0, m0, &full[s]);
        tma3d(st + S::A_BYTES, &tma_b, p0, n0, tap, &full[s]);
      } else {
        tma2d(st, &tma_a, kb * BK, m0, &full[s]);
        tma2d(st + S::A_BYTES, &tma_b, kb * BK, n0, &full[s]);
      }
    }
    if (kb < nk) {  // aborted: bounded wait for the copies in flight
      for (int i = kb - STAGES > 0 ? kb - STAGES : 0; i < kb; i++) {
        const long long t0 = clock64();
        while (!mbar_try(&full[i % STAGES], (uint32_t)((i / STAGES) & 1)) && clock64() - t0 < (1LL << 24)) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {  // ------------------------------------ MMA issuer
    constexpr uint32_t IDESC = idesc_bf16(BN);
    int kb = 0;
    for (; kb < nk; kb++) {
      const int s = kb % STAGES;
      if (!mbar_wait(&full[s], (uint32_t)((kb / STAGES) & 1), g.status, abort_flag)) break;
      fence_after();
      const uint32_t a0 = saddr(sm + s * S::STAGE), b0 = a0 + S::A_BYTES;
#pragma unroll
      for (int kk = 0; kk < BK / 16; kk++)
        mma_bf16(tbase, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), IDESC, (kb | kk) != 0);
      mma_commit(&empty[s]);  // stage free once these MMAs have read it
    }
    mma_commit(&accf[0]);  // accumulator complete (or, after an abort, every issued MMA done)
  }
  __syncwarp();

  // ---------------------------------------------------------------------- epilogue
  const bool ok = mbar_wait(&accf[0], 0, g.status, abort_flag) && !*abort_flag;
  fence_after();
  if (ok) {
    const int row = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < BN; c0 += 32) {
      float v[32];
      tmem_ld32(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (row < g.M) {
#pragma unroll
        for (int i = 0; i < 32; i++) {
          float x = v[i];
          if (g.bias) x += __ldg(g.bias + n0 + c0 + i);
          if (g.relu) x = fmaxf(x, 0.f);
          v[i] = x;
        }
        if (MODE == WGRAD && g.part) {  // this split's slice: plain stores, summed in order later
          float* d = g.part + ((long long)split * g.M + row) * g.ldd + tap * g.Cin + n0 + c0;
#pragma unroll
          for (int i = 0; i < 32; i += 4) *reinterpret_cast<float4*>(d + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        } else if (MODE == WGRAD) {
          float* d = reinterpret_cast<float*>(g.D) + (long long)row * g.ldd + tap * g.Cin + n0 + c0;
#pragma unroll
          for (int i = 0; i < 32; i++) atomicAdd(d + i, v[i]);
        } else if (g.d_bf16) {
          __nv_bfloat16* d = reinterpret_cast<__nv_bfloat16*>(g.D) + (long long)row * g.ldd + n0 + c0;
#pragma unroll
          for (int i = 0; i < 32; i += 8)
            *reinterpret_cast<uint4*>(d + i) =
                make_uint4(pack_bf16(v[i], v[i + 1]), pack_bf16(v[i + 2], v[i + 3]), pack_bf16(v[i + 4], v[i + 5]),
                           pack_bf16(v[i + 6], v[i + 7]));
        } else {
          float* d = reinterpret_cast<float*>(g.D) + (long long)row * g.ldd + n0 + c0;
#pragma unroll
          for (int i = 0; i < 32; i += 4) *reinterpret_cast<float4*>(d + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TMEM_COLS) : "memory");
}

}  // namespace prior

// ------------------------------------------------------------------ host side
namespace {

__device__ int g_prior_status;

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// BF16 tensor map with the 128-byte swizzle; dims/box innermost first.
bool make_map(CUtensorMap* m, const void* base, int rank, const cuuint64_t* dims, const cuuint32_t* box) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t strides[4];
  cuuint64_t s = 2;
  for (int i = 0; i + 1 < rank; i++) {
    s *= dims[i];
    strides[i] = s;
  }
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int* status_ptr(int* status) {
  if (status) return status;
  void* p = nullptr;
  return cudaGetSymbolAddress(&p, g_prior_status) == cudaSuccess ? reinterpret_cast<int*>(p) : nullptr;
}

template <int BN, int MODE>
int launch(const CUtensorMap& ma, const CUtensorMap& mb, const prior::Args& g, cudaStream_t st) {
  constexpr int STAGES = 3;  // 96 KB at BN = 128: two CTAs per SM overlap one's epilogue with the other's MMAs
  using S = prior::Smem<BN, STAGES>;
  auto kern = prior::gemm_kernel<BN, STAGES, MODE>;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::bytes) != cudaSuccess)
      return PRIOR_ERR_CUDA;
    attr = true;
  }
  dim3 grid((g.M + prior::BM - 1) / prior::BM, g.N / BN, MODE == prior::WGRAD ? g.ntap * g.splits : 1);
  kern<<<grid, 128, S::bytes, st>>>(ma, mb, g);
  return cudaGetLastError() == cudaSuccess ? PRIOR_OK : PRIOR_ERR_CUDA;
}

template <int MODE>
int dispatch(int bn, const CUtensorMap& ma, const CUtensorMap& mb, const prior::Args& g, cudaStream_t st) {
  switch (bn) {
    case 32: return launch<32, MODE>(ma, mb, g, st);
    case 64: return launch<64, MODE>(ma, mb, g, st);
    case 128: return launch<128, MODE>(ma, mb, g, st);
    case 256: return launch<256, MODE>(ma, mb, g, st);
  }
  return PRIOR_ERR_ARG;
}

int tile_n(int N) {
  if (N == 32 || N == 64 || N == 128 || N == 256) return N;
  if (N > 0 && N % 128 == 0) return 128;
  return N > 0 && N % 64 == 0 ? 64 : 0;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace

extern "C" {

int prior_gemm_bf16(const void* A, const void* B, void* D, int M, int N, int K, int ldd, int d_bf16,
                    const float* bias, int relu, int* status, void* stream) {
  const int bn = tile_n(N);
  if (!A || !B || !D || M <= 0 || K <= 0 || M % prior::BM || K % prior::BK || !bn || ldd < N || ldd % 8)
    return PRIOR_ERR_ARG;
  if (!aligned16(A) || !aligned16(B) || !aligned16(D) || (bias && (reinterpret_cast<uintptr_t>(bias) & 3)))
    return PRIOR_ERR_ARG;
  prior::Args g = {};
  g.M = M;
  g.N = N;
  g.K = K;
  g.ldd = ldd;
  g.D = D;
  g.d_bf16 = d_bf16 != 0;
  g.bias = bias;
  g.relu = relu != 0;
  g.status = status_ptr(status);
  if (!g.status) return PRIOR_ERR_CUDA;
  CUtensorMap ma, mb;
  const cuuint64_t da[2] = {(cuuint64_t)K, (cuuint64_t)M}, db[2] = {(cuuint64_t)K, (cuuint64_t)N};
  const cuuint32_t ba[2] = {prior::BK, prior::BM}, bb[2] = {prior::BK, (cuuint32_t)bn};
  if (!make_map(&ma, A, 2, da, ba) || !make_map(&mb, B, 2, db, bb)) return PRIOR_ERR_ARG;
  return dispatch<prior::GEMM>(bn, ma, mb, g, (cudaStream_t)stream);
}

int prior_conv3x3_bf16(const void* X, const void* Wt, void* Y, int nimg, int H, int W, int Cin, int Cout,
                       int y_bf16, const float* bias, int relu, int* status, void* stream) {
  const int bn = tile_n(Cout);
  if (!X || !Wt || !Y || nimg <= 0 || H <= 0 || W <= 0 || Cin <= 0 || Cin % prior::BK || !bn) return PRIOR_ERR_ARG;
  const bool w_ok = W % 128 == 0 || (W <= 128 && (W & (W - 1)) == 0);
  const int TW = W < 128 ? W : 128, TH = prior::BM / TW;
  if (!w_ok || H % TH) return PRIOR_ERR_ARG;
  if (!aligned16(X) || !aligned16(Wt) || !aligned16(Y) || (bias && (reinterpret_cast<uintptr_t>(bias) & 3)))
    return PRIOR_ERR_ARG;
  prior::Args g = {};
  g.M = nimg * H * W;
  g.N = Cout;
  g.K = 9 * Cin;
  g.ldd = Cout;
  g.D = Y;
  g.d_bf16 = y_bf16 != 0;
  g.bias = bias;
  g.relu = relu != 0;
  g.H = H;
  g.W = W;
  g.Cin = Cin;
  g.TW = TW;
  g.TH = TH;
  g.status = status_ptr(status);
  if (!g.status) return PRIOR_ERR_CUDA;
  CUtensorMap ma, mb;
  const cuuint64_t da[4] = {(cuuint64_t)Cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)nimg};
  const cuuint32_t ba[4] = {prior::BK, (cuuint32_t)TW, (cuuint32_t)TH, 1};
  const cuuint64_t db[2] = {(cuuint64_t)(9 * Cin), (cuuint64_t)Cout};
  const cuuint32_t bb[2] = {prior::BK, (cuuint32_t)bn};
  if (!make_map(&ma, X, 4, da, ba) || !make_map(&mb, Wt, 2, db, bb)) return PRIOR_ERR_ARG;
  return dispatch<prior::CONV>(bn, ma, mb, g, (cudaStream_t)stream);
}

}  // extern "C"

namespace {

// dW[i] += sum over s = 0 .. splits-1 of part[s][i], in that order.
__global__ void split_sum_kernel(const float* __restrict__ part, int splits, long long n, float* dW) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float acc = dW[i];
    for (int s = 0; s < splits; s++) acc += part[(long long)s * n + i];
    dW[i] = acc;
  }
}

int wgrad(const void* dYt, const void* Xs, float* dW, float* work, int P, int Cout, int Cin, int ntap, int splits,
          int* status, void* stream) {
  const int bn = tile_n(Cin);
  const int mp = (Cout + prior::BM - 1) / prior::BM * prior::BM;
  if (!dYt || !Xs || !dW || P <= 0 || P % prior::BK || Cout <= 0 || !bn || splits < 1 || splits > 65535 / ntap)
    return PRIOR_ERR_ARG;
  if (!aligned16(dYt) || !aligned16(Xs) || !aligned16(dW)) return PRIOR_ERR_ARG;
  prior::Args g = {};
  g.M = Cout;
  g.N = Cin;
  g.K = P;
  g.ldd = ntap * Cin;
  g.D = dW;
  g.Cin = Cin;
  g.ntap = ntap;
  g.splits = splits < P / prior::BK ? splits : P / prior::BK;
  g.part = work;
  if (work && !aligned16(work)) return PRIOR_ERR_ARG;
  g.status = status_ptr(status);
  if (!g.status) return PRIOR_ERR_CUDA;
  CUtensorMap ma, mb;
  const cuuint64_t da[2] = {(cuuint64_t)P, (cuuint64_t)mp};
  const cuuint32_t ba[2] = {prior::BK, prior::BM};
  const cuuint64_t db[3] = {(cuuint64_t)P, (cuuint64_t)Cin, (cuuint64_t)ntap};
  const cuuint32_t bb[3] = {prior::BK, (cuuint32_t)bn, 1};
  if (!make_map(&ma, dYt, 2, da, ba) || !make_map(&mb, Xs, 3, db, bb)) return PRIOR_ERR_ARG;
  const int rc = dispatch<prior::WGRAD>(bn, ma, mb, g, (cudaStream_t)stream);
  if (rc != PRIOR_OK || !work) return rc;
  const long long n = (long long)Cout * ntap * Cin;
  const long long blocks = (n + 255) / 256;
  split_sum_kernel<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, (cudaStream_t)stream>>>(work, g.splits, n, dW);
  return cudaGetLastError() == cudaSuccess ? PRIOR_OK : PRIOR_ERR_CUDA;
}

}  // namespace

extern "C" {

int prior_conv3x3_wgrad_bf16(const void* dYt, const void* X9, float* dW, float* work, int P, int Cout, int Cin,
                             int splits, int* status, void* stream) {
  return wgrad(dYt, X9, dW, work, P, Cout, Cin, 9, splits, status, stream);
}

int prior_conv3x3x3_bf16(const void* X, const void* Wt, void* Y, int nimg, int D, int H, int W, int Cin, int Cout,
                         int y_bf16, const float* bias, int relu, int* status, void* stream) {
  const int bn = tile_n(Cout);
  if (!X || !Wt || !Y || nimg <= 0 || D <= 0 || H <= 0 || W <= 0 || Cin <= 0 || Cin % prior::BK || !bn)
    return PRIOR_ERR_ARG;
  // a tile is 128 consecutive voxels of one volume: TW whole-width columns,
  // TH whole rows, TD whole planes
  int TW, TH, TD;
  if (W >= 128) {
    if (W % 128) return PRIOR_ERR_ARG;
    TW = 128, TH = 1, TD = 1;
  } else {
    if (W & (W - 1)) return PRIOR_ERR_ARG;
    TW = W;
    if (H * W >= 128) {
      TH = 128 / W, TD = 1;
      if (H % TH) return PRIOR_ERR_ARG;
    } else {
      if (H & (H - 1)) return PRIOR_ERR_ARG;
      TH = H, TD = 128 / (H * W);
      if (D % TD) return PRIOR_ERR_ARG;
    }
  }
  if (!aligned16(X) || !aligned16(Wt) || !aligned16(Y) || (bias && (reinterpret_cast<uintptr_t>(bias) & 3)))
    return PRIOR_ERR_ARG;
  prior::Args g = {};
  g.M = nimg * D * H * W;
  g.N = Cout;
  g.K = 27 * Cin;
  g.ldd = Cout;
  g.D = Y;
  g.d_bf16 = y_bf16 != 0;
  g.bias = bias;
  g.relu = relu != 0;
  g.Dd = D;
  g.H = H;
  g.W = W;
  g.Cin = Cin;
  g.TW = TW;
  g.TH = TH;
  g.TD = TD;
  g.status = status_ptr(status);
  if (!g.status) return PRIOR_ERR_CUDA;
  CUtensorMap ma, mb;
  const cuuint64_t da[5] = {(cuuint64_t)Cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)nimg};
  const cuuint32_t ba[5] = {prior::BK, (cuuint32_t)TW, (cuuint32_t)TH, (cuuint32_t)TD, 1};
  const cuuint64_t db[2] = {(cuuint64_t)(27 * Cin), (cuuint64_t)Cout};
  const cuuint32_t bb[2] = {prior::BK, (cuuint32_t)bn};
  if (!make_map(&ma, X, 5, da, ba) || !make_map(&mb, Wt, 2, db, bb)) return PRIOR_ERR_ARG;
  return dispatch<prior::CONV3>(bn, ma, mb, g, (cudaStream_t)stream);
}

int prior_conv3x3x3_wgrad_bf16(const void* dYt, const void* X27, float* dW, float* work, int P, int Cout, int Cin,
                               int splits, int* status, void* stream) {
  return wgrad(dYt, X27, dW, work, P, Cout, Cin, 27, splits, status, stream);
}

int prior_last_status(void* stream) {
  int* p = status_ptr(nullptr);
  if (!p) return PRIOR_ERR_CUDA;
  int v = 0;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess ||
      cudaMemcpy(&v, p, 4, cudaMemcpyDeviceToHost) != cudaSuccess || cudaMemset(p, 0, 4) != cudaSuccess)
    return PRIOR_ERR_CUDA;
  return v;
}

}  // extern "C"
