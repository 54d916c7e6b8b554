// prior_ops.cu -- the memory-bound layers of the learned prior's U-Net (the
// denoiser g_theta of Sec. 2.2) around its tensor-core convolutions, each one
// pass over NHWC activations with 16-byte accesses:
//   prior_first_conv_bf16 -- the network input (the noisy model scaled to
//       y = x_t / sqrt(abar_t), edge-padded to the tiled shape, plus the
//       noise-level channel) built on the fly and convolved 3x3 from its 2
//       channels to Cout on the CUDA cores (18 MACs per output: the tensor-core
//       kernel would have to pad the 2 channels to a 64-channel block);
//   prior_pool2_bf16      -- 2 x 2 average pooling (FP32 sum, one rounding);
//   prior_upcat_bf16      -- nearest x2 upsampling of the coarse level joined
//       with the skip connection along channels (the decoder's input);
//   prior_output          -- x0-hat = y + (1x1 output) + bias on the physical
//       part of the padded grid;
// and their forms over NDHWC volumes for the 3D network (prior_first_conv3d_bf16,
// 27 taps x 2 channels per output; prior_pool2_3d_bf16, 2 x 2 x 2;
// prior_upcat3d_bf16; prior_output3d).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "prior.h"

namespace {

constexpr int kThreads = 256;

int grid_blocks(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  return (int)(b < (1LL << 30) ? (b > 0 ? b : 1) : (1LL << 30));
}

__device__ __forceinline__ float bf16_round(float v) { return __bfloat162float(__float2bfloat16(v)); }

// One thread per output pixel and group of 8 output channels.  The 3 x 3 x 2
// inputs of the pixel are rebuilt from x (replicate padding to Hp x Wp, then
// the convolution's zero padding outside), rounded to BF16 as the network's
// input is, and the weights (BF16, [Cout][9][2]) are read through shared
// memory; FP32 accumulation in tap-major order, then bias, ReLU and one BF16
// rounding per output.
__global__ void first_conv_kernel(const float* __restrict__ x, int nimg, int H, int W, int Hp, int Wp, float scale,
                                  const float* __restrict__ sigma, const __nv_bfloat16* __restrict__ Wt,
                                  const float* __restrict__ bias, int Cout, int relu, __nv_bfloat16* __restrict__ Y) {
  extern __shared__ float wsh[];  // [Cout][18] then bias [Cout]
  for (int i = threadIdx.x; i < Cout * 18; i += blockDim.x) wsh[i] = __bfloat162float(Wt[i]);
  for (int i = threadIdx.x; i < Cout; i += blockDim.x) wsh[Cout * 18 + i] = bias ? bias[i] : 0.f;
  __syncthreads();
  const int groups = Cout / 8;
  const long long total = (long long)nimg * Hp * Wp * groups;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(t % groups);
    const long long pix = t / groups;
    const int w = (int)(pix % Wp);
    const int h = (int)((pix / Wp) % Hp);
    const int n = (int)(pix / ((long long)Wp * Hp));
    const float sg = bf16_round(sigma[n]);
    float in0[9], in1[9];
#pragma unroll
    for (int dy = 0; dy < 3; dy++)
#pragma unroll
      for (int dx = 0; dx < 3; dx++) {
        const int yy = h + dy - 1, xx = w + dx - 1;
        const bool inside = yy >= 0 && yy < Hp && xx >= 0 && xx < Wp;
        const int cy = min(max(yy, 0), H - 1), cx = min(max(xx, 0), W - 1);
        in0[dy * 3 + dx] = inside ? bf16_round(scale * x[((long long)n * H + cy) * W + cx]) : 0.f;
        in1[dy * 3 + dx] = inside ? sg : 0.f;
      }
    __align__(16) __nv_bfloat16 out[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const int o = g * 8 + j;
      const float* wo = wsh + o * 18;
      float acc = 0.f;
#pragma unroll
      for (int tap = 0; tap < 9; tap++) {
        acc = fmaf(wo[2 * tap], in0[tap], acc);
        acc = fmaf(wo[2 * tap + 1], in1[tap], acc);
      }
      acc += wsh[Cout * 18 + o];
      if (relu) acc = fmaxf(acc, 0.f);
      out[j] = __float2bfloat16(acc);
    }
    *reinterpret_cast<uint4*>(Y + pix * Cout + g * 8) = *reinterpret_cast<const uint4*>(out);
  }
}

// Y[n][h][w][c] = bf16(mean of X over the 2 x 2 block), 8 channels per thread.
__global__ void pool2_kernel(const __nv_bfloat16* __restrict__ X, int nimg, int H, int W, int C,
                             __nv_bfloat16* __restrict__ Y) {
  const int Ho = H / 2, Wo = W / 2, groups = C / 8;
  const long long total = (long long)nimg * Ho * Wo * groups;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(t % groups);
    const long long pix = t / groups;
    const int w = (int)(pix % Wo);
    const int h = (int)((pix / Wo) % Ho);
    const int n = (int)(pix / ((long long)Wo * Ho));
    float acc[8];
#pragma unroll
    for (int j = 0; j < 8; j++) acc[j] = 0.f;
#pragma unroll
    for (int dy = 0; dy < 2; dy++)
#pragma unroll
      for (int dx = 0; dx < 2; dx++) {
        const uint4 v = *reinterpret_cast<const uint4*>(
            X + (((long long)n * H + 2 * h + dy) * W + 2 * w + dx) * C + g * 8);
        const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
        for (int j = 0; j < 8; j++) acc[j] += __bfloat162float(e[j]);
      }
    __align__(16) __nv_bfloat16 out[8];
#pragma unroll
    for (int j = 0; j < 8; j++) out[j] = __float2bfloat16(0.25f * acc[j]);
    *reinterpret_cast<uint4*>(Y + pix * C + g * 8) = *reinterpret_cast<const uint4*>(out);
  }
}

// Y[n][h][w][:C1] = Lo[n][h/2][w/2][:], Y[n][h][w][C1:] = Skip[n][h][w][:] (exact copies).
__global__ void upcat_kernel(const __nv_bfloat16* __restrict__ Lo, int C1, const __nv_bfloat16* __restrict__ Skip,
                             int C2, int nimg, int H, int W, __nv_bfloat16* __restrict__ Y) {
  const int C = C1 + C2, groups = C / 8;
  const long long total = (long long)nimg * H * W * groups;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(t % groups);
    const long long pix = t / groups;
    const int w = (int)(pix % W);
    const int h = (int)((pix / W) % H);
    const int n = (int)(pix / ((long long)W * H));
    const int c = g * 8;
    uint4 v;
    if (c < C1)
      v = *reinterpret_cast<const uint4*>(Lo + (((long long)n * (H / 2) + h / 2) * (W / 2) + w / 2) * C1 + c);
    else
      v = *reinterpret_cast<const uint4*>(Skip + pix * C2 + (c - C1));
    *reinterpret_cast<uint4*>(Y + pix * C + c) = v;
  }
}

// out[n][h][w] = scale * x[n][h][w] + D[((n * Hp + h) * Wp + w) * ldd] + bo.
__global__ void output_kernel(const float* __restrict__ D, int ldd, const float* __restrict__ x, int nimg, int H,
                              int W, int Hp, int Wp, float scale, float bo, float* __restrict__ out) {
  const long long total = (long long)nimg * H * W;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int w = (int)(t % W);
    const int h = (int)((t / W) % H);
    const int n = (int)(t / ((long long)W * H));
    out[t] = scale * x[t] + D[(((long long)n * Hp + h) * Wp + w) * ldd] + bo;
  }
}

// ---- 3D forms (NDHWC volumes of the 3D network), same conventions ----

// First layer over volumes: 27 taps x 2 channels per output (tap-major order,
// dz slowest), replicate padding of x from [D][H][W] to [Dp][Hp][Wp], zero
// padding around that.  Weights [Cout][27][2] through shared memory.
__global__ void first_conv3d_kernel(const float* __restrict__ x, int nimg, int D, int H, int W, int Dp, int Hp,
                                    int Wp, float scale, const float* __restrict__ sigma,
                                    const __nv_bfloat16* __restrict__ Wt, const float* __restrict__ bias, int Cout,
                                    int relu, __nv_bfloat16* __restrict__ Y) {
  extern __shared__ float wsh[];  // [Cout][54] then bias [Cout]
  for (int i = threadIdx.x; i < Cout * 54; i += blockDim.x) wsh[i] = __bfloat162float(Wt[i]);
  for (int i = threadIdx.x; i < Cout; i += blockDim.x) wsh[Cout * 54 + i] = bias ? bias[i] : 0.f;
  __syncthreads();
  const int groups = Cout / 8;
  const long long total = (long long)nimg * Dp * Hp * Wp * groups;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(t % groups);
    const long long pix = t / groups;
    const int w = (int)(pix % Wp);
    const int h = (int)((pix / Wp) % Hp);
    const int d = (int)((pix / ((long long)Wp * Hp)) % Dp);
    const int n = (int)(pix / ((long long)Wp * Hp * Dp));
    const float sg = bf16_round(sigma[n]);
    float in0[27];
    bool inside[27];
#pragma unroll
    for (int dz = 0; dz < 3; dz++)
#pragma unroll
      for (int dy = 0; dy < 3; dy++)
#pragma unroll
        for (int dx = 0; dx < 3; dx++) {
          const int zz = d + dz - 1, yy = h + dy - 1, xx = w + dx - 1;
          const int tap = (dz * 3 + dy) * 3 + dx;
          inside[tap] = zz >= 0 && zz < Dp && yy >= 0 && yy < Hp && xx >= 0 && xx < Wp;
          const int cz = min(max(zz, 0), D - 1), cy = min(max(yy, 0), H - 1), cx = min(max(xx, 0), W - 1);
          in0[tap] = inside[tap] ? bf16_round(scale * x[(((long long)n * D + cz) * H + cy) * W + cx]) : 0.f;
        }
    __align__(16) __nv_bfloat16 out[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const int o = g * 8 + j;
      const float* wo = wsh + o * 54;
      float acc = 0.f;
#pragma unroll
      for (int tap = 0; tap < 27; tap++) {
        acc = fmaf(wo[2 * tap], in0[tap], acc);
        acc = fmaf(wo[2 * tap + 1], inside[tap] ? sg : 0.f, acc);
      }
      acc += wsh[Cout * 54 + o];
      if (relu) acc = fmaxf(acc, 0.f);
      out[j] = __float2bfloat16(acc);
    }
    *reinterpret_cast<uint4*>(Y + pix * Cout + g * 8) = *reinterpret_cast<const uint4*>(out);
  }
}

// Y[n][d][h][w][c] = bf16(mean of X over the 2 x 2 x 2 block), 8 channels per thread.
__global__ void pool2_3d_kernel(const __nv_bfloat16* __restrict__ X, int nimg, int D, int H, int W, int C,
                                __nv_bfloat16* __restrict__ Y) {
  const int Do = D / 2, Ho = H / 2, Wo = W / 2, groups = C / 8;
  const long long total = (long long)nimg * Do * Ho * Wo * groups;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(t % groups);
    const long long pix = t / groups;
    const int w = (int)(pix % Wo);
    const int h = (int)((pix / Wo) % Ho);
    const int d = (int)((pix / ((long long)Wo * Ho)) % Do);
    const int n = (int)(pix / ((long long)Wo * Ho * Do));
    float acc[8];
#pragma unroll
    for (int j = 0; j < 8; j++) acc[j] = 0.f;
#pragma unroll
    for (int dz = 0; dz < 2; dz++)
#pragma unroll
      for (int dy = 0; dy < 2; dy++)
#pragma unroll
        for (int dx = 0; dx < 2; dx++) {
          const uint4 v = *reinterpret_cast<const uint4*>(
              X + ((((long long)n * D + 2 * d + dz) * H + 2 * h + dy) * W + 2 * w + dx) * C + g * 8);
          const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
          for (int j = 0; j < 8; j++) acc[j] += __bfloat162float(e[j]);
        }
    __align__(16) __nv_bfloat16 out[8];
#pragma unroll
    for (int j = 0; j < 8; j++) out[j] = __float2bfloat16(0.125f * acc[j]);
    *reinterpret_cast<uint4*>(Y + pix * C + g * 8) = *reinterpret_cast<const uint4*>(out);
  }
}

// Y[n][d][h][w][:C1] = Lo[n][d/2][h/2][w/2][:], Y[...][C1:] = Skip[n][d][h][w][:] (exact copies).
__global__ void upcat3d_kernel(const __nv_bfloat16* __restrict__ Lo, int C1, const __nv_bfloat16* __restrict__ Skip,
                               int C2, int nimg, int D, int H, int W, __nv_bfloat16* __restrict__ Y) {
  const int C = C1 + C2, groups = C / 8;
  const long long total = (long long)nimg * D * H * W * groups;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(t % groups);
    const long long pix = t / groups;
    const int w = (int)(pix % W);
    const int h = (int)((pix / W) % H);
    const int d = (int)((pix / ((long long)W * H)) % D);
    const int n = (int)(pix / ((long long)W * H * D));
    const int c = g * 8;
    uint4 v;
    if (c < C1)
      v = *reinterpret_cast<const uint4*>(
          Lo + ((((long long)n * (D / 2) + d / 2) * (H / 2) + h / 2) * (W / 2) + w / 2) * C1 + c);
    else
      v = *reinterpret_cast<const uint4*>(Skip + pix * C2 + (c - C1));
    *reinterpret_cast<uint4*>(Y + pix * C + c) = v;
  }
}

// out[n][d][h][w] = scale * x[n][d][h][w] + Dm[(((n * Dp + d) * Hp + h) * Wp + w) * ldd] + bo.
__global__ void output3d_kernel(const float* __restrict__ Dm, int ldd, const float* __restrict__ x, int nimg, int D,
                                int H, int W, int Dp, int Hp, int Wp, float scale, float bo, float* __restrict__ out) {
  const long long total = (long long)nimg * D * H * W;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int w = (int)(t % W);
    const int h = (int)((t / W) % H);
    const int d = (int)((t / ((long long)W * H)) % D);
    const int n = (int)(t / ((long long)W * H * D));
    out[t] = scale * x[t] + Dm[((((long long)n * Dp + d) * Hp + h) * Wp + w) * ldd] + bo;
  }
}

bool a16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace

extern "C" {

int prior_first_conv_bf16(const float* x, int nimg, int H, int W, int Hp, int Wp, float scale, const float* sigma,
                          const void* Wt, const float* bias, int Cout, int relu, void* Y, void* stream) {
  if (!x || !sigma || !Wt || !Y || nimg < 1 || H < 1 || W < 1 || Hp < H || Wp < W) return PRIOR_ERR_ARG;
  if (Cout < 8 || Cout % 8 || Cout > 256 || !a16(Y)) return PRIOR_ERR_ARG;
  const size_t sh = (size_t)(Cout * 19) * 4;
  first_conv_kernel<<<grid_blocks((long long)nimg * Hp * Wp * (Cout / 8)), kThreads, sh, (cudaStream_t)stream>>>(
      x, nimg, H, W, Hp, Wp, scale, sigma, reinterpret_cast<const __nv_bfloat16*>(Wt), bias, Cout, relu,
      reinterpret_cast<__nv_bfloat16*>(Y));
  return cudaGetLastError() == cudaSuccess ? PRIOR_OK : PRIOR_ERR_CUDA;
}

int prior_pool2_bf16(const void* X, int nimg, int H, int W, int C, void* Y, void* stream) {
  if (!X || !Y || nimg < 1 || H < 2 || W < 2 || H % 2 || W % 2 || C < 8 || C % 8 || !a16(X) || !a16(Y))
    return PRIOR_ERR_ARG;
  pool2_kernel<<<grid_blocks((long long)nimg * (H / 2) * (W / 2) * (C / 8)), kThreads, 0, (cudaStream_t)stream>>>(
      reinterpret_cast<const __nv_bfloat16*>(X), nimg, H, W, C, reinterpret_cast<__nv_bfloat16*>(Y));
  return cudaGetLastError() == cudaSuccess ? PRIOR_OK : PRIOR_ERR_CUDA;
}

int prior_upcat_bf16(const void* Lo, int C1, const void* Skip, int C2, int nimg, int H, int W, void* Y,
                     void* stream) {
  if (!Lo || !Skip || !Y || nimg < 1 || H < 2 || W < 2 || H % 2 || W % 2 || C1 < 8 || C1 % 8 || C2 < 8 ||
      C2 % 8 || !a16(Lo) || !a16(Skip) || !a16(Y))
    return PRIOR_ERR_ARG;
  upcat_kernel<<<grid_blocks((long long)nimg * H * W * ((C1 + C2) / 8)), kThreads, 0, (cudaStream_t)stream>>>(
      reinterpret_cast<const __nv_bfloat16*>(Lo), C1, reinterpret_cast<const __nv_bfloat16*>(Skip), C2, nimg, H, W,
      reinterpret_cast<__nv_bfloat16*>(Y));
  return cudaGetLastError() == cudaSuccess ? PRIOR_OK : PRIOR_ERR_CUDA;
}

int prior_output(const float* D, int ldd, const float* x, int nimg, int H, int W, int Hp, int Wp, float scale,
                 float bo, float* out, void* stream) {
  if (!D || !x || !out || nimg < 1 || H < 1 || W < 1 || Hp < H || Wp < W || ldd < 1) return PRIOR_ERR_ARG;
  output_kernel<<<grid_blocks((long long)nimg * H * W), kThreads, 0, (cudaStream_t)stream>>>(D, ldd, x, nimg, H, W,
                                                                                           Hp, Wp, scale, bo, out);
  return cudaGetLastError() == cudaSuccess ? PRIOR_OK : PRIOR_ERR_CUDA;
}

int prior_first_conv3d_bf16(const float* x, int nimg, int D, int H, int W, int Dp, int Hp, int Wp, float scale,
                            const float* sigma, const void* Wt, const float* bias, int Cout, int relu, void* Y,
                            void* stream) {
  if (!x || !sigma || !Wt || !Y || nimg < 1 || D < 1 || H < 1 || W < 1 || Dp < D || Hp < H || Wp < W)
    return PRIOR_ERR_ARG;
  if (Cout < 8 || Cout % 8 || Cout > 128 || !a16(Y)) return PRIOR_ERR_ARG;
  const size_t sh = (size_t)(Cout * 55) * 4;
  first_conv3d_kernel<<<grid_blocks((long long)nimg * Dp * Hp * Wp * (Cout / 8)), kThreads, sh,
                        (cudaStream_t)stream>>>(x, nimg, D, H, W, Dp, Hp, Wp, scale, sigma,
                                                reinterpret_cast<const __nv_bfloat16*>(Wt), bias, Cout, relu,
                                                reinterpret_cast<__nv_bfloat16*>(Y));
  return cudaGetLastError() == cudaSuccess ? PRIOR_OK : PRIOR_ERR_CUDA;
}

int prior_pool2_3d_bf16(const void* X, int nimg, int D, int H, int W, int C, void* Y, void* stream) {
  if (!X || !Y || nimg < 1 || D < 2 || H < 2 || W < 2 || D % 2 || H % 2 || W % 2 || C < 8 || C % 8 || !a16(X) ||
      !a16(Y))
    return PRIOR_ERR_ARG;
  pool2_3d_kernel<<<grid_blocks((long long)nimg * (D / 2) * (H / 2) * (W / 2) * (C / 8)), kThreads, 0,
                    (cudaStream_t)stream>>>(reinterpret_cast<const __nv_bfloat16*>(X), nimg, D, H, W, C,
                                            reinterpret_cast<__nv_bfloat16*>(Y));
  return cudaGetLastError() == cudaSuccess ? PRIOR_OK : PRIOR_ERR_CUDA;
}

int prior_upcat3d_bf16(const void* Lo, int C1, const void* Skip, int C2, int nimg, int D, int H, int W, void* Y,
                       void* stream) {
  if (!Lo || !Skip || !Y || nimg < 1 || D < 2 || H < 2 || W < 2 || D % 2 || H % 2 || W % 2 || C1 < 8 || C1 % 8 ||
      C2 < 8 || C2 % 8 || !a16(Lo) || !a16(Skip) || !a16(Y))
    return PRIOR_ERR_ARG;
  upcat3d_kernel<<<grid_blocks((long long)nimg * D * H * W * ((C1 + C2) / 8)), kThreads, 0, (cudaStream_t)stream>>>(
      reinterpret_cast<const __nv_bfloat16*>(Lo), C1, reinterpret_cast<const __nv_bfloat16*>(Skip), C2, nimg, D, H,
      W, reinterpret_cast<__nv_bfloat16*>(Y));
  return cudaGetLastError() == cudaSuccess ? PRIOR_OK : PRIOR_ERR_CUDA;
}

int prior_output3d(const float* Dm, int ldd, const float* x, int nimg, int D, int H, int W, int Dp, int Hp, int Wp,
                   float scale, float bo, float* out, void* stream) {
  if (!Dm || !x || !out || nimg < 1 || D < 1 || H < 1 || W < 1 || Dp < D || Hp < H || Wp < W || ldd < 1)
    return PRIOR_ERR_ARG;
  output3d_kernel<<<grid_blocks((long long)nimg * D * H * W), kThreads, 0, (cudaStream_t)stream>>>(
      Dm, ldd, x, nimg, D, H, W, Dp, Hp, Wp, scale, bo, out);
  return cudaGetLastError() == cudaSuccess ? PRIOR_OK : PRIOR_ERR_CUDA;
}

}  // extern "C"
