// prior.h -- C ABI of the tensor-core kernels of the learned prior: the
// network g_theta that predicts the clean model from a noisy one (Sec. 2.2,
// eq. for x0-hat; trained on velocity-model patches, Sec. 3.1).  The network
// is a small U-Net of 3x3 (3D models: 3x3x3) convolutions; these entry points run its
// contractions in BF16 with FP32 accumulation on the tensor cores.
//
// Conventions: all pointers are device pointers owned by the caller and
// 16-byte aligned; calls are asynchronous on `stream` (a cudaStream_t, null =
// legacy default stream).  A return value < 0 is an argument or launch error
// and nothing was launched, except PRIOR_ERR_CUDA, which carries a failed
// launch.  Device-side timeouts of the kernels' bounded waits are recorded in
// *status (a device int the caller zeroes; null selects an internal word read
// by prior_last_status).
#pragma once
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum prior_status {
  PRIOR_OK = 0,
  PRIOR_ERR_ARG = -1,
  PRIOR_ERR_CUDA = -4,
  PRIOR_ERR_TIMEOUT = -6,
};

// D = A * B^T (+ bias) (ReLU if relu != 0).
//   A: [M][K] BF16 row-major (K contiguous); B: [N][K] BF16 row-major;
//   D: [M][ldd] FP32 (d_bf16 = 0) or BF16 (d_bf16 = 1); bias: [N] FP32 or null.
// Requires M % 128 == 0, K % 64 == 0 and N in {32, 64, 128, 256} or a
// multiple of 64; ldd >= N and ldd % 8 == 0.
int prior_gemm_bf16(const void* A, const void* B, void* D, int M, int N, int K, int ldd, int d_bf16,
                    const float* bias, int relu, int* status, void* stream);

// Y = conv3x3(X, Wt) (+ bias) (ReLU if relu != 0), stride 1, zero padding 1
// ("same" size), cross-correlation as in the usual CNN definition:
//   Y[n][y][x][o] = sum_{dy,dx in 0..2} sum_c Wt[o][dy*3+dx][c] * X[n][y+dy-1][x+dx-1][c].
//   X: [nimg][H][W][Cin] BF16 (NHWC); Wt: [Cout][9][Cin] BF16;
//   Y: [nimg][H][W][Cout] FP32 (y_bf16 = 0) or BF16 (y_bf16 = 1); bias: [Cout] FP32 or null.
// Requires Cin % 64 == 0; Cout in {32, 64, 128, 256} or a multiple of 64;
// W a power of two <= 128 or a multiple of 128; H * min(W, 128) a multiple of 128.
// The data gradient of this layer is the same call on the output gradient
// with weights Wt'[c][8 - t][o] = Wt[o][t][c].
int prior_conv3x3_bf16(const void* X, const void* Wt, void* Y, int nimg, int H, int W, int Cin, int Cout,
                       int y_bf16, const float* bias, int relu, int* status, void* stream);

// Weight gradient of prior_conv3x3_bf16, accumulated:
//   dW[o][t][c] += sum_p dYt[o][p] * X9[t][c][p],
// where X9[t][c][p] = X[n][y+dy-1][x+dx-1][c] (zero off the image) for pixel
// p = (n, y, x) and tap t = dy*3 + dx, i.e. the input's tap-shifted copies.
//   dYt: [ceil(Cout/128)*128][P] BF16 (channel-major output gradient; rows
//        >= Cout are read but not used); X9: [9][Cin][P] BF16;
//   dW: [Cout][9][Cin] FP32, accumulated (zero it first).
// The pixels are split into `splits` ranges per tap for parallelism.  With a
// workspace `work` of splits * Cout * 9 * Cin floats (16-byte aligned), each
// range stores its partial sum in its own slice and a second kernel adds the
// slices to dW in range order: the result is the same on every run.  With
// work = null the ranges add into dW with FP32 atomics, whose order (and so
// the last bits) varies between runs.  Requires P % 64 == 0 and Cin in
// {32, 64, 128, 256} or a multiple of 64.
int prior_conv3x3_wgrad_bf16(const void* dYt, const void* X9, float* dW, float* work, int P, int Cout, int Cin,
                             int splits, int* status, void* stream);

// 3D counterpart of prior_conv3x3_bf16 for volume patches (the prior of the
// 3D models): same-size 3x3x3 cross-correlation with zero padding 1,
//   Y[n][z][y][x][o] = sum_{dz,dy,dx in 0..2} sum_c Wt[o][dz*9+dy*3+dx][c] X[n][z+dz-1][y+dy-1][x+dx-1][c].
//   X: [nimg][D][H][W][Cin] BF16 (NDHWC); Wt: [Cout][27][Cin] BF16;
//   Y: [nimg][D][H][W][Cout] FP32 (y_bf16 = 0) or BF16 (y_bf16 = 1); bias: [Cout] FP32 or null.
// Requires Cin % 64 == 0; Cout as prior_conv3x3_bf16; W a multiple of 128,
// or a power of two < 128 with H * W a multiple of 128, or H and W powers of
// two with H * W < 128 and D * H * W a multiple of 128.  The data gradient
// is the same call with weights Wt'[c][26 - t][o] = Wt[o][t][c].
int prior_conv3x3x3_bf16(const void* X, const void* Wt, void* Y, int nimg, int D, int H, int W, int Cin, int Cout,
                         int y_bf16, const float* bias, int relu, int* status, void* stream);

// Weight gradient of prior_conv3x3x3_bf16, accumulated:
//   dW[o][t][c] += sum_p dYt[o][p] * X27[t][c][p],
// with X27 the input's 27 tap-shifted copies (t = dz*9 + dy*3 + dx) and the
// other conventions of prior_conv3x3_wgrad_bf16 (splits <= 2427; work of
// splits * Cout * 27 * Cin floats, or null).
int prior_conv3x3x3_wgrad_bf16(const void* dYt, const void* X27, float* dW, float* work, int P, int Cout, int Cin,
                               int splits, int* status, void* stream);

// The memory-bound layers around the convolutions (csrc/prior_ops.cu); all
// activations are BF16 NHWC with C a multiple of 8, pointers 16-byte aligned.
//
// First layer of the network: the input image is the noisy model scaled,
// y = scale * x (x_t / sqrt(abar_t) for scale = 1/sqrt(abar_t), Sec. 2.2),
// edge-replicated from [H][W] to the tiled shape [Hp][Wp], as channel 0, and
// the noise level sigma[n] as channel 1, both rounded to BF16; then the same
// 3x3 convolution as prior_conv3x3_bf16 (zero padding 1 around [Hp][Wp]),
//   Y[n][h][w][o] = relu?(bias[o] + sum_{dy,dx} sum_{c<2} Wt[o][dy*3+dx][c] * in_c(h+dy-1, w+dx-1)),
// with FP32 accumulation on the CUDA cores (18 products per output).
//   x: [nimg][H][W] FP32; sigma: [nimg] FP32; Wt: [Cout][9][2] BF16; bias: [Cout] FP32 or null;
//   Y: [nimg][Hp][Wp][Cout] BF16; 8 <= Cout <= 256, Cout % 8 == 0.
int prior_first_conv_bf16(const float* x, int nimg, int H, int W, int Hp, int Wp, float scale, const float* sigma,
                          const void* Wt, const float* bias, int Cout, int relu, void* Y, void* stream);

// 2 x 2 average pooling: Y[n][h][w][c] = BF16(FP32 sum of X[n][2h..2h+1][2w..2w+1][c] / 4).
//   X: [nimg][H][W][C]; Y: [nimg][H/2][W/2][C]; H, W even.
int prior_pool2_bf16(const void* X, int nimg, int H, int W, int C, void* Y, void* stream);

// Decoder input: nearest x2 upsampling of the coarse level joined with the skip
// connection along channels (exact copies):
//   Y[n][h][w][c] = Lo[n][h/2][w/2][c] for c < C1, Skip[n][h][w][c - C1] otherwise.
//   Lo: [nimg][H/2][W/2][C1]; Skip: [nimg][H][W][C2]; Y: [nimg][H][W][C1 + C2]; H, W even.
int prior_upcat_bf16(const void* Lo, int C1, const void* Skip, int C2, int nimg, int H, int W, void* Y,
                     void* stream);

// Network output on the physical part of the padded grid:
//   out[n][h][w] = scale * x[n][h][w] + D[((n*Hp + h)*Wp + w) * ldd] + bo,
// D the FP32 result of the 1x1 output layer over the padded grid (column 0 of
// rows of ldd floats), x and out [nimg][H][W] FP32.
int prior_output(const float* D, int ldd, const float* x, int nimg, int H, int W, int Hp, int Wp, float scale,
                 float bo, float* out, void* stream);

// The same four layers over volumes, for the 3D network (NDHWC, [nimg][D][H][W][C]):
//   prior_first_conv3d_bf16: x [nimg][D][H][W] FP32 edge-replicated to [Dp][Hp][Wp];
//     the 3x3x3 convolution of prior_conv3x3x3_bf16 (tap = dz*9 + dy*3 + dx) over
//     the 2-channel input, Wt [Cout][27][2] BF16, 54 products per output;
//     Y [nimg][Dp][Hp][Wp][Cout] BF16; 8 <= Cout <= 128, Cout % 8 == 0.
//   prior_pool2_3d_bf16: 2 x 2 x 2 average (FP32 sum / 8, one rounding); D, H, W even.
//   prior_upcat3d_bf16: Y[n][d][h][w][c] = Lo[n][d/2][h/2][w/2][c] for c < C1,
//     Skip[n][d][h][w][c - C1] otherwise; D, H, W even.
//   prior_output3d: out[n][d][h][w] = scale * x[n][d][h][w] + D[(((n*Dp + d)*Hp + h)*Wp + w) * ldd] + bo.
// Errors as above: PRIOR_ERR_ARG for a null or unaligned pointer or a size out
// of range (nothing launched), PRIOR_ERR_CUDA if the launch fails.
int prior_first_conv3d_bf16(const float* x, int nimg, int D, int H, int W, int Dp, int Hp, int Wp, float scale,
                            const float* sigma, const void* Wt, const float* bias, int Cout, int relu, void* Y,
                            void* stream);
int prior_pool2_3d_bf16(const void* X, int nimg, int D, int H, int W, int C, void* Y, void* stream);
int prior_upcat3d_bf16(const void* Lo, int C1, const void* Skip, int C2, int nimg, int D, int H, int W, void* Y,
                       void* stream);
int prior_output3d(const float* Dm, int ldd, const float* x, int nimg, int D, int H, int W, int Dp, int Hp, int Wp,
                   float scale, float bo, float* out, void* stream);

// Reads and clears the internal status word (synchronises the stream).
int prior_last_status(void* stream);

#ifdef __cplusplus
}
#endif
