// noalloc.cu -- fwi_residual_misfit_noalloc: the encoded residual and misfit
// for callers that must not allocate device memory.
//
// Its scratch (FP64 per-block partial sums, the copied encoding and the
// derived shot lists) lives in one file-scope device array of
// FWI_NOALLOC_MAX_BYTES, which every GPU that loads this library keeps until
// the process exits.  Host code cannot use the array's name as a device
// address, so on the first call on each device (with that device current) the
// address is looked up once with cudaGetSymbolAddress and cached.  Every call
// reuses the same array and keeps the last call's contents; each call writes
// every piece of it before reading it (the per-block partial sums are stores,
// not accumulations), so nothing needs clearing.  Calls that overlap on the
// GPU (different streams, or different host threads) race on it.
#include <string.h>

#include "fwi_internal.cuh"

namespace {

constexpr int NOALLOC_NBLK = 64;
constexpr int MAX_DEVICES = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[FWI_NOALLOC_MAX_BYTES];
void* g_scratch_addr[MAX_DEVICES] = {};

int scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return FWI_ERR_CUDA;
  if (dev < 0 || dev >= MAX_DEVICES) return FWI_ERR_ARG;
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return FWI_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return FWI_OK;
}

size_t up256(size_t n) { return (n + 255) / 256 * 256; }

// Shot lists of every wavefield b = s * nsg + j from the copied encoding:
// shots perm[s][off_j .. off_j + sg[j]) with the weights w[s][shot id].
__global__ void noalloc_lists_kernel(int nsamp, int ns, int nsg, const int* __restrict__ perm,
                                     const int8_t* __restrict__ w, const int* __restrict__ sg, int* shot_off,
                                     int* shot_id, float* shot_w) {
  const int B = nsamp * nsg;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const int s = b / nsg, j = b - s * nsg;
  int tot = 0, off = 0;
  for (int k = 0; k < nsg; k++) {
    if (k < j) off += sg[k];
    tot += sg[k];
  }
  const int base = s * tot + off;
  shot_off[b] = base;
  if (b == B - 1) shot_off[B] = nsamp * tot;
  for (int k = 0; k < sg[j]; k++) {
    const int id = perm[s * ns + off + k];
    shot_id[base + k] = id;
    shot_w[base + k] = (float)w[s * ns + id];
  }
}

}  // namespace

extern "C" int fwi_residual_misfit_noalloc(const float* d_pred, const float* d_obs, int nsamp, int ns, int nt, int nr,
                                           const int32_t* perm, const int8_t* w, const int32_t* sg_sizes, int nsg,
                                           double sigma_y, double scale, float* rhat, double* misfit, void* stream) {
  if (!d_pred || !d_obs || !perm || !w || !sg_sizes || !rhat || !misfit) return FWI_ERR_ARG;
  if (nsamp < 1 || ns < 1 || nt < 1 || nr < 1 || nsg < 1 || !(sigma_y > 0)) return FWI_ERR_ARG;
  long long tot = 0;
  for (int j = 0; j < nsg; j++) {
    if (sg_sizes[j] < 1) return FWI_ERR_ARG;
    tot += sg_sizes[j];
  }
  if (tot > ns) return FWI_ERR_ARG;
  for (long long i = 0; i < (long long)nsamp * ns; i++)
    if (perm[i] < 0 || perm[i] >= ns || (w[i] != 1 && w[i] != -1)) return FWI_ERR_ARG;
  if (!(scale > 0)) scale = (double)ns / (double)tot;

  // scratch layout, each piece 256-byte aligned
  const long long B = (long long)nsamp * nsg;
  const size_t o_part = 0;
  const size_t o_off = o_part + up256((size_t)B * NOALLOC_NBLK * 8);
  const size_t o_id = o_off + up256((size_t)(B + 1) * 4);
  const size_t o_w = o_id + up256((size_t)(nsamp * tot) * 4);
  const size_t o_perm = o_w + up256((size_t)(nsamp * tot) * 4);
  const size_t o_wt = o_perm + up256((size_t)nsamp * ns * 4);
  const size_t o_sg = o_wt + up256((size_t)nsamp * ns);
  const size_t need = o_sg + up256((size_t)nsg * 4);
  if (need > (size_t)FWI_NOALLOC_MAX_BYTES || B > (1 << 30)) return FWI_ERR_ARG;

  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != FWI_OK) return rc;
  unsigned char* S = static_cast<unsigned char*>(base);
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(S + o_perm, perm, (size_t)nsamp * ns * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(S + o_wt, w, (size_t)nsamp * ns, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(S + o_sg, sg_sizes, (size_t)nsg * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return FWI_ERR_CUDA;
  noalloc_lists_kernel<<<(int)((B + 127) / 128), 128, 0, st>>>(
      nsamp, ns, nsg, reinterpret_cast<const int*>(S + o_perm), reinterpret_cast<const int8_t*>(S + o_wt),
      reinterpret_cast<const int*>(S + o_sg), reinterpret_cast<int*>(S + o_off), reinterpret_cast<int*>(S + o_id),
      reinterpret_cast<float*>(S + o_w));
  if (cudaGetLastError() != cudaSuccess) return FWI_ERR_CUDA;
  const double inv_s2 = 1.0 / (sigma_y * sigma_y);
  if (fwi::launch_residual((int)B, nt, nr, d_pred, d_obs, reinterpret_cast<const int*>(S + o_off),
                           reinterpret_cast<const int*>(S + o_id), reinterpret_cast<const float*>(S + o_w), inv_s2,
                           rhat, reinterpret_cast<double*>(S + o_part), NOALLOC_NBLK, st) != cudaSuccess)
    return FWI_ERR_CUDA;
  if (fwi::launch_misfit(nsamp, nsg, reinterpret_cast<const double*>(S + o_part), NOALLOC_NBLK, scale * 0.5 * inv_s2,
                         misfit, nullptr, st) != cudaSuccess)
    return FWI_ERR_CUDA;
  return FWI_OK;
}
