// aux.cu -- the light kernels around the time-step loop: velocity padding,
// Ricker table, encoded residual and misfit, source-point imaging term,
// gradient fold, Langevin step, DDPM re-noise and the smoothness prior.
#include <math.h>

#include "fwi_internal.cuh"

namespace fwi {

// Blocks of 256 threads for a grid-stride loop over n elements: enough for
// every element, at most `per_sm` resident blocks on each SM of the current
// device (the SM count is queried once per device).
static int num_sms() {
  static int cached[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
  if (dev < 64 && cached[dev] > 0) return cached[dev];
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
  if (dev < 64) cached[dev] = n;
  return n;
}

static inline int grid_for(long long n, int per_sm) {
  const long long cap = (long long)num_sms() * per_sm;
  const long long b = (n + 255) / 256;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

// ------------------------------------------------------------------ setup --

// cc = v^2 dt^2 / (1 + gamma dt) on the padded grid, velocity edge-replicated
// into the sponge, gamma dt = gz[z] + gy[y] + gx[x] from the per-axis table.
// Velocities above vmax_cfl (the stability bound checked at creation) are
// flagged in the status word.
__global__ void expand_kernel(const Layout L, const float* __restrict__ vel, int nsamp, double dt,
                              const float* __restrict__ gtab, float* c, float vmax_cfl, int* status) {
  const long long npad = (long long)L.nzp * L.nyp * L.nxp;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npad * nsamp;
       i += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(i / npad);
    long long k = i - (long long)s * npad;
    const int x = (int)(k % L.nxp);
    k /= L.nxp;
    const int y = (int)(k % L.nyp);
    const int z = (int)(k / L.nyp);
    const int pz = min(max(z - L.nb, 0), L.nz - 1);
    const int px = min(max(x - L.nb, 0), L.nx - 1);
    const int py = L.ndim == 3 ? min(max(y - L.nb, 0), L.ny - 1) : 0;
    const float v = vel[(long long)s * L.phys + ((long long)pz * (L.ndim == 3 ? L.ny : 1) + py) * L.nx + px];
    if (!(v <= vmax_cfl) || !(v > 0.f)) atomicCAS(status, 0, (int)FWI_ERR_CFL);
    const float g = gtab[z] + (L.ndim == 3 ? gtab[L.nzp + y] : 0.f) + gtab[L.nzp + L.nyp + x];
    c[(long long)s * L.field + L.off(z, y, x)] = (float)((double)v * (double)v * dt * dt) * __fdividef(1.0f, 1.0f + g);
  }
}

cudaError_t launch_expand(const Layout& L, const float* vel, int nsamp, double dt, const float* gtab, float* c,
                          float vmax_cfl, int* status, cudaStream_t st) {
  const long long n = (long long)L.nzp * L.nyp * L.nxp * nsamp;
  const int blocks = grid_for(n, 32);
  expand_kernel<<<blocks, 256, 0, st>>>(L, vel, nsamp, dt, gtab, c, vmax_cfl, status);
  return cudaGetLastError();
}

// Ricker samples f(n dt), evaluated in FP64 and rounded once.
__global__ void wavelet_kernel(int nt, double dt, double f0, double t0, float* wav) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nt) return;
  const double a = M_PI * f0 * (n * dt - t0);
  wav[n] = (float)((1.0 - 2.0 * a * a) * exp(-a * a));
}

cudaError_t launch_wavelet(int nt, double dt, double f0, double t0, float* wav, cudaStream_t st) {
  wavelet_kernel<<<(nt + 255) / 256, 256, 0, st>>>(nt, dt, f0, t0, wav);
  return cudaGetLastError();
}

// ---------------------------------------------------------- residual/misfit --

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// r = d_pred - sum_{i in B_b} w_i d_obs_i (encoded observed data formed on the
// fly), rhat = r / sigma^2 (adjoint source), and per-block partial sums of r^2
// in FP64 (fixed reduction order: deterministic).
// rhat may alias dpred (fwi_gradient computes in place): each element is read
// and then written by the same thread, and neither pointer is __restrict__.
__global__ void residual_kernel(int nt, int nr, const float* dpred, const float* __restrict__ dobs,
                                const int* __restrict__ shot_off, const int* __restrict__ shot_id,
                                const float* __restrict__ shot_w, double inv_sigma2, float* rhat, double* part,
                                int nblk) {
  const int b = blockIdx.y;
  const long long ne = (long long)nt * nr;
  const int i0 = shot_off[b], i1 = shot_off[b + 1];
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne;
       e += (long long)gridDim.x * blockDim.x) {
    float enc = 0.f;
    for (int i = i0; i < i1; i++) enc = fmaf(shot_w[i], __ldg(dobs + (long long)shot_id[i] * ne + e), enc);
    const float r = dpred[(long long)b * ne + e] - enc;
    rhat[(long long)b * ne + e] = (float)(r * inv_sigma2);
    acc += (double)r * (double)r;
  }
  __shared__ double sh[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < blockDim.x / 32 ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) part[(long long)b * nblk + blockIdx.x] = v;
  }
}

cudaError_t launch_residual(int B, int nt, int nr, const float* dpred, const float* dobs, const int* shot_off,
                            const int* shot_id, const float* shot_w, double inv_sigma2, float* rhat, double* part,
                            int nblk, cudaStream_t st) {
  residual_kernel<<<dim3(nblk, B), 256, 0, st>>>(nt, nr, dpred, dobs, shot_off, shot_id, shot_w, inv_sigma2, rhat,
                                                 part, nblk);
  return cudaGetLastError();
}

// misfit[s] = factor * sum over the sample's supergathers and blocks of the
// partials, in a fixed order; NaN/Inf is flagged in the status word.
__global__ void misfit_kernel(int nsg, const double* __restrict__ part, int nblk, double factor, double* misfit,
                              int* status) {
  const int s = blockIdx.x;
  const int n = nsg * nblk;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[(long long)s * n + i];
  __shared__ double sh[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < blockDim.x / 32 ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) {
      misfit[s] = factor * v;
      if (status && !isfinite(v)) atomicCAS(status, 0, (int)FWI_ERR_NONFINITE);
    }
  }
}

cudaError_t launch_misfit(int nsamp, int nsg, const double* part, int nblk, double factor, double* misfit,
                          int* status, cudaStream_t st) {
  misfit_kernel<<<nsamp, 256, 0, st>>>(nsg, part, nblk, factor, misfit, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- imaging --

// Source-point term of the imaging condition: for every merged source entry e
// of wavefield b, tmp[b][e] = amp_e * sum_k q^k(x_e) f((k-1) dt), one warp per entry.
__global__ void source_dot_kernel(int nt, int E, const float* __restrict__ qsrc, const float* __restrict__ wav,
                                  const int* __restrict__ src_cnt, const float* __restrict__ src_amp, float* tmp) {
  const int b = blockIdx.y;
  const int e = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (e >= src_cnt[b]) return;
  double acc = 0.0;
  for (int k = lane; k < nt; k += 32) acc += (double)qsrc[((long long)b * nt + k) * E + e] * (double)wav[k];
  acc = warp_sum(acc);
  if (lane == 0) tmp[(long long)b * E + e] = (float)(acc * src_amp[(long long)b * E + e]);
}

// Adds tmp into the imaging accumulators in a fixed (supergather, entry)
// order; wavefield b's accumulator is b / wf_per_acc (one per wavefield, per
// pair of supergathers, or per sample).
__global__ void source_add_kernel(int nsg, int E, const int* __restrict__ src_cnt,
                                  const long long* __restrict__ src_pos, const float* __restrict__ tmp, float* grad,
                                  long long field, int wf_per_acc) {
  const int s = blockIdx.x;
  if (threadIdx.x != 0) return;
  for (int j = 0; j < nsg; j++) {
    const int b = s * nsg + j;
    float* g = grad + (long long)(b / wf_per_acc) * field;
    for (int e = 0; e < src_cnt[b]; e++) g[src_pos[(long long)b * E + e]] += tmp[(long long)b * E + e];
  }
}

cudaError_t launch_source_imaging(int B, int nsg, int nt, int E, const float* qsrc, const float* wav,
                                  const int* src_cnt, const long long* src_pos, const float* src_amp, float* tmp,
                                  float* grad, long long field, int wf_per_acc, cudaStream_t st) {
  if (E <= 0) return cudaSuccess;
  source_dot_kernel<<<dim3((E + 7) / 8, B), 256, 0, st>>>(nt, E, qsrc, wav, src_cnt, src_amp, tmp);
  source_add_kernel<<<B / nsg, 32, 0, st>>>(nsg, E, src_cnt, src_pos, tmp, grad, field, wf_per_acc);
  return cudaGetLastError();
}

// grad_v[phys] = scale * (2 / v) * sum of G over the padded cells that replicate
// the physical cell (adjoint of edge replication; dc/dv = 2 v dt^2 and G holds
// c * dJ/dc), summed over the g_per_sample accumulators of each sample.
__global__ void finalize_kernel(const Layout L, const float* __restrict__ vel, const float* __restrict__ G,
                                int nsamp, int g_per_sample, double scale, float* grad) {
  const int ny = L.ndim == 3 ? L.ny : 1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L.phys * nsamp;
       i += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(i / L.phys);
    long long k = i - (long long)s * L.phys;
    const int ix = (int)(k % L.nx);
    k /= L.nx;
    const int iy = (int)(k % ny);
    const int iz = (int)(k / ny);
    const int z0 = iz == 0 ? 0 : iz + L.nb, z1 = iz == L.nz - 1 ? L.nzp - 1 : iz + L.nb;
    const int x0 = ix == 0 ? 0 : ix + L.nb, x1 = ix == L.nx - 1 ? L.nxp - 1 : ix + L.nb;
    int y0 = 0, y1 = 0;
    if (L.ndim == 3) {
      y0 = iy == 0 ? 0 : iy + L.nb;
      y1 = iy == L.ny - 1 ? L.nyp - 1 : iy + L.nb;
    }
    double acc = 0.0;
    for (int j = 0; j < g_per_sample; j++) {
      const float* Gs = G + (long long)(s * g_per_sample + j) * L.field;
      for (int z = z0; z <= z1; z++)
        for (int y = y0; y <= y1; y++)
          for (int x = x0; x <= x1; x++) acc += Gs[L.off(z, y, x)];
    }
    grad[i] = (float)(scale * 2.0 * acc / (double)vel[i]);
  }
}

cudaError_t launch_finalize(const Layout& L, const float* vel, const float* G, int nsamp, int g_per_sample,
                            double scale, float* grad, cudaStream_t st) {
  const long long n = L.phys * nsamp;
  const int blocks = grid_for(n, 32);
  finalize_kernel<<<blocks, 256, 0, st>>>(L, vel, G, nsamp, g_per_sample, scale, grad);
  return cudaGetLastError();
}

// ----------------------------------------------------------- sampler steps --

// SplitMix64 output function and the counter-based normal stream.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double normal_at(uint64_t key, uint64_t i) {
  const uint64_t G = 0x9e3779b97f4a7c15ULL;
  const uint64_t a = mix64(key + (2 * i + 1) * G);
  const uint64_t b = mix64(key + (2 * i + 2) * G);
  const double u1 = (double)((a >> 11) + 1) * 0x1.0p-53;
  const double u2 = (double)(b >> 11) * 0x1.0p-53;
  return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

__global__ void langevin_kernel(float* z, const float* __restrict__ g, long long n, double eta, double nu,
                                double vmin, double vmax, uint64_t key) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double v = (double)z[i] - eta * (double)g[i];
    if (nu != 0.0) v += nu * normal_at(key, (uint64_t)i);
    z[i] = (float)fmin(fmax(v, vmin), vmax);
  }
}

cudaError_t launch_langevin(float* z, const float* g, long long n, double eta, double nu, double vmin, double vmax,
                            uint64_t seed, uint64_t counter, cudaStream_t st) {
  const uint64_t key = [&] {
    auto m = [](uint64_t x) {
      x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
      x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
      return x ^ (x >> 31);
    };
    return m(seed ^ m(counter));
  }();
  const int blocks = grid_for(n, 16);
  langevin_kernel<<<blocks, 256, 0, st>>>(z, g, n, eta, nu, vmin, vmax, key);
  return cudaGetLastError();
}

// Preconditioned Langevin step, pass 1: running moments per element
//   v <- alpha v + (1 - alpha) g^2,   m <- beta1 m + (1 - beta1) g   (m optional)
// and per-block FP64 partial sums of the bias-corrected second moment
// vh = v * inv_cv of each sample (blockIdx.y), over the values as stored in
// FP32 so that pass 2 sees the same numbers; fixed reduction order.
__global__ void precond_moments_kernel(const float* __restrict__ g, float* __restrict__ v, float* __restrict__ m,
                                       long long per, double alpha, double beta1, double inv_cv, double* part,
                                       int nblk) {
  const int s = blockIdx.y;
  const long long o = (long long)s * per;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < per; i += (long long)gridDim.x * blockDim.x) {
    const double gi = (double)g[o + i];
    const float vn = (float)(alpha * (double)v[o + i] + (1.0 - alpha) * gi * gi);
    v[o + i] = vn;
    if (m) m[o + i] = (float)(beta1 * (double)m[o + i] + (1.0 - beta1) * gi);
    acc += (double)vn * inv_cv;
  }
  __shared__ double sh[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < blockDim.x / 32 ? sh[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) part[(long long)s * nblk + blockIdx.x] = t;
  }
}

// Pass 2: r = sqrt(mean vh) of the sample (its nblk partials summed in a
// fixed order), G = 1/(sqrt(vh) + eps r) (0 where that is 0), drift d = g or
// the bias-corrected first moment, and
//   z <- clamp(z - eta G d + nu sqrt(G) xi, vmin, vmax),
// xi number s * per + i of the counter-based normal stream.
__global__ void precond_update_kernel(float* z, const float* __restrict__ g, const float* __restrict__ v,
                                      const float* __restrict__ m, long long per, const double* __restrict__ part,
                                      int nblk, double inv_cv, double inv_cm, double eps, double eta, double nu,
                                      double vmin, double vmax, uint64_t key) {
  const int s = blockIdx.y;
  const long long o = (long long)s * per;
  __shared__ double r_sh;
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 32) t += part[(long long)s * nblk + b];
    t = warp_sum(t);
    if (threadIdx.x == 0) r_sh = sqrt(t / (double)per);
  }
  __syncthreads();
  const double er = eps * r_sh;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < per; i += (long long)gridDim.x * blockDim.x) {
    const double den = sqrt((double)v[o + i] * inv_cv) + er;
    const double G = den > 0.0 ? 1.0 / den : 0.0;
    const double d = m ? (double)m[o + i] * inv_cm : (double)g[o + i];
    double x = (double)z[o + i] - eta * G * d;
    if (nu != 0.0) x += nu * sqrt(G) * normal_at(key, (uint64_t)(o + i));
    z[o + i] = (float)fmin(fmax(x, vmin), vmax);
  }
}

cudaError_t launch_langevin_precond(float* z, const float* g, float* v, float* m, int nsamp, long long per,
                                    double alpha, double beta1, double eps, long long k, double eta, double nu,
                                    double vmin, double vmax, uint64_t seed, uint64_t counter, double* part,
                                    int nblk, cudaStream_t st) {
  const double cv = k > 0 ? 1.0 - pow(alpha, (double)k) : 1.0;
  const double cm = k > 0 ? 1.0 - pow(beta1, (double)k) : 1.0;
  auto mx = [](uint64_t x) {
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
    return x ^ (x >> 31);
  };
  const uint64_t key = mx(seed ^ mx(counter));
  const int per_blocks = grid_for(per, 16);
  precond_moments_kernel<<<dim3(nblk, nsamp), 256, 0, st>>>(g, v, m, per, alpha, beta1, 1.0 / cv, part, nblk);
  const int ub = (per_blocks + nsamp - 1) / nsamp > 0 ? (per_blocks + nsamp - 1) / nsamp : 1;
  precond_update_kernel<<<dim3(ub, nsamp), 256, 0, st>>>(z, g, v, m, per, part, nblk, 1.0 / cv, 1.0 / cm, eps,
                                                         eta, nu, vmin, vmax, key);
  return cudaGetLastError();
}

__global__ void renoise_kernel(float* xp, const float* __restrict__ xt, const float* __restrict__ x0, long long n,
                               double c0, double ct, double sd, uint64_t key) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double v = c0 * (double)x0[i] + ct * (double)xt[i];
    if (sd != 0.0) v += sd * normal_at(key, (uint64_t)i);
    xp[i] = (float)v;
  }
}

cudaError_t launch_renoise(float* xp, const float* xt, const float* x0, long long n, double c0, double ct, double sd,
                           uint64_t seed, uint64_t counter, cudaStream_t st) {
  auto m = [](uint64_t x) {
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
    return x ^ (x >> 31);
  };
  const uint64_t key = m(seed ^ m(counter));
  const int blocks = grid_for(n, 16);
  renoise_kernel<<<blocks, 256, 0, st>>>(xp, xt, x0, n, c0, ct, sd, key);
  return cudaGetLastError();
}

// grad += lam * (sum over face neighbours inside the grid of (u_i - u_j)/h_a^2) + mu * u_i,
// u = z - zref: the gradient of lam/2 sum_faces ((u_j - u_i)/h_a)^2 + mu/2 sum u^2.
__global__ void prior_kernel(const Layout L, const float* __restrict__ z, const float* __restrict__ zref, int nsamp,
                             double lam, double mu, double ihz2, double ihy2, double ihx2, float* grad) {
  const int ny = L.ndim == 3 ? L.ny : 1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L.phys * nsamp;
       i += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(i / L.phys);
    const long long k0 = i - (long long)s * L.phys;
    long long k = k0;
    const int ix = (int)(k % L.nx);
    k /= L.nx;
    const int iy = (int)(k % ny);
    const int iz = (int)(k / ny);
    const float* zs = z + (long long)s * L.phys;
    const double u = (double)zs[k0] - (double)zref[k0];
    double lap = 0.0;
    auto nb = [&](long long kk, double ih2) { lap += (u - ((double)zs[kk] - (double)zref[kk])) * ih2; };
    const long long sz = (long long)ny * L.nx, sy = L.nx;
    if (iz > 0) nb(k0 - sz, ihz2);
    if (iz < L.nz - 1) nb(k0 + sz, ihz2);
    if (L.ndim == 3) {
      if (iy > 0) nb(k0 - sy, ihy2);
      if (iy < ny - 1) nb(k0 + sy, ihy2);
    }
    if (ix > 0) nb(k0 - 1, ihx2);
    if (ix < L.nx - 1) nb(k0 + 1, ihx2);
    grad[i] = (float)((double)grad[i] + lam * lap + mu * u);
  }
}

cudaError_t launch_prior(const Layout& L, const float* z, const float* zref, int nsamp, double lam, double mu,
                         double hz, double hy, double hx, float* grad, cudaStream_t st) {
  const long long n = L.phys * nsamp;
  const int blocks = grid_for(n, 16);
  prior_kernel<<<blocks, 256, 0, st>>>(L, z, zref, nsamp, lam, mu, 1.0 / (hz * hz), 1.0 / (hy * hy),
                                       1.0 / (hx * hx), grad);
  return cudaGetLastError();
}

}  // namespace fwi
