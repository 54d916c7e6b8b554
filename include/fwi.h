/*
 * fwi.h -- C ABI of the GB300 library for the encoded simultaneous-source
 * wave-equation likelihood gradient used by diffusion-based posterior
 * sampling for full waveform inversion (Taufik & Alkhalifah, arXiv 2512.12797).
 *
 * The library computes, on one GPU, the quantities the sampler of Sec. 2.3
 * calls at every Langevin refinement step:
 *   - encoded predicted data  F~_j(x) = sum_{i in B_j} w_i F_i(x)        (Sec. 2.1, encoded-shot definitions)
 *   - encoded misfit          Phi~_j  = 1/(2 sigma_y^2) ||d~_j - F~_j(x)||^2   (Sec. 2.1)
 *   - its velocity gradient by the adjoint-state method, scaled to the
 *     unbiased estimator (N_s/m) grad Phi~                               (Sec. 2.1, unbiased gradient)
 *   - the Langevin refinement update                                    (Sec. 2.3 (ii))
 *   - the DDPM re-noise draw                                            (Sec. 2.3 (iii))
 *
 * Discrete forward operator F_i (the paper says only that it solves the
 * acoustic wave equation on the acquisition geometry, Sec. 2.1; this is the
 * library's reading): constant-density damped acoustic equation
 *     p_tt + 2 gamma p_t = v^2 (lap p + s),
 * 8th-order central differences in space, leapfrog in time, a sponge of nb
 * cells on every side with gamma = gmax sum_a (depth_a/nb)^2,
 * gmax = 3 sponge_vmax ln(1/sponge_R) / (2 nb h_min), velocity edge-replicated
 * into the sponge, zero field outside the padded grid, p^0 = p^-1 = 0,
 *     p^{n+1} = [2 p^n - (1 - gamma dt) p^{n-1} + v^2 dt^2 (L p^n + s^n)] / (1 + gamma dt),
 * source term s^n = sum_i w_i f(n dt) delta_{x_i} / (cell volume) with the Ricker
 * f(t) = (1 - 2 pi^2 f0^2 (t - t0)^2) exp(-pi^2 f0^2 (t - t0)^2), records
 * d[n][r] = p^{n+1}(x_r) for n = 0..nt-1.  The gradient is the exact gradient of
 * this discrete misfit (discretise-then-differentiate).
 *
 * Conventions for every entry point
 *   - Arrays are row-major with x fastest: physical velocity models are
 *     [nsamp][nz][nx] (2D) or [nsamp][nz][ny][nx] (3D), float32, m/s.
 *   - "device" pointers are CUDA device memory owned by the caller; "host"
 *     pointers are ordinary host memory owned by the caller.  The library never
 *     frees caller memory and keeps no caller pointer after a call returns.
 *   - stream is a cudaStream_t (NULL = legacy default stream).  Device work is
 *     enqueued asynchronously on it; calls return once the work is enqueued.
 *     Calls on one context use one stream.  The calls of a context do not
 *     wait for the device, with three exceptions: the first fwi_forward or
 *     fwi_gradient for a given number of wavefields times the step-kernel
 *     variants (see fwi_set_kernel_variants); the per-call point lists and
 *     step descriptors go through 4 pinned staging buffers each, used in
 *     turn, so an upload waits for the copy issued 4 uploads earlier (the
 *     host can run 4 gradient chunks ahead); and the profiling and status
 *     queries below synchronise as documented.
 *   - Return value: FWI_OK or a negative fwi_status.  Argument, geometry,
 *     stability and allocation errors are detected on the host and returned
 *     before anything is enqueued.  Errors found on the device (non-finite
 *     misfit, a wait that ran out) are recorded in a per-context status word
 *     read by fwi_last_device_status.  No C++ exception crosses this ABI.
 *   - The library is not thread-safe per context; distinct contexts may be
 *     used from distinct threads.
 */
#ifndef FWI_H
#define FWI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FWI_OK = 0,
    FWI_ERR_ARG = -1,        /* invalid argument or geometry */
    FWI_ERR_CFL = -2,        /* sponge_vmax violates the leapfrog stability bound */
    FWI_ERR_OOM = -3,        /* device or pinned allocation failed / budget too small */
    FWI_ERR_CUDA = -4,       /* a CUDA runtime call failed */
    FWI_ERR_NONFINITE = -5,  /* device status: misfit was NaN or Inf */
    FWI_ERR_TIMEOUT = -6,    /* device status: a bounded wait ran out */
    FWI_ERR_BOUNDS = -7      /* device status: an index check failed (reserved for a debug build
                                with device index checks; this version sets it nowhere: every
                                index the kernels use is validated on the host) */
} fwi_status;

/* Physical grid, time axis, wavelet and sponge.  ny/hy are ignored in 2D. */
typedef struct fwi_grid {
    int ndim;                /* 2 or 3 */
    int nz, ny, nx;          /* physical nodes (z is depth) */
    double hz, hy, hx;       /* spacing [m] */
    int nb;                  /* sponge cells added on every side (>= 0) */
    double dt;               /* time step [s] */
    int nt;                  /* time steps = samples per trace */
    double f0, t0;           /* Ricker peak frequency [Hz] and delay [s] */
    double sponge_vmax;      /* velocity [m/s] that sets the sponge strength; also
                                the largest velocity the stability check admits */
    double sponge_R;         /* target reflection coefficient in (0, 1) */
} fwi_grid;

/* Acquisition geometry: node indices (iz, iy, ix) on the physical grid, host
 * memory, [n][3] int32 (iy ignored in 2D).  Receivers must be distinct nodes;
 * several shots may share a node. */
typedef struct fwi_geom {
    int ns;
    const int32_t* src;
    int nr;
    const int32_t* rec;
} fwi_geom;

typedef struct fwi_ctx fwi_ctx;

/*
 * Create a context for one grid and geometry.  The context owns all device
 * workspace: a pool of wavefield slots (forward ring, checkpoints, snapshot
 * buffer, adjoint ring), padded c = v^2 dt^2, gradient accumulators, receiver
 * records.  max_wavefields bounds nsamp * nsg per call.  workspace_budget_bytes
 * bounds the wavefield pool; 0 means "most of the free device memory".  A larger
 * pool lets fwi_gradient keep more snapshots and recompute fewer time steps.
 * Returns FWI_ERR_CFL if sponge_vmax^2 dt^2 * 6.5016 * sum_a 1/h_a^2 > 4
 * (6.5016 = largest eigenvalue of the 1D 8th-order stencil, at kh = pi).
 */
int fwi_create(const fwi_grid* grid, const fwi_geom* geom, int max_wavefields,
               size_t workspace_budget_bytes, fwi_ctx** out);
void fwi_destroy(fwi_ctx* ctx);

/*
 * Supergather encoding for FWI iteration `iter` (Sec. 2.1 encoded shots; the
 * source subsets and weights are redrawn every FWI iteration, Sec. 3.2).
 * Host only.  Outputs perm_out[ns] (a permutation of shot ids; supergather j is
 * the next sg_sizes[j] entries) and w_out[ns] (+1/-1 weight of shot id i).
 * Definition (bit-exact): mix64 = SplitMix64 output function; key =
 * mix64(seed ^ mix64(iter)); u_j = mix64(key + (j+1) * 0x9e3779b97f4a7c15);
 * w_i = (u_i >> 63) ? -1 : +1; Fisher-Yates for i = ns-1..1 with
 * j = (u_{ns + ns-1-i} * (i+1)) >> 64 (128-bit product), swap(perm[i], perm[j]).
 */
int fwi_encode(uint64_t seed, uint64_t iter, int ns, int32_t* perm_out, int8_t* w_out);

/*
 * Encoded forward modelling F~_j(x) for nsamp velocity models and nsg
 * supergathers each (Sec. 2.1, encoded-shot definitions).
 *   vel      device [nsamp][phys]        velocity models (m/s)
 *   perm, w  host   [nsamp][ns]          encoding of each sample (as fwi_encode)
 *   sg_sizes host   [nsg]                shots per supergather, sum <= ns
 *   d_pred   device [nsamp][nsg][nt][nr] output records
 * Every velocity must lie in (0, sponge_vmax], the bound the stability
 * condition was checked against in fwi_create; any other value (or a NaN)
 * records FWI_ERR_CFL in the device status word (fwi_last_device_status) and
 * that call's outputs are not valid (the 2D step kernels leave at their next
 * dependency check; the 3D ones finish their bounded loops).  The same holds
 * for fwi_gradient and fwi_adjoint.
 */
int fwi_forward(fwi_ctx* ctx, const float* vel, int nsamp, const int32_t* perm,
                const int8_t* w, const int32_t* sg_sizes, int nsg, float* d_pred, void* stream);

/*
 * Encoded misfit and its velocity gradient (Sec. 2.1: encoded misfit,
 * adjoint-state gradient, unbiased scaling), one forward and one adjoint solve
 * per supergather, forward wavefields checkpointed and recomputed as the
 * workspace allows.
 *   d_obs    device [ns][nt][nr]   observed single-shot records d_i
 *   sigma_y  noise standard deviation (> 0)
 *   scale    multiplies misfit and gradient (the paper's N_s/m); <= 0 selects
 *            N_s / sum(sg_sizes)
 *   grad     device [nsamp][phys]  OVERWRITTEN with scale * sum_j dPhi~_j/dv
 *   misfit   device [nsamp] double OVERWRITTEN with scale * sum_j Phi~_j
 */
int fwi_gradient(fwi_ctx* ctx, const float* vel, int nsamp, const int32_t* perm,
                 const int8_t* w, const int32_t* sg_sizes, int nsg, const float* d_obs,
                 double sigma_y, double scale, float* grad, double* misfit, void* stream);

/*
 * Transposed Jacobian of the encoded records (the adjoint-state method of
 * Sec. 2.1 with an arbitrary adjoint source): for each sample s,
 *   grad[s] = sum_j (dF~_j(v_s)/dv_s)^T d_cot[s][j]
 * where F~_j is the record fwi_forward returns for supergather j.  It is
 * fwi_gradient with the cotangent in place of the scaled residual
 * (d~_j - F~_j)/sigma_y^2 and with scale 1: same forward solve with
 * checkpointing, same adjoint solve and imaging, no misfit.  This is the
 * backward of the records as a differentiable function of velocity.
 *   d_cot    device [nsamp][nsg][nt][nr]  cotangent of the records (read only)
 *   grad     device [nsamp][phys]         OVERWRITTEN
 * Other arguments and errors as fwi_forward.
 */
int fwi_adjoint(fwi_ctx* ctx, const float* vel, int nsamp, const int32_t* perm, const int8_t* w,
                const int32_t* sg_sizes, int nsg, const float* d_cot, float* grad, void* stream);

/*
 * Clean-space Langevin refinement step (Sec. 2.3 (ii), with the independent
 * noise scale of the modified refinement step, Sec. 2.3 closing paragraph):
 *   z <- clamp(z - eta * grad + nu * xi, vmin, vmax)
 * on n contiguous float32 device values; xi_i is standard normal number i of
 * stream (seed, counter): Box-Muller on 53-bit uniforms u1 = ((a >> 11) + 1) 2^-53,
 * u2 = (b >> 11) 2^-53 with a, b outputs 2i, 2i+1 of the SplitMix64 stream keyed
 * mix64(seed ^ mix64(counter)).  The plain sampler uses nu = sqrt(2 eta).
 */
int langevin_step(float* z, const float* grad, int64_t n, double eta, double nu, double vmin,
                  double vmax, uint64_t seed, uint64_t counter, void* stream);

/*
 * Preconditioned clean-space Langevin step (Sec. 2.3 (ii) with a diagonal
 * preconditioner; Sec. 5 requires the noise to be matched to any
 * preconditioning, and Sec. 3.2 refines with Adam).  For each sample s of
 * nsamp, over its phys = nz*ny*nx elements i (layout [nsamp][phys], float32,
 * device), at step number k >= 1 (k = 0: no bias correction):
 *   v_i <- alpha v_i + (1 - alpha) g_i^2                     (second moment, in/out)
 *   m_i <- beta1 m_i + (1 - beta1) g_i                       (first moment, in/out; only if m != NULL)
 *   vh_i = v_i / (1 - alpha^k),  mh_i = m_i / (1 - beta1^k)
 *   r_s  = sqrt(mean_i vh_i)                                  (per-sample scale)
 *   G_i  = 1 / (sqrt(vh_i) + eps r_s)                        (0 where the denominator is 0)
 *   d_i  = mh_i if m != NULL else g_i
 *   z_i <- clamp(z_i - eta G_i d_i + nu sqrt(G_i) xi_i, vmin, vmax)
 * xi_i is normal number s*phys + i of stream (seed, counter), as in
 * langevin_step.  With m == NULL and nu = sqrt(2 eta) this is preconditioned
 * SGLD (Li et al. 2016): eta is a step in model units (m/s) and the injected
 * noise has the variance the preconditioner implies; another nu scales the
 * noise independently (Sec. 2.3 closing paragraph).  With m != NULL and nu = 0
 * it is an Adam step (the deterministic refinement, Sec. 3.2).
 *   z, v, m device [nsamp][phys] float32, owned by the caller; v and m hold
 *           the moments between calls (start them at zero)
 *   grad    device [nsamp][phys] float32 (read only)
 * Two launches on `stream`: the moments with per-block FP64 partial sums of
 * vh into the context's reduction buffer (deterministic order), then the
 * update.  Calls on one context share that buffer with fwi_gradient: issue
 * them on one stream.  FWI_ERR_ARG: null pointer, nsamp outside
 * [1, max_wavefields], alpha outside [0, 1], beta1 outside [0, 1) when m is
 * given, negative eps/eta/nu, vmin > vmax, or alpha = 1 with k > 0.
 */
int langevin_step_precond(fwi_ctx* ctx, float* z, const float* grad, float* v, float* m, int nsamp,
                          double alpha, double beta1, double eps, int64_t k, double eta, double nu,
                          double vmin, double vmax, uint64_t seed, uint64_t counter, void* stream);

/*
 * DDPM re-noise to the next level (Sec. 2.3 (iii), DDPM posterior mean and
 * variance), elementwise on n float32 device values:
 *   x_prev = sqrt(abar_prev) beta_t/(1-abar_t) x0 + sqrt(1-beta_t)(1-abar_prev)/(1-abar_t) x_t
 *            + sqrt((1-abar_prev)/(1-abar_t) beta_t) xi
 * abar_* are the paper's cumulative alpha; requires abar_t < 1 and
 * |abar_t - abar_prev (1 - beta_t)| <= 1e-9.  xi as in langevin_step.
 */
int renoise(float* x_prev, const float* x_t, const float* x0, int64_t n, double abar_t,
            double abar_prev, double beta_t, uint64_t seed, uint64_t counter, void* stream);

/*
 * Gradient of the Gaussian smoothness prior of the plain-Langevin baseline
 *   Phi_p(z) = lam/2 sum_faces ((u_j - u_i)/h_a)^2 + mu/2 sum u_i^2,  u = z - zref,
 * ADDED into grad (device [nsamp][phys]); zref device [phys] is shared by all samples.
 */
int smooth_prior_grad(fwi_ctx* ctx, const float* z, const float* zref, int nsamp, double lam,
                      double mu, float* grad, void* stream);

/*
 * Encoded residual and misfit for callers that cannot allocate device memory.
 * The paper has no counterpart: this is an interface for users of the library.
 * Some callers must not call cudaMalloc: plug-ins whose host application owns
 * the device memory pool and forbids allocations of its own, and tight loops
 * that cannot absorb the implicit device synchronisation of an allocation.
 * This entry point allocates nothing and needs no context; it computes what
 * fwi_gradient computes between its forward and adjoint passes:
 *   rhat[b][n][r] = (d_pred[b][n][r] - sum_{i in B_b} w_i d_obs[i][n][r]) / sigma_y^2
 *   misfit[s]     = scale * sum_j 1/(2 sigma_y^2) ||d~_j - F~_j||^2
 *   d_pred  device [nsamp][nsg][nt][nr]   encoded predicted records (e.g. from fwi_forward)
 *   d_obs   device [ns][nt][nr]           observed single-shot records
 *   perm, w host [nsamp][ns], sg_sizes host [nsg]: the encoding, as in fwi_gradient;
 *           copied before the call returns, so they may be freed afterwards
 *   rhat    device [nsamp][nsg][nt][nr]   output (may equal d_pred: computed in place)
 *   misfit  device [nsamp] double         output
 *   scale   <= 0 selects N_s / sum(sg_sizes)
 * Its scratch (FP64 partial sums, the copied encoding, shot lists) lives in
 * one static device array of FWI_NOALLOC_MAX_BYTES that every GPU which loads
 * the library holds until the process exits; calls whose scratch would exceed
 * it (roughly nsamp*nsg*512 + nsamp*ns*13 bytes) return FWI_ERR_ARG.  The
 * first call on each device looks up the array's device address with that
 * device current (cudaGetSymbolAddress) and caches it; make that first call
 * before any stream capture.  Every call reuses the same array and keeps the
 * last call's contents, so calls that overlap on the GPU (on different streams
 * or from different host threads) race; serialise them.  A non-finite value
 * in d_pred or d_obs makes the misfit non-finite; rhat can overflow to +-Inf
 * when |r| / sigma_y^2 exceeds the FP32 range.
 */
#define FWI_NOALLOC_MAX_BYTES (1u << 20)
int fwi_residual_misfit_noalloc(const float* d_pred, const float* d_obs, int nsamp, int ns, int nt, int nr,
                                const int32_t* perm, const int8_t* w, const int32_t* sg_sizes, int nsg,
                                double sigma_y, double scale, float* rhat, double* misfit, void* stream);

/* Human-readable name of a status code. */
const char* fwi_status_string(int status);

/* Text of the CUDA runtime error behind the most recent FWI_ERR_CUDA returned
 * by any entry point of this library (process-wide; "no error" if none). */
const char* fwi_last_cuda_error(void);

/* Synchronises `stream`, returns the device status word (FWI_OK or the first
 * device-side error) and clears it. */
int fwi_last_device_status(fwi_ctx* ctx, void* stream);

/* Checkpoint plan of the last fwi_gradient call: snapshot segment length,
 * number of segments, forward steps recomputed, wavefield slots used (all
 * per chunk of samples, see fwi_chunking). */
int fwi_plan_info(fwi_ctx* ctx, int* segment_len, int* nsegments, int64_t* recomputed_steps,
                  int* slots_used, int* slots_available);

/* Checkpoint schedule of fwi_gradient for nt steps and a pool of `slots`
 * wavefield slots (host only, no device work; the paper is silent on
 * checkpointing).  Slot 0 always holds zeros; the forward pass keeps
 * checkpoint pairs and the last segment's snapshots, and each earlier segment
 * is recomputed from its checkpoint before its adjoint steps.  Returns the
 * plan's segment length, number of segments, recomputed steps and slots used,
 * the number of step descriptors in *nsteps and, if desc_out is not null,
 * the descriptors in launch order as rows of 7 ints
 *   {launch, kind (0 forward, 1 adjoint), cur, prev, out, snap, t}:
 * a forward step t reads p^t (cur, with halo) and p^{t-1} (prev) and writes
 * p^{t+1}; an adjoint step t reads q^{t+2} (cur, with halo), q^{t+3} (prev)
 * and the snapshot p^t (snap, with halo) and writes q^{t+1}.  All steps with
 * the same launch index run in one launch in 2D.  FWI_ERR_OOM if no plan fits
 * `slots`, FWI_ERR_ARG if cap < *nsteps. */
int fwi_checkpoint_schedule(int nt, int64_t slots, int32_t* desc_out, int cap, int* nsteps, int* segment_len,
                            int* nsegments, int64_t* recomputed, int* slots_used);

/* Samples per chunk of the last fwi_gradient call.  When the checkpoint plan
 * of all nsamp*nsg wavefields does not fit the workspace (large 3D batches),
 * fwi_gradient processes the samples in chunks, choosing the chunk size that
 * minimises (chunks) x (2 nt + recomputed steps) x (time of one step launch). */
int fwi_chunking(fwi_ctx* ctx, int* samples_per_chunk);

/* Step-kernel variants.  2D: bit 0 the TMA ring depth, bit 1 the tile shape
 * (128 x 32 or 128 x 24; the same arithmetic per point).  3D: variant bits
 *   bit 0  CTA order: all tiles of one wavefield back to back, or the tile of
 *          every wavefield of the launch side by side (a sample's supergathers
 *          then share its cc reads through L2);
 *   bit 1  one z level per march step, or two computed together;
 *   bit 2  tile shape: 64 x 16 columns of one wavefield, or 64 x 8 columns of
 *          two supergathers of one sample per CTA (cc shared; in the adjoint
 *          one imaging accumulator per pair), when a sample has an even
 *          number of supergathers;
 *   bit 3  one CTA per column, or a persistent grid of one CTA per SM that
 *          runs its columns back to back;
 *   bit 4  (with bit 3) one launch per time step, or all steps of a phase in
 *          one cooperative launch, a column's step starting once its 3 x 3
 *          tile neighbourhood has finished the step before (progress flags
 *          in device memory); bit 4 without bit 3 is rejected.
 * By default the first fwi_forward / fwi_gradient call for a given
 * (nsamp*nsg, nsg) times every variant on that shape (synchronising the stream
 * while it does) and keeps the fastest; the variants it chooses among give
 * bit-identical results.  The 3D adjoint's tile shape (bit 2) is not tuned:
 * the pair form sums the imaging term in another order, so it is used only
 * when forced.  fwi_set_kernel_variants forces a variant index (-1 restores
 * autotuning; FWI_ERR_ARG beyond the variant count); fwi_kernel_variants
 * reports the chosen indices and names and, in ms[0..31] (2D: the first
 * nvariants), the per-step time
 * of each variant measured by the tuner (-1: not run). */
int fwi_set_kernel_variants(fwi_ctx* ctx, int fwd, int adj);
int fwi_kernel_variants(fwi_ctx* ctx, int* fwd, int* adj, const char** fwd_name, const char** adj_name,
                        float* fwd_ms, float* adj_ms, int* nvariants);

/* Per-phase device timing of the last call made with profiling on (CUDA events
 * on the call's stream): ms[0] forward, ms[1] residual+misfit, ms[2] adjoint
 * incl. recompute, ms[3] finalize; launches[0..3] = kernel launches per phase.
 * Synchronises on the events. */
int fwi_set_profiling(fwi_ctx* ctx, int on);
int fwi_phase_times(fwi_ctx* ctx, float* ms, int64_t* launches);

#ifdef __cplusplus
}
#endif
#endif /* FWI_H */
