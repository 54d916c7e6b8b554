/*
 * fwi_oracle.c -- plain FP64 CPU oracle for the encoded wave-equation
 * likelihood gradient of diffusion-based posterior sampling for FWI
 * (Taufik & Alkhalifah, arXiv 2512.12797).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  It shares no code,
 * header, table or helper with the CUDA library; it is written to be read
 * against the paper and the discrete scheme, not to be fast.
 *
 * The paper states the forward operator only as "numerically solving the
 * acoustic wave equation" (Sec. 2.1), so the discrete scheme below is a
 * reading that fixes every free choice:
 *   - constant-density damped acoustic equation p_tt + 2 g p_t = v^2 (lap p + s),
 *     explicit leapfrog in time, 8th-order central differences in space
 *     (coefficients -205/72, 8/5, -1/5, 8/315, -1/560 per axis);
 *   - sponge: nb padding cells on every side, damping
 *     g(x) = gmax * sum_a (d_a(x)/nb)^2, gmax = 3 vmax ln(1/R) / (2 nb hmin);
 *     velocity edge-replicated into the padding; field zero outside the padded grid;
 *   - update p^{n+1} = [2 p^n - (1 - g dt) p^{n-1} + c (L p^n + s^n)] / (1 + g dt),
 *     c = v^2 dt^2, p^0 = p^{-1} = 0;
 *   - recording d[n][r] = p^{n+1}(x_r), n = 0..nt-1;
 *   - source term s^n = sum_i w_i f(n dt) delta_{x_i} / (cell volume), with the
 *     Ricker f(t) = (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2).
 * The adjoint is the exact transpose of this recursion (adjoint-state method,
 * Sec. 2.1 unbiased-gradient paragraph), written in the multiplier lambda:
 *   lambda^k = (2/(1+g dt)) lambda^{k+1} + L( c/(1+g dt) lambda^{k+1} )
 *              - ((1-g dt)/(1+g dt)) lambda^{k+2} + R^T dJ/dd[k-1],
 *   dJ/dc(x) = sum_n lambda^{n+1}(x) (L p^n + s^n)(x) / (1 + g(x) dt).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int ndim, nz, ny, nx;
    double hz, hy, hx;
    int nb;
    double dt;
    int nt;
    double f0, t0, sponge_vmax, sponge_R;
} or_grid;

/* ---------------------------------------------------------------- grid -- */

static void pdims(const or_grid* g, long* pz, long* py, long* px) {
    *pz = g->nz + 2L * g->nb;
    *px = g->nx + 2L * g->nb;
    *py = (g->ndim == 3) ? g->ny + 2L * g->nb : 1;
}

long or_npad(const or_grid* g) {
    long pz, py, px;
    pdims(g, &pz, &py, &px);
    return pz * py * px;
}

double or_cell_volume(const or_grid* g) {
    return g->ndim == 3 ? g->hz * g->hy * g->hx : g->hz * g->hx;
}

/* Linear index on the padded grid of physical node (iz, iy, ix). */
long or_pad_index(const or_grid* g, int iz, int iy, int ix) {
    long pz, py, px;
    pdims(g, &pz, &py, &px);
    long jy = (g->ndim == 3) ? iy + g->nb : 0;
    return ((long)(iz + g->nb) * py + jy) * px + (ix + g->nb);
}

/* Depth of padded index i into the sponge along an axis of n physical cells. */
static int pad_depth(long i, int n, int nb) {
    if (i < nb) return (int)(nb - i);
    if (i >= nb + n) return (int)(i - (nb + n - 1));
    return 0;
}

/* Damping profile gamma(x) on the padded grid. */
void or_sponge(const or_grid* g, double* gamma) {
    long pz, py, px;
    pdims(g, &pz, &py, &px);
    double hmin = g->hz < g->hx ? g->hz : g->hx;
    if (g->ndim == 3 && g->hy < hmin) hmin = g->hy;
    double gmax = g->nb > 0 ? 3.0 * g->sponge_vmax * log(1.0 / g->sponge_R) / (2.0 * g->nb * hmin) : 0.0;
    for (long z = 0; z < pz; z++)
        for (long y = 0; y < py; y++)
            for (long x = 0; x < px; x++) {
                double s = 0.0, d;
                if (g->nb > 0) {
                    d = (double)pad_depth(z, g->nz, g->nb) / g->nb; s += d * d;
                    d = (double)pad_depth(x, g->nx, g->nb) / g->nb; s += d * d;
                    if (g->ndim == 3) { d = (double)pad_depth(y, g->ny, g->nb) / g->nb; s += d * d; }
                }
                gamma[(z * py + y) * px + x] = gmax * s;
            }
}

/* Clamp a padded index back to the physical cell it replicates. */
static long to_phys(long i, int n, int nb) {
    long j = i - nb;
    if (j < 0) j = 0;
    if (j > n - 1) j = n - 1;
    return j;
}

/* Edge-replicate the physical velocity [nz][ny][nx] into the padded grid. */
void or_pad_velocity(const or_grid* g, const double* v, double* vpad) {
    long pz, py, px;
    pdims(g, &pz, &py, &px);
    int ny = g->ndim == 3 ? g->ny : 1;
    for (long z = 0; z < pz; z++)
        for (long y = 0; y < py; y++)
            for (long x = 0; x < px; x++) {
                long sz = to_phys(z, g->nz, g->nb);
                long sy = g->ndim == 3 ? to_phys(y, g->ny, g->nb) : 0;
                long sx = to_phys(x, g->nx, g->nb);
                vpad[(z * py + y) * px + x] = v[(sz * ny + sy) * g->nx + sx];
            }
}

/* Adjoint of the replication composed with the chain rule c = v^2 dt^2:
 * gv[phys] = sum over padded cells replicating it of 2 v dt^2 gc[pad]. */
void or_fold_gradient(const or_grid* g, const double* v, const double* gc, double* gv) {
    long pz, py, px;
    pdims(g, &pz, &py, &px);
    int ny = g->ndim == 3 ? g->ny : 1;
    long nphys = (long)g->nz * ny * g->nx;
    for (long i = 0; i < nphys; i++) gv[i] = 0.0;
    for (long z = 0; z < pz; z++)
        for (long y = 0; y < py; y++)
            for (long x = 0; x < px; x++) {
                long sz = to_phys(z, g->nz, g->nb);
                long sy = g->ndim == 3 ? to_phys(y, g->ny, g->nb) : 0;
                long sx = to_phys(x, g->nx, g->nb);
                long k = (sz * ny + sy) * g->nx + sx;
                gv[k] += 2.0 * v[k] * g->dt * g->dt * gc[(z * py + y) * px + x];
            }
}

/* ------------------------------------------------------------ operator -- */

static const double A8[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};

/* 8th-order Laplacian on the padded grid, field taken as zero outside it. */
void or_lap8(const or_grid* g, const double* p, double* out) {
    long pz, py, px;
    pdims(g, &pz, &py, &px);
    double iz2 = 1.0 / (g->hz * g->hz), ix2 = 1.0 / (g->hx * g->hx), iy2 = 1.0 / (g->hy * g->hy);
#pragma omp parallel for schedule(static)
    for (long z = 0; z < pz; z++)
        for (long y = 0; y < py; y++)
            for (long x = 0; x < px; x++) {
                long c = (z * py + y) * px + x;
                double sz = A8[0] * p[c], sx = A8[0] * p[c], sy = A8[0] * p[c];
                for (int k = 1; k <= 4; k++) {
                    if (z + k < pz) sz += A8[k] * p[c + k * py * px];
                    if (z - k >= 0) sz += A8[k] * p[c - k * py * px];
                    if (x + k < px) sx += A8[k] * p[c + k];
                    if (x - k >= 0) sx += A8[k] * p[c - k];
                    if (g->ndim == 3) {
                        if (y + k < py) sy += A8[k] * p[c + k * px];
                        if (y - k >= 0) sy += A8[k] * p[c - k * px];
                    }
                }
                out[c] = sz * iz2 + sx * ix2 + (g->ndim == 3 ? sy * iy2 : 0.0);
            }
}

/* Ricker wavelet samples f(n dt), n = 0..nt-1. */
void or_ricker(const or_grid* g, double* f) {
    for (int n = 0; n < g->nt; n++) {
        double a = M_PI * g->f0 * (n * g->dt - g->t0);
        f[n] = (1.0 - 2.0 * a * a) * exp(-a * a);
    }
}

/*
 * Forward propagation.  Sources: nsrc padded indices with source-term series
 * src_ts[i][n] = s_i^n (already weighted and divided by the cell volume).
 * Output d[n][r] = p^{n+1}(rec_idx[r]).  If snaps != NULL it receives
 * p^0 .. p^{nt-1} as snaps[n][npad].
 */
int or_forward(const or_grid* g, const double* vpad, int nsrc, const long* src_idx,
               const double* src_ts, int nrec, const long* rec_idx, double* d, double* snaps) {
    long np = or_npad(g);
    double* gam = malloc(np * sizeof(double));
    double* pm = calloc(np, sizeof(double));
    double* p = calloc(np, sizeof(double));
    double* pn = malloc(np * sizeof(double));
    double* L = malloc(np * sizeof(double));
    if (!gam || !pm || !p || !pn || !L) return -3;
    or_sponge(g, gam);
    double dt = g->dt;
    for (int n = 0; n < g->nt; n++) {
        if (snaps) memcpy(snaps + (long)n * np, p, np * sizeof(double));
        or_lap8(g, p, L);
        for (int i = 0; i < nsrc; i++) L[src_idx[i]] += src_ts[(long)i * g->nt + n];
#pragma omp parallel for schedule(static)
        for (long k = 0; k < np; k++) {
            double c = vpad[k] * vpad[k] * dt * dt;
            pn[k] = (2.0 * p[k] - (1.0 - gam[k] * dt) * pm[k] + c * L[k]) / (1.0 + gam[k] * dt);
        }
        for (int r = 0; r < nrec; r++) d[(long)n * nrec + r] = pn[rec_idx[r]];
        double* t = pm; pm = p; p = pn; pn = t;
    }
    free(gam); free(pm); free(p); free(pn); free(L);
    return 0;
}

/*
 * Adjoint propagation (exact transpose of or_forward) driven by
 * adj[n][r] = dJ/dd[n][r].  Needs snaps (p^0..p^{nt-1}) when grad_c != NULL.
 *   grad_c[npad]     += dJ/dc
 *   src_grad[i][n]    = dJ/ds_i^n = c/(1+g dt) lambda^{n+1} at source i   (if != NULL)
 */
int or_adjoint(const or_grid* g, const double* vpad, const double* snaps, int nsrc,
               const long* src_idx, const double* src_ts, int nrec, const long* rec_idx,
               const double* adj, double* grad_c, double* src_grad) {
    long np = or_npad(g);
    double* gam = malloc(np * sizeof(double));
    double* l2 = calloc(np, sizeof(double));   /* lambda^{k+2} */
    double* l1 = calloc(np, sizeof(double));   /* lambda^{k+1} */
    double* l0 = malloc(np * sizeof(double));  /* lambda^{k}   */
    double* t = malloc(np * sizeof(double));
    double* Lt = malloc(np * sizeof(double));
    double* Lp = malloc(np * sizeof(double));
    if (!gam || !l2 || !l1 || !l0 || !t || !Lt || !Lp) return -3;
    or_sponge(g, gam);
    double dt = g->dt;
    for (int k = g->nt; k >= 1; k--) {
        for (long j = 0; j < np; j++) {
            double c = vpad[j] * vpad[j] * dt * dt;
            t[j] = c / (1.0 + gam[j] * dt) * l1[j];
        }
        or_lap8(g, t, Lt);
#pragma omp parallel for schedule(static)
        for (long j = 0; j < np; j++)
            l0[j] = 2.0 / (1.0 + gam[j] * dt) * l1[j] + Lt[j]
                    - (1.0 - gam[j] * dt) / (1.0 + gam[j] * dt) * l2[j];
        for (int r = 0; r < nrec; r++) l0[rec_idx[r]] += adj[(long)(k - 1) * nrec + r];
        if (grad_c) {
            or_lap8(g, snaps + (long)(k - 1) * np, Lp);
            for (int i = 0; i < nsrc; i++) Lp[src_idx[i]] += src_ts[(long)i * g->nt + (k - 1)];
#pragma omp parallel for schedule(static)
            for (long j = 0; j < np; j++) grad_c[j] += l0[j] * Lp[j] / (1.0 + gam[j] * dt);
        }
        if (src_grad)
            for (int i = 0; i < nsrc; i++) {
                long j = src_idx[i];
                double c = vpad[j] * vpad[j] * dt * dt;
                src_grad[(long)i * g->nt + (k - 1)] = c / (1.0 + gam[j] * dt) * l0[j];
            }
        double* s = l2; l2 = l1; l1 = l0; l0 = s;
    }
    free(gam); free(l2); free(l1); free(l0); free(t); free(Lt); free(Lp);
    return 0;
}

/*
 * Tangent-linear model: data perturbation dd[n][r] produced by a perturbation
 * dc[npad] of c = v^2 dt^2, linearised about the stored forward (snaps).
 */
int or_tangent(const or_grid* g, const double* vpad, const double* snaps, int nsrc,
               const long* src_idx, const double* src_ts, const double* dc, int nrec,
               const long* rec_idx, double* dd) {
    long np = or_npad(g);
    double* gam = malloc(np * sizeof(double));
    double* qm = calloc(np, sizeof(double));
    double* q = calloc(np, sizeof(double));
    double* qn = malloc(np * sizeof(double));
    double* Lq = malloc(np * sizeof(double));
    double* Lp = malloc(np * sizeof(double));
    if (!gam || !qm || !q || !qn || !Lq || !Lp) return -3;
    or_sponge(g, gam);
    double dt = g->dt;
    for (int n = 0; n < g->nt; n++) {
        or_lap8(g, q, Lq);
        or_lap8(g, snaps + (long)n * np, Lp);
        for (int i = 0; i < nsrc; i++) Lp[src_idx[i]] += src_ts[(long)i * g->nt + n];
        for (long k = 0; k < np; k++) {
            double c = vpad[k] * vpad[k] * dt * dt;
            qn[k] = (2.0 * q[k] - (1.0 - gam[k] * dt) * qm[k] + c * Lq[k] + dc[k] * Lp[k])
                    / (1.0 + gam[k] * dt);
        }
        for (int r = 0; r < nrec; r++) dd[(long)n * nrec + r] = qn[rec_idx[r]];
        double* s = qm; qm = q; q = qn; qn = s;
    }
    free(gam); free(qm); free(q); free(qn); free(Lq); free(Lp);
    return 0;
}

/* -------------------------------------------------------------- random -- */

/* SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014). */
uint64_t or_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static const uint64_t GOLDEN = 0x9e3779b97f4a7c15ULL;

/* j-th output (0-based) of a SplitMix64 generator whose state starts at s. */
uint64_t or_splitmix(uint64_t s, uint64_t j) { return or_mix64(s + (j + 1) * GOLDEN); }

/* Stream key for (seed, counter). */
uint64_t or_stream_key(uint64_t seed, uint64_t counter) { return or_mix64(seed ^ or_mix64(counter)); }

/*
 * Supergather encoding for one FWI iteration (Sec. 2.1, encoded shots;
 * random re-selection every iteration, Sec. 3.2).  With key = stream(seed, iter):
 *   w[i]   = +1 if the top bit of output i is 0, else -1         (i = 0..ns-1)
 *   perm   = Fisher-Yates shuffle of 0..ns-1: for i = ns-1 down to 1,
 *            j = floor(u * (i+1) / 2^64) with u = output ns + (ns-1-i), swap.
 * Supergather j is the next sg_sizes[j] entries of perm.
 */
void or_encode(uint64_t seed, uint64_t iter, int ns, int* perm, int8_t* w) {
    uint64_t key = or_stream_key(seed, iter);
    for (int i = 0; i < ns; i++) w[i] = (or_splitmix(key, (uint64_t)i) >> 63) ? -1 : 1;
    for (int i = 0; i < ns; i++) perm[i] = i;
    for (int i = ns - 1; i >= 1; i--) {
        uint64_t u = or_splitmix(key, (uint64_t)ns + (uint64_t)(ns - 1 - i));
        uint64_t j = (uint64_t)(((unsigned __int128)u * (unsigned __int128)(i + 1)) >> 64);
        int t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
}

/* Standard normal number `index` of stream (seed, counter): Box-Muller on two
 * 53-bit uniforms u1 in (0,1], u2 in [0,1) taken from outputs 2*index, 2*index+1. */
double or_gauss(uint64_t seed, uint64_t counter, uint64_t index) {
    uint64_t key = or_stream_key(seed, counter);
    double u1 = (double)((or_splitmix(key, 2 * index) >> 11) + 1) * 0x1.0p-53;
    double u2 = (double)(or_splitmix(key, 2 * index + 1) >> 11) * 0x1.0p-53;
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

/* ----------------------------------------------------- sampler updates -- */

/* Clean-space Langevin step (Sec. 2.3 (ii)) with independent noise scale nu
 * (Sec. 2.3, modification of DAPS) and a clamp to [vmin, vmax]:
 *   z <- clamp(z - eta * grad + nu * xi, vmin, vmax),  xi_i = gauss(seed, counter, i). */
void or_langevin(double* z, const double* grad, long n, double eta, double nu, double vmin,
                 double vmax, uint64_t seed, uint64_t counter) {
    for (long i = 0; i < n; i++) {
        double v = z[i] - eta * grad[i] + nu * or_gauss(seed, counter, (uint64_t)i);
        z[i] = v < vmin ? vmin : (v > vmax ? vmax : v);
    }
}

/* Preconditioned Langevin step.  The paper's conclusion (Sec. 5) requires the
 * refinement to stay a stochastic Langevin step "with noise matched to any
 * preconditioning"; this is the diagonal preconditioner of preconditioned
 * SGLD (Li et al. 2016, RMSprop second moment) with the noise scaled by the
 * square root of the same preconditioner, and, with a first moment, the Adam
 * update the paper's experiments use for deterministic refinement (Sec. 3.2).
 * For each of nsamp samples of `per` elements, at step number k:
 *   v_i <- alpha v_i + (1 - alpha) g_i^2
 *   m_i <- beta1 m_i + (1 - beta1) g_i                  (only when m != NULL)
 *   vh_i = v_i / (1 - alpha^k),  mh_i = m_i / (1 - beta1^k)   (k = 0: no correction)
 *   r    = sqrt(mean over the sample of vh_i)
 *   G_i  = 1 / (sqrt(vh_i) + eps r)                     (0 where the denominator is 0)
 *   d_i  = mh_i when m != NULL, else g_i
 *   z_i <- clamp(z_i - eta G_i d_i + nu sqrt(G_i) xi_i, vmin, vmax)
 * xi_i = gauss(seed, counter, s * per + i).  With nu = sqrt(2 eta) and a
 * constant G the chain targets exp(-Phi) up to the O(eta) bias of the
 * unadjusted step (Sec. 2.3 (ii)); another nu is the paper's independent
 * noise scale (Sec. 2.3, modification of DAPS). */
void or_langevin_precond(double* z, const double* grad, double* v, double* m, int nsamp, long per,
                         double alpha, double beta1, double eps, long k, double eta, double nu,
                         double vmin, double vmax, uint64_t seed, uint64_t counter) {
    double cv = k > 0 ? 1.0 - pow(alpha, (double)k) : 1.0;
    double cm = k > 0 ? 1.0 - pow(beta1, (double)k) : 1.0;
    for (int s = 0; s < nsamp; s++) {
        long o = (long)s * per;
        double msum = 0.0;
        for (long i = 0; i < per; i++) {
            double g = grad[o + i];
            v[o + i] = alpha * v[o + i] + (1.0 - alpha) * g * g;
            if (m) m[o + i] = beta1 * m[o + i] + (1.0 - beta1) * g;
            msum += v[o + i] / cv;
        }
        double r = sqrt(msum / (double)per);
        for (long i = 0; i < per; i++) {
            double den = sqrt(v[o + i] / cv) + eps * r;
            double G = den > 0.0 ? 1.0 / den : 0.0;
            double d = m ? m[o + i] / cm : grad[o + i];
            double x = z[o + i] - eta * G * d + nu * sqrt(G) * or_gauss(seed, counter, (uint64_t)(o + i));
            z[o + i] = x < vmin ? vmin : (x > vmax ? vmax : x);
        }
    }
}

/* DDPM re-noise (Sec. 2.3 (iii), posterior mean and variance):
 *   btilde = (1 - abar_prev) / (1 - abar_t) * beta_t
 *   mu     = sqrt(abar_prev) beta_t / (1 - abar_t) x0 + sqrt(1 - beta_t)(1 - abar_prev)/(1 - abar_t) x_t
 *   x_prev = mu + sqrt(btilde) xi. */
void or_renoise(double* x_prev, const double* x_t, const double* x0, long n, double abar_t,
                double abar_prev, double beta_t, uint64_t seed, uint64_t counter) {
    double bt = (1.0 - abar_prev) / (1.0 - abar_t) * beta_t;
    double c0 = sqrt(abar_prev) * beta_t / (1.0 - abar_t);
    double ct = sqrt(1.0 - beta_t) * (1.0 - abar_prev) / (1.0 - abar_t);
    for (long i = 0; i < n; i++)
        x_prev[i] = c0 * x0[i] + ct * x_t[i] + sqrt(bt) * or_gauss(seed, counter, (uint64_t)i);
}

/* Gaussian smoothness prior of the plain-Langevin baseline:
 *   Phi_p(z) = lam/2 sum_edges ((u_j - u_i)/h_a)^2 + mu/2 sum u_i^2,  u = z - zref,
 * summing over every pair of face neighbours inside the physical grid.
 * Returns Phi_p and adds its gradient into grad. */
double or_smooth_prior(const or_grid* g, const double* z, const double* zref, double lam,
                       double mu, double* grad) {
    int ny = g->ndim == 3 ? g->ny : 1;
    long n = (long)g->nz * ny * g->nx;
    double phi = 0.0;
    for (long i = 0; i < n; i++) {
        double u = z[i] - zref[i];
        phi += 0.5 * mu * u * u;
        grad[i] += mu * u;
    }
    for (int a = 0; a < 3; a++) {
        if (a == 1 && g->ndim != 3) continue;
        double h = a == 0 ? g->hz : (a == 1 ? g->hy : g->hx);
        long st = a == 0 ? (long)ny * g->nx : (a == 1 ? g->nx : 1);
        for (long iz = 0; iz < g->nz; iz++)
            for (long iy = 0; iy < ny; iy++)
                for (long ix = 0; ix < g->nx; ix++) {
                    long i = (iz * ny + iy) * g->nx + ix;
                    int last = a == 0 ? iz == g->nz - 1 : (a == 1 ? iy == ny - 1 : ix == g->nx - 1);
                    if (last) continue;
                    double du = ((z[i + st] - zref[i + st]) - (z[i] - zref[i])) / h;
                    phi += 0.5 * lam * du * du;
                    grad[i + st] += lam * du / h;
                    grad[i] -= lam * du / h;
                }
    }
    return phi;
}

/* Threads of the spatial loops: n > 0 sets them; returns the number in use
 * (1 without OpenMP).  Timing only: results do not depend on it. */
int or_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
