"""Pins of the FP64 CPU oracle against facts fixed by mathematics and physics.

The paper prints no solver, traces or worked example, so each oracle function
is pinned to something other than itself: closed-form Green's functions, the
textbook truncation error of the 8th-order stencil, exact algebraic identities
of the adjoint-state method and of the encoding (Sec. 2.1), DDPM identities
(Sec. 2.2-2.3), published SplitMix64 outputs, and brute-force finite
differences on tiny grids.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad

import oracle as O
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _ricker(t, f0, t0):
    a = np.pi * f0 * (t - t0)
    return (1 - 2 * a * a) * np.exp(-a * a)


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


# ----------------------------------------------------------------- random --

def test_splitmix64_published_outputs():
    vals = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt")) if l[0].isdigit()]
    assert [O.splitmix(1234567, j) for j in range(5)] == vals


def test_encoding_is_permutation_and_pm1():
    for it in range(20):
        perm, w = O.encode(42, it, 100)
        assert sorted(perm.tolist()) == list(range(100))
        assert set(np.unique(w).tolist()) <= {-1, 1}


def test_encoding_weight_balance_chi2():
    # +-1 weights must be fair coins (zero mean, unit variance: Sec. 2.1 unbiasedness).
    ws = np.concatenate([O.encode(7, it, 200)[1] for it in range(200)])
    n = ws.size
    k = int((ws == 1).sum())
    chi2 = (k - n / 2) ** 2 / (n / 2) + ((n - k) - n / 2) ** 2 / (n / 2)
    assert chi2 < 10.8  # p = 0.001, 1 dof


def test_fisher_yates_uniform_chi2():
    # Uniform supergather selection (Sec. 2.1): all 4! orders equally likely.
    counts = {}
    N = 4800
    for it in range(N):
        p = tuple(O.encode(3, it, 4)[0].tolist())
        counts[p] = counts.get(p, 0) + 1
    assert len(counts) == 24
    e = N / 24
    chi2 = sum((c - e) ** 2 / e for c in counts.values())
    assert chi2 < 49.7  # p = 0.001, 23 dof


def test_gauss_moments():
    x = O.gauss(11, 5, 40000)
    assert abs(x.mean()) < 0.02
    assert abs(x.var() - 1.0) < 0.03
    assert abs(np.mean(x ** 4) - 3.0) < 0.15
    # streams differ by counter
    assert not np.allclose(O.gauss(11, 6, 10), x[:10])


# ------------------------------------------------------------------ stencil --

def _grid(ndim, n=24, h=7.0, nb=0):
    return O.Grid(ndim, n, n, n, h, h * 1.3, h * 0.8, nb, 1e-3, 1, 10.0, 0.15, 2000.0)


@pytest.mark.parametrize("ndim", [2, 3])
def test_lap8_exact_on_degree9_polynomials(ndim):
    g = _grid(ndim, n=22 if ndim == 3 else 30)
    rng = np.random.default_rng(0)
    ax = [np.arange(s, dtype=np.float64) for s in g.pshape]
    hs = [g.hz, g.hy, g.hx] if ndim == 3 else [g.hz, g.hx]
    coords = np.meshgrid(*[a * h for a, h in zip(ax, hs)], indexing="ij")
    p = np.zeros(g.pshape)
    lap = np.zeros(g.pshape)
    for a, X in enumerate(coords):
        c = rng.normal(0, 1, 10)
        X0 = X - X.mean()
        s = 50.0
        p += sum(c[k] * (X0 / s) ** k for k in range(10))
        lap += sum(c[k] * k * (k - 1) * (X0 / s) ** (k - 2) / s ** 2 for k in range(2, 10))
    L = O.lap8(g, p)
    inner = tuple(slice(4, -4) for _ in g.pshape)
    assert np.max(np.abs(L[inner] - lap[inner])) < 1e-9 * np.max(np.abs(lap[inner]))


def test_lap8_leading_truncation_error():
    # 2p-order central second difference: error -(2 (p!)^2/(2p+2)!) h^{2p} f^{(2p+2)};
    # p = 4: -h^8/3150 f^(10).  For f = x^10 at x = 0: L f = -10!/3150 h^8 = -1152 h^8.
    h = 0.5
    g = O.Grid(2, 1, 1, 9, 1e8, 1.0, h, 0, 1e-3, 1, 10.0, 0.1, 1.0)  # hz huge: 1-row grid
    x = (np.arange(9) - 4) * h
    p = np.tile(x ** 10, (1, 1))
    L = O.lap8(g, p.reshape(1, 9))
    assert math.isclose(L[0, 4], -1152 * h ** 8, rel_tol=1e-12)


def test_lap8_eighth_order_on_sine():
    errs = []
    for n in (32, 64):
        h = 2 * np.pi / n
        g = O.Grid(2, 1, 1, n + 8, 1e8, 1.0, h, 0, 1e-3, 1, 10.0, 0.1, 1.0)  # hz huge: 1-row grid
        x = (np.arange(n + 8) - 4) * h
        L = O.lap8(g, np.sin(3 * x).reshape(1, -1))[0, 4:-4]
        errs.append(np.max(np.abs(L + 9 * np.sin(3 * x[4:-4]))))
    order = math.log2(errs[0] / errs[1])
    assert 7.5 < order < 8.5


# ----------------------------------------------------------------- forward --

def test_ricker_shape():
    g = O.Grid(2, 4, 1, 4, 1, 1, 1, 0, 1e-4, 4000, 12.0, 0.125, 1.0)
    f = O.ricker(g)
    assert math.isclose(f[1250], 1.0, rel_tol=1e-15)       # peak at t0
    tz = 0.125 + 1 / (np.pi * 12.0 * math.sqrt(2))         # zero crossing
    assert abs(np.interp(tz, np.arange(4000) * 1e-4, f)) < 2e-3
    assert abs(f.sum() * 1e-4) < 1e-6                      # zero mean


def test_forward_2d_matches_green_function():
    # Homogeneous medium: p(r,t) = (1/2pi) int_0^inf f(t - (r/v) cosh u) du
    # for (1/v^2) p_tt - lap p = f(t) delta(x); d[n] approximates p((n+1) dt).
    v, h, f0, t0, dt, n, nb, nt = 2000.0, 10.0, 10.0, 0.15, 1e-3, 161, 20, 600
    g = O.Grid(2, n, 1, n, h, h, h, nb, dt, nt, f0, t0, v)
    c = n // 2
    offs = [20, 40]
    rec = np.array([[c, 0, c + o] for o in offs])
    d = O.forward_shot(g, np.full((n, n), v, np.float32), np.array([[c, 0, c]]), [1.0], rec)
    tt = (np.arange(nt) + 1) * dt
    for j, o in enumerate(offs):
        r = o * h
        an = np.array([quad(lambda u: _ricker(T - r / v * np.cosh(u), f0, t0), 0,
                            np.arccosh(max(T * v / r, 1.0)), limit=200)[0] / (2 * np.pi)
                       if T > r / v else 0.0 for T in tt])
        assert _rel(d[:, j], an) < 1e-2


def test_forward_3d_matches_green_function():
    # p(r,t) = f(t - r/v) / (4 pi r) in 3D.
    v, h, f0, t0, dt, n, nb, nt = 2000.0, 10.0, 10.0, 0.15, 1e-3, 61, 10, 350
    g = O.Grid(3, n, n, n, h, h, h, nb, dt, nt, f0, t0, v)
    c = n // 2
    offs = [10, 14]
    rec = np.array([[c, c, c + o] for o in offs])
    d = O.forward_shot(g, np.full((n, n, n), v, np.float32), np.array([[c, c, c]]), [1.0], rec)
    tt = (np.arange(nt) + 1) * dt
    for j, o in enumerate(offs):
        an = _ricker(tt - o * h / v, f0, t0) / (4 * np.pi * o * h)
        assert _rel(d[:, j], an) < 2e-2


def test_leapfrog_second_order_in_time():
    # Self-convergence under dt halving on one grid: ratio of successive
    # differences -> 2^2 for a second-order scheme.
    n, h, v = 81, 10.0, 2000.0
    outs = []
    for k in range(3):
        dt = 1e-3 / 2 ** k
        nt = 300 * 2 ** k
        g = O.Grid(2, n, 1, n, h, h, h, 10, dt, nt, 10.0, 0.15, v)
        d = O.forward_shot(g, np.full((n, n), v, np.float32), np.array([[40, 0, 40]]), [1.0],
                           np.array([[40, 0, 60]]))
        outs.append(d[2 ** k - 1::2 ** k, 0])     # samples at t = (m+1) * 1 ms
    r = np.linalg.norm(outs[0] - outs[1]) / np.linalg.norm(outs[1] - outs[2])
    assert 3.6 < r < 4.4


def test_sponge_absorbs_reflections():
    # Trace near the boundary of a padded grid vs the same node on a grid large
    # enough that nothing returns within the window: the difference is what the
    # boundary sends back.  The damping sponge must cut it several-fold against a
    # hard (undamped, zero-halo) boundary and keep cutting it as it widens.
    # R = 1e-3 bounds only what crosses the whole sponge and returns (the
    # round-trip attenuation exp(-2 int gamma/v) = R at normal incidence); the
    # damping profile's own gradient reflects more.  Measured relative L2:
    # hard wall 1.10, 20 cells 0.209, 40 cells 0.035, 60 cells 0.011 -- the
    # bounds below hold these with a margin, so a profile off by a factor
    # (gamma_max, the (d/nb)^2 shape) fails them.
    v, h, dt, nt, f0 = 2000.0, 10.0, 1e-3, 800, 10.0
    n = 81
    N = 3 * n
    G = O.Grid(2, N, 1, N, h, h, h, 20, dt, nt, f0, 0.15, v)
    big = O.forward_shot(G, np.full((N, N), v, np.float32), np.array([[40 + n, 0, 40 + n]]), [1.0],
                         np.array([[40 + n, 0, 70 + n]]))

    def refl(nb, vref):
        g = O.Grid(2, n, 1, n, h, h, h, nb, dt, nt, f0, 0.15, vref)
        s = O.forward_shot(g, np.full((n, n), v, np.float32), np.array([[40, 0, 40]]), [1.0],
                           np.array([[40, 0, 70]]))
        return np.linalg.norm(s - big) / np.linalg.norm(big)

    hard, r20, r40 = refl(20, 1e-9), refl(20, v), refl(40, v)
    assert hard > 0.8
    assert 0.15 < r20 < 0.23
    assert 0.02 < r40 < 0.045
    assert r40 < 0.25 * r20


def test_encoded_forward_is_weighted_sum_of_shots():
    # Sec. 2.1: F~(x) = sum_{i in B} w_i F_i(x), exactly (the operator is linear in the source).
    w_ = synth.tiny2d(ns=4, nt=200)
    g = O.Grid.from_workload(w_)
    v = synth.models.random_smooth_model(w_.shape, 1, 1500, 2500)
    perm, w = O.encode(5, 0, w_.ns)
    enc = O.encoded_forward(g, v, w_.src, w_.rec, perm, w, [4])[0]
    ssum = sum(w[i] * O.forward_shot(g, v, w_.src[i:i + 1], [1.0], w_.rec) for i in range(4))
    assert np.max(np.abs(enc - ssum)) < 1e-13 * np.max(np.abs(ssum))


# ----------------------------------------------------------------- adjoint --

def _tiny(ndim):
    w_ = synth.tiny2d(nt=120) if ndim == 2 else synth.tiny3d(nt=80)
    g = O.Grid.from_workload(w_)
    v = synth.models.random_smooth_model(w_.shape, 3, 1500, 2500)
    return w_, g, v


@pytest.mark.parametrize("ndim", [2, 3])
def test_source_to_receiver_adjoint_dot(ndim):
    # <S f, d> = <f, S^T d> for the linear map from source series to records.
    w_, g, v = _tiny(ndim)
    rng = np.random.default_rng(1)
    vpad = O.pad_velocity(g, v)
    src_idx = O.pad_index(g, w_.src)
    rec_idx = O.pad_index(g, w_.rec)
    f = rng.normal(0, 1, (len(src_idx), g.nt))
    dd = rng.normal(0, 1, (g.nt, len(rec_idx)))
    Sf = O.forward_raw(g, vpad, src_idx, f, rec_idx)
    _, STd = O.adjoint_raw(g, vpad, None, src_idx, f, rec_idx, dd, want_grad=False, want_src=True)
    lhs, rhs = np.sum(Sf * dd), np.sum(f * STd)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("ndim", [2, 3])
def test_tangent_linear_adjoint_dot(ndim):
    # <J dc, dd> = <dc, J^T dd>: the gradient routine is the exact transpose of
    # the linearised forward map.
    w_, g, v = _tiny(ndim)
    rng = np.random.default_rng(2)
    vpad = O.pad_velocity(g, v)
    src_idx = O.pad_index(g, w_.src)
    rec_idx = O.pad_index(g, w_.rec)
    ts = O.source_series(g, np.ones(len(src_idx)))
    _, snaps = O.forward_raw(g, vpad, src_idx, ts, rec_idx, keep_snaps=True)
    dc = rng.normal(0, 1, g.npad) * 1e-9
    dd = rng.normal(0, 1, (g.nt, len(rec_idx)))
    Jdc = O.tangent_raw(g, vpad, snaps, src_idx, ts, dc, rec_idx)
    JTdd, _ = O.adjoint_raw(g, vpad, snaps, src_idx, ts, rec_idx, dd)
    lhs, rhs = np.sum(Jdc * dd), np.sum(dc * JTdd)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


@pytest.mark.parametrize("ndim", [2, 3])
def test_gradient_matches_central_differences(ndim):
    w_, g, v = _tiny(ndim)
    truth = synth.models.random_smooth_model(w_.shape, 4, 1500, 2500)
    d_obs = np.stack([O.forward_shot(g, truth, w_.src[i:i + 1], [1.0], w_.rec) for i in range(w_.ns)])
    perm, w = O.encode(9, 1, w_.ns)
    sig = 0.5
    phi, grad = O.gradient(g, v, w_.src, w_.rec, d_obs, perm, w, w_.sg_sizes, sig)
    rng = np.random.default_rng(5)
    dv = rng.normal(0, 1, v.shape)
    vd = v.astype(np.float64)

    def J(x):
        return O.gradient(g, x, w_.src, w_.rec, d_obs, perm, w, w_.sg_sizes, sig)[0]

    dirn = float(np.sum(grad * dv))
    e1, e2 = 1.0, 0.5
    fd1 = (J(vd + e1 * dv) - J(vd - e1 * dv)) / (2 * e1)
    fd2 = (J(vd + e2 * dv) - J(vd - e2 * dv)) / (2 * e2)
    err1, err2 = abs(fd1 - dirn), abs(fd2 - dirn)
    assert err2 < 1e-4 * abs(dirn)
    assert err1 / err2 > 3.0  # O(eps^2) convergence of the central difference


def test_records_vjp_matches_central_differences():
    # <dF~/dv dv, dd> from central differences of the encoded records alone
    # equals <dv, records_vjp(dd)>, with O(eps^2) convergence; two uneven
    # supergathers, so the sum over supergathers is exercised.
    w_ = synth.tiny2d(nt=120, ns=4)
    g = O.Grid.from_workload(w_)
    v = synth.models.random_smooth_model(w_.shape, 3, 1500, 2500).astype(np.float64)
    perm, w = O.encode(4, 2, w_.ns)
    sg = [3, 1]
    rng = np.random.default_rng(8)
    dd = rng.normal(0, 1, (len(sg), g.nt, len(w_.rec)))
    dv = rng.normal(0, 1, v.shape)
    dirn = float(np.sum(O.records_vjp(g, v, w_.src, w_.rec, perm, w, sg, dd) * dv))

    def F(x):
        return O.encoded_forward(g, x, w_.src, w_.rec, perm, w, sg)

    errs = []
    for e in (1.0, 0.5):
        fd = float(np.sum((F(v + e * dv) - F(v - e * dv)) * dd)) / (2 * e)
        errs.append(abs(fd - dirn))
    assert errs[1] < 1e-4 * abs(dirn)
    assert errs[0] / errs[1] > 3.0


def test_gradient_is_records_vjp_of_scaled_residual():
    # Sec. 2.1: the misfit gradient is the transposed Jacobian applied to
    # (F~_j - d~_j)/sigma^2, times the supergather scaling.
    w_ = synth.tiny2d(nt=100, ns=4)
    g = O.Grid.from_workload(w_)
    v = synth.models.random_smooth_model(w_.shape, 6, 1500, 2500)
    d_obs = synth.random_records(w_, 3)
    perm, w = O.encode(2, 5, w_.ns)
    sg, sig, scale = [2, 1], 0.7, 1.3
    _, grad = O.gradient(g, v, w_.src, w_.rec, d_obs, perm, w, sg, sig, scale)
    r = O.encoded_forward(g, v, w_.src, w_.rec, perm, w, sg) - O.encoded_data(d_obs, perm, w, sg)
    vjp = O.records_vjp(g, v, w_.src, w_.rec, perm, w, sg, r / sig ** 2)
    assert _rel(grad, scale * vjp) < 1e-12


def test_encoded_estimator_unbiased_exactly():
    # Sec. 2.1: E_w[Phi~] = Phi and E_w[grad Phi~] = grad Phi for zero-mean,
    # unit-variance weights: averaging over all 2^M sign patterns cancels the
    # cross terms exactly.
    w_ = synth.tiny2d(ns=3, nt=100)
    g = O.Grid.from_workload(w_)
    v = synth.models.random_smooth_model(w_.shape, 6, 1500, 2500)
    truth = synth.models.random_smooth_model(w_.shape, 7, 1500, 2500)
    d_obs = np.stack([O.forward_shot(g, truth, w_.src[i:i + 1], [1.0], w_.rec) for i in range(3)])
    perm = np.arange(3, dtype=np.int32)
    phis, grads = [], []
    for signs in itertools.product([-1, 1], repeat=3):
        p, gr = O.gradient(g, v, w_.src, w_.rec, d_obs, perm, np.array(signs, np.int8), [3], 1.0)
        phis.append(p)
        grads.append(gr)
    full = O.full_misfit(g, v, w_.src, w_.rec, d_obs, 1.0)
    gfull = sum(O.gradient(g, v, w_.src, w_.rec, d_obs, np.array([i], np.int32), np.ones(3, np.int8), [1],
                           1.0, scale=1.0)[1] for i in range(3))
    assert math.isclose(np.mean(phis), full, rel_tol=1e-11)
    assert np.max(np.abs(np.mean(grads, 0) - gfull)) < 1e-10 * np.max(np.abs(gfull))


def test_subset_scaling_unbiased_exactly():
    # (N_s/m) scaling with a uniformly drawn subset B, |B| = m (Sec. 2.1):
    # averaging over all subsets and sign patterns returns the full-shot misfit.
    w_ = synth.tiny2d(ns=4, nt=80)
    g = O.Grid.from_workload(w_)
    v = synth.models.random_smooth_model(w_.shape, 8, 1500, 2500)
    truth = synth.models.random_smooth_model(w_.shape, 9, 1500, 2500)
    d_obs = np.stack([O.forward_shot(g, truth, w_.src[i:i + 1], [1.0], w_.rec) for i in range(4)])
    vals = []
    for B in itertools.combinations(range(4), 2):
        rest = [i for i in range(4) if i not in B]
        perm = np.array(list(B) + rest, np.int32)
        for s in itertools.product([-1, 1], repeat=2):
            w = np.ones(4, np.int8)
            w[list(B)] = s
            vals.append(O.gradient(g, v, w_.src, w_.rec, d_obs, perm, w, [2], 1.0)[0])
    full = O.full_misfit(g, v, w_.src, w_.rec, d_obs, 1.0)
    assert math.isclose(np.mean(vals), full, rel_tol=1e-11)


# ----------------------------------------------------------------- sampler --

def test_langevin_ula_stationary_variance():
    # Quadratic Phi = z^2/(2 s^2): the unadjusted Langevin chain
    # z' = z - eta z/s^2 + sqrt(2 eta) xi has stationary variance s^2 / (1 - eta/(2 s^2)).
    s2, eta, n = 4.0, 1.0, 20000
    z = np.zeros(n)
    acc = []
    for k in range(400):
        z = O.langevin(z, z / s2, eta, math.sqrt(2 * eta), -1e30, 1e30, 99, k)
        if k >= 100:
            acc.append(z.var())
    expect = s2 / (1 - eta / (2 * s2))
    assert abs(np.mean(acc) - expect) < 0.02 * expect


def test_langevin_clamps_and_descends():
    z = np.array([1000.0, 2000.0, 3000.0])
    out = O.langevin(z, np.array([1.0, 0.0, -1.0]), 100.0, 0.0, 1500.0, 3050.0, 1, 1)
    assert out.tolist() == [1500.0, 2000.0, 3050.0]


def test_precond_langevin_matched_noise_stationary_variance():
    # Quadratic Phi = z^2/(2 s^2) with a constant diagonal preconditioner G
    # (alpha = 1 freezes v; k = 0 drops the bias correction; eps = 0 makes
    # G = 1/sqrt(v)).  z' = z - eta G z/s^2 + sqrt(2 eta) sqrt(G) xi is the
    # unadjusted chain with step eta G, whose stationary variance is
    # s^2 / (1 - eta G/(2 s^2)) (Sec. 5: noise matched to the preconditioning).
    # Three groups with G = 0.25, 1, 3 give three different variances; noise
    # that ignored G, or a G taken from v instead of sqrt(v), misses them.
    s2, eta, n = 4.0, 1.0, 20000
    Gs = [0.25, 1.0, 3.0]
    v = np.concatenate([np.full(n, 1.0 / G ** 2) for G in Gs])[None]
    z = np.zeros_like(v)
    acc = []
    for k in range(400):
        z, v, _ = O.langevin_precond(z, z / s2, v, None, eta, math.sqrt(2 * eta), -1e30, 1e30, 21, k, k=0,
                                     alpha=1.0, eps=0.0)
        if k >= 100:
            acc.append([z[0, j * n:(j + 1) * n].var() for j in range(3)])
    got = np.mean(acc, axis=0)
    for G, var in zip(Gs, got):
        expect = s2 / (1 - eta * G / (2 * s2))
        assert abs(var - expect) < 0.03 * expect, (G, var, expect)


def test_precond_langevin_closed_form_steps_and_per_sample_scale():
    # A constant gradient g gives, after k steps, v_k = (1 - alpha^k) g^2 and
    # m_k = (1 - beta1^k) g, so the bias-corrected moments are exactly g^2 and
    # g and every step moves z by -eta g / (|g| + eps RMS(g)), with RMS taken
    # over the sample.  Sample 1's gradient is 1000 x sample 0's: both move
    # alike (the preconditioner removes the gradient's scale, per sample).
    rng = np.random.default_rng(5)
    g0 = rng.normal(0, 1, 50)
    g0[7] = 0.0
    grad = np.stack([g0, 1000.0 * g0])
    eta, eps = 5.0, 1e-3
    for use_m in (False, True):
        z = np.full((2, 50), 2500.0)
        v = np.zeros_like(z)
        m = np.zeros_like(z) if use_m else None
        expect = z.copy()
        for k in range(1, 4):
            z, v, m = O.langevin_precond(z, grad, v, m, eta, 0.0, 0.0, 1e9, 3, k, k=k, alpha=0.999, beta1=0.9,
                                         eps=eps)
            for s in range(2):
                r = np.sqrt(np.mean(grad[s] ** 2))
                expect[s] -= eta * grad[s] / (np.abs(grad[s]) + eps * r)
            assert np.max(np.abs(z - expect)) < 1e-9, (use_m, k)
        assert np.max(np.abs(z[0] - z[1])) < 1e-9
        assert z[0, 7] == 2500.0


def test_precond_langevin_reduces_to_plain_step():
    # G = 1 everywhere (v = 1 frozen, no bias correction, eps = 0): the
    # preconditioned step is the plain Langevin step with the same noise.
    rng = np.random.default_rng(6)
    z = rng.normal(2500, 300, (2, 40))
    g = rng.normal(0, 1, (2, 40))
    got, _, _ = O.langevin_precond(z, g, np.ones_like(z), None, 7.0, 3.0, 1600.0, 3400.0, 8, 9, k=0, alpha=1.0,
                                   eps=0.0)
    ref = O.langevin(z.ravel(), g.ravel(), 7.0, 3.0, 1600.0, 3400.0, 8, 9).reshape(2, 40)
    assert np.max(np.abs(got - ref)) < 1e-9
    # a sample whose gradient and moment are all zero does not move (G = 0, no NaN)
    zz, _, _ = O.langevin_precond(z, np.zeros_like(z), np.zeros_like(z), None, 7.0, 3.0, 0.0, 1e9, 8, 9, k=1)
    assert np.array_equal(zz, z)


def test_renoise_at_first_level_returns_x0():
    # abar_0 = 1: beta~_1 = 0 and mu~_1 = x0 exactly.
    beta, abar = O.ddpm_schedule()
    x0 = np.linspace(-1, 1, 50)
    xt = np.cos(np.arange(50.0))
    out = O.renoise(xt, x0, abar[0], 1.0, beta[0], 3, 4)
    assert np.max(np.abs(out - x0)) < 1e-12


def test_renoise_preserves_ddpm_marginal():
    # If x_t ~ q(x_t | x0) = N(sqrt(abar_t) x0, 1 - abar_t), a draw from the DDPM
    # posterior q(x_{t-1} | x_t, x0) has marginal N(sqrt(abar_{t-1}) x0, 1 - abar_{t-1}).
    # Checked on the linear schedule (level 300) and on a coarse two-level
    # schedule with beta_t = 0.5, where every coefficient matters at O(1).
    beta, abar = O.ddpm_schedule()
    cases = [(abar[299], abar[298], beta[299]), (0.6 * 0.5, 0.6, 0.5)]
    n = 60000
    for k, (ab_t, ab_p, b_t) in enumerate(cases):
        x0 = np.full(n, 0.7)
        eps = np.random.default_rng(k).normal(0, 1, n)
        xt = math.sqrt(ab_t) * x0 + math.sqrt(1 - ab_t) * eps
        out = O.renoise(xt, x0, ab_t, ab_p, b_t, 17, 2)
        assert abs(out.mean() - math.sqrt(ab_p) * 0.7) < 0.01
        assert abs(out.var() - (1 - ab_p)) < 0.015 * (1 - ab_p) + 0.002
        # the pair (x_t, x_{t-1}) has covariance sqrt(1 - beta_t) (1 - abar_{t-1})
        cov = np.mean((out - out.mean()) * (xt - xt.mean()))
        assert abs(cov - math.sqrt(1 - b_t) * (1 - ab_p)) < 0.015


def test_smooth_prior_gradient_brute_force():
    g = O.Grid(2, 6, 1, 7, 10.0, 1.0, 12.0, 2, 1e-3, 1, 10.0, 0.1, 2000.0)
    rng = np.random.default_rng(3)
    z = rng.normal(2000, 100, (6, 7))
    zr = rng.normal(2000, 100, (6, 7))
    phi, grad = O.smooth_prior(g, z, zr, 3.0, 0.2)
    # direct definition: squared forward differences along each axis
    u = z - zr
    direct = 0.5 * 3.0 * (np.sum((np.diff(u, axis=0) / 10.0) ** 2) + np.sum((np.diff(u, axis=1) / 12.0) ** 2)) \
        + 0.5 * 0.2 * np.sum(u ** 2)
    assert math.isclose(phi, direct, rel_tol=1e-12)
    num = np.zeros_like(z)
    for idx in np.ndindex(z.shape):
        e = np.zeros_like(z)
        e[idx] = 1e-3
        num[idx] = (O.smooth_prior(g, z + e, zr, 3.0, 0.2)[0] - O.smooth_prior(g, z - e, zr, 3.0, 0.2)[0]) / 2e-3
    assert np.max(np.abs(num - grad)) < 1e-6 * np.max(np.abs(grad))


def test_ddpm_schedule_definition():
    beta, abar = O.ddpm_schedule()
    assert len(beta) == 1000 and math.isclose(beta[0], 1e-4) and math.isclose(beta[-1], 0.02)
    assert math.isclose(abar[9], float(np.prod(1 - beta[:10])), rel_tol=1e-14)


def test_results_do_not_depend_on_the_thread_count():
    # the OpenMP loops write disjoint elements and every reduction is serial,
    # so the timing baseline's thread setting cannot change a result
    w_ = synth.tiny2d(nt=80, ns=4)
    g = O.Grid.from_workload(w_)
    v = synth.models.random_smooth_model(w_.shape, 2, 1500, 2500)
    perm, w = O.encode(1, 1, w_.ns)
    d_obs = synth.random_records(w_, 4)
    n0 = O.threads()
    try:
        O.threads(1)
        one = O.gradient(g, v, w_.src, w_.rec, d_obs, perm, w, [2, 2], 0.5)
        O.threads(max(2, n0))
        many = O.gradient(g, v, w_.src, w_.rec, d_obs, perm, w, [2, 2], 0.5)
    finally:
        O.threads(n0)
    assert one[0] == many[0] and np.array_equal(one[1], many[1])
