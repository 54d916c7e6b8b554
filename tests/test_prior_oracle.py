"""Pins of oracle/prior_oracle.py (the FP64 definitions the learned prior's
tensor-core kernels are checked against) against hand values and brute force."""
import numpy as np

from oracle import prior_oracle as PO


def test_gemm_hand_values():
    A = np.array([[1.0, 2.0, 3.0], [0.0, -1.0, 4.0]])
    B = np.array([[1.0, 0.0, 0.0], [1.0, 1.0, 1.0], [2.0, -1.0, 0.5]])
    expect = np.array([[1.0, 6.0, 1.5], [0.0, 3.0, 3.0]])  # row i of A . row j of B
    assert np.array_equal(PO.gemm(A, B), expect)


def _conv_brute(X, Wt):
    n, H, W, C = X.shape
    O = Wt.shape[0]
    Y = np.zeros((n, H, W, O))
    for b in range(n):
        for y in range(H):
            for x in range(W):
                for o in range(O):
                    acc = 0.0
                    for dy in range(3):
                        for dx in range(3):
                            yy, xx = y + dy - 1, x + dx - 1
                            if 0 <= yy < H and 0 <= xx < W:
                                for c in range(C):
                                    acc += Wt[o, dy * 3 + dx, c] * X[b, yy, xx, c]
                    Y[b, y, x, o] = acc
    return Y


def test_conv3x3_matches_brute_force():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((2, 5, 4, 3))
    Wt = rng.standard_normal((2, 9, 3))
    assert np.allclose(PO.conv3x3(X, Wt), _conv_brute(X, Wt), rtol=0, atol=1e-12)


def test_conv3x3_delta_reproduces_the_taps():
    # a unit impulse at (y0, x0, c) reaches output (y0 - dy + 1, x0 - dx + 1) through tap (dy, dx)
    X = np.zeros((1, 7, 7, 2))
    X[0, 3, 3, 1] = 1.0
    Wt = np.arange(2 * 9 * 2, dtype=float).reshape(2, 9, 2)
    Y = PO.conv3x3(X, Wt)
    for dy in range(3):
        for dx in range(3):
            assert np.array_equal(Y[0, 3 - dy + 1, 3 - dx + 1], Wt[:, dy * 3 + dx, 1])
    assert np.count_nonzero(np.abs(Y).sum(-1)) == 9


def test_conv3x3_zero_padding_on_constant_image():
    X = np.ones((1, 4, 5, 1))
    Wt = np.ones((1, 9, 1))
    Y = PO.conv3x3(X, Wt)[0, :, :, 0]
    assert Y[0, 0] == 4 and Y[0, 2] == 6 and Y[2, 2] == 9 and Y[3, 4] == 4


def test_conv_gradients_satisfy_the_adjoint_identities():
    # <conv(X, W), G> = <X, dgrad(G, W)> = <W, wgrad(G, X)>: the conv is bilinear
    rng = np.random.default_rng(1)
    X = rng.standard_normal((2, 6, 5, 3))
    Wt = rng.standard_normal((4, 9, 3))
    G = rng.standard_normal((2, 6, 5, 4))
    lhs = float(np.sum(PO.conv3x3(X, Wt) * G))
    assert abs(lhs - float(np.sum(X * PO.conv3x3_dgrad(G, Wt)))) < 1e-10 * max(1.0, abs(lhs))
    assert abs(lhs - float(np.sum(Wt * PO.conv3x3_wgrad(G, X)))) < 1e-10 * max(1.0, abs(lhs))


def test_conv_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((1, 4, 4, 2))
    Wt = rng.standard_normal((2, 9, 2))
    G = rng.standard_normal((1, 4, 4, 2))
    loss = lambda X_, W_: float(np.sum(_conv_brute(X_, W_) * G))
    dX, dW = PO.conv3x3_dgrad(G, Wt), PO.conv3x3_wgrad(G, X)
    e = 1e-6
    for idx in [(0, 0, 0, 0), (0, 3, 2, 1), (0, 1, 3, 0)]:
        Xe = X.copy(); Xe[idx] += e
        assert abs((loss(Xe, Wt) - loss(X, Wt)) / e - dX[idx]) < 1e-5
    for idx in [(0, 0, 0), (1, 4, 1), (0, 8, 1)]:
        We = Wt.copy(); We[idx] += e
        assert abs((loss(X, We) - loss(X, Wt)) / e - dW[idx]) < 1e-5



def _conv3_brute(X, Wt):
    n, D, H, W, C = X.shape
    O = Wt.shape[0]
    Y = np.zeros((n, D, H, W, O))
    for b in range(n):
        for z in range(D):
            for y in range(H):
                for x in range(W):
                    for o in range(O):
                        acc = 0.0
                        for dz in range(3):
                            for dy in range(3):
                                for dx in range(3):
                                    zz, yy, xx = z + dz - 1, y + dy - 1, x + dx - 1
                                    if 0 <= zz < D and 0 <= yy < H and 0 <= xx < W:
                                        for c in range(C):
                                            acc += Wt[o, dz * 9 + dy * 3 + dx, c] * X[b, zz, yy, xx, c]
                        Y[b, z, y, x, o] = acc
    return Y


def test_conv3x3x3_matches_brute_force():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((1, 3, 4, 5, 2))
    Wt = rng.standard_normal((2, 27, 2))
    assert np.allclose(PO.conv3x3x3(X, Wt), _conv3_brute(X, Wt), rtol=0, atol=1e-12)


def test_conv3x3x3_delta_reproduces_the_taps():
    X = np.zeros((1, 5, 5, 5, 1))
    X[0, 2, 2, 2, 0] = 1.0
    Wt = np.arange(27, dtype=float).reshape(1, 27, 1) + 1.0
    Y = PO.conv3x3x3(X, Wt)
    for t in range(27):
        dz, dy, dx = t // 9, (t // 3) % 3, t % 3
        assert Y[0, 3 - dz, 3 - dy, 3 - dx, 0] == Wt[0, t, 0]
    assert np.count_nonzero(Y) == 27


def test_conv3x3x3_with_only_the_middle_plane_is_the_2d_conv():
    # weights zero outside dz = 1 act plane by plane as the (pinned) 3x3 conv
    rng = np.random.default_rng(4)
    X = rng.standard_normal((2, 3, 5, 4, 3))
    W2 = rng.standard_normal((2, 9, 3))
    W3 = np.zeros((2, 27, 3))
    W3[:, 9:18, :] = W2
    Y3 = PO.conv3x3x3(X, W3)
    Y2 = PO.conv3x3(X.reshape(6, 5, 4, 3), W2).reshape(2, 3, 5, 4, 2)
    assert np.allclose(Y3, Y2, rtol=0, atol=1e-12)


def test_conv3x3x3_zero_padding_on_constant_volume():
    Y = PO.conv3x3x3(np.ones((1, 3, 4, 5, 1)), np.ones((1, 27, 1)))[0, :, :, :, 0]
    assert Y[0, 0, 0] == 8 and Y[1, 1, 1] == 27 and Y[1, 0, 2] == 18 and Y[2, 3, 4] == 8


def test_conv3x3x3_gradients_satisfy_the_adjoint_identities():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((2, 3, 4, 5, 3))
    Wt = rng.standard_normal((4, 27, 3))
    G = rng.standard_normal((2, 3, 4, 5, 4))
    lhs = float(np.sum(PO.conv3x3x3(X, Wt) * G))
    assert abs(lhs - float(np.sum(X * PO.conv3x3x3_dgrad(G, Wt)))) < 1e-10 * max(1.0, abs(lhs))
    assert abs(lhs - float(np.sum(Wt * PO.conv3x3x3_wgrad(G, X)))) < 1e-10 * max(1.0, abs(lhs))
