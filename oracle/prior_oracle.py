"""Oracle of the learned prior's contractions -- TEST INFRASTRUCTURE ONLY.

Plain FP64 numpy definitions that the tensor-core kernels are checked
against; nothing in the product path imports this module.

gemm(A, B)        D = A B^T, the definition written with numpy's matmul.
conv3x3(X, Wt)    same-size 3x3 cross-correlation with zero padding, written as
                  the nine shifted, weighted sums of the convolution layer of
                  the denoising network (Sec. 2.2: g_theta is a CNN/U-Net on
                  velocity-model images):
                  Y[n, y, x, o] = sum_{dy, dx} sum_c Wt[o, dy*3+dx, c] X[n, y+dy-1, x+dx-1, c].
"""
import numpy as np


def gemm(A, B):
    return np.asarray(A, np.float64) @ np.asarray(B, np.float64).T


def conv3x3(X, Wt):
    X = np.asarray(X, np.float64)
    Wt = np.asarray(Wt, np.float64)
    n, H, W, C = X.shape
    O = Wt.shape[0]
    Xp = np.zeros((n, H + 2, W + 2, C))
    Xp[:, 1:H + 1, 1:W + 1, :] = X
    Y = np.zeros((n, H, W, O))
    for dy in range(3):
        for dx in range(3):
            # tap (dy, dx) reads the input shifted by (dy - 1, dx - 1)
            Y += Xp[:, dy:dy + H, dx:dx + W, :] @ Wt[:, dy * 3 + dx, :].T
    return Y
