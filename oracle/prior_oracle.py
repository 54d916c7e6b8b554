"""Oracle of the learned prior's contractions -- TEST INFRASTRUCTURE ONLY.

Plain FP64 numpy definitions that the tensor-core kernels are checked
against; nothing in the product path imports this module.

gemm(A, B)        D = A B^T, the definition written with numpy's matmul.
conv3x3(X, Wt)    same-size 3x3 cross-correlation with zero padding, written as
                  the nine shifted, weighted sums of the convolution layer of
                  the denoising network (Sec. 2.2: g_theta is a CNN/U-Net on
                  velocity-model images):
                  Y[n, y, x, o] = sum_{dy, dx} sum_c Wt[o, dy*3+dx, c] X[n, y+dy-1, x+dx-1, c].
conv3x3x3(X, Wt)  the same layer for volumes (the prior of the 3D models), 27
                  shifted, weighted sums:
                  Y[n, z, y, x, o] = sum_{dz, dy, dx} sum_c Wt[o, dz*9+dy*3+dx, c] X[n, z+dz-1, y+dy-1, x+dx-1, c].
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


def conv3x3_dgrad(dY, Wt):
    """Input gradient of conv3x3, written as the scatter of every output
    gradient back through the nine taps: dX[n, y+dy-1, x+dx-1, c] +=
    sum_o dY[n, y, x, o] Wt[o, dy*3+dx, c] (contributions off the image dropped)."""
    dY = np.asarray(dY, np.float64)
    Wt = np.asarray(Wt, np.float64)
    n, H, W, O = dY.shape
    C = Wt.shape[2]
    dXp = np.zeros((n, H + 2, W + 2, C))
    for dy in range(3):
        for dx in range(3):
            dXp[:, dy:dy + H, dx:dx + W, :] += dY @ Wt[:, dy * 3 + dx, :]
    return dXp[:, 1:H + 1, 1:W + 1, :]


def conv3x3_wgrad(dY, X):
    """Weight gradient of conv3x3: dW[o, dy*3+dx, c] = sum over pixels of
    dY[n, y, x, o] X[n, y+dy-1, x+dx-1, c] (zero off the image)."""
    dY = np.asarray(dY, np.float64)
    X = np.asarray(X, np.float64)
    n, H, W, O = dY.shape
    C = X.shape[3]
    Xp = np.zeros((n, H + 2, W + 2, C))
    Xp[:, 1:H + 1, 1:W + 1, :] = X
    dW = np.zeros((O, 9, C))
    for dy in range(3):
        for dx in range(3):
            dW[:, dy * 3 + dx, :] = dY.reshape(-1, O).T @ Xp[:, dy:dy + H, dx:dx + W, :].reshape(-1, C)
    return dW


def _pad3(X):
    n, D, H, W, C = X.shape
    Xp = np.zeros((n, D + 2, H + 2, W + 2, C))
    Xp[:, 1:D + 1, 1:H + 1, 1:W + 1, :] = X
    return Xp


def conv3x3x3(X, Wt):
    X = np.asarray(X, np.float64)
    Wt = np.asarray(Wt, np.float64)
    n, D, H, W, C = X.shape
    Xp = _pad3(X)
    Y = np.zeros((n, D, H, W, Wt.shape[0]))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                # tap (dz, dy, dx) reads the input shifted by (dz - 1, dy - 1, dx - 1)
                Y += Xp[:, dz:dz + D, dy:dy + H, dx:dx + W, :] @ Wt[:, dz * 9 + dy * 3 + dx, :].T
    return Y


def conv3x3x3_dgrad(dY, Wt):
    """Input gradient of conv3x3x3: the scatter of every output gradient back
    through the 27 taps (contributions off the volume dropped)."""
    dY = np.asarray(dY, np.float64)
    Wt = np.asarray(Wt, np.float64)
    n, D, H, W, O = dY.shape
    dXp = np.zeros((n, D + 2, H + 2, W + 2, Wt.shape[2]))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                dXp[:, dz:dz + D, dy:dy + H, dx:dx + W, :] += dY @ Wt[:, dz * 9 + dy * 3 + dx, :]
    return dXp[:, 1:D + 1, 1:H + 1, 1:W + 1, :]


def conv3x3x3_wgrad(dY, X):
    """Weight gradient of conv3x3x3: dW[o, dz*9+dy*3+dx, c] = sum over voxels
    of dY[n, z, y, x, o] X[n, z+dz-1, y+dy-1, x+dx-1, c] (zero off the volume)."""
    dY = np.asarray(dY, np.float64)
    X = np.asarray(X, np.float64)
    n, D, H, W, O = dY.shape
    C = X.shape[4]
    Xp = _pad3(X)
    dW = np.zeros((O, 27, C))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                dW[:, dz * 9 + dy * 3 + dx, :] = (dY.reshape(-1, O).T
                                                  @ Xp[:, dz:dz + D, dy:dy + H, dx:dx + W, :].reshape(-1, C))
    return dW
