"""The island criterion of a mixed pass, restated in numpy from its definition (include/qmcfi.h, FP64 islands):
a lattice point is an island at level L when prod over the sector's singular variables of (k_j + 1) / n is below
10^-(L+1), k_j = floor(n x_j) the integer part of the shifted lattice coordinate.  The product is taken in FP32,
factor by factor, each operation correctly rounded, floored at 1e-30 after each factor; its island bin is the
number of levels it is an island at.  numpy's float32 operations round as the device's correctly rounded ones
do, so this gives the device's decision bit for bit."""
import numpy as np

LEVELS = 6
BINS = LEVELS + 1
XI = np.array([1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6], dtype=np.float32)


def shift_floor(delta: float, n: int) -> int:
    a = np.floor(np.float64(delta) * np.float64(n))
    return int(n - 1) if a >= n else int(a)


def shifted_indices(idx, n: int, z, delta):
    """k_j = (i z_j mod n + floor(n delta_j)) mod n per point (rows) and dimension (columns)"""
    idx = np.asarray(idx, dtype=np.uint64)
    cols = []
    for zj, dj in zip(z, delta):
        r = (idx * np.uint64(zj)) % np.uint64(n)
        cols.append((r + np.uint64(shift_floor(dj, n))) % np.uint64(n))
    return np.stack(cols, axis=1).astype(np.uint64)


def keys(k, mask: int, n: int):
    rn = np.float32(1.0) / np.float32(n)
    c = np.ones(k.shape[0], dtype=np.float32)
    for j in range(k.shape[1]):
        if (mask >> j) & 1:
            f = (k[:, j] + np.uint64(1)).astype(np.float32) * rn
            c = np.maximum((c * f).astype(np.float32), np.float32(1e-30))
    return c


def bins(key):
    return (key[:, None] < XI[None, :]).sum(axis=1)


def sing_mask(sec) -> int:
    """bit j set when the sector's endpoint exponent of variable j is -1 (oracle sector)"""
    return sum(1 << j for j, a in enumerate(np.asarray(sec.A)) if int(a) == -1)
