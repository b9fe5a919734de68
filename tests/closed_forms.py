"""Closed-form Laplacian spectra of structured graphs (textbook results).

Path P_n: 2 - 2 cos(pi k / n); cycle C_n: 2 - 2 cos(2 pi k / n); complete K_n:
0 and n (n-1 times); star K_{1,n-1}: 0, 1 (n-2 times), n; hypercube Q_r: 2j with
multiplicity C(r, j); Cartesian products (grids) add the factors' eigenvalues
(the Laplacian of a Cartesian product is the Kronecker sum of the factors').
"""
import math

import numpy as np


def path(n):
    return np.sort(2.0 - 2.0 * np.cos(np.pi * np.arange(n) / n))


def cycle(n):
    return np.sort(2.0 - 2.0 * np.cos(2.0 * np.pi * np.arange(n) / n))


def complete(n):
    return np.array([0.0] + [float(n)] * (n - 1))


def star(n):
    return np.array([0.0] + [1.0] * (n - 2) + [float(n)])


def hypercube(r):
    return np.sort(np.concatenate([np.full(math.comb(r, j), 2.0 * j) for j in range(r + 1)]))


def product(*factors):
    out = np.zeros(1)
    for f in factors:
        out = (out[:, None] + np.asarray(f)[None, :]).ravel()
    return np.sort(out)


def grid2d(nx, ny):
    return product(path(nx), path(ny))


def grid3d(nx, ny, nz):
    return product(path(nx), path(ny), path(nz))
