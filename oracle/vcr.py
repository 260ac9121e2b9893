"""FP64 oracle of the vessel continuity regulariser (Methods, vessel continuity regularisation):

    R_VCR(x) = R_H(x) + beta R_TV(x)
    R_H(x)   = sum_i sqrt( sum_{p,q in {x,y,z}} (D_pq x)_i^2 + eps )
    R_TV(x)  = sum_i sqrt( sum_{d in {x,y,z}} (D_d x)_i^2 + eps )

TEST INFRASTRUCTURE ONLY: loaded by tests/ (and nothing in the product package).  It shares no
code with the CUDA library.

The paper leaves the difference operators, the boundary rule and eps open; the readings taken:
  - D_d: central first difference (x[i + e_d] - x[i - e_d]) / 2;
  - D_pp: x[i + e_p] - 2 x[i] + x[i - e_p];
  - D_pq (p != q): (x[i+e_p+e_q] - x[i+e_p-e_q] - x[i-e_p+e_q] + x[i-e_p-e_q]) / 4, which appears
    twice in the sum over (p, q) (D_pq = D_qp);
  - Neumann boundaries: every neighbour index is clamped to the volume, per axis;
  - unit (voxel) spacing; eps inside each square root.
Each operator is an explicit sparse matrix built from those stencils; the gradient is
grad R = sum_k D_k^T (w_k * D_k x) with w = 1 / sqrt(...) of the term the operator belongs to.
Volumes are (nz, ny, nx) arrays, x fastest.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _shift(dims, off):
    """(S x)[i] = x[clamp(i + off)] per axis, as a sparse matrix (off = (ox, oy, oz))."""
    nz, ny, nx = dims
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    jx = np.clip(ix + off[0], 0, nx - 1)
    jy = np.clip(iy + off[1], 0, ny - 1)
    jz = np.clip(iz + off[2], 0, nz - 1)
    rows = ((iz * ny + iy) * nx + ix).ravel()
    cols = ((jz * ny + jy) * nx + jx).ravel()
    M = nx * ny * nz
    return sp.csr_matrix((np.ones(M), (rows, cols)), shape=(M, M))


def operators(dims):
    """Returns (first, hessian): first = [D_x, D_y, D_z]; hessian = [(D, multiplicity)] over
    (xx, yy, zz, xy, xz, yz), the mixed ones counted twice in the Frobenius sum."""
    e = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    S = lambda *o: _shift(dims, o)
    add = lambda a, b, s=1: tuple(a[t] + s * b[t] for t in range(3))
    neg = lambda a: tuple(-c for c in a)
    M = int(np.prod(dims))
    I = sp.identity(M, format="csr")
    first = [0.5 * (S(*e[d]) - S(*neg(e[d]))) for d in range(3)]
    hess = [(S(*e[p]) - 2.0 * I + S(*neg(e[p])), 1.0) for p in range(3)]
    for p, q in ((0, 1), (0, 2), (1, 2)):
        D = 0.25 * (S(*add(e[p], e[q])) - S(*add(e[p], e[q], -1)) - S(*add(neg(e[p]), e[q]))
                    + S(*add(neg(e[p]), e[q], -1)))
        hess.append((D, 2.0))
    return first, hess


def value_and_grad(x, beta, eps=1e-8):
    """R_VCR(x) and its gradient (same shape as x), FP64."""
    x = np.asarray(x, dtype=np.float64)
    dims = x.shape
    v = x.ravel()
    first, hess = operators(dims)
    hx = [D @ v for D, _ in hess]
    sH = sum(m * h * h for (_, m), h in zip(hess, hx))
    dx = [D @ v for D in first]
    sT = sum(d * d for d in dx)
    rH, rT = np.sqrt(sH + eps), np.sqrt(sT + eps)
    value = float(np.sum(rH) + beta * np.sum(rT))
    g = sum(m * (D.T @ (h / rH)) for (D, m), h in zip(hess, hx))
    g = g + beta * sum(D.T @ (d / rT) for D, d in zip(first, dx))
    return value, g.reshape(dims)
