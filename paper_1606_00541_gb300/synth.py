"""Seeded synthetic inputs: matrices, right-hand sides and subdomain partitions.

This module holds no arithmetic of the solver method (no factorization, no level analysis, no
triangular solve).  It only builds the test problems, and it is the one module that both the
CUDA path (benchmark, smoke check) and the CPU oracle's tests read their inputs from.

Grid order is lexicographic with x fastest: g = x + nx * (y + ny * z).  Every CSR row is sorted
by ascending column, as the solver requires (Sec. 2).  All generators return
``(rowptr int32[n+1], col int32[nnz], val float64[nnz])``.

Workloads (stand-ins for the paper's matrices, Sec. 4):
  * ``poisson2d_5pt(64, 64)``: 2D 5-point Poisson, 4 on the diagonal and -1 off it.
  * ``fv7_lognormal(m, sigma=2)``: 3D 7-point finite-volume matrix with ln k ~ N(0, sigma^2) per
    cell, harmonic face transmissibility 2 k1 k2 / (k1 + k2), and Dirichlet boundary faces adding
    2 k_c to the diagonal (an SPD M-matrix).  Stands in for the heterogeneous reservoir matrix
    (SPE10, Example 3) and the 7-point CFD matrix (atmosmodd, Example 2), whose data are not here.
    ``poisson3d_7pt(100)`` reproduces the size of Example 1 exactly (n = 10^6, nnz = 6,940,000).
  * ``stencil27_jitter(m)``: 3D 27-point stencil, a_ij = -(1 + 0.3 u_e) with u_e ~ U[-1, 1] drawn
    once per undirected edge (so A is symmetric), a_ii = 1.05 * sum_j |a_ij|.
"""
from __future__ import annotations

import numpy as np


def _rng(seed):
    return np.random.default_rng(np.random.PCG64(seed))


def _assemble(cols, vals, mask):
    """cols/vals/mask: (n, s) arrays with the s candidate entries of each row already in
    ascending column order; mask selects the entries that exist."""
    counts = mask.sum(axis=1)
    rp = np.zeros(cols.shape[0] + 1, dtype=np.int64)
    np.cumsum(counts, out=rp[1:])
    return rp.astype(np.int32), cols[mask].astype(np.int32), vals[mask].astype(np.float64)


def poisson2d_5pt(nx, ny=None):
    ny = nx if ny is None else ny
    n = nx * ny
    g = np.arange(n, dtype=np.int64)
    x, y = g % nx, g // nx
    offs = [(-nx, y > 0), (-1, x > 0), (0, np.ones(n, bool)), (1, x < nx - 1), (nx, y < ny - 1)]
    cols = np.stack([g + o for o, _ in offs], axis=1)
    mask = np.stack([m for _, m in offs], axis=1)
    vals = np.where(cols == g[:, None], 4.0, -1.0)
    return _assemble(cols, vals, mask)


def _grid3(m):
    n = m * m * m
    g = np.arange(n, dtype=np.int64)
    return n, g, g % m, (g // m) % m, g // (m * m)


def poisson3d_7pt(m):
    """7-point Poisson on an m^3 grid: 6 on the diagonal, -1 off it."""
    n, g, x, y, z = _grid3(m)
    s = m * m
    offs = [(-s, z > 0), (-m, y > 0), (-1, x > 0), (0, np.ones(n, bool)), (1, x < m - 1), (m, y < m - 1),
            (s, z < m - 1)]
    cols = np.stack([g + o for o, _ in offs], axis=1)
    mask = np.stack([k for _, k in offs], axis=1)
    vals = np.where(cols == g[:, None], 6.0, -1.0)
    return _assemble(cols, vals, mask)


def lognormal_perm(m, sigma=2.0, seed=0):
    """Cell permeability k with ln k ~ N(0, sigma^2), i.i.d. per cell."""
    return np.exp(_rng(seed).normal(0.0, sigma, size=m * m * m))


def fv7_lognormal(m, sigma=2.0, seed=0, perm=None):
    k = lognormal_perm(m, sigma, seed) if perm is None else perm
    return fv7_lognormal_box(m, m, m, perm=k)


def fv7_lognormal_box(nx, ny, nz, perm):
    """7-point finite-volume matrix on an nx x ny x nz grid (x fastest) for cell permeability
    `perm`: harmonic face averages, Dirichlet faces at the boundary (2 k)."""
    n = nx * ny * nz
    g = np.arange(n, dtype=np.int64)
    x, y, z = g % nx, (g // nx) % ny, g // (nx * ny)
    k = np.asarray(perm, dtype=np.float64)
    s = nx * ny
    nbr = [(-s, z > 0), (-nx, y > 0), (-1, x > 0), (1, x < nx - 1), (nx, y < ny - 1), (s, z < nz - 1)]
    diag = np.zeros(n)
    off_vals = []
    for o, ok in nbr:
        kn = np.where(ok, k[np.clip(g + o, 0, n - 1)], 1.0)
        t = np.where(ok, 2.0 * k * kn / (k + kn), 0.0)      # harmonic face average
        tb = np.where(ok, 0.0, 2.0 * k)                      # Dirichlet boundary face
        diag += t + tb
        off_vals.append(-t)
    cols = np.stack([g - s, g - nx, g - 1, g, g + 1, g + nx, g + s], axis=1)
    vals = np.stack(off_vals[:3] + [diag] + off_vals[3:], axis=1)
    mask = np.stack([nbr[0][1], nbr[1][1], nbr[2][1], np.ones(n, bool), nbr[3][1], nbr[4][1], nbr[5][1]], axis=1)
    return _assemble(cols, vals, mask)


def stencil27_jitter(m, jitter=0.3, dominance=1.05, seed=0):
    n, g, x, y, z = _grid3(m)
    rng = _rng(seed)
    offsets = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    # one uniform draw per undirected edge: stored on the cell with the larger index (positive
    # offset seen from the smaller one), read back by the other endpoint
    pos = [o for o in offsets if (o[0] * m * m + o[1] * m + o[2]) > 0]
    u = {o: rng.uniform(-1.0, 1.0, size=n) for o in pos}
    cols, vals, mask = [], [], []
    for dz, dy, dx in offsets:
        d = dz * m * m + dy * m + dx
        ok = (x + dx >= 0) & (x + dx < m) & (y + dy >= 0) & (y + dy < m) & (z + dz >= 0) & (z + dz < m)
        c = g + d
        if d == 0:
            cols.append(c); vals.append(np.zeros(n)); mask.append(np.ones(n, bool))
            continue
        if d > 0:
            ue = u[(dz, dy, dx)]
        else:
            ue = u[(-dz, -dy, -dx)][np.clip(c, 0, n - 1)]
        cols.append(c)
        vals.append(np.where(ok, -(1.0 + jitter * ue), 0.0))
        mask.append(ok)
    cols = np.stack(cols, axis=1)
    vals = np.stack(vals, axis=1)
    mask = np.stack(mask, axis=1)
    dcol = offsets.index((0, 0, 0))
    vals[:, dcol] = dominance * np.abs(np.where(mask, vals, 0.0)).sum(axis=1)
    return _assemble(cols, vals, mask)


def uniform_vector(n, seed, nrhs=1, lo=-1.0, hi=1.0):
    """b (or x_true) ~ U[lo, hi], shape (n,) or row-major (n, nrhs) with column q drawn from seed + q."""
    if nrhs == 1:
        return _rng(seed).uniform(lo, hi, size=n)
    return np.stack([_rng(seed + q).uniform(lo, hi, size=n) for q in range(nrhs)], axis=1)


def box_partition(m, cuts):
    """Box subdomains of an m^3 grid: the same per-axis cut lengths on x, y and z (they must sum
    to m).  Returns (part[n] int32 with the subdomain of each cell, number of subdomains).  With
    cuts [25, 39, 25, 39] on 128^3 this gives 64 boxes of 25^3 .. 39^3 cells."""
    cuts = list(cuts)
    assert sum(cuts) == m
    edges = np.cumsum([0] + cuts)
    axis_id = np.searchsorted(edges, np.arange(m), side="right") - 1
    nc = len(cuts)
    n, g, x, y, z = _grid3(m)
    part = axis_id[x] + nc * (axis_id[y] + nc * axis_id[z])
    return part.astype(np.int32), nc ** 3


def grid_boxes(m, nb):
    """Partition of an m^3 grid into nb = (bx, by, bz) boxes of near-equal extent per axis (box k
    of an axis covers cells floor(k m / b) .. floor((k+1) m / b) - 1).  (1, 12, 12) gives 144 x-pencils
    of 128 x 10..11 x 10..11 cells on 128^3.  Returns (part[n] int32, number of boxes)."""
    n, g, x, y, z = _grid3(m)
    ids = [(c * b) // m for c, b in zip((x, y, z), nb)]
    part = ids[0] + nb[0] * (ids[1] + nb[1] * ids[2])
    return part.astype(np.int32), int(nb[0] * nb[1] * nb[2])


def random_lower(n, density, seed, unit_diag=False, uplo=0, dominance=None):
    """Random sparse triangular matrix for property tests: each strictly-triangular entry is
    present with probability ``density``; off-diagonal values ~ U[-1, 1]; the diagonal is
    1 when ``unit_diag`` else U[1, 2] (or ``dominance`` * row abs-sum when given)."""
    rng = _rng(seed)
    rows, cols, vals = [], [], []
    for i in range(n):
        if uplo == 0:
            cand = np.nonzero(rng.random(i) < density)[0]
        else:
            cand = i + 1 + np.nonzero(rng.random(n - 1 - i) < density)[0]
        ov = rng.uniform(-1.0, 1.0, size=len(cand))
        d = 1.0 if unit_diag else rng.uniform(1.0, 2.0)
        if dominance is not None:
            d = dominance * max(np.abs(ov).sum(), 1.0)
        c = np.concatenate([cand, [i]]) if uplo == 0 else np.concatenate([[i], cand])
        vv = np.concatenate([ov, [d]]) if uplo == 0 else np.concatenate([[d], ov])
        rows.append(np.full(len(c), i))
        cols.append(c)
        vals.append(vv)
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, rows + 1, 1)
    return np.cumsum(rp).astype(np.int32), cols.astype(np.int32), vals.astype(np.float64)


def random_sparse(n, density, seed, dominance=1.5):
    """Random sparse (nonsymmetric pattern) diagonally dominant matrix for factorization tests."""
    rng = _rng(seed)
    rp = [0]
    cols, vals = [], []
    for i in range(n):
        c = np.nonzero(rng.random(n) < density)[0]
        c = c[c != i]
        v = rng.uniform(-1.0, 1.0, size=len(c))
        d = dominance * max(np.abs(v).sum(), 1.0)
        cc = np.concatenate([c, [i]])
        vv = np.concatenate([v, [d]])
        o = np.argsort(cc, kind="stable")
        cols.append(cc[o])
        vals.append(vv[o])
        rp.append(rp[-1] + len(cc))
    return np.array(rp, dtype=np.int32), np.concatenate(cols).astype(np.int32), np.concatenate(vals)
