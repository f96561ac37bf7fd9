"""Finite-difference diffusion matrices, box partitions and seeded vectors.

Conventions (one reading of Section 6, where the paper uses finite elements):
  * Dirichlet boundary nodes are eliminated; only interior nodes are unknowns.
  * Lexicographic numbering idx = i + nx*(j + ny*k).
  * Stencils are unscaled by h^2: 5-point [4; -1 x 4], 7-point [6; -1 x 6].
  * Variable coefficient: node-wise kappa, face coefficient is the harmonic
    mean 2 k_i k_j / (k_i + k_j), a face to the boundary uses k_i, and the
    diagonal is the sum of the face coefficients of the node.
  * CSR arrays: rowptr int32 (n+1), col int32 (nnz, ascending within a row),
    val float64 (nnz).
"""
from __future__ import annotations

import numpy as np


def _stencil_csr(shape, face_coef):
    """Assemble the CSR matrix of a nearest-neighbour stencil on a box grid.

    shape     -- (nx,) (nx, ny) or (nx, ny, nz) interior grid
    face_coef -- callable(axis, lo_mask_index_arrays) -> see below; here a list
                 per axis of arrays c_minus, c_plus of shape `shape` giving the
                 coefficient of the face towards -axis / +axis of each node
                 (the boundary faces included: they add to the diagonal only).
    """
    dims = len(shape)
    n = int(np.prod(shape))
    # lexicographic: first axis fastest
    strides = [1]
    for d in range(1, dims):
        strides.append(strides[-1] * shape[d - 1])
    idx = np.arange(n, dtype=np.int64).reshape(shape[::-1])  # (nz, ny, nx)
    coords = np.unravel_index(np.arange(n), shape[::-1])      # arrays k, j, i
    coords = coords[::-1]                                       # i, j, k order
    c_minus, c_plus = face_coef
    diag = np.zeros(n)
    for d in range(dims):
        diag += c_minus[d].reshape(-1) + c_plus[d].reshape(-1)
    # neighbour slots in ascending column order:
    # -z, -y, -x, self, +x, +y, +z  (for lexicographic numbering)
    cols = []
    vals = []
    valid = []
    for d in reversed(range(dims)):
        ok = coords[d] > 0
        cols.append(np.arange(n, dtype=np.int64) - strides[d])
        vals.append(-c_minus[d].reshape(-1))
        valid.append(ok)
    cols.append(np.arange(n, dtype=np.int64))
    vals.append(diag)
    valid.append(np.ones(n, dtype=bool))
    for d in range(dims):
        ok = coords[d] < shape[d] - 1
        cols.append(np.arange(n, dtype=np.int64) + strides[d])
        vals.append(-c_plus[d].reshape(-1))
        valid.append(ok)
    cols = np.stack(cols, axis=1)
    vals = np.stack(vals, axis=1)
    valid = np.stack(valid, axis=1)
    counts = valid.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("matrix too large for int32 row pointers")
    col = cols[valid].astype(np.int32)
    val = vals[valid].astype(np.float64)
    del idx
    return rowptr.astype(np.int32), col, val


def poisson2d(nx: int, ny: int):
    """5-point Dirichlet Laplacian on an nx x ny interior grid (unscaled)."""
    shape = (nx, ny)
    ones = np.ones(shape[::-1])
    c = [ones, ones]
    return _stencil_csr(shape, (c, c))


def poisson3d(nx: int, ny: int, nz: int):
    """7-point Dirichlet Laplacian on an nx x ny x nz interior grid (unscaled)."""
    shape = (nx, ny, nz)
    ones = np.ones(shape[::-1])
    c = [ones, ones, ones]
    return _stencil_csr(shape, (c, c))


def diffusion3d(kappa: np.ndarray):
    """7-point -div(kappa grad u) with node-wise kappa of shape (nz, ny, nx).

    Face coefficient between nodes i and j: 2 k_i k_j / (k_i + k_j); a face
    to the Dirichlet boundary uses k_i.
    """
    k = np.asarray(kappa, dtype=np.float64)
    nz, ny, nx = k.shape
    shape = (nx, ny, nz)
    c_minus = []
    c_plus = []
    for d, ax in zip(range(3), (2, 1, 0)):  # d: x,y,z  -> array axis
        km = k.copy()
        kp = k.copy()
        sl_lo = [slice(None)] * 3
        sl_hi = [slice(None)] * 3
        sl_lo[ax] = slice(0, -1)
        sl_hi[ax] = slice(1, None)
        a = k[tuple(sl_lo)]
        b = k[tuple(sl_hi)]
        h = 2.0 * a * b / (a + b)
        kp[tuple(sl_lo)] = h
        km[tuple(sl_hi)] = h
        c_minus.append(km)
        c_plus.append(kp)
    return _stencil_csr(shape, (c_minus, c_plus))


def rotated_anisotropic2d(nx: int, ny: int, theta: float = 3 * np.pi / 16, eps: float = 1e-3):
    """-div(K grad u) on the unit square, K = Q diag(1, eps) Q^T with Q the
    rotation by theta, Dirichlet boundary, nx*ny interior nodes, i fastest.

    9-point finite differences (unscaled by h^2): with k11 = cos^2 + eps sin^2,
    k22 = sin^2 + eps cos^2, k12 = (1 - eps) cos sin, centre 2 k11 + 2 k22,
    east/west -k11, north/south -k22, and the mixed derivative as
    -2 k12 (u_NE - u_NW - u_SE + u_SW) / 4: NE/SW -k12/2, NW/SE +k12/2.
    """
    c, s = np.cos(theta), np.sin(theta)
    k11 = c * c + eps * s * s
    k22 = s * s + eps * c * c
    k12 = (1.0 - eps) * c * s
    n = nx * ny
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    ii = ii.reshape(-1)
    jj = jj.reshape(-1)
    rows, cols, vals = [np.arange(n)], [np.arange(n)], [np.full(n, 2.0 * k11 + 2.0 * k22)]
    for di, dj, a in ((-1, 0, -k11), (1, 0, -k11), (0, -1, -k22), (0, 1, -k22),
                      (1, 1, -0.5 * k12), (-1, -1, -0.5 * k12), (-1, 1, 0.5 * k12), (1, -1, 0.5 * k12)):
        i2, j2 = ii + di, jj + dj
        ok = (i2 >= 0) & (i2 < nx) & (j2 >= 0) & (j2 < ny)
        rows.append(np.nonzero(ok)[0])
        cols.append(j2[ok] * nx + i2[ok])
        vals.append(np.full(int(ok.sum()), a))
    r = np.concatenate(rows)
    cidx = np.concatenate(cols)
    v = np.concatenate(vals)
    order = np.lexsort((cidx, r))
    r, cidx, v = r[order], cidx[order], v[order]
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr.astype(np.int32), cidx.astype(np.int32), v


def weak_link_chain(n_left: int = 8, n_right: int = 8, link: float = 0.25, y_diag: float = 1.0):
    """1D chain whose middle point y = n_left is attached to its two chain
    neighbours only through positive (weak) entries: rows away from y are
    [-1, 2, -1] (entries towards y omitted), row y is [+link, y_diag, +link]
    and its neighbours hold the symmetric +link. Irreducibly diagonally
    dominant with a positive diagonal (SPD) for link < 1 and y_diag > 2 link. This is
    the shape of the example of Section 4.2 in which a fine point has no
    interpolation connection between two injected C points.
    Returns rowptr, col (int32), val (float64) in CSR."""
    n = n_left + 1 + n_right
    y = n_left
    rows, cols, vals = [], [], []
    for i in range(n):
        for j in (i - 1, i, i + 1):
            if j < 0 or j >= n:
                continue
            if i == j:
                a = y_diag if i == y else 2.0
            elif i == y or j == y:
                a = link
            else:
                a = -1.0
            rows.append(i)
            cols.append(j)
            vals.append(a)
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, np.asarray(rows) + 1, 1)
    return np.cumsum(rowptr).astype(np.int32), np.asarray(cols, np.int32), np.asarray(vals, np.float64)


def checkerboard_kappa(n: int, blocks: int, seed: int, values=(1.0, 1e3)):
    """Piecewise-constant kappa on an n^3 grid: blocks^3 cubes, i.i.d. values."""
    rng = np.random.default_rng(seed)
    pick = rng.integers(0, 2, size=(blocks, blocks, blocks))
    table = np.asarray(values, dtype=np.float64)[pick]
    edge = -(-n // blocks)
    k = np.repeat(np.repeat(np.repeat(table, edge, 0), edge, 1), edge, 2)
    return np.ascontiguousarray(k[:n, :n, :n])


def gaussian_random_field(n: int, length: float = 0.1, variance: float = 1.0, seed: int = 0):
    """Zero-mean Gaussian random field on the interior nodes of the unit cube
    (h = 1/(n+1)), shape (n, n, n): white noise smoothed by a separable
    Gaussian filter whose covariance exp(-d^2 / (2 length^2)) corresponds to a
    filter width length / sqrt(2) per axis, renormalised to the requested
    variance (sample variance)."""
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((n, n, n))
    h = 1.0 / (n + 1)
    sigma = length / np.sqrt(2.0) / h            # in grid points
    r = int(np.ceil(4 * sigma))
    t = np.arange(-r, r + 1)
    k = np.exp(-0.5 * (t / sigma) ** 2)
    k /= k.sum()
    g = noise
    for ax in range(3):
        g = np.apply_along_axis(lambda v: np.convolve(v, k, mode="same"), ax, g)
    g -= g.mean()
    g *= np.sqrt(variance / g.var())
    return g


def lognormal_kappa(n: int, length: float = 0.1, variance: float = 1.0, seed: int = 0):
    """kappa = exp(g) with g a Gaussian random field (gaussian_random_field)."""
    return np.exp(gaussian_random_field(n, length, variance, seed))


def box_partition(shape, box):
    """Subdomain id of every unknown for a partition into boxes.

    shape -- interior grid (nx, ny[, nz]); box -- box edge lengths.
    Boxes are numbered lexicographically (first axis fastest), like unknowns.
    Returns (part int32[n], nsub).
    """
    shape = tuple(int(s) for s in shape)
    box = tuple(int(b) for b in box)
    nb = [-(-s // b) for s, b in zip(shape, box)]
    grids = np.meshgrid(*[np.arange(s) // b for s, b in zip(shape, box)],
                        indexing="ij")  # each of shape `shape`
    pid = np.zeros(shape, dtype=np.int64)
    mult = 1
    for d in range(len(shape)):
        pid += grids[d] * mult
        mult *= nb[d]
    # flatten in lexicographic order (first axis fastest)
    part = pid.transpose(tuple(reversed(range(len(shape))))).reshape(-1)
    return part.astype(np.int32), int(mult)


def batched_poisson(nsys: int = 64, edges=(32, 48, 64, 80, 96), box: int = 16, nrhs: int = 4, seed: int = 0):
    """Independent 3D 7-point Poisson systems as one block-diagonal matrix.

    Each system's edge length is drawn uniformly from `edges` (seeded); its
    unknowns are partitioned into boxes of `box`^3 (uneven boxes at the ends
    when box does not divide the edge), numbered after the previous systems'.
    Returns rowptr, col, val (int32/int32/float64), part (int32), nsub,
    B (n x nrhs, U[-1,1] from the seed), the edge list and the row offsets."""
    rng = np.random.default_rng(seed)
    picks = [int(edges[i]) for i in rng.integers(0, len(edges), size=nsys)]
    rps, cis, vs, parts = [], [], [], []
    row0 = 0
    nnz0 = 0
    sub0 = 0
    offs = [0]
    for e in picks:
        rp, ci, v = poisson3d(e, e, e)
        part, ns = box_partition((e, e, e), (box, box, box))
        rps.append(rp[:-1].astype(np.int64) + nnz0)
        cis.append(ci.astype(np.int64) + row0)
        vs.append(v)
        parts.append(part.astype(np.int64) + sub0)
        row0 += len(rp) - 1
        nnz0 += len(ci)
        sub0 += ns
        offs.append(row0)
    rowptr = np.concatenate(rps + [np.array([nnz0], np.int64)])
    if nnz0 >= 2**31:
        raise ValueError("batch too large for int32 row pointers")
    B = rng.uniform(-1.0, 1.0, size=(row0, nrhs))
    return (rowptr.astype(np.int32), np.concatenate(cis).astype(np.int32), np.concatenate(vs),
            np.concatenate(parts).astype(np.int32), int(sub0), B, picks, np.array(offs))


def uniform_rhs(n: int, seed: int):
    """b ~ U[-1, 1] from numpy.random.default_rng(seed)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=n)


def grid_shape_of(name: str):
    return WORKLOADS[name]["shape"]


WORKLOADS = {
    # 2D 5-point Poisson 64x64, 4x4 boxes of 16x16, padding 1 on every level
    "poisson2d_64": dict(shape=(64, 64), box=(16, 16), padding=1, n_fac=2),
    # 3D 7-point Poisson 128^3, 8x8x8 boxes of 16^3, padding 2 on every level
    "poisson3d_128": dict(shape=(128, 128, 128), box=(16, 16, 16), padding=2,
                          n_fac=2),
    # 3D 7-point -div(kappa grad u) on 256^3, kappa constant on 8^3 blocks of
    # 32^3 nodes, i.i.d. {1, 1e3} with p = 1/2; 4096 boxes of 16^3, padding 2;
    # FP32 AlgFAC inside FP64 refinement
    "kappa3d_256": dict(shape=(256, 256, 256), box=(16, 16, 16), padding=2, n_fac=2,
                        kappa_blocks=8, precision=1),
    # 2D rotated anisotropic diffusion (theta = 3 pi / 16, eps = 1e-3, 9-point
    # finite differences) on 512^2, 256 boxes of 32^2, padding 2, FP64
    "aniso2d_512": dict(shape=(512, 512), box=(32, 32), padding=2, n_fac=2,
                        aniso=(3 * np.pi / 16, 1e-3)),
    # 64 independent 3D 7-point Poisson systems, edges i.i.d. from
    # {32, 48, 64, 80, 96}, boxes of 16^3, 4 right-hand sides each, FP32
    # AlgFAC inside FP64 refinement
    "batched_64": dict(nsys=64, edges=(32, 48, 64, 80, 96), box=(16, 16, 16), padding=2, n_fac=2,
                       nrhs=4, precision=1),
}


def workload(name: str, seed: int = 0, shape=None, box=None, nsys=None):
    """Matrix, partition and right-hand side of a named synthetic workload
    (shape, box, nsys: smaller variants of it for profiling and tests)."""
    w = dict(WORKLOADS[name])
    if nsys is not None:
        w["nsys"] = int(nsys)
    if shape is not None:
        w["shape"] = tuple(shape)
    if box is not None:
        w["box"] = tuple(box)
    if "nsys" in w:
        rp, ci, v, part, nsub, B, picks, offs = batched_poisson(
            w["nsys"], edges=w["edges"], box=w["box"][0], nrhs=w["nrhs"], seed=seed)
        return dict(rowptr=rp, col=ci, val=v, part=part, nsub=nsub, B=B, b=np.ascontiguousarray(B[:, 0]),
                    padding=w["padding"], n_fac=w["n_fac"], edges=picks, offsets=offs, nrhs=w["nrhs"],
                    precision=w["precision"], box=w["box"], name=name, seed=seed)
    shape = w["shape"]
    if "kappa_blocks" in w:
        kappa = checkerboard_kappa(shape[0], w["kappa_blocks"], seed)
        rp, ci, v = diffusion3d(kappa)
    elif "aniso" in w:
        rp, ci, v = rotated_anisotropic2d(shape[0], shape[1], *w["aniso"])
    elif len(shape) == 2:
        rp, ci, v = poisson2d(*shape)
    else:
        rp, ci, v = poisson3d(*shape)
    part, nsub = box_partition(shape, w["box"])
    b = uniform_rhs(int(np.prod(shape)), seed)
    return dict(rowptr=rp, col=ci, val=v, part=part, nsub=nsub, b=b,
                padding=w["padding"], n_fac=w["n_fac"], shape=shape,
                box=w["box"], name=name, seed=seed, precision=w.get("precision", 0))
