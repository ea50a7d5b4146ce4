"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the preconditioner: it only builds problem
matrices (CSR, full symmetric pattern), partitions of the unknowns into
non-overlapping subdomains, and right-hand sides.  Everything is deterministic
for a given seed (numpy PCG64 streams).

Problem shapes follow the paper's experiments where they are stated: a sparse
SPD matrix A and a graph partition into N disjoint sets (Sec. 2.1); the 3D
diffusion generator mimics the high-contrast coefficient of Fig. 2a
(coefficient extruded in one direction, contrast up to 1e6).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    """Square sparse matrix in CSR form: int64 row pointers, int32 column
    indices (ascending within each row), float64 values."""

    n: int
    rowptr: np.ndarray
    colind: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def _csr_from_coo(n, rows, cols, vals) -> CSR:
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    key = rows * n + cols
    order = np.argsort(key, kind="stable")
    key, vals = key[order], vals[order]
    uniq, start = np.unique(key, return_index=True)
    summed = np.add.reduceat(vals, start) if len(vals) else vals
    r = (uniq // n).astype(np.int64)
    c = (uniq % n).astype(np.int32)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int64)
    return CSR(n, rowptr, c, summed.astype(np.float64))


def laplace2d(m: int) -> CSR:
    """5-point Dirichlet Laplacian on an m x m grid of interior nodes.

    Node (x, y) has index y*m + x; the stencil is [4, -1, -1, -1, -1] with the
    boundary eliminated.  Its eigenvalues are 4 - 2cos(j pi/(m+1)) -
    2cos(k pi/(m+1)), j, k = 1..m.
    """
    n = m * m
    idx = np.arange(n).reshape(m, m)  # [y, x]
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [np.full(n, 4.0)]
    for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
        ys, xs = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
        ny, nx = ys + dy, xs + dx
        ok = (ny >= 0) & (ny < m) & (nx >= 0) & (nx < m)
        rows.append(idx[ys[ok], xs[ok]])
        cols.append(idx[ny[ok], nx[ok]])
        vals.append(np.full(int(ok.sum()), -1.0))
    return _csr_from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def disjoint_blocks(m: int, nblocks: int):
    """nblocks uncoupled copies of the m x m 2D Laplacian, copy b scaled by
    b + 1, and the partition with one subdomain per copy (returns (A, part)).
    Every subdomain then has empty overlap and extension sets."""
    L = laplace2d(m)
    rows = np.repeat(np.arange(L.n, dtype=np.int64), np.diff(L.rowptr))
    R, Cc, V = [], [], []
    for b in range(nblocks):
        R.append(rows + b * L.n)
        Cc.append(L.colind.astype(np.int64) + b * L.n)
        V.append(L.val * (b + 1))
    A = _csr_from_coo(nblocks * L.n, np.concatenate(R), np.concatenate(Cc), np.concatenate(V))
    return A, np.repeat(np.arange(nblocks, dtype=np.int32), L.n)


def box_partition_2d(m: int, box: int) -> np.ndarray:
    """Partition of the m x m grid of laplace2d into (m/box)^2 square boxes,
    numbered row-major; returns part[node] in [0, N)."""
    assert m % box == 0
    nb = m // box
    ys, xs = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    return ((ys // box) * nb + xs // box).ravel().astype(np.int32)


def box_groups_2d(nb: int, g: int) -> np.ndarray:
    """Groups of g x g neighbouring boxes of an nb x nb row-major box
    partition (second-level subdomains of the multilevel form): box
    i = by * nb + bx goes to group (by // g) * ceil(nb / g) + bx // g."""
    ng = -(-nb // g)
    by, bx = np.divmod(np.arange(nb * nb), nb)
    return ((by // g) * ng + bx // g).astype(np.int32)


def _gaussian_field(shape, corr: float, rng) -> np.ndarray:
    """Unit-variance Gaussian random field: white noise convolved with a
    separable Gaussian kernel of correlation length `corr` (truncated at
    3*corr), periodic wrap, then renormalised."""
    g = rng.standard_normal(shape)
    half = int(np.ceil(3 * corr))
    t = np.arange(-half, half + 1, dtype=np.float64)
    k = np.exp(-0.5 * (t / corr) ** 2)
    k /= k.sum()
    for ax in range(len(shape)):
        acc = np.zeros_like(g)
        for off, w in zip(t.astype(int), k):
            acc += w * np.roll(g, off, axis=ax)
        g = acc
    g -= g.mean()
    g /= g.std()
    return g


def diffusion_coefficient_3d(m: int, sigma: float, corr: float, n_channels: int,
                             seed: int, channel_value: float = 1e6) -> np.ndarray:
    """Cell coefficient kappa[z, y, x] = exp(sigma * g) with g a unit-variance
    correlated Gaussian field, plus `n_channels` straight one-cell channels of
    value `channel_value` along x at seeded (y, z) positions."""
    rng = np.random.Generator(np.random.PCG64(seed))
    kappa = np.exp(sigma * _gaussian_field((m, m, m), corr, rng))
    if n_channels:
        pos = rng.choice(m * m, size=min(n_channels, m * m), replace=False)
        for p in pos:
            kappa[p // m, p % m, :] = channel_value
    return kappa


def diffusion3d(m: int, sigma: float = 2.0, corr: float = 8.0, n_channels: int = 16,
                seed: int = 0, channel_value: float = 1e6) -> CSR:
    """7-point cell-centred finite-volume diffusion on an m^3 grid (h = 1) with
    homogeneous Dirichlet boundary.  Interior face coefficient: harmonic mean
    of the two cell coefficients; boundary face: 2*kappa_cell (half-cell
    distance).  Cell (x, y, z) has index (z*m + y)*m + x."""
    kappa = diffusion_coefficient_3d(m, sigma, corr, n_channels, seed, channel_value)
    n = m ** 3
    idx = np.arange(n).reshape(m, m, m)
    diag = np.zeros((m, m, m))
    rows, cols, vals = [], [], []
    for ax in range(3):
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, m - 1)
        hi[ax] = slice(1, m)
        ka, kb = kappa[tuple(lo)], kappa[tuple(hi)]
        t = 2.0 * ka * kb / (ka + kb)
        diag[tuple(lo)] += t
        diag[tuple(hi)] += t
        ia, ib = idx[tuple(lo)].ravel(), idx[tuple(hi)].ravel()
        rows += [ia, ib]
        cols += [ib, ia]
        vals += [-t.ravel(), -t.ravel()]
        for face in (0, m - 1):
            sl = [slice(None)] * 3
            sl[ax] = slice(face, face + 1)
            diag[tuple(sl)] += 2.0 * kappa[tuple(sl)]
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    return _csr_from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def _q1_elasticity_stiffness(nu: float) -> np.ndarray:
    """24 x 24 stiffness of a unit-cube trilinear (Q1) hexahedron for isotropic
    linear elasticity with Young's modulus 1 and Poisson ratio nu, by 2x2x2
    Gauss quadrature.  Local node a = (ax, ay, az) in {0,1}^3 has index
    ax + 2 ay + 4 az; dof 3a + component."""
    lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = 1.0 / (2.0 * (1.0 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2.0 * mu
    D[np.arange(3, 6), np.arange(3, 6)] = mu
    corners = np.array([[ax, ay, az] for az in (0, 1) for ay in (0, 1) for ax in (0, 1)], dtype=float)
    sgn = 2.0 * corners - 1.0  # reference coordinates of the corners, +-1
    g = 1.0 / np.sqrt(3.0)
    K = np.zeros((24, 24))
    for qx in (-g, g):
        for qy in (-g, g):
            for qz in (-g, g):
                q = np.array([qx, qy, qz])
                # dN_a/dxi_k = sgn_ak / 8 * prod_{l != k} (1 + sgn_al q_l); x = (xi + 1) / 2
                dN = np.zeros((8, 3))
                for a in range(8):
                    f = 1.0 + sgn[a] * q
                    for k in range(3):
                        dN[a, k] = sgn[a, k] / 8.0 * np.prod(np.delete(f, k))
                dN *= 2.0  # d/dx = 2 d/dxi on a unit cube
                B = np.zeros((6, 24))
                for a in range(8):
                    bx, by, bz = dN[a]
                    B[0, 3 * a] = bx
                    B[1, 3 * a + 1] = by
                    B[2, 3 * a + 2] = bz
                    B[3, 3 * a], B[3, 3 * a + 1] = by, bx
                    B[4, 3 * a + 1], B[4, 3 * a + 2] = bz, by
                    B[5, 3 * a], B[5, 3 * a + 2] = bz, bx
                K += B.T @ D @ B / 8.0  # weight 1, det J = 1/8
    return 0.5 * (K + K.T)


def elasticity3d(ne: int, e_soft: float = 1.0, e_stiff: float = 1e5, layer: int = 4, nu: float = 0.3):
    """3D linear elasticity on ne^3 unit Q1 hexahedra, 3 dofs per node, with
    Young's modulus alternating e_soft / e_stiff every `layer` element layers
    along x, Poisson ratio nu, and the nodes of the face x = 0 clamped (their
    dofs removed).  Returns (A, f, coords): A the SPD stiffness (CSR), f the
    load of a unit body force (0, 0, -1) per unit volume (1/8 of each element's
    volume to each of its nodes), and the node coordinates of each dof.
    Node (x, y, z) has index x + (ne+1) y + (ne+1)^2 z; dofs are numbered
    node-major over the free nodes."""
    Ke = _q1_elasticity_stiffness(nu)
    m = ne + 1
    ex, ey, ez = np.meshgrid(np.arange(ne), np.arange(ne), np.arange(ne), indexing="ij")
    ex, ey, ez = ex.ravel(), ey.ravel(), ez.ravel()
    young = np.where((ex // layer) % 2 == 0, e_soft, e_stiff)
    corner = np.array([[ax, ay, az] for az in (0, 1) for ay in (0, 1) for ax in (0, 1)])
    nodes = ((ex[:, None] + corner[None, :, 0]) + m * (ey[:, None] + corner[None, :, 1])
             + m * m * (ez[:, None] + corner[None, :, 2]))  # (nel, 8)
    free = np.ones(m ** 3, dtype=bool)
    free[np.arange(m ** 3) % m == 0] = False  # x = 0
    node_id = -np.ones(m ** 3, dtype=np.int64)
    node_id[free] = np.arange(int(free.sum()))
    dofs = (3 * node_id[nodes][:, :, None] + np.arange(3)[None, None, :]).reshape(len(ex), 24)
    keep = (node_id[nodes][:, :, None] >= 0).repeat(3, axis=2).reshape(len(ex), 24)
    rows = np.broadcast_to(dofs[:, :, None], (len(ex), 24, 24))
    cols = np.broadcast_to(dofs[:, None, :], (len(ex), 24, 24))
    vals = young[:, None, None] * Ke[None, :, :]
    mask = keep[:, :, None] & keep[:, None, :]
    n = 3 * int(free.sum())
    A = _csr_from_coo(n, rows[mask], cols[mask], vals[mask])
    f = np.zeros(n)
    zdof = dofs[:, 2::3]
    zkeep = keep[:, 2::3]
    np.add.at(f, zdof[zkeep], -1.0 / 8.0)
    fx = np.flatnonzero(free)
    coords = np.stack([fx % m, (fx // m) % m, fx // (m * m)], axis=1).repeat(3, axis=0)
    return A, f, coords


def box_partition_dofs(coords: np.ndarray, boxes) -> np.ndarray:
    """Partition dofs by the node's position in a grid of boxes: boxes =
    (bx, by, bz) node counts per box along x, y, z.  Subdomains are numbered
    x-fastest and renumbered to be contiguous (empty boxes dropped)."""
    c = np.asarray(coords)
    b = np.asarray(boxes)
    cell = c // b
    nb = cell.max(axis=0) + 1
    raw = cell[:, 0] + nb[0] * (cell[:, 1] + nb[1] * cell[:, 2])
    _, part = np.unique(raw, return_inverse=True)
    return part.astype(np.int32)


def _neighbors(A: CSR, v: int) -> np.ndarray:
    return A.colind[A.rowptr[v]:A.rowptr[v + 1]]


def bfs_partition(A: CSR, N: int, seed: int, min_size: int, max_size: int) -> np.ndarray:
    """Seeded multi-source BFS region growing on the graph of A.

    N distinct random seeds; regions grow in round-robin order, one frontier
    node at a time, claiming unclaimed neighbours in random order, and stop at
    max_size.  Nodes left over join an adjacent region.  Regions smaller than
    min_size are merged into their smallest adjacent region; regions larger
    than max_size are split by BFS from their farthest node.  Returns part
    with values in [0, N') (N' may differ from N after merges/splits)."""
    n = A.n
    rng = np.random.Generator(np.random.PCG64(seed))
    part = np.full(n, -1, dtype=np.int64)
    seeds = rng.choice(n, size=N, replace=False)
    frontiers = [[int(s)] for s in seeds]
    heads = [0] * N
    sizes = np.ones(N, dtype=np.int64)
    for r, s in enumerate(seeds):
        part[s] = r
    active = True
    while active:
        active = False
        for r in range(N):
            if sizes[r] >= max_size or heads[r] >= len(frontiers[r]):
                continue
            v = frontiers[r][heads[r]]
            heads[r] += 1
            nb = _neighbors(A, v)
            nb = nb[part[nb] < 0]
            rng.shuffle(nb)
            for u in nb:
                if sizes[r] >= max_size:
                    break
                if part[u] < 0:
                    part[u] = r
                    sizes[r] += 1
                    frontiers[r].append(int(u))
            active = True
    # leftovers: attach to any claimed neighbour (repeat until none left)
    while (part < 0).any():
        for v in np.flatnonzero(part < 0):
            nb = _neighbors(A, v)
            claimed = nb[part[nb] >= 0]
            if len(claimed):
                part[v] = part[claimed[0]]
    part = _merge_small(A, part, min_size)
    part = _split_large(A, part, max_size)
    # renumber densely
    _, part = np.unique(part, return_inverse=True)
    return part.astype(np.int32)


def _region_adjacency(A: CSR, part: np.ndarray, r: int) -> np.ndarray:
    nodes = np.flatnonzero(part == r)
    nb = np.concatenate([_neighbors(A, v) for v in nodes]) if len(nodes) else np.zeros(0, np.int64)
    other = np.unique(part[nb])
    return other[other != r]


def _merge_small(A: CSR, part: np.ndarray, min_size: int) -> np.ndarray:
    part = part.copy()
    while True:
        labels, counts = np.unique(part, return_counts=True)
        small = labels[counts < min_size]
        if len(small) == 0 or len(labels) == 1:
            return part
        r = int(small[np.argmin(counts[counts < min_size])])
        adj = _region_adjacency(A, part, r)
        if len(adj) == 0:
            return part
        sz = np.array([np.sum(part == a) for a in adj])
        part[part == r] = adj[int(np.argmin(sz))]


def _split_large(A: CSR, part: np.ndarray, max_size: int) -> np.ndarray:
    part = part.copy()
    next_label = int(part.max()) + 1
    changed = True
    while changed:
        changed = False
        labels, counts = np.unique(part, return_counts=True)
        for r, c in zip(labels, counts):
            if c <= max_size:
                continue
            nodes = np.flatnonzero(part == r)
            inside = np.zeros(A.n, dtype=bool)
            inside[nodes] = True
            # farthest node from the first node by BFS inside the region
            far = _bfs_order(A, int(nodes[0]), inside)[-1]
            order = _bfs_order(A, far, inside)
            take = np.array(order[: c // 2], dtype=np.int64)
            part[take] = next_label
            next_label += 1
            changed = True
    return part


def _bfs_order(A: CSR, start: int, inside: np.ndarray) -> list:
    seen = {start}
    order = [start]
    head = 0
    while head < len(order):
        v = order[head]
        head += 1
        for u in _neighbors(A, v):
            u = int(u)
            if inside[u] and u not in seen:
                seen.add(u)
                order.append(u)
    return order


def rhs(n: int, seed: int, nrhs: int = 1) -> np.ndarray:
    """Right-hand side(s) with entries uniform in [-1, 1]; shape (n,) or
    (nrhs, n) (row k is right-hand side k, seed + k)."""
    out = np.empty((nrhs, n))
    for k in range(nrhs):
        rng = np.random.Generator(np.random.PCG64(seed + k))
        out[k] = rng.uniform(-1.0, 1.0, n)
    return out[0] if nrhs == 1 else out


# Named workloads (sizes as stated with the paper's experiments' shapes).
def workload_c1():
    """2D 5-point Laplacian, 64x64 interior nodes (n = 4096), 16 boxes of
    16x16, overlap 1, tau = 50, b uniform[-1, 1] with seed 0."""
    m = 64
    return dict(A=laplace2d(m), part=box_partition_2d(m, 16), N=16, overlap=1, tau=50.0,
                b=rhs(m * m, 0), name="laplace2d_64x64_16box_ov1_tau50")


def workload_diffusion3d(m: int = 32, N: int = 16, lo: int = 1024, hi: int = 4096, overlap: int = 2,
                         tau: float = 100.0, sigma: float = 2.0, corr: float = 8.0, n_channels: int = 16,
                         seed: int = 0):
    """3D 7-point channelled diffusion on an m^3 grid (lognormal coefficient,
    correlation length corr, n_channels one-cell channels of 1e6 along x),
    N seeded BFS subdomains of lo..hi cells, overlap layers, tau, b uniform
    [-1, 1] (seed 0): the shape of the paper-scale diffusion configuration at
    a size one GPU sets up in seconds in both precision forms."""
    A = diffusion3d(m, sigma=sigma, corr=corr, n_channels=n_channels, seed=seed)
    part = bfs_partition(A, N, seed, lo, hi)
    Nn = int(part.max()) + 1
    name = f"diffusion3d_{m}^3_sigma{sigma:g}_ch{n_channels}_bfs{Nn}_{lo}-{hi}_ov{overlap}_tau{tau:g}"
    return dict(A=A, part=part, N=Nn, overlap=overlap, tau=tau, b=rhs(A.n, 0), name=name)
