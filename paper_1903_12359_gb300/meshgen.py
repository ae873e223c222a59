"""Seeded synthetic meshes shaped like the dense surfaces PGCP is run on.

This module only builds inputs (vertex coordinates, faces and a face
partition); it contains none of the parameterization arithmetic, so both the
CPU oracle tests and the CUDA path tests can draw from it.

Workloads (all deterministic for a given seed, ``numpy.random.default_rng``):

* ``polar_disk_mesh``: the small disk case -- a centre vertex plus 40 rings x 64
  sectors over the unit disk, radii jittered by +-2 % on the inner rings (at
  most 0.4 ring spacings, so rings never cross), lifted
  by z = 0.3 sin(3x) cos(2y) and cut along the x = 0 diameter (2 subdomains).
* ``heightfield_disk_mesh``: N points (boundary ring on r = 1, rows of points
  along straight cut lines, uniform interior points), Delaunay-triangulated,
  lifted by a sum of 8 Gaussians and cut along the lines into grid cells.
* ``icosphere_sh_mesh``: an icosahedron subdivided ``subdiv`` times, radius
  1 + 0.2 * sum of real spherical harmonics up to degree 6, cut into octants.
* ``uneven_batch``: many height-field disks of log-uniform size, each cut into
  4..32 grid cells of uneven size.

The paper's scanned meshes (Face, Nefertiti, Asian Dragon, ...) are not
available; these generators stand in for them with the same size, topology
(simply-connected open or genus-0 closed) and partition structure.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components


@dataclass
class Mesh:
    """A triangle mesh plus a face partition (labels need not be canonical)."""

    V: np.ndarray            # float64 [nv, 3]
    F: np.ndarray            # int32 [nf, 3], counter-clockwise seen from outside / +z
    face_labels: np.ndarray  # int32 [nf]
    kind: str                # "open" or "closed"
    name: str = ""

    @property
    def nv(self) -> int:
        return int(self.V.shape[0])

    @property
    def nf(self) -> int:
        return int(self.F.shape[0])

    def cut_edges(self) -> np.ndarray:
        return labels_to_cut_edges(self.F, self.face_labels)


# --------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------

def _interior_edge_pairs(F: np.ndarray, nv: int):
    """Return (f0, f1, u, v): the two faces of every interior edge (u < v)."""
    he = np.stack([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]], axis=1).reshape(-1, 2)
    a = np.minimum(he[:, 0], he[:, 1]).astype(np.int64)
    b = np.maximum(he[:, 0], he[:, 1]).astype(np.int64)
    key = a * nv + b
    order = np.argsort(key, kind="stable")
    ks = key[order]
    same = ks[1:] == ks[:-1]
    i0 = order[:-1][same]
    i1 = order[1:][same]
    return i0 // 3, i1 // 3, a[i0], b[i0]


def labels_to_cut_edges(F: np.ndarray, labels: np.ndarray) -> np.ndarray:
    """Cut-edge list (int32 [n, 2], u < v) separating faces of different labels."""
    nv = int(F.max()) + 1
    f0, f1, u, v = _interior_edge_pairs(F, nv)
    diff = labels[f0] != labels[f1]
    return np.stack([u[diff], v[diff]], axis=1).astype(np.int32)


def _morton_keys(P: np.ndarray, bits: int = 20) -> np.ndarray:
    lo = P.min(axis=0)
    span = np.maximum(P.max(axis=0) - lo, 1e-300)
    q = ((P - lo) / span * ((1 << bits) - 1)).astype(np.uint64)
    key = np.zeros(P.shape[0], dtype=np.uint64)
    d = P.shape[1]
    for bit in range(bits):
        for c in range(d):
            key |= ((q[:, c] >> np.uint64(bit)) & np.uint64(1)) << np.uint64(bit * d + c)
    return key


def _reorder_spatially(V: np.ndarray, F: np.ndarray, P: np.ndarray):
    """Renumber vertices by Morton order of P and sort faces by their vertices.

    Scanned meshes are stored with spatial locality; random point clouds are
    not, so the generators restore it (the numbering itself carries no meaning
    for the method).
    """
    perm = np.argsort(_morton_keys(P), kind="stable")
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    V2 = V[perm]
    F2 = inv[F]
    fk = np.sort(F2, axis=1)
    forder = np.lexsort((fk[:, 2], fk[:, 1], fk[:, 0]))
    return V2, F2[forder].astype(np.int32), forder


def _orient_ccw_xy(P2: np.ndarray, F: np.ndarray) -> np.ndarray:
    a, b, c = P2[F[:, 0]], P2[F[:, 1]], P2[F[:, 2]]
    area = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    F = F.copy()
    neg = area < 0
    F[neg] = F[neg][:, [0, 2, 1]]
    return F


def _region_boundary_degree(F: np.ndarray, labels: np.ndarray, nv: int):
    """Per (vertex, label): number of region-boundary edges incident to it."""
    he = np.stack([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]], axis=1).reshape(-1, 2)
    hf = np.repeat(np.arange(F.shape[0]), 3)
    a = np.minimum(he[:, 0], he[:, 1]).astype(np.int64)
    b = np.maximum(he[:, 0], he[:, 1]).astype(np.int64)
    lab = labels[hf].astype(np.int64)
    L = int(labels.max()) + 1
    key = (a * nv + b) * L + lab
    uk, cnt = np.unique(key, return_counts=True)
    bnd = uk[cnt == 1]
    lab_b = bnd % L
    e = bnd // L
    u = e // nv
    v = e % nv
    vk = np.concatenate([u * L + lab_b, v * L + lab_b])
    vks, vcnt = np.unique(vk, return_counts=True)
    return vks // L, vks % L, vcnt


def repair_labels(F: np.ndarray, labels: np.ndarray, max_rounds: int = 50) -> np.ndarray:
    """Make every label region one connected, pinch-free, simply-connected piece.

    Faces of minor connected components are given the label of a neighbouring
    face; faces at a pinch vertex (a vertex with more than two region-boundary
    edges of one label) are moved to the neighbouring label.  Input-generation
    step only.
    """
    labels = labels.astype(np.int32).copy()
    nf = F.shape[0]
    nv = int(F.max()) + 1
    f0, f1, _, _ = _interior_edge_pairs(F, nv)
    for _ in range(max_rounds):
        changed = False
        same = labels[f0] == labels[f1]
        g = coo_matrix((np.ones(int(same.sum())), (f0[same], f1[same])), shape=(nf, nf))
        ncomp, comp = connected_components(g, directed=False)
        if ncomp > labels.max() + 1:
            # keep the largest component of every label
            sizes = np.bincount(comp, minlength=ncomp)
            comp_label = np.zeros(ncomp, dtype=np.int64)
            comp_label[comp] = labels
            best = {}
            for c in np.argsort(-sizes, kind="stable"):
                best.setdefault(int(comp_label[c]), int(c))
            keep = np.zeros(ncomp, dtype=bool)
            keep[list(best.values())] = True
            bad = ~keep[comp]
            # relabel bad faces from a neighbour in a kept component
            for _inner in range(1000):
                if not bad.any():
                    break
                m0 = bad[f0] & ~bad[f1]
                m1 = bad[f1] & ~bad[f0]
                tgt = np.concatenate([f0[m0], f1[m1]])
                src = np.concatenate([f1[m0], f0[m1]])
                if tgt.size == 0:
                    break
                labels[tgt] = labels[src]
                bad[tgt] = False
            changed = True
        vtx, lab, deg = _region_boundary_degree(F, labels, nv)
        pinch = deg > 2
        if pinch.any():
            pv = set(zip(vtx[pinch].tolist(), lab[pinch].tolist()))
            # move one face of the pinched region at each pinch vertex
            moved = 0
            vf = {}
            for c in range(3):
                for fi in np.nonzero(np.isin(F[:, c], vtx[pinch]))[0]:
                    vf.setdefault(int(F[fi, c]), []).append(int(fi))
            for (v, l) in sorted(pv):
                faces = [fi for fi in vf.get(v, []) if labels[fi] == l]
                for fi in faces:
                    # neighbours of fi with a different label
                    others = np.concatenate([f1[f0 == fi], f0[f1 == fi]])
                    others = others[labels[others] != l]
                    if others.size:
                        labels[fi] = labels[others[0]]
                        moved += 1
                        break
            if moved:
                changed = True
        if not changed:
            return labels
    raise RuntimeError("label repair did not converge")


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def polar_disk_mesh(rings: int = 40, sectors: int = 64, jitter: float = 0.02, seed: int = 0) -> Mesh:
    """Small disk case: polar grid over the unit disk, 2 pieces split at x = 0."""
    rng = np.random.default_rng(seed)
    nv = 1 + rings * sectors
    V = np.zeros((nv, 3))
    ang = 2.0 * np.pi * np.arange(sectors) / sectors
    for i in range(1, rings + 1):
        r = np.full(sectors, i / rings)
        if i < rings:
            # multiplicative jitter, capped at 0.4 ring spacings so that
            # neighbouring rings never cross (the planar grid stays embedded)
            dr = r * rng.uniform(-jitter, jitter, size=sectors)
            r = r + np.clip(dr, -0.4 / rings, 0.4 / rings)
        idx = 1 + (i - 1) * sectors + np.arange(sectors)
        V[idx, 0] = r * np.cos(ang)
        V[idx, 1] = r * np.sin(ang)

    def vid(i, j):
        return 0 if i == 0 else 1 + (i - 1) * sectors + (j % sectors)

    faces = []
    for j in range(sectors):
        faces.append((0, vid(1, j), vid(1, j + 1)))
    for i in range(1, rings):
        for j in range(sectors):
            a, b = vid(i, j), vid(i, j + 1)
            c, d = vid(i + 1, j + 1), vid(i + 1, j)
            faces.append((a, d, c))   # split along (i,j)-(i+1,j+1)
            faces.append((a, c, b))
    F = np.array(faces, dtype=np.int32)
    if np.any(F != _orient_ccw_xy(V[:, :2], F)):
        raise RuntimeError("polar grid folded")
    V[:, 2] = 0.3 * np.sin(3.0 * V[:, 0]) * np.cos(2.0 * V[:, 1])
    cx = V[F, 0].mean(axis=1)
    labels = (cx < 0).astype(np.int32)
    return Mesh(V, F, labels, "open", f"polar_disk_{rings}x{sectors}_s{seed}")


def _gaussian_bumps(rng, P2: np.ndarray, n: int = 8) -> np.ndarray:
    a = rng.uniform(0.05, 0.3, size=n)
    s = rng.uniform(0.1, 0.4, size=n)
    rr = np.sqrt(rng.uniform(0, 1, size=n))
    tt = rng.uniform(0, 2 * np.pi, size=n)
    c = np.stack([rr * np.cos(tt), rr * np.sin(tt)], axis=1)
    z = np.zeros(P2.shape[0])
    for i in range(n):
        d2 = ((P2 - c[i]) ** 2).sum(axis=1)
        z += a[i] * np.exp(-d2 / (2.0 * s[i] ** 2))
    return z


def _line_points(c: float, h: float, vertical: bool, cross: np.ndarray):
    """Vertex row along the cut line x = c (or y = c) inside the unit disk.

    Points at spacing ~h between the two circle crossings (the crossings
    themselves are boundary points), plus the grid crossings in ``cross``.
    """
    half = math.sqrt(max(1.0 - c * c, 0.0))
    n = max(int(math.ceil(2.0 * half / h)), 2)
    t = np.linspace(-half, half, n + 1)[1:-1]
    t = np.union1d(t, cross[(cross > -half) & (cross < half)])
    # drop row points too close to a crossing (keeps the spacing >= h/2)
    keep = np.ones(t.size, dtype=bool)
    for x in cross:
        near = (np.abs(t - x) < 0.5 * h) & (t != x)
        keep &= ~near
    t = t[keep]
    if vertical:
        return np.stack([np.full(t.size, c), t], axis=1)
    return np.stack([t, np.full(t.size, c)], axis=1)


def heightfield_disk_mesh(N: int, seed: int = 0, nx: int = 4, ny: int = 2, uneven: bool = False,
                          min_share: float = 0.1) -> Mesh:
    """Delaunay height field over the unit disk, cut along a grid of straight lines.

    n_b = round(2 sqrt(pi N)) points on r = 1 (angle jitter +-1/4 spacing, plus
    the points where cut lines meet the circle), a row of points at spacing
    h = sqrt(pi / N) along every cut line, and uniform random points in
    r <= 1 - h/2 outside a band of half-width h/2 around each cut line (so the
    Delaunay triangulation keeps every row segment as an edge and the cuts are
    straight vertex paths).  Height: a sum of 8 Gaussians.  Cut lines sit at
    equal (or, with ``uneven``, random sorted) fractions of [-0.9, 0.9] in x
    (nx - 1 lines) and y (ny - 1 lines); the pieces are the grid cells.
    """
    from scipy.spatial import Delaunay

    rng = np.random.default_rng(seed)
    h = math.sqrt(math.pi / N)

    def cuts(n):
        if n <= 1:
            return np.zeros(0)
        if not uneven:
            return -0.9 + 1.8 * np.arange(1, n) / n
        while True:
            q = np.sort(rng.uniform(0, 1, size=n - 1))
            sh = np.diff(np.concatenate([[0.0], q, [1.0]]))
            if sh.min() >= min_share:
                return -0.9 + 1.8 * q

    cx, cy = cuts(nx), cuts(ny)
    nb = int(round(2.0 * math.sqrt(math.pi * N)))
    t = (np.arange(nb) + rng.uniform(-0.25, 0.25, size=nb)) * (2 * np.pi / nb)
    # circle crossings of the cut lines become boundary points
    extra = []
    for c in cx:
        a = math.acos(c)
        extra += [a, -a]
    for c in cy:
        a = math.asin(c)
        extra += [a, math.pi - a]
    if extra:
        extra = np.mod(np.array(extra), 2 * np.pi)
        d = np.abs(np.angle(np.exp(1j * (t[:, None] - extra[None, :]))))
        t = t[d.min(axis=1) > 0.5 * (2 * np.pi / nb)]
        t = np.concatenate([t, extra])
    B = np.stack([np.cos(t), np.sin(t)], axis=1)
    rows = [_line_points(c, h, True, cy) for c in cx] + [_line_points(c, h, False, cx) for c in cy]
    R = np.concatenate(rows, axis=0) if rows else np.zeros((0, 2))
    if R.size:
        R = np.unique(np.round(R, 15), axis=0)
    ni = max(N - B.shape[0] - R.shape[0], 0)
    pts = []
    while sum(p.shape[0] for p in pts) < ni:
        m = 2 * (ni - sum(p.shape[0] for p in pts)) + 16
        r = (1.0 - 0.5 * h) * np.sqrt(rng.uniform(0, 1, size=m))
        th = rng.uniform(0, 2 * np.pi, size=m)
        P = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
        ok = np.ones(m, dtype=bool)
        for c in cx:
            ok &= np.abs(P[:, 0] - c) >= 0.5 * h
        for c in cy:
            ok &= np.abs(P[:, 1] - c) >= 0.5 * h
        pts.append(P[ok])
    I = np.concatenate(pts, axis=0)[:ni] if ni else np.zeros((0, 2))
    P2 = np.concatenate([B, R, I], axis=0)
    tri = Delaunay(P2)
    F = _orient_ccw_xy(P2, tri.simplices.astype(np.int32))
    z = _gaussian_bumps(rng, P2)
    V = np.concatenate([P2, z[:, None]], axis=1)
    V, F, _ = _reorder_spatially(V, F, P2)
    c = V[F, :2].mean(axis=1)
    lab = np.searchsorted(cx, c[:, 0]) + nx * np.searchsorted(cy, c[:, 1])
    labels = validate_pieces(F, repair_labels(F, _compact_labels(lab.astype(np.int32))))
    return Mesh(V, F, labels, "open", f"heightfield_N{N}_{nx}x{ny}_s{seed}")


def _piece_ok(F: np.ndarray, faces: np.ndarray) -> bool:
    """One piece is a topological disk: one boundary loop, no pinch, V - E + F = 1."""
    Fi = F[faces]
    he = np.stack([Fi[:, [0, 1]], Fi[:, [1, 2]], Fi[:, [2, 0]]], axis=1).reshape(-1, 2).astype(np.int64)
    a, b = np.minimum(he[:, 0], he[:, 1]), np.maximum(he[:, 0], he[:, 1])
    nv = int(Fi.max()) + 1
    key = a * nv + b
    uk, inv, cnt = np.unique(key, return_inverse=True, return_counts=True)
    bnd = he[cnt[inv] == 1]
    if bnd.shape[0] == 0 or np.unique(bnd[:, 0]).size != bnd.shape[0]:
        return False
    nxt = dict(zip(bnd[:, 0].tolist(), bnd[:, 1].tolist()))
    start = bnd[0, 0]
    v, n = nxt[start], 1
    while v != start and n <= len(nxt):
        v = nxt.get(v, start)
        n += 1
    if n != len(nxt):
        return False
    return np.unique(Fi).size - uk.size + Fi.shape[0] == 1


def validate_pieces(F: np.ndarray, labels: np.ndarray, max_rounds: int = 64) -> np.ndarray:
    """Merge every piece that is not a topological disk into the neighbour it
    shares most edges with (input-generation step; guards against rare
    triangulations where a cut row is crossed)."""
    labels = _compact_labels(labels)
    nv = int(F.max()) + 1
    f0, f1, _, _ = _interior_edge_pairs(F, nv)
    for _ in range(max_rounds):
        bad = [L for L in range(int(labels.max()) + 1) if not _piece_ok(F, np.nonzero(labels == L)[0])]
        if not bad:
            return labels
        L = bad[0]
        m0 = (labels[f0] == L) & (labels[f1] != L)
        m1 = (labels[f1] == L) & (labels[f0] != L)
        nb = np.concatenate([labels[f1[m0]], labels[f0[m1]]])
        if nb.size == 0:
            raise RuntimeError("isolated piece")
        labels[labels == L] = np.bincount(nb).argmax()
        labels = repair_labels(F, _compact_labels(labels))
    raise RuntimeError("piece validation did not converge")


def _compact_labels(lab: np.ndarray) -> np.ndarray:
    _, inv = np.unique(lab, return_inverse=True)
    return inv.astype(np.int32)


def _icosahedron():
    p = (1.0 + math.sqrt(5.0)) / 2.0
    V = np.array([[-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
                  [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
                  [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1]], dtype=np.float64)
    F = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    return V / np.linalg.norm(V, axis=1, keepdims=True), F


def _subdivide(V, F):
    nv = V.shape[0]
    e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]], axis=0)
    a = np.minimum(e[:, 0], e[:, 1])
    b = np.maximum(e[:, 0], e[:, 1])
    key = a * nv + b
    uk, inv = np.unique(key, return_inverse=True)
    ua, ub = uk // nv, uk % nv
    M = 0.5 * (V[ua] + V[ub])
    M /= np.linalg.norm(M, axis=1, keepdims=True)
    nf = F.shape[0]
    m01 = nv + inv[:nf]
    m12 = nv + inv[nf:2 * nf]
    m20 = nv + inv[2 * nf:]
    v0, v1, v2 = F[:, 0], F[:, 1], F[:, 2]
    F2 = np.concatenate([np.stack([v0, m01, m20], 1), np.stack([v1, m12, m01], 1),
                         np.stack([v2, m20, m12], 1), np.stack([m01, m12, m20], 1)], axis=0)
    return np.concatenate([V, M], axis=0), F2


def real_sph_harm(l: int, m: int, theta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Real orthonormal spherical harmonic (theta polar angle, phi azimuth)."""
    from scipy.special import lpmv
    am = abs(m)
    norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
    P = lpmv(am, l, np.cos(theta))
    if m == 0:
        return norm * P
    if m > 0:
        return math.sqrt(2.0) * norm * P * np.cos(m * phi)
    return math.sqrt(2.0) * norm * P * np.sin(am * phi)


def icosphere_sh_mesh(subdiv: int = 8, seed: int = 0, lmax: int = 6, amp: float = 0.2) -> Mesh:
    """Genus-0 closed surface: deformed icosphere cut into the 8 octants."""
    V, F = _icosahedron()
    for _ in range(subdiv):
        V, F = _subdivide(V, F)
    theta = np.arccos(np.clip(V[:, 2], -1.0, 1.0))
    phi = np.arctan2(V[:, 1], V[:, 0])
    s = seed
    while True:
        rng = np.random.default_rng(s)
        r = np.ones(V.shape[0])
        for l in range(lmax + 1):
            for m in range(-l, l + 1):
                r += amp * rng.normal() / (l + 1) ** 2 * real_sph_harm(l, m, theta, phi)
        if r.min() >= 0.2:
            break
        s += 10007
    U = V * r[:, None]
    U, F, _ = _reorder_spatially(U, F.astype(np.int32), V)
    Vs = U / np.linalg.norm(U, axis=1, keepdims=True)
    c = Vs[F].mean(axis=1)
    lab = (c[:, 0] < 0).astype(np.int32) + 2 * (c[:, 1] < 0) + 4 * (c[:, 2] < 0)
    labels = validate_pieces(F, repair_labels(F, lab.astype(np.int32)))
    return Mesh(U, F, labels, "closed", f"icosphere_sd{subdiv}_s{seed}")


def uneven_batch_params(n_mesh: int = 256, seed: int = 0, nmin: int = 5000, nmax: int = 200000,
                        kmin: int = 4, kmax: int = 32) -> list:
    """(N, nx, ny, mesh seed) of each mesh of ``uneven_batch``, without meshing.

    Each mesh draws N log-uniform in [nmin, nmax] and K ~ U{kmin..kmax}, and is
    cut by an nx x ny grid (nx = ceil(sqrt K), ny = ceil(K / nx)) of straight
    lines at random positions (cells outside the disk vanish).
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_mesh):
        N = int(math.floor(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        K = int(rng.integers(kmin, kmax + 1))
        nx = int(math.ceil(math.sqrt(K)))
        ny = int(math.ceil(K / nx))
        out.append((N, nx, ny, seed * 100003 + i))
    return out


def uneven_mesh(params) -> Mesh:
    """One mesh of ``uneven_batch`` from its ``uneven_batch_params`` entry."""
    N, nx, ny, s = params
    return heightfield_disk_mesh(N, seed=s, nx=nx, ny=ny, uneven=True)


def uneven_batch(n_mesh: int = 256, seed: int = 0, nmin: int = 5000, nmax: int = 200000,
                 kmin: int = 4, kmax: int = 32) -> list:
    """Many height-field disks, log-uniform sizes, 4..32 pieces of uneven size."""
    return [uneven_mesh(p) for p in uneven_batch_params(n_mesh, seed, nmin, nmax, kmin, kmax)]


def he_normal(seed: int, shapes) -> np.ndarray:
    """Seeded initial parameters: N(0, 2 / fan_in) for matrices (rows = inputs),
    zeros for vectors, concatenated in order (float64)."""
    rng = np.random.default_rng(seed)
    parts = []
    for shp in shapes:
        if len(shp) == 2:
            parts.append(rng.normal(0.0, math.sqrt(2.0 / shp[0]), size=shp).reshape(-1))
        else:
            parts.append(np.zeros(shp))
    return np.concatenate(parts)
