"""The PGCP pipeline, Algorithm 3 (test infrastructure).

partition (Sec. 4.1) -> DNCP per piece, translated to the local frame (Sec. 4.2)
-> partial welds one piece at a time (Alg. 1, Alg. 2, Fig. 7) -> optional disk
(geodesic algorithm on the global boundary, Sec. 4.4.1) or sphere (closed weld
of the last piece, Sec. 4.4.2) -> Laplace solve per piece with the welded
boundary (Sec. 4.5) -> gather (lowest label wins) -> stereographic projection
for the sphere.

Readings (listed in full in the design notes; the CUDA library follows them):
* auxiliary points of a weld of B onto A: a_{m+1} and b_{n+1} are the
  components' reference points (0 for a single DNCP piece, -1 -- the value
  the normalisation gives A's reference -- for a welded component),
  a_{m+2} = b_{n+2} = inf;
* welds run by levels of disjoint pairs (see mesh.weld_schedule);
* the final normalisation takes the midpoint of a~_{m+2} and b~_{n+2}
  (the paper's "a~_{n+2}" is read as b~_{n+2});
* the closed weld of a sphere normalises with p1 = a~_{m+1} -> 0,
  p2 = b~_{n+1} -> inf, a~_{floor(k/2)} -> 1; the pieces of its B component
  are then held in the chart w = 1/z; the projection (2x, -2y, |z|^2 - 1)/(1 + |z|^2), i.e.
  (2 Re w, 2 Im w, 1 - |w|^2)/(1 + |w|^2) in that chart, keeps orientation.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.sparse.linalg import spsolve

from .common import OracleError
from .dncp import dncp
from .laplacian import cotan_laplacian
from .mesh import partition, weld_schedule
from . import welding as W


@dataclass
class Result:
    part: object
    welds: list
    L: list = field(default_factory=list)         # per piece CSR (PSD cotan)
    local: list = field(default_factory=list)     # per piece DNCP coords (complex, local frame)
    ref: list = field(default_factory=list)       # per piece reference vertex (local id)
    weld_chains: list = field(default_factory=list)  # per weld: (A_chain, B_chain)
    welded: list = field(default_factory=list)    # per piece: complex coords after welds (+disk)
    welded_inf: list = field(default_factory=list)
    disk_chain: list = None
    final: list = field(default_factory=list)     # per piece coords after the Laplace solve
    out: np.ndarray = None                        # gathered [nv, 2] or [nv, 3]
    sphere_w_pieces: list = field(default_factory=list)   # pieces held in the w = 1/z chart
    seam_mismatch: float = 0.0


def _weld_phase1(res: Result, wd, sphere_close: bool):
    """Algorithms 1-2 on the weld's sequence points (read from the current
    boundary coordinates of its pieces): the two chains and the final images
    of the arc points on each side."""
    P = res.part
    k = wd.k
    members = wd.members
    b_members = wd.b_members

    def loop_coords(pieces, ids):
        # each loop point from the copy in the lowest-label piece of the side holding it
        pos = {}
        for pc in pieces:
            for li, g in enumerate(P.verts[pc].tolist()):
                pos.setdefault(g, (pc, li))
        re_ = np.empty(ids.size)
        im_ = np.empty(ids.size)
        for j, g in enumerate(ids.tolist()):
            pc, li = pos[g]
            re_[j] = res.welded[pc].real[li]
            im_[j] = res.welded[pc].imag[li]
        return re_, im_

    a_re, a_im = loop_coords(members, wd.a)
    b_re, b_im = loop_coords(b_members, wd.b)
    # reference points: 0 in a single piece's DNCP frame, -1 (where the
    # normalisation sends A's reference) for a welded component
    ref_A = 0.0 if wd.a_single else -1.0
    ref_B = 0.0 if wd.b_single else -1.0
    Aarc = W.Pts(a_re[:k + 1], a_im[:k + 1])
    Barc = W.Pts(b_re[:k + 1], b_im[:k + 1])
    gA, Aimg = W.intermediate_form(Aarc, k, +1.0)
    gB, Bimg = W.intermediate_form(Barc, k, -1.0)
    hs, X, Y = W.weld_maps(Aimg, Bimg, k)
    # auxiliary points through each side's chain
    auxA = W.apply_chain(gA + hs, W.Pts([ref_A, 0.0], [0.0, 0.0], [False, True]))
    auxB = W.apply_chain(gB + hs, W.Pts([ref_B, 0.0], [0.0, 0.0], [False, True]))
    if auxA.inf.any() or auxB.inf.any():
        raise OracleError("NUMERIC", "auxiliary point mapped to infinity")
    p1 = complex(auxA.re[0], auxA.im[0])
    p2 = complex(auxB.re[0], auxB.im[0])
    if sphere_close:
        q = complex(X.re[k // 2], X.im[k // 2])
        TA = W.rec_sphere_frame(p1, p2, q, invert=False)
        TB = W.rec_sphere_frame(p1, p2, q, invert=True)
    else:
        p3 = complex((auxA.re[1] + auxB.re[1]) * 0.5, (auxA.im[1] + auxB.im[1]) * 0.5)
        TA = TB = W.rec_normalize(p1, p2, p3)
    arc_A = W.apply_rec(TA, X)      # final images of the arc points (C side)
    arc_B = W.apply_rec(TB, Y)      # same points in B's chart (sphere) / same values
    chainA = gA + hs + [TA]
    chainB = gB + hs + [TB]
    res.weld_chains.append((chainA, chainB))
    return chainA, chainB, arc_A, arc_B


def _weld_phase2(res: Result, wd, ph1, map_interior: bool, pieces=None):
    """The weld's chains applied to the points of its pieces (all, or those
    in ``pieces``); the arc points take their phase-1 images."""
    P = res.part
    k = wd.k
    chainA, chainB, arc_A, arc_B = ph1
    arc_pos = {g: j for j, g in enumerate(wd.a[:k + 1].tolist())}
    # apply to every point of every involved piece
    for pc, chain, arc in [(pc, chainA, arc_A) for pc in wd.members] + [(pc, chainB, arc_B) for pc in wd.b_members]:
        if pieces is not None and pc not in pieces:
            continue
        g_ids = P.verts[pc]
        on_loop = np.zeros(g_ids.size, dtype=bool)
        gl = {g: li for li, g in enumerate(g_ids.tolist())}
        for g in P.loops[pc].tolist():
            on_loop[gl[g]] = True
        sel = on_loop if not map_interior else np.ones(g_ids.size, dtype=bool)
        arc_here = np.array([g in arc_pos for g in g_ids.tolist()])
        todo = np.nonzero(sel & ~arc_here)[0]
        cur = W.Pts(res.welded[pc].real[todo], res.welded[pc].imag[todo], res.welded_inf[pc][todo])
        new = W.apply_chain(chain, cur)
        zr = res.welded[pc].real.copy()
        zi = res.welded[pc].imag.copy()
        zinf = res.welded_inf[pc].copy()
        zr[todo], zi[todo], zinf[todo] = new.re, new.im, new.inf
        for li in np.nonzero(arc_here)[0]:
            j = arc_pos[int(g_ids[li])]
            zr[li], zi[li], zinf[li] = arc.re[j], arc.im[j], arc.inf[j]
        if not map_interior:
            # interior points are not needed (only boundary coordinates are kept)
            zr[~on_loop] = np.nan
            zi[~on_loop] = np.nan
        res.welded[pc] = zr + 1j * zi
        res.welded_inf[pc] = zinf


def _weld_once(res: Result, wd, map_interior: bool, sphere_close: bool):
    _weld_phase2(res, wd, _weld_phase1(res, wd, sphere_close), map_interior)
    return res


def _disk_phase1(res: Result):
    """The geodesic algorithm on the global boundary loop: its chain and the
    images of the loop points."""
    P = res.part
    # global boundary loop = C's loop after all welds (or the single piece's loop)
    C_loop = res.welds[-1].new_loop if res.welds else P.loops[0]
    pos = {}
    for pc in range(P.K):
        for li, g in enumerate(P.verts[pc].tolist()):
            pos.setdefault(g, (pc, li))
    zr = np.array([res.welded[pos[g][0]].real[pos[g][1]] for g in C_loop.tolist()])
    zi = np.array([res.welded[pos[g][0]].imag[pos[g][1]] for g in C_loop.tolist()])
    # C's reference point: -1 after any weld (the normalisation sends it there),
    # 0 for a single piece (its DNCP frame)
    cref = -1.0 if res.welds else 0.0
    chain, img = W.geodesic_disk(W.Pts(zr, zi), W.Pts([cref], [0.0]))
    res.disk_chain = chain
    return chain, img, C_loop


def _disk_phase2(res: Result, ph1, map_interior: bool, pieces=None):
    """The disk chain applied to the points of the pieces (all, or those in
    ``pieces``); the global boundary points take their phase-1 images."""
    P = res.part
    chain, img, C_loop = ph1
    bpos = {g: j for j, g in enumerate(C_loop.tolist())}
    for pc in range(P.K):
        if pieces is not None and pc not in pieces:
            continue
        g_ids = P.verts[pc]
        gl = {g: li for li, g in enumerate(g_ids.tolist())}
        on_loop = np.zeros(g_ids.size, dtype=bool)
        for g in P.loops[pc].tolist():
            on_loop[gl[g]] = True
        sel = on_loop if not map_interior else np.ones(g_ids.size, dtype=bool)
        isb = np.array([g in bpos for g in g_ids.tolist()])
        todo = np.nonzero(sel & ~isb)[0]
        cur = W.Pts(res.welded[pc].real[todo], res.welded[pc].imag[todo])
        new = W.apply_chain(chain, cur)
        z = res.welded[pc].copy()
        z[todo] = new.complex()
        for li in np.nonzero(isb)[0]:
            j = bpos[int(g_ids[li])]
            z[li] = complex(img.re[j], img.im[j])
        res.welded[pc] = z


def _disk_step(res: Result, map_interior: bool):
    _disk_phase2(res, _disk_phase1(res), map_interior)


def harmonic_solve(L, loop_local: np.ndarray, ub: np.ndarray) -> np.ndarray:
    """Laplace equation with Dirichlet boundary (Sec. 4.5): L_II u_I = -L_IB u_B."""
    n = L.shape[0]
    isb = np.zeros(n, dtype=bool)
    isb[loop_local] = True
    I = np.nonzero(~isb)[0]
    B = loop_local
    u = np.zeros(n, dtype=np.complex128)
    u[B] = ub
    if I.size:
        LII = L[I][:, I].tocsc()
        LIB = L[I][:, B]
        rx = -(LIB @ ub.real)
        ry = -(LIB @ ub.imag)
        u[I] = spsolve(LII, rx) + 1j * spsolve(LII, ry)
    return u


def stereo_from_plane(z: np.ndarray) -> np.ndarray:
    """Inverse stereographic projection of the z chart, orientation-preserving
    (counter-clockwise in the plane is counter-clockwise seen from outside):
    (2x, -2y, |z|^2 - 1) / (1 + |z|^2)."""
    x, y = z.real, z.imag
    r2 = x * x + y * y
    d = 1.0 + r2
    return np.stack([2.0 * x / d, -2.0 * y / d, (r2 - 1.0) / d], axis=1)


def stereo_from_inverted(w: np.ndarray) -> np.ndarray:
    """Same sphere point from the chart w = 1/z: (2 Re w, 2 Im w, 1 - |w|^2)/(1 + |w|^2)."""
    x, y = w.real, w.imag
    r2 = x * x + y * y
    d = 1.0 + r2
    return np.stack([2.0 * x / d, 2.0 * y / d, (1.0 - r2) / d], axis=1)


def _local_piece(args):
    """Cotangent Laplacian and DNCP map of one piece (a pool task)."""
    X, Fl, ll = args
    L = cotan_laplacian(X, Fl)
    u, ref = dncp(X, Fl, ll, L)
    return L, u, ref


def _final_piece(args):
    """Laplace solve of one piece with its welded boundary (a pool task)."""
    L, ll, ub = args
    return harmonic_solve(L, ll, ub)


def pgcp(V, F, cut_edges=None, face_labels=None, variant: str = "disk",
         map_interior: bool = False, local=None, workers: int = 1) -> Result:
    """Run Algorithm 3.  ``variant`` is "free", "disk" or "sphere".

    ``local`` (tests only): per-piece complex coordinates to use instead of the
    DNCP solve, so the welding can be compared on identical inputs.
    ``workers`` > 1: the per-piece DNCP and Laplace solves run in a pool of that
    many spawned processes, one piece per task -- the parallel scheme of the
    paper's experiments (one subdomain per parallel worker, Section 5.6).  The
    arithmetic of every piece is the same as with workers = 1.
    """
    V = np.asarray(V, dtype=np.float64)
    P = partition(V, F, cut_edges=cut_edges, face_labels=face_labels)
    welds = weld_schedule(P, closed_surface=(variant == "sphere"))
    res = Result(part=P, welds=welds)
    pool = None
    if workers > 1 and P.K > 1:
        import multiprocessing as mp
        pool = mp.get_context("spawn").Pool(min(workers, P.K))
    try:
        return _pgcp_stages(res, V, P, welds, variant, map_interior, local, pool)
    finally:
        if pool is not None:
            pool.close()
            pool.join()


def _pgcp_stages(res, V, P, welds, variant, map_interior, local, pool):
    loop_local = [np.searchsorted(P.verts[i], P.loops[i]) for i in range(P.K)]
    if local is None:
        tasks = [(V[P.verts[i]], P.local_F[i], loop_local[i]) for i in range(P.K)]
        solved = pool.map(_local_piece, tasks, chunksize=1) if pool is not None else [_local_piece(t) for t in tasks]
    for i in range(P.K):
        ll = loop_local[i]
        if local is None:
            L, u, ref = solved[i]
        else:
            L = cotan_laplacian(V[P.verts[i]], P.local_F[i])
            u, ref = np.asarray(local[i], dtype=np.complex128), -1
        res.L.append(L)
        res.local.append(u)
        res.ref.append(ref)
        res.welded.append(u.copy())
        res.welded_inf.append(np.zeros(u.size, dtype=bool))
    for wd in welds:
        _weld_once(res, wd, map_interior, sphere_close=wd.closed)
    if variant == "sphere":
        res.sphere_w_pieces = list(welds[-1].b_members)
    if variant == "disk":
        _disk_step(res, map_interior)
    # final Laplace solves with the welded boundary
    tasks = []
    for i in range(P.K):
        ub = res.welded[i][loop_local[i]]
        if np.any(res.welded_inf[i][loop_local[i]]) or not np.all(np.isfinite(ub)):
            raise OracleError("NUMERIC", f"piece {i}: non-finite welded boundary")
        tasks.append((res.L[i], loop_local[i], ub))
    res.final = pool.map(_final_piece, tasks, chunksize=1) if pool is not None else [_final_piece(t) for t in tasks]
    # gather: lowest label wins
    nv = V.shape[0]
    if variant == "sphere":
        out = np.full((nv, 3), np.nan)
    else:
        out = np.full((nv, 2), np.nan)
    mism = 0.0
    for i in range(P.K):
        g = P.verts[i]
        if variant == "sphere":
            xyz = stereo_from_inverted(res.final[i]) if i in res.sphere_w_pieces else stereo_from_plane(res.final[i])
            have = ~np.isnan(out[g, 0])
            if have.any():
                mism = max(mism, float(np.abs(out[g[have]] - xyz[have]).max()))
            out[g[~have]] = xyz[~have]
        else:
            xy = np.stack([res.final[i].real, res.final[i].imag], axis=1)
            have = ~np.isnan(out[g, 0])
            if have.any():
                mism = max(mism, float(np.abs(out[g[have]] - xy[have]).max()))
            out[g[~have]] = xy[~have]
    res.out = out
    res.seam_mismatch = mism
    return res
