"""Surface partition, boundary loops and the welding order (test infrastructure).

Section 4.1 (surface partition): faces are joined when they share an edge that
is neither a cut edge nor a boundary edge; the connected components of that
face graph are the submeshes S_i = (V_i, F_i) with properties (i)-(iv).

Readings where the paper is silent (the same in the CUDA library):
* component label = rank of the component's smallest face id;
* V_i lists the vertices of F_i in ascending global id, F_i the faces in
  ascending global id;
* a boundary loop runs u -> v as the edge appears in its face's cyclic order
  (counter-clockwise, interior on the left) and starts at its smallest global id;
* every piece must be a topological disk: V - E + F = 1, one boundary loop,
  two boundary edges at every boundary vertex.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

from .common import OracleError


@dataclass
class Partition:
    nv: int
    nf: int
    K: int
    face_label: np.ndarray             # int32 [nf], canonical labels 0..K-1
    faces: list = field(default_factory=list)   # per piece: ascending global face ids
    verts: list = field(default_factory=list)   # per piece: ascending global vertex ids
    loops: list = field(default_factory=list)   # per piece: global ids, ccw, canonical start
    local_F: list = field(default_factory=list)  # per piece: int [nf_i, 3] local vertex ids


def _half_edges(F: np.ndarray):
    he = np.stack([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]], axis=1).reshape(-1, 2).astype(np.int64)
    hf = np.repeat(np.arange(F.shape[0], dtype=np.int64), 3)
    return he, hf


def partition(V: np.ndarray, F: np.ndarray, cut_edges=None, face_labels=None) -> Partition:
    """Partition (V, F) along the cut-edge set (Section 4.1).

    ``cut_edges``: int [n, 2] undirected edges; or ``face_labels``: int [nf],
    where every edge between faces of different labels is a cut edge.
    """
    V = np.asarray(V, dtype=np.float64)
    F = np.asarray(F, dtype=np.int64)
    nv, nf = V.shape[0], F.shape[0]
    if F.ndim != 2 or F.shape[1] != 3 or nf == 0:
        raise OracleError("ARG", "faces must be [nf, 3], nf > 0")
    if F.min() < 0 or F.max() >= nv:
        raise OracleError("ARG", "face index out of range")
    if np.any(F[:, 0] == F[:, 1]) or np.any(F[:, 1] == F[:, 2]) or np.any(F[:, 0] == F[:, 2]):
        raise OracleError("ARG", "face with a repeated vertex")
    he, hf = _half_edges(F)
    a = np.minimum(he[:, 0], he[:, 1])
    b = np.maximum(he[:, 0], he[:, 1])
    key = a * nv + b
    uk, inv, cnt = np.unique(key, return_inverse=True, return_counts=True)
    if cnt.max() > 2:
        raise OracleError("NONMANIFOLD", "an edge is shared by more than two faces")
    # the two half-edges of an interior edge must run in opposite directions
    order = np.argsort(inv, kind="stable")
    inv_s = inv[order]
    pair = inv_s[1:] == inv_s[:-1]
    h0 = order[:-1][pair]
    h1 = order[1:][pair]
    if np.any(he[h0, 0] == he[h1, 0]):
        raise OracleError("ARG", "faces are not consistently oriented")
    f0, f1 = hf[h0], hf[h1]
    # which interior edges are cut
    if face_labels is not None:
        fl = np.asarray(face_labels)
        if fl.shape[0] != nf:
            raise OracleError("ARG", "face_labels must have nf entries")
        is_cut = fl[f0] != fl[f1]
    else:
        is_cut = np.zeros(f0.shape[0], dtype=bool)
        if cut_edges is not None and len(cut_edges):
            ce = np.asarray(cut_edges, dtype=np.int64).reshape(-1, 2)
            ck = np.minimum(ce[:, 0], ce[:, 1]) * nv + np.maximum(ce[:, 0], ce[:, 1])
            pos = np.searchsorted(uk, ck)
            ok = (pos < uk.size)
            ok[ok] = uk[pos[ok]] == ck[ok]
            if not np.all(ok):
                raise OracleError("ARG", "a cut edge is not an edge of the mesh")
            cut_ids = np.zeros(uk.size, dtype=bool)
            cut_ids[pos] = True
            is_cut = cut_ids[inv[h0]]
    keep = ~is_cut
    g = coo_matrix((np.ones(int(keep.sum())), (f0[keep], f1[keep])), shape=(nf, nf))
    ncomp, comp = connected_components(g, directed=False)
    # canonical label = rank of the component's smallest face id
    first_face = np.full(ncomp, nf, dtype=np.int64)
    np.minimum.at(first_face, comp, np.arange(nf))
    rank = np.empty(ncomp, dtype=np.int64)
    rank[np.argsort(first_face, kind="stable")] = np.arange(ncomp)
    label = rank[comp].astype(np.int32)
    K = int(ncomp)
    P = Partition(nv=nv, nf=nf, K=K, face_label=label)
    for i in range(K):
        fi = np.nonzero(label == i)[0]
        vi = np.unique(F[fi].ravel())
        Fl = np.searchsorted(vi, F[fi])
        P.faces.append(fi)
        P.verts.append(vi)
        P.local_F.append(Fl)
        P.loops.append(_piece_loop(F[fi], vi, i))
    return P


def _piece_loop(Fi: np.ndarray, vi: np.ndarray, piece: int) -> np.ndarray:
    """Boundary loop of one piece; checks the disk topology (Section 4.1)."""
    nf_i = Fi.shape[0]
    he, _ = _half_edges(Fi)
    a = np.minimum(he[:, 0], he[:, 1])
    b = np.maximum(he[:, 0], he[:, 1])
    nvv = int(max(vi.max(), Fi.max())) + 1
    key = a * nvv + b
    uk, inv, cnt = np.unique(key, return_inverse=True, return_counts=True)
    bnd = cnt[inv] == 1
    bu, bv = he[bnd, 0], he[bnd, 1]
    E = uk.size
    chi = vi.size - E + nf_i
    if bu.size == 0:
        raise OracleError("TOPOLOGY", f"piece {piece} has no boundary (not a disk)")
    nxt = {}
    for u, v in zip(bu.tolist(), bv.tolist()):
        if u in nxt:
            raise OracleError("TOPOLOGY", f"piece {piece} is pinched at vertex {u}")
        nxt[u] = v
    if len(set(bv.tolist())) != bv.size:
        raise OracleError("TOPOLOGY", f"piece {piece} is pinched")
    start = min(nxt)
    loop = [start]
    v = nxt[start]
    while v != start:
        loop.append(v)
        if len(loop) > len(nxt):
            raise OracleError("TOPOLOGY", f"piece {piece}: broken boundary loop")
        v = nxt[v]
    if len(loop) != len(nxt):
        raise OracleError("TOPOLOGY", f"piece {piece} has more than one boundary loop")
    if chi != 1:
        raise OracleError("TOPOLOGY", f"piece {piece} has Euler characteristic {chi}, not 1")
    return np.array(loop, dtype=np.int64)


# --------------------------------------------------------------------------
# welding order (Figure 7 caption: pieces are welded one at a time)
# --------------------------------------------------------------------------

@dataclass
class Weld:
    piece: int              # lowest label of B, the component joined to A
    a: np.ndarray           # A's loop rotated so a[0..k] is the shared arc (global ids)
    b: np.ndarray           # B's loop reversed, rotated so b[j] == a[j] for j <= k
    k: int                  # number of shared edges
    closed: bool            # the whole loop is shared (closed welding, Section 4.4.2)
    members: list           # pieces of A (ascending)
    new_loop: np.ndarray    # loop of A u B after this weld (ccw, canonical start)
    b_members: list = field(default_factory=list)   # pieces of B (ascending)
    a_single: bool = True   # A is one unwelded piece (its reference point is 0, else -1)
    b_single: bool = True
    level: int = 0          # welds of one level join disjoint components


@dataclass
class _Comp:
    members: list
    loop: np.ndarray
    single: bool


def _rotate_canonical(loop: np.ndarray) -> np.ndarray:
    i = int(np.argmin(loop))
    return np.concatenate([loop[i:], loop[:i]])


def _pair_weld(A: _Comp, B: _Comp, closed_final: bool):
    """The weld of B onto A, or None unless their loops share exactly one
    contiguous arc of >= 2 edges and touch nowhere else (A u B is then a
    disk); on a closed surface the final two components share the whole loop."""
    A_loop, B_loop = A.loop, B.loop
    b_edges = set(zip(B_loop.tolist(), np.roll(B_loop, -1).tolist()))
    m1 = A_loop.size
    nxt = np.roll(A_loop, -1)
    shared = np.array([(int(v), int(u)) in b_edges for u, v in zip(A_loop, nxt)])
    if not shared.any():
        return None
    rb = B_loop[::-1]

    def plan(a, b, k, closed, new_loop):
        return Weld(piece=B.members[0], a=a, b=b, k=k, closed=closed, members=list(A.members), new_loop=new_loop,
                    b_members=list(B.members), a_single=A.single, b_single=B.single)

    if shared.all():
        if not (closed_final and B_loop.size == m1):
            return None
        a = A_loop.copy()
        j = int(np.nonzero(rb == a[0])[0][0])
        b = np.concatenate([rb[j:], rb[:j]])
        if not np.array_equal(a, b):
            return None
        return plan(a, b, m1 - 1, True, np.zeros(0, dtype=np.int64))
    starts = np.nonzero(shared & ~np.roll(shared, 1))[0]
    if starts.size != 1:
        return None
    i0 = int(starts[0])
    rs = np.roll(shared, -i0)
    k = int(np.argmin(rs))
    if k < 2:
        return None
    a = np.concatenate([A_loop[i0:], A_loop[:i0]])
    if set(A_loop.tolist()) & set(B_loop.tolist()) != set(a[:k + 1].tolist()):
        return None
    j = int(np.nonzero(rb == a[0])[0][0])
    b = np.concatenate([rb[j:], rb[:j]])
    if not np.array_equal(a[:k + 1], b[:k + 1]):
        return None
    new_loop = _rotate_canonical(np.concatenate([a[k:], a[:1], b[k + 1:][::-1]]))
    return plan(a, b, k, False, new_loop)


def weld_schedule(P: Partition, closed_surface: bool) -> list:
    """Order of the partial welds, by levels.

    Reading: the paper welds one piece at a time onto a growing component
    (Fig. 7), but Algorithm 2 joins any two disks that share one boundary arc.
    Sequential welding composes K elementary chains on the first piece's
    boundary, and with 16-36 pieces the crowding of that boundary makes the
    FP64 zipper lose the order of the arc.  Here components are instead paired
    level by level, so a piece's boundary passes through about log2 K welds:
    * the components start as the pieces, ordered by lowest label;
    * in each level, every unpaired component, in that order, is paired with
      the first later unpaired component that shares ONE contiguous arc of >= 2
      edges of its loop and touches it nowhere else, so the union stays a disk;
      the earlier component is A, the later one B;
    * the welds of a level join disjoint components;
    * on a closed surface the last two components share their whole loops and
      are joined by a closed weld.
    """
    K = P.K
    if K == 1:
        return []
    comps = [_Comp([i], P.loops[i].copy(), True) for i in range(K)]
    welds = []
    level = 0
    while len(comps) > 1:
        final2 = closed_surface and len(comps) == 2
        used = [False] * len(comps)
        merged = []
        for i in range(len(comps)):
            if used[i]:
                continue
            for j in range(i + 1, len(comps)):
                if used[j]:
                    continue
                w = _pair_weld(comps[i], comps[j], final2)
                if w is None:
                    continue
                w.level = level
                welds.append(w)
                used[i] = used[j] = True
                merged.append(_Comp(sorted(comps[i].members + comps[j].members), w.new_loop, False))
                break
        if not merged:
            raise OracleError("SCHEDULE", "no two components share one contiguous arc")
        comps = sorted(merged + [c for c, u in zip(comps, used) if not u], key=lambda c: c.members[0])
        level += 1
    if closed_surface and not welds[-1].closed:
        raise OracleError("SCHEDULE", "closed surface did not end with a closed weld")
    return welds
