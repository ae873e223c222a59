"""Pins for the oracle's partition, boundary loops and weld order (Section 4.1).

Checked against a hand-derived 9-vertex case, properties (i)-(iv), a brute
force component search and the disk-topology errors.
"""
import json
import os

import numpy as np
import pytest

from oracle import OracleError
from oracle.mesh import partition, weld_schedule
from paper_1903_12359_gb300 import meshgen

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_hand_derived_grid():
    g = json.load(open(os.path.join(GOLD, "grid3x3_cut.json")))
    P = partition(g["V"], g["F"], cut_edges=g["cut_edges"])
    assert P.K == g["expected_K"]
    assert P.face_label.tolist() == g["expected_face_label"]
    assert [v.tolist() for v in P.verts] == g["expected_verts"]
    assert [l.tolist() for l in P.loops] == g["expected_loops"]
    ws = weld_schedule(P, closed_surface=False)
    assert len(ws) == 1
    w, e = ws[0], g["expected_welds"][0]
    assert (w.piece, w.k) == (e["piece"], e["k"])
    assert w.a.tolist() == e["a"] and w.b.tolist() == e["b"]
    assert w.new_loop.tolist() == e["new_loop"]


def _brute_components(F, cut):
    """Flood fill over faces sharing a non-cut edge (pure Python, tiny meshes)."""
    nf = len(F)
    edges = {}
    for f, t in enumerate(F):
        for c in range(3):
            u, v = int(t[c]), int(t[(c + 1) % 3])
            edges.setdefault((min(u, v), max(u, v)), []).append(f)
    cutset = {(min(u, v), max(u, v)) for u, v in cut}
    adj = [[] for _ in range(nf)]
    for e, fs in edges.items():
        if len(fs) == 2 and e not in cutset:
            adj[fs[0]].append(fs[1])
            adj[fs[1]].append(fs[0])
    label = [-1] * nf
    k = 0
    for f in range(nf):          # ascending face id: labels are canonical
        if label[f] >= 0:
            continue
        stack = [f]
        label[f] = k
        while stack:
            x = stack.pop()
            for y in adj[x]:
                if label[y] < 0:
                    label[y] = k
                    stack.append(y)
        k += 1
    return np.array(label)


@pytest.mark.parametrize("nx,ny,seed", [(2, 2, 0), (3, 1, 1), (2, 3, 2)])
def test_partition_properties(nx, ny, seed):
    m = meshgen.heightfield_disk_mesh(600, seed=seed, nx=nx, ny=ny)
    cut = m.cut_edges()
    P = partition(m.V, m.F, cut_edges=cut)
    # brute force components, canonical labels
    assert np.array_equal(P.face_label, _brute_components(m.F, cut))
    # (i) union of vertex sets, (ii) union of face sets, (iv) disjoint faces
    assert np.array_equal(np.unique(np.concatenate(P.verts)), np.arange(m.nv))
    allf = np.concatenate(P.faces)
    assert allf.size == m.nf and np.array_equal(np.sort(allf), np.arange(m.nf))
    # (iii) V_i cap V_j lies on both boundaries
    for i in range(P.K):
        for j in range(i + 1, P.K):
            common = set(P.verts[i].tolist()) & set(P.verts[j].tolist())
            assert common <= set(P.loops[i].tolist()) & set(P.loops[j].tolist())
    # loops: ccw (positive area in the xy plane for these height fields), start at min id
    for i in range(P.K):
        lp = P.loops[i]
        assert lp[0] == lp.min() and np.unique(lp).size == lp.size
        x, y = m.V[lp, 0], m.V[lp, 1]
        assert 0.5 * np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y) > 0


def test_face_labels_equal_cut_edges():
    m = meshgen.polar_disk_mesh()
    a = partition(m.V, m.F, cut_edges=m.cut_edges())
    b = partition(m.V, m.F, face_labels=m.face_labels)
    assert np.array_equal(a.face_label, b.face_label)
    assert a.K == 2 and [v.size for v in a.verts] == [1321, 1321]


def test_errors():
    g = json.load(open(os.path.join(GOLD, "grid3x3_cut.json")))
    V, F = np.array(g["V"]), np.array(g["F"])
    with pytest.raises(OracleError) as e:
        partition(V, F, cut_edges=[[0, 8]])
    assert e.value.code == "ARG"
    bad = F.copy()
    bad[0] = bad[0][[0, 2, 1]]
    with pytest.raises(OracleError) as e:
        partition(V, bad)
    assert e.value.code == "ARG"
    nm = np.concatenate([F, [[0, 1, 8]]])
    with pytest.raises(OracleError) as e:
        partition(np.concatenate([V, [[5, 5, 5]]]), nm[:, :], cut_edges=None)
    assert e.value.code in ("NONMANIFOLD", "ARG")
    # a piece that is an annulus is not a disk
    m = meshgen.polar_disk_mesh(rings=4, sectors=8)
    lab = np.zeros(m.nf, dtype=np.int32)
    lab[:8] = 1                      # the centre fan is its own piece
    with pytest.raises(OracleError) as e:
        partition(m.V, m.F, face_labels=lab)
    assert e.value.code == "TOPOLOGY"


def test_weld_schedule_grid_and_sphere():
    m = meshgen.heightfield_disk_mesh(3000, seed=3, nx=4, ny=2)
    P = partition(m.V, m.F, face_labels=m.face_labels)
    ws = weld_schedule(P, closed_surface=False)
    assert len(ws) == P.K - 1
    for w in ws:
        assert w.k >= 2 and np.array_equal(w.a[:w.k + 1], w.b[:w.k + 1])
    s = meshgen.icosphere_sh_mesh(subdiv=3, seed=0)
    P = partition(s.V, s.F, face_labels=s.face_labels)
    ws = weld_schedule(P, closed_surface=True)
    assert len(ws) == 7 and ws[-1].closed and not any(w.closed for w in ws[:-1])
