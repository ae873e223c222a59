"""The multilevel preconditioner of the double-float solves (the DNCP systems
of Section 4.2 and the final Laplace solve of Section 4.5; the preconditioner
is the library's) against the Jacobi-only solve and the oracle.

- Both preconditioners solve every piece to the tolerance and match the
  oracle's sparse direct solve to 1e-8 absolute: the preconditioner changes the
  iteration, never the answer.
- On a mesh with pieces of tens of thousands of vertices the multilevel form
  needs several times fewer iterations.
- Odd shapes: pieces of a few dozen rows, a batch of pieces of very different
  sizes (runs cut at piece ends and every 4096 rows), the sphere (curved
  pieces).
"""
import numpy as np
import pytest

from oracle.dncp import dncp as o_dncp
from oracle.mesh import partition as o_partition
from paper_1903_12359_gb300 import meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1903_12359_gb300 import build
    build.build()
    from paper_1903_12359_gb300 import api as a
    return a


def _local(api, m, precond, closed=False, tol=1e-13):
    ctx = api.Context(variant=2 if closed else 1, precision=0, tol=tol, local_precision=api.DF64_REFINED,
                      local_precond=precond)
    part = ctx.partition(m.V, m.F, face_labels=m.face_labels, closed=closed)
    part.local_param()
    return part.coords(0).cpu().numpy(), part.get_stats()


def _oracle_err(m, u):
    P = o_partition(m.V, m.F, face_labels=m.face_labels)
    voff = np.concatenate([[0], np.cumsum([v.size for v in P.verts])])
    worst = 0.0
    for i in range(P.K):
        ll = np.searchsorted(P.verts[i], P.loops[i])
        ref, _ = o_dncp(m.V[P.verts[i]], P.local_F[i], ll)
        worst = max(worst, float(np.abs(u[voff[i]:voff[i + 1]] - ref).max()))
    return worst


@pytest.mark.parametrize("name", ["polar", "grid4x2_3k", "grid2x2_40k", "sphere", "tiny_pieces"])
def test_both_preconditioners_match_the_direct_solve(api, name):
    closed = False
    if name == "polar":
        m = meshgen.polar_disk_mesh()
    elif name == "grid4x2_3k":
        m = meshgen.heightfield_disk_mesh(3000, seed=3, nx=4, ny=2)
    elif name == "grid2x2_40k":
        m = meshgen.heightfield_disk_mesh(40000, seed=5, nx=2, ny=2)
    elif name == "sphere":
        m, closed = meshgen.icosphere_sh_mesh(subdiv=3, seed=1), True
    else:   # 6 x 4 grid on 600 vertices: pieces of a few dozen rows
        m = meshgen.heightfield_disk_mesh(600, seed=2, nx=6, ny=4)
    iters = {}
    for precond in (0, 1):
        u, st = _local(api, m, precond, closed)
        assert st["dncp_relres"] <= 1e-13, (precond, st["dncp_relres"])
        err = _oracle_err(m, u)
        # forward error <= cond(A~) * relres * |u|: cond is 6e7-1e8 on the
        # 10k-row pieces of grid2x2_40k, so 1e-8 still sits three orders below it
        assert err < 1e-8, (name, precond, err)
        iters[precond] = st["dncp_iters"]
    print(name, "dncp iterations: multilevel", iters[0], "jacobi", iters[1])


def test_multilevel_cuts_the_iterations(api):
    m = meshgen.heightfield_disk_mesh(150000, seed=1, nx=2, ny=2)
    u_ml, st_ml = _local(api, m, 0, tol=1e-10)
    u_j, st_j = _local(api, m, 1, tol=1e-10)
    assert st_ml["dncp_relres"] <= 1e-10 and st_j["dncp_relres"] <= 1e-10
    # both solutions agree to the accuracy the 1e-10 residual allows
    assert np.abs(u_ml - u_j).max() < 1e-6
    print("150k dncp iterations: multilevel", st_ml["dncp_iters"], "jacobi", st_j["dncp_iters"],
          "pcg ms", st_ml["pcg_ms"], st_j["pcg_ms"])
    assert 3 * st_ml["dncp_iters"] <= st_j["dncp_iters"], (st_ml["dncp_iters"], st_j["dncp_iters"])


def test_uneven_batch_pieces(api):
    """Pieces of very different sizes in one batch: every piece converges and
    the maps equal those of the Jacobi solve to the solve's accuracy."""
    ms = [meshgen.uneven_mesh(p) for p in meshgen.uneven_batch_params(n_mesh=6, seed=3, nmin=2000, nmax=30000)]
    out = {}
    for precond in (0, 1):
        ctx = api.Context(variant=1, precision=0, tol=1e-12, local_precision=api.DF64_REFINED, local_precond=precond)
        part = ctx.partition_batch([(m.V, m.F, m.face_labels) for m in ms])
        part.local_param()
        st = part.get_stats()
        assert st["dncp_relres"] <= 1e-12
        out[precond] = part.coords(0).cpu().numpy()
    assert np.abs(out[0] - out[1]).max() < 1e-8


def test_final_laplace_solve_with_the_multilevel_preconditioner(api):
    """The double-float final solve (Section 4.5's Laplace equation with the
    welded boundary) takes the same preconditioner: the same map as the
    Jacobi-only solve within the accuracy its residual allows, the oracle's map
    within the parity bar, and several times fewer iterations."""
    from oracle.pipeline import pgcp as o_pgcp
    m = meshgen.heightfield_disk_mesh(40000, seed=5, nx=2, ny=2)
    out, iters = {}, {}
    for precond in (0, 1):
        ctx = api.Context(variant=api.DISK, precision=api.DF64_REFINED, tol=1e-13,
                          local_precision=api.DF64_REFINED, local_precond=precond)
        part = ctx.partition(m.V, m.F, face_labels=m.face_labels)
        part.local_param()
        part.weld()
        out[precond] = part.global_solve().cpu().numpy()
        st = part.stats
        assert st["final_relres"] <= 1e-13
        iters[precond] = st["final_iters"]
    print("40k final-solve iterations: multilevel", iters[0], "jacobi", iters[1])
    assert np.abs(out[0] - out[1]).max() < 1e-8
    ref = o_pgcp(m.V, m.F, face_labels=m.face_labels, variant="disk").out
    assert np.abs(out[0] - ref).max() < 1e-8
    assert 3 * iters[0] <= iters[1], iters


def test_unreachable_tolerance_fails_after_bounded_work(api):
    """A tolerance below the double-float floor ends in NO_CONVERGENCE after the
    refinement steps, each cut short once it stalls (2,048 iterations without
    halving the residual norm squared), not after max_iters per step."""
    m = meshgen.heightfield_disk_mesh(150000, seed=1, nx=2, ny=2)
    ctx = api.Context(variant=1, precision=0, tol=1e-16, local_precision=api.DF64_REFINED)
    part = ctx.partition(m.V, m.F, face_labels=m.face_labels)
    with pytest.raises(api.PgcpError) as e:
        part.local_param()
    assert e.value.code == "NO_CONVERGENCE"
    st = part.get_stats()
    print("tol 1e-16: dncp iterations", st["dncp_iters"], "relres", st["dncp_relres"])
    assert st["dncp_iters"] < 40000, st["dncp_iters"]
    assert st["dncp_relres"] < 1e-11
