"""The learned warm start on the GPU (BF16 tensor-core network, C ABI) against
the FP64 oracle network (oracle/mpnn.py): features, prediction, gradients;
then training and its use in the final solve, where the plain method verifies
every prediction (fallback per piece)."""
import numpy as np
import pytest
import torch
from scipy.sparse import csr_matrix

from oracle import mpnn as om
from paper_1903_12359_gb300 import meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1903_12359_gb300 import build
    build.build()
    from paper_1903_12359_gb300 import api as a
    return a


def _solved_part(api, m, warm=1, gnn=None, interior_fp64=0):
    ctx = api.Context(variant=api.DISK, precision=0, tol=1e-12, warm_start=warm, interior_map_fp64=interior_fp64)
    if gnn is not None:
        ctx.set_gnn(gnn)
    part = ctx.partition(m.V, m.F, face_labels=m.face_labels)
    part.local_param()
    part.weld()
    out = part.global_solve()
    return ctx, part, out


def _oracle_graph(m):
    """The oracle's own pipeline on the mesh (Algorithm 3 with the interior
    mapped through the welding chains): block-diagonal cotan Laplacian of the
    pieces, boundary flags, row offsets of the pieces and the weld map u_w of
    every vertex copy, all computed by the oracle."""
    from scipy.sparse import block_diag
    from oracle.pipeline import pgcp as o_pgcp
    ref = o_pgcp(m.V, m.F, face_labels=m.face_labels, variant="disk", map_interior=True)
    P = ref.part
    L = block_diag(ref.L).tocsr()
    voff = np.concatenate([[0], np.cumsum([v.size for v in P.verts])])
    is_bnd = np.zeros(voff[-1], dtype=bool)
    for i in range(P.K):
        is_bnd[voff[i] + np.searchsorted(P.verts[i], P.loops[i])] = True
    c = np.concatenate(ref.welded)
    return L, is_bnd, voff, np.column_stack([c.real, c.imag])


def _bf16(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def _theta_as_gpu_uses(theta):
    """Matrices rounded to bf16 (the tensor cores read bf16), biases FP32."""
    out = theta.astype(np.float32).astype(np.float64)
    o = 0
    for shp in om.param_shapes():
        k = int(np.prod(shp))
        if len(shp) == 2:
            out[o:o + k] = _bf16(out[o:o + k])
        o += k
    return out


@pytest.fixture(scope="module")
def case(api):
    m = meshgen.heightfield_disk_mesh(3000, seed=3, nx=4, ny=2)
    # FP64 interior weld map on the GPU, as in the oracle
    ctx, part, out = _solved_part(api, m, interior_fp64=1)
    L, is_bnd, voff, uw = _oracle_graph(m)
    gv = part.partition_arrays()[1].cpu().numpy()
    assert np.array_equal(gv, voff)              # the same pieces, rows in the same order
    return dict(m=m, ctx=ctx, part=part, L=L, is_bnd=is_bnd, voff=voff, uw=uw)


def test_parameter_count(api):
    assert api.num_gnn_params() == om.n_params() == 35152
    assert sum(int(np.prod(s)) for s in api.GNN_PARAM_SHAPES) == 35152


def test_features_match_oracle(api, case):
    feat, tgt, sig = api.gnn_inputs(case["part"])
    feat, sig = feat.cpu().numpy(), sig.cpu().numpy()
    voff, L, is_bnd, uw = case["voff"], case["L"], case["is_bnd"], case["uw"]
    for i in range(voff.size - 1):
        a, b = voff[i], voff[i + 1]
        F, s = om.features(L[a:b, a:b], is_bnd[a:b], uw[a:b])
        assert abs(sig[i] - s) <= 1e-5 * s
        assert np.all(np.abs(feat[a:b] - F) <= 2.0 ** -8 * np.abs(F) + 1e-6)


def test_prediction_and_gradient_match_oracle(api, case):
    theta = 0.5 * meshgen.he_normal(11, om.param_shapes())
    theta[-16:] = 0.05
    gnn = api.Gnn(case["ctx"], theta)
    part = case["part"]
    feat, tgt, sig = api.gnn_inputs(part)
    F = feat.cpu().numpy().astype(np.float64)          # the bf16 values the network sees
    T = tgt.cpu().numpy().astype(np.float64)
    P = om.aggregation(case["L"])
    inner = ~case["is_bnd"]
    th = _theta_as_gpu_uses(theta)
    # prediction: u_w + sigma * out
    x0 = gnn.predict(part).cpu().numpy()
    out = om.forward(th, F, P)
    s_row = np.repeat(sig.cpu().numpy(), np.diff(case["voff"]))
    ref = case["uw"].copy()
    ref[inner] += s_row[inner, None] * out[inner, 0:2]
    corr = np.abs(ref[inner] - case["uw"][inner]).max()
    assert np.abs(x0[inner] - ref[inner]).max() <= 5e-2 * corr
    # boundary rows keep the welded values (GPU FP64 welds of the GPU DNCP map
    # against the oracle's welds of its direct solve)
    assert np.abs(x0[~inner] - case["uw"][~inner]).max() < 1e-9
    # gradient: per parameter block, relative L2 error of the BF16 network
    g, loss = gnn.grad(part)
    go = om.gradient(th, F, P, T, inner)
    lo = om.loss(th, F, P, T, inner)
    assert abs(loss - lo) <= 2e-2 * lo
    o = 0
    for shp in om.param_shapes():
        k = int(np.prod(shp))
        a, b = g[o:o + k].astype(np.float64), go[o:o + k]
        assert np.linalg.norm(a - b) <= 5e-2 * np.linalg.norm(b) + 1e-12, (shp, np.linalg.norm(a - b), np.linalg.norm(b))
        o += k
    cos = float(g.astype(np.float64) @ go / (np.linalg.norm(g) * np.linalg.norm(go)))
    assert cos > 0.999


def test_training_lowers_the_loss_and_learned_start_is_verified(api, case):
    theta = meshgen.he_normal(12, om.param_shapes())
    gnn = api.Gnn(case["ctx"], theta)
    part = case["part"]
    l0 = gnn.train_step(part, 1e-3)
    for _ in range(60):
        l1 = gnn.train_step(part, 1e-3)
    assert l1 < 0.5 * l0
    # the final solve from the learned start reaches the same map
    ctx2, part2, out2 = _solved_part(api, case["m"], warm=api.WARM_LEARNED, gnn=gnn)
    ref = _solved_part(api, case["m"])[2]
    assert torch.allclose(out2, ref, atol=1e-9, rtol=0)
    assert 0 <= part2.stats["learned_pieces"] <= part2.info()["K"]


def test_bad_network_falls_back_to_the_weld_map(api, case):
    theta = 1e3 * meshgen.he_normal(13, om.param_shapes())
    gnn = api.Gnn(case["ctx"], theta)
    ctx2, part2, out2 = _solved_part(api, case["m"], warm=api.WARM_LEARNED, gnn=gnn)
    assert part2.stats["learned_pieces"] == 0
    ref = _solved_part(api, case["m"])[2]
    assert torch.allclose(out2, ref, atol=1e-9, rtol=0)


def test_learned_start_without_network_is_an_argument_error(api, case):
    ctx = api.Context(variant=api.DISK, precision=0, tol=1e-12, warm_start=api.WARM_LEARNED)
    part = ctx.partition(case["m"].V, case["m"].F, face_labels=case["m"].face_labels)
    part.local_param()
    part.weld()
    with pytest.raises(api.PgcpError) as e:
        part.global_solve()
    assert e.value.code == "ARG"
