"""The area distortion metric and the Mobius area step (Section 6.2) through
the C ABI, against the oracle (oracle/area.py):
* mean |d_area| equals the oracle's on the same coordinates;
* a planar disk mapped by a known automorphism (or free Mobius map) is mapped
  back: the inverse parameter, d_area ~ 0;
* on pipeline outputs the step takes the oracle's parameter and reaches its
  objective, and maps U as the oracle's formula does;
* a batch gives each mesh its single-mesh result;
* on the sphere (ball automorphisms, chordal areas) the same checks, and a
  variant that does not fit the part is refused.
"""
import numpy as np
import pytest
import torch

from oracle import area as AR
from paper_1903_12359_gb300 import meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1903_12359_gb300 import build
    build.build()
    from paper_1903_12359_gb300 import api as a
    return a


def _solve(api, m, variant):
    ctx = api.Context(variant=variant, precision=api.FP32_REFINED, tol=1e-12)
    part = ctx.partition(m.V, m.F, face_labels=m.face_labels)
    part.local_param()
    part.weld()
    return ctx, part, part.global_solve()


def test_metric_matches_the_oracle(api):
    m = meshgen.heightfield_disk_mesh(20000, seed=31, nx=4, ny=2)
    ctx, part, U = _solve(api, m, api.DISK)
    got = part.area_distortion(U)[0]
    ref = np.abs(AR.area_distortion(m.V, m.F, U.cpu().numpy())).mean()
    assert abs(got - ref) < 1e-12 * max(1.0, ref)
    assert part.area_distortion(U)[0] == got          # fixed-order sums: the same bits


@pytest.mark.parametrize("variant,p0", [("disk", 0.35 + 0.2j), ("free", 0.25 - 0.15j)])
def test_known_map_is_undone(api, variant, p0):
    m = meshgen.polar_disk_mesh(rings=12, sectors=24, seed=1)
    flat = m.V.copy()
    flat[:, 2] = 0.0
    ctx = api.Context(variant=api.DISK)
    part = ctx.partition(flat, m.F, face_labels=m.face_labels)
    w = AR.mobius(variant, p0, flat[:, 0] + 1j * flat[:, 1])
    U = torch.tensor(np.stack([w.real, w.imag], axis=1), device="cuda")
    r = part.area_mobius(U, api.DISK if variant == "disk" else api.FREE)[0]
    assert r["status"] == "OK" and r["before"] > 0.05 and r["after"] < 1e-6, r
    assert abs(r["param"] + p0) < 1e-6
    assert np.abs(U.cpu().numpy() - flat[:, :2]).max() < 1e-5


@pytest.mark.parametrize("variant", ["disk", "free"])
def test_step_matches_the_oracle_on_pipeline_output(api, variant):
    m = meshgen.heightfield_disk_mesh(12000, seed=32, nx=3, ny=2) if variant == "disk" else \
        meshgen.heightfield_disk_mesh(6000, seed=33, nx=2, ny=1)
    ctx, part, U = _solve(api, m, api.DISK if variant == "disk" else api.FREE)
    U0 = U.cpu().numpy()
    r = part.area_mobius(U, api.DISK if variant == "disk" else api.FREE)[0]
    p, before, after, evals, W = AR.area_step(m.V, m.F, U0, variant)
    assert r["status"] == "OK"
    assert abs(r["before"] - before) < 1e-12 * before
    assert abs(r["after"] - after) < 1e-9 * before and r["after"] <= r["before"]
    assert abs(r["param"] - p) < 1e-5, (r["param"], p)
    w = AR.mobius(variant, r["param"], U0[:, 0] + 1j * U0[:, 1])
    assert np.abs(U.cpu().numpy() - np.stack([w.real, w.imag], axis=1)).max() < 1e-12


def test_batch_equals_single_meshes(api):
    ms = [meshgen.heightfield_disk_mesh(3000 + 1500 * i, seed=40 + i, nx=2, ny=2) for i in range(2)]
    singles, Us = [], []
    for x in ms:
        _, p1, U1 = _solve(api, x, api.DISK)
        Us.append(U1.clone())
        singles.append(p1.area_mobius(U1, api.DISK)[0])
    ctx = api.Context(variant=api.DISK, precision=api.FP32_REFINED, tol=1e-12)
    part = ctx.partition_batch([(x.V, x.F, x.face_labels) for x in ms])
    U = torch.cat(Us).contiguous()                 # the same coordinates as the single runs
    rb = part.area_mobius(U, api.DISK)
    for i in range(len(ms)):
        assert rb[i]["param"] == singles[i]["param"] and rb[i]["after"] == singles[i]["after"]


def _sphere_part(api, m):
    ctx = api.Context(variant=api.SPHERE, precision=api.FP32_REFINED, tol=1e-12)
    return ctx, ctx.partition(m.V, m.F, face_labels=m.face_labels, closed=True)


def test_sphere_known_automorphism_is_undone(api):
    m = meshgen.icosphere_sh_mesh(subdiv=3, seed=0, amp=0.0)
    S = m.V / np.linalg.norm(m.V, axis=1, keepdims=True)
    a0 = np.array([0.25, 0.1, -0.3])
    ctx, part = _sphere_part(api, m)
    U = torch.tensor(AR.ball_automorphism(a0, S), device="cuda")
    r = part.area_mobius(U, api.SPHERE)[0]
    assert r["status"] == "OK" and r["before"] > 0.1 and r["after"] < 1e-6, r
    assert np.abs(np.array(r["param3"]) + a0).max() < 1e-5
    Y = U.cpu().numpy()
    idx = np.arange(0, m.nv, 7)
    assert np.abs(Y[idx] @ Y[idx].T - S[idx] @ S[idx].T).max() < 1e-5


def test_sphere_step_matches_the_oracle_and_wrong_variants_are_refused(api):
    m = meshgen.icosphere_sh_mesh(subdiv=4, seed=2)
    ctx, part = _sphere_part(api, m)
    part.local_param()
    part.weld()
    U = part.global_solve()
    U0 = U.cpu().numpy()
    got = part.area_distortion(U)[0]
    assert abs(got - np.abs(AR.sphere_area_distortion(m.V, m.F, U0)).mean()) < 1e-12 * max(1.0, got)
    r = part.area_mobius(U, api.SPHERE)[0]
    a, before, after, evals, Y = AR.area_step(m.V, m.F, U0, "sphere")
    assert r["status"] == "OK" and abs(r["before"] - before) < 1e-12 * before
    assert abs(r["after"] - after) < 1e-9 * before and r["after"] <= r["before"]
    assert np.abs(np.array(r["param3"]) - a).max() < 1e-5, (r["param3"], a)
    assert np.abs(U.cpu().numpy() - AR.ball_automorphism(np.array(r["param3"]), U0)).max() < 1e-12
    assert np.abs(np.linalg.norm(U.cpu().numpy(), axis=1) - 1.0).max() < 1e-13
    with pytest.raises(api.PgcpError) as e:
        part.area_mobius(U, api.DISK)
    assert e.value.code == "ARG"
    d = meshgen.heightfield_disk_mesh(3000, seed=3, nx=2, ny=2)
    _, dp, DU = _solve(api, d, api.DISK)
    with pytest.raises(api.PgcpError) as e:
        dp.area_mobius(DU, api.SPHERE)
    assert e.value.code == "ARG"
