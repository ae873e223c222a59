"""pgcp_metrics_noalloc (fixed static device scratch, no allocation) against
pgcp_metrics on the same part and coordinates, two calls in a row each.

Order statistics, max, flips and max |mu| must agree bit for bit; mean and sd
come from atomic sums in a different order, so 1e-12 relative.  The file name
puts it last in collection so that it also runs after every other GPU test.
"""
import numpy as np
import pytest
import torch

from paper_1903_12359_gb300 import meshgen

pytestmark = pytest.mark.gpu

EXACT = ("median", "iqr", "max", "n_corners", "flips", "max_mu")
CLOSE = ("mean", "sd")


@pytest.fixture(scope="module")
def api():
    from paper_1903_12359_gb300 import build
    build.build()
    from paper_1903_12359_gb300 import api as a
    return a


def _solved(api, m, variant):
    ctx = api.Context(variant=variant, precision=0, tol=1e-12)
    part = ctx.partition(m.V, m.F, face_labels=m.face_labels, closed=(variant == 2))
    part.local_param()
    part.weld()
    out = part.global_solve()
    return ctx, part, out


def _compare(ref, got):
    for k in EXACT:
        assert got[k] == ref[k], (k, got[k], ref[k])
    for k in CLOSE:
        assert abs(got[k] - ref[k]) <= 1e-12 * max(abs(ref[k]), 1.0), (k, got[k], ref[k])


@pytest.mark.parametrize("kind", ["disk", "sphere"])
def test_noalloc_metrics_equal_pooled_metrics_twice(api, kind):
    if kind == "disk":
        m, variant = meshgen.heightfield_disk_mesh(3000, seed=3, nx=4, ny=2), 1
    else:
        m, variant = meshgen.icosphere_sh_mesh(subdiv=3, seed=1), 2
    ctx, part, out = _solved(api, m, variant)
    ref = part.metrics(out)
    a0 = api.alloc_count()
    first = part.metrics_noalloc(out)
    second = part.metrics_noalloc(out)
    # the library's own counter of device allocations does not move
    assert api.alloc_count() == a0
    _compare(ref, first)
    _compare(ref, second)
    assert ref["n_corners"] == 3 * m.nf


def test_noalloc_metrics_several_tiles_and_perturbed_input(api):
    """A part spanning many radix-sort tiles; the second call gets different
    coordinates, so stale scratch from the first would show."""
    m = meshgen.heightfield_disk_mesh(40000, seed=5, nx=4, ny=2)
    ctx, part, out = _solved(api, m, 1)
    g = torch.Generator(device="cpu").manual_seed(7)
    noisy = out + 1e-3 * torch.randn(out.shape, generator=g, dtype=torch.float64).to(out.device)
    for U in (out, noisy):
        _compare(part.metrics(U), part.metrics_noalloc(U))


def test_noalloc_metrics_rejects_parts_over_the_limit(api):
    m = meshgen.heightfield_disk_mesh(140000, seed=2, nx=2, ny=2)
    assert m.nf > api.METRICS_NOALLOC_MAX_FACES
    ctx = api.Context(variant=1)
    part = ctx.partition(m.V, m.F, face_labels=m.face_labels)
    U = torch.zeros((m.nv, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(api.PgcpError) as e:
        part.metrics_noalloc(U)
    assert e.value.code == "ARG"
    assert str(api.METRICS_NOALLOC_MAX_FACES) in str(e.value)
    # the library stays usable after the refusal
    small = meshgen.polar_disk_mesh(rings=6, sectors=16)
    ctx2, p2, o2 = _solved(api, small, 1)
    _compare(p2.metrics(o2), p2.metrics_noalloc(o2))
