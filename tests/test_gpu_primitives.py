"""Device primitives at partition scale (6M corners of a 1M-vertex mesh):
stable radix sort and exclusive scan against numpy, through the C ABI."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1903_12359_gb300 import build
    build.build()
    from paper_1903_12359_gb300 import api
    return api.Context()


@pytest.mark.parametrize("n,bits", [(1000, 8), (5000, 23), (6_000_000, 23), (3_000_000, 64), (777_777, 3)])
def test_radix_sort_stable(ctx, n, bits):
    rng = np.random.default_rng(n + bits)
    hi = (1 << bits) if bits < 64 else (1 << 63)
    keys = rng.integers(0, min(hi, 1 << 62), size=n, dtype=np.int64).astype(np.uint64)
    if bits < 64:
        keys %= np.uint64(1 << bits)
    vals = np.arange(n, dtype=np.int32)
    kd = torch.as_tensor(keys.view(np.int64), device="cuda")
    vd = torch.as_tensor(vals, device="cuda")
    ctx.selftest_sort(kd, vd, bits)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(kd.cpu().numpy().view(np.uint64), keys[order])
    assert np.array_equal(vd.cpu().numpy(), vals[order])


@pytest.mark.parametrize("n", [1, 2047, 2048, 2049, 5_000_000, 6_000_001])
def test_exclusive_scan(ctx, n):
    rng = np.random.default_rng(n)
    x = rng.integers(0, 5, size=n, dtype=np.int32)
    out, tot = ctx.selftest_scan(torch.as_tensor(x, device="cuda"))
    ref = np.concatenate([[0], np.cumsum(x.astype(np.int64))[:-1]])
    assert np.array_equal(out.cpu().numpy(), ref) and tot == int(x.sum())
