"""The allocation-free comparison entry point (gs_compare_noalloc) gives the
same records as gs_compare, on two calls in a row through the C ABI.

It exists for callers that may not allocate device memory while running
(flight/embedded renderers with a no-allocation rule after start-up, or a
process whose allocator owns all of HBM); its scratch is a fixed array inside
the library, reused by every call, so the second call checks that each call
starts from cleared accumulators.  This file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _pairs(seed, K, H, W):
    rng = np.random.default_rng(seed)
    a = rng.uniform(-0.1, 1.1, size=(K, H, W, 3)).astype(np.float32)
    b = a + (rng.normal(0, 0.02, size=a.shape) * (rng.uniform(size=a.shape) < 0.4)).astype(np.float32)
    a[0, 1, 2, 0] = np.nan
    return a, b


def test_noalloc_compare_matches_compare_twice():
    import torch
    import paper_2606_21791_gb300 as P
    P.build()
    from paper_2606_21791_gb300 import gs as G
    G.load_library()
    for call, (seed, K, H, W) in enumerate([(11, 3, 70, 93), (12, 5, 48, 64)]):
        a, b = _pairs(seed, K, H, W)
        da = torch.from_numpy(a.reshape(-1).copy()).cuda()
        db = torch.from_numpy(b.reshape(-1).copy()).cuda()
        ref = G.device_bytes(K * 24)
        out = G.device_bytes(K * 24)
        G.gs_compare(da, db, H, W, K, ref)
        G.gs_compare_noalloc(da, db, H, W, K, out)
        torch.cuda.synchronize()
        r = G.from_device(ref, G.RESULT_DTYPE)
        o = G.from_device(out, G.RESULT_DTYPE)
        assert np.array_equal(o["footprint"], r["footprint"]), call
        assert np.array_equal(o["nonfinite"], r["nonfinite"]), call
        assert np.array_equal(o["maxabs"], r["maxabs"]), call
        assert np.all(np.abs(o["sse"] - r["sse"]) <= 1e-6 * r["sse"] + 1e-9), call
        assert o["nonfinite"][0] == 1 and (o["footprint"] > 0).all()
    with pytest.raises(G.GsError) as e:
        G.gs_compare_noalloc(da, db, H, W, 65, out)
    assert e.value.status == G.GS_ERR_ARG
