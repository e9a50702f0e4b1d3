"""Autotuning on the GPU: the tensor-core product's tile width (stbem_tc_tune)
is timed once per shape, recorded in the tune cache and its file, and taken
from there afterwards; products with the tuned width stay within the
tensor-core bound against the oracle."""
import numpy as np
import pytest

from oracle import solve as OS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1811_05224_gb300 as P
    return P.Context(0)


def test_tc_tune_records_and_reuses(ctx, tmp_path):
    import paper_1811_05224_gb300 as P
    rng = np.random.default_rng(3)
    nt, nx, B = 300, 64, 2
    A = torch.as_tensor(rng.standard_normal((nt, nx, nx))).cuda()
    x = torch.as_tensor(rng.standard_normal((B, nt, nx))).cuda()
    Ab, xb = P.to_bf16(ctx, A), P.to_bf16(ctx, x)
    f = tmp_path / "tune.txt"
    try:
        P.tune_cache(f)
        P.tune_cache_clear()
        tn, cached = P.tc_tune(ctx, Ab, xb)
        assert tn in (128, 256) and not cached
        assert ("|tc_plain|nt=%d|nx=%d|rhs=%d\tbn=%d" % (nt, nx, B, tn)) in f.read_text()
        assert P.tc_tune(ctx, Ab, xb) == (tn, True)
        # a fresh table reloaded from the file
        P.tune_cache_clear()
        P.tune_cache(f)
        assert P.tc_tune(ctx, Ab, xb) == (tn, True)
        y = P.apply_tc(ctx, Ab, xb).cpu().numpy()
        A64, x64 = Ab.double().cpu().numpy(), xb.double().cpu().numpy()
        for b in range(B):
            ref = OS.toeplitz_apply(A64, x64[b])
            mag = OS.toeplitz_apply(np.abs(A64), np.abs(x64[b]))
            steps = nt * ((nx + 63) // 64)
            assert np.all(np.abs(y[b] - ref) <= 16 * steps * 2.0 ** -24 * mag + 1e-30)
        # one step tile: only the 128-wide tile is a candidate
        tn1, _ = P.tc_tune(ctx, Ab[:100].contiguous(), xb[:, :100].contiguous())
        assert tn1 == 128
    finally:
        P.tune_cache(None)
        P.tune_cache_clear()
