"""Time-sharded chi^2 on the GPU: one rank (no process group) equals the
whole-observation chi^2, and the per-rank chunks of a two-rank split,
evaluated one after the other, add up to it."""
import numpy as np
import pytest

import oracle
import rime_synth
from gpu_cases import TOL, gpu_ctx, make_case, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_sharded_chi2_matches_whole(precision):
    import paper_1501_07719_gb300 as R
    from paper_1501_07719_gb300 import shard
    inp = make_case(rime_synth.custom(12, 9, 4, 5, 3, seed_index=82), precision)
    prec = R.RIME_FP64 if precision == "f64" else R.RIME_FP32
    r = gpu_ctx(inp, precision)
    whole = r.chi2()
    r.close()
    assert shard.sharded_chi2(inp, prec) == pytest.approx(whole, rel=1e-12)
    parts = 0.0
    for rank in range(2):
        t0, t1 = shard.time_chunk(inp["ntime"], rank, 2)
        sl = shard.slice_observation(inp, t0, t1)
        rs = gpu_ctx(sl, precision)
        parts += rs.chi2()
        rs.close()
    assert rel_err(parts, whole) <= 1e-12
    assert rel_err(whole, oracle.Problem(inp, data=inp["data"]).chi2()) <= TOL[precision]["chi2"]
