"""Per-chain residuals (rime_chains_*): a proposal's chi^2 evaluated as the
predict of its moved sources (new values and the current ones with negated
Stokes vectors) against the chain's resident residual D - V equals the
oracle's chi^2 of the chain's whole proposed sky model, over several rounds
of proposals and partial acceptance, through both direct-sum kernels and in
both precisions; and the ensemble sampler scored this way follows the
oracle-scored chain."""
import numpy as np
import pytest

import oracle
import rime_synth
from gpu_cases import JINC, TOL, gpu_ctx, make_case, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _perturb(rng, src, rows):
    out = {k: np.array(v[rows], copy=True) for k, v in src.items()}
    out["lm"] += rng.normal(0, 2e-4, out["lm"].shape)
    out["stokes"] *= 1 + rng.normal(0, 0.05, (len(rows), 1))
    out["alpha"] += rng.normal(0, 0.1, len(rows))
    if "shape" in out:
        ext = out["shape"][:, 0] > 0
        out["shape"][ext, :2] *= 1.1
        out["shape"][ext, 2] += 0.2
    return out


CASES = {
    "9ant-f64": dict(wl=rime_synth.custom(9, 3, 4, 3, 3, seed_index=95), precision="f64", pointing_sigma=0.002),
    "9ant-f32": dict(wl=rime_synth.custom(9, 3, 4, 3, 3, seed_index=95), precision="f32", pointing_sigma=0.002),
    "50ant-tiled-f32": dict(wl=rime_synth.custom(50, 2, 3, 2, 3, seed_index=96), precision="f32", kernel="tiled"),
    "12ant-disks-jinc-f64": dict(wl=rime_synth.custom(12, 2, 3, 2, 4, seed_index=97), precision="f64",
                                 disk_fraction=0.5, **JINC),
}


@pytest.mark.parametrize("case", list(CASES))
def test_chain_proposals_match_oracle_over_rounds(case):
    import paper_1501_07719_gb300 as R
    kw = dict(CASES[case])
    precision, kernel = kw.pop("precision"), kw.pop("kernel", None)
    inp = make_case(precision=precision, **kw)
    r = gpu_ctx(inp, precision)
    if kernel == "tiled":
        r.set_kernel(R.RIME_KERNEL_TILED)
    K, moved = 5, np.array([1, 4])
    models = [{k: np.array(v, copy=True) for k, v in inp["sources"].items()} for _ in range(K)]
    r.chains_init(K)
    rng = np.random.default_rng(4)
    for rnd in range(3):
        prop = [_perturb(rng, m, moved) for m in models]
        cat = lambda ms: {k: np.concatenate([m[k] for m in ms]) for k in ms[0]}
        cur = [{k: v[moved] for k, v in m.items()} for m in models]
        got = r.chains_propose(len(moved), cat(prop), cat(cur)).cpu().numpy()
        for c in range(K):
            full = {k: np.array(v, copy=True) for k, v in models[c].items()}
            for k in full:
                full[k][moved] = prop[c][k]
            want = oracle.Problem(inp, sources=full, data=inp["data"]).chi2()
            assert rel_err(got[c], want) <= TOL[precision]["chi2"], (rnd, c, got[c], want)
        accept = rng.uniform(size=K) < 0.6
        accept[rnd % K] = True
        r.chains_accept(accept.astype(np.int32))
        for c in np.flatnonzero(accept):
            for k in models[c]:
                models[c][k][moved] = prop[c][k]
    r.close()


def test_chain_call_order_and_argument_errors():
    import paper_1501_07719_gb300 as R
    inp = make_case(rime_synth.custom(6, 2, 2, 3, 0, seed_index=98), "f64")
    r = gpu_ctx(inp, "f64")
    one = {k: v[:1] for k, v in inp["sources"].items()}
    with pytest.raises(R.RimeError) as e:
        r.chains_accept(np.ones(2, dtype=np.int32))
    assert e.value.status == R._abi.RIME_E_STATE
    r.nchains = 2
    with pytest.raises(R.RimeError) as e:
        r.chains_propose(1, one, one)
    assert e.value.status == R._abi.RIME_E_STATE      # before rime_chains_init
    r.chains_init(2)
    with pytest.raises(R.RimeError) as e:
        r.chains_propose(1, one, one)                 # needs 2 chains x 1 source
    assert e.value.status == R._abi.RIME_E_INVALID
    with pytest.raises(R.RimeError):
        R._abi.rime_chains_init(r.ctx, 0)
    r.close()


def test_delta_sampler_matches_oracle_scored_chain():
    from paper_1501_07719_gb300 import sampler
    inp = make_case(rime_synth.custom(8, 3, 4, 2, 1, seed_index=91), "f64")
    steps = {"l": 3e-5, "m": 3e-5, "I": 0.01, "alpha": 0.02}
    r = gpu_ctx(inp, "f64")
    gpu = sampler.EnsembleMetropolis(r, inp["sources"], 6, steps, seed=7, delta=True)
    ora = sampler.EnsembleMetropolis(
        None, inp["sources"], 6, steps, seed=7,
        chi2_fn=lambda models: np.array([oracle.Problem(inp, sources=m, data=inp["data"]).chi2() for m in models]))
    a, b = gpu.run(25), ora.run(25)
    r.close()
    np.testing.assert_array_equal(a["accept"], b["accept"])
    assert 0 < a["accept"].sum() < a["accept"].size
    assert np.all(np.abs(a["chi2"] - b["chi2"]) <= 1e-10 * np.abs(b["chi2"]))
