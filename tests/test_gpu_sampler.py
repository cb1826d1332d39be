"""Sampler-in-the-loop drivers on the GPU: an ensemble Metropolis run scored
by the batched chi^2 follows, proposal for proposal, the same run scored by
the FP64 oracle; the MAP fit by the adjoint gradient recovers the sky model."""
import numpy as np
import pytest

import oracle
import rime_synth
from gpu_cases import gpu_ctx, make_case, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


STEPS = {"l": 3e-5, "m": 3e-5, "I": 0.01, "alpha": 0.02}


def test_ensemble_chain_matches_oracle_scored_chain():
    from paper_1501_07719_gb300 import sampler
    inp = make_case(rime_synth.custom(8, 3, 4, 2, 1, seed_index=91), "f64")
    r = gpu_ctx(inp, "f64")
    gpu = sampler.EnsembleMetropolis(r, inp["sources"], 6, STEPS, seed=7)
    ora = sampler.EnsembleMetropolis(
        None, inp["sources"], 6, STEPS, seed=7,
        chi2_fn=lambda models: np.array([oracle.Problem(inp, sources=m, data=inp["data"]).chi2() for m in models]))
    a, b = gpu.run(25), ora.run(25)
    r.close()
    np.testing.assert_array_equal(a["accept"], b["accept"])
    assert 0 < a["accept"].sum() < a["accept"].size
    for p in STEPS:
        np.testing.assert_array_equal(gpu.theta[p], ora.theta[p])
    assert np.all(np.abs(a["chi2"] - b["chi2"]) <= 1e-10 * np.abs(b["chi2"]))


def test_ensemble_fp32_batched_scoring_equals_one_set_calls():
    from paper_1501_07719_gb300 import sampler
    inp = make_case(rime_synth.custom(16, 3, 4, 3, 2, seed_index=92), "f32")
    r = gpu_ctx(inp, "f32")
    r2 = gpu_ctx(inp, "f32")

    def one_by_one(models):
        out = []
        for m in models:
            r2.set_sources(m)
            out.append(r2.chi2())
        return np.array(out)
    a = sampler.EnsembleMetropolis(r, inp["sources"], 5, STEPS, seed=3).run(15)
    b = sampler.EnsembleMetropolis(None, inp["sources"], 5, STEPS, seed=3, chi2_fn=one_by_one).run(15)
    r.close()
    r2.close()
    np.testing.assert_array_equal(a["accept"], b["accept"])
    assert np.all(np.abs(a["chi2"] - b["chi2"]) <= 1e-12 * np.abs(b["chi2"]))


def test_map_fit_recovers_the_sky_model():
    from paper_1501_07719_gb300 import sampler
    inp = make_case(rime_synth.custom(12, 4, 6, 3, 2, seed_index=93), "f64")
    truth = inp["sources"]
    start = {k: np.array(v) for k, v in truth.items()}
    rng = np.random.default_rng(2)
    start["lm"] = truth["lm"] + rng.normal(0, 2e-6, truth["lm"].shape)
    start["stokes"] = truth["stokes"] * 1.02
    start["alpha"] = truth["alpha"] + 0.02
    r = gpu_ctx(inp, "f64")
    fitted, trace = sampler.fit_map(r, start, max_iter=200)
    chi_truth = oracle.Problem(inp, data=inp["data"]).chi2()
    r.close()
    assert trace[-1] < trace[0]
    # the fit reaches the truth's chi^2 or below (it also fits the noise:
    # about 2 sigma^2 w = 2.5e-4 per fitted parameter)
    assert min(trace) <= chi_truth
    err0 = np.abs(start["lm"] - truth["lm"]).max()
    err1 = np.abs(fitted["lm"] - truth["lm"]).max()
    assert err1 < 0.2 * err0, (err0, err1)
    want = oracle.Problem(inp, sources=fitted, data=inp["data"]).chi2()
    assert want <= chi_truth and rel_err(want, min(trace)) <= 1e-6
