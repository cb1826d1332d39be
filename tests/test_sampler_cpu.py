"""The ensemble Metropolis driver's host logic with stand-in scorers (no
GPU): acceptance rule, bounds, determinism, and that chains sample a known
Gaussian posterior."""
import numpy as np
import pytest

from paper_1501_07719_gb300 import sampler


def _sky(n=3):
    return dict(lm=np.zeros((n, 2)), stokes=np.tile([1.0, 0.0, 0.0, 0.0], (n, 1)), alpha=np.full(n, -0.7),
                shape=np.zeros((n, 3)))


def test_log_likelihood_is_eq7():
    assert sampler.log_likelihood(10.0, 4.0) == -7.0


def test_flat_scorer_accepts_every_proposal_in_bounds():
    s = sampler.EnsembleMetropolis(None, _sky(), 5, {"I": 0.5}, seed=3, bounds={"I": (0.0, 1.2)},
                                   chi2_fn=lambda models: np.zeros(len(models)))
    for _ in range(20):
        acc = s.step()
        assert np.all(s.theta["I"] >= 0.0) and np.all(s.theta["I"] <= 1.2)
    # proposals outside the bounds were rejected, inside ones accepted
    assert 0 < s.naccept.sum() < 5 * 20


def test_chains_are_deterministic_under_a_seed():
    f = lambda models: np.array([np.sum((m["lm"][:, 0] - 1e-3) ** 2) / 1e-8 for m in models])
    runs = []
    for _ in range(2):
        s = sampler.EnsembleMetropolis(None, _sky(), 4, {"l": 1e-4}, seed=11, chi2_fn=f)
        runs.append(s.run(30))
    np.testing.assert_array_equal(runs[0]["accept"], runs[1]["accept"])
    np.testing.assert_array_equal(runs[0]["chi2"], runs[1]["chi2"])


def test_chains_sample_a_gaussian_posterior():
    # chi^2 = ((l - mu) / sigma)^2 for each source: the posterior of l is N(mu, sigma^2)
    mu, sigma = 2e-3, 5e-4
    f = lambda models: np.array([np.sum(((m["lm"][:, 0] - mu) / sigma) ** 2) for m in models])
    s = sampler.EnsembleMetropolis(None, _sky(2), 64, {"l": 1.5 * sigma}, seed=5, chi2_fn=f)
    s.run(400)                                 # burn-in
    out = s.run(2000, thin=10)
    l = out["samples"]["l"].ravel()
    assert abs(l.mean() - mu) < 0.05 * sigma * 10 and abs(l.std() - sigma) < 0.1 * sigma
    rate = out["accept"].mean()
    assert 0.2 < rate < 0.7


@pytest.mark.parametrize("start", [1e-3, 1e3])
def test_adapt_brings_the_acceptance_rate_near_its_target(start):
    # proposal widths 1000x too small (accept ~1) or too large (accept ~0)
    mu, sigma = 2e-3, 5e-4
    f = lambda models: np.array([np.sum(((m["lm"][:, 0] - mu) / sigma) ** 2) for m in models])
    s = sampler.EnsembleMetropolis(None, _sky(2), 64, {"l": start * sigma}, seed=7, chi2_fn=f)
    scale = s.adapt(150, target=0.3)
    assert scale.shape == (150,)
    rate = s.run(200)["accept"].mean()
    assert 0.15 < rate < 0.5, rate


def test_unknown_parameter_is_rejected():
    with pytest.raises(ValueError):
        sampler.EnsembleMetropolis(None, _sky(), 2, {"flux": 1.0}, seed=0, chi2_fn=lambda m: np.zeros(len(m)))


def test_delta_scoring_needs_the_gpu_context():
    # residual-based scoring keeps state on the GPU: no stand-in scorer, no None context
    with pytest.raises(ValueError):
        sampler.EnsembleMetropolis(None, _sky(), 2, {"l": 1e-4}, seed=0, delta=True)
    with pytest.raises(ValueError):
        sampler.EnsembleMetropolis(object(), _sky(), 2, {"l": 1e-4}, seed=0, delta=True,
                                   chi2_fn=lambda m: np.zeros(len(m)))


def test_moved_rows_are_chain_major_and_carry_the_moved_parameters():
    class FakeRime:
        def set_sources(self, src):
            self.src = src

        def chi2(self):
            return 1.0

        def chains_init(self, k):
            self.k = k

    sky = _sky(4)
    sky["shape"][2] = [2e-5, 1e-5, 0.3]
    steps = {"l": np.array([0.0, 1e-4, 0.0, 2e-4]), "I": np.array([0.0, 0.1, 0.0, 0.0])}
    s = sampler.EnsembleMetropolis(FakeRime(), sky, 3, steps, seed=0, delta=True)
    np.testing.assert_array_equal(s.moved, [1, 3])       # sources with a non-zero step
    theta = {p: s.theta[p] + np.arange(3)[:, None] * 10.0 for p in s.theta}
    rows = s._moved_rows(theta)
    assert rows["lm"].shape == (6, 2) and rows["stokes"].shape == (6, 4) and rows["shape"].shape == (6, 3)
    for c in range(3):
        for j, src in enumerate((1, 3)):
            r = 2 * c + j
            assert rows["lm"][r, 0] == sky["lm"][src, 0] + 10.0 * c
            assert rows["lm"][r, 1] == sky["lm"][src, 1]       # m is not moved
            assert rows["stokes"][r, 0] == sky["stokes"][src, 0] + 10.0 * c
            np.testing.assert_array_equal(rows["shape"][r], sky["shape"][src])
