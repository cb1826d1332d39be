"""Sampler-in-the-loop drivers of the BIRO iteration (Sec. 2.3 and the BIRO
flow of Fig. 3): the library scores proposed sky models, the host keeps the
chain.

With Gaussian noise, -2 ln L = chi^2 + sum ln(2 pi / w) (eq. 7); the second
term does not depend on the sky model, so with flat priors inside bounds a
Metropolis proposal is accepted with probability min(1, exp(-(chi2' - chi2)
/ 2)).

* ``EnsembleMetropolis``: K independent random-walk Metropolis chains; the K
  proposals of one step are scored by one batched chi^2 call
  (``rime_chi2_batched``), so a sampler iteration is one persistent launch;
  or, with ``delta=True``, against per-chain residuals kept on the GPU
  (``rime_chains_*``): a proposal then costs the predict of the moved
  sources only.
* ``fit_map``: maximum-likelihood fit of the sky model by L-BFGS on the
  adjoint gradient (``RimeChi2``, ``rime_chi2_grad``).
"""
from __future__ import annotations

import numpy as np

# the parameters a chain may move: name -> (sky-model array, column or None)
PARAMS = {"l": ("lm", 0), "m": ("lm", 1), "I": ("stokes", 0), "Q": ("stokes", 1), "U": ("stokes", 2),
          "V": ("stokes", 3), "alpha": ("alpha", None), "major": ("shape", 0), "minor": ("shape", 1),
          "pa": ("shape", 2)}


def log_likelihood(chi2, ln_norm: float):
    """ln L of eq. 7 from chi^2 and sum ln(2 pi / w) (``Rime.ln_norm``)."""
    return -0.5 * (np.asarray(chi2, dtype=np.float64) + ln_norm)


class EnsembleMetropolis:
    """K random-walk Metropolis chains over chosen parameters of every source.

    rime:    a Rime context holding the observation, data, weights and gains
    sources: the starting sky model (SoA dict: lm, stokes, alpha, shape);
             every chain starts there
    steps:   {parameter name: proposal standard deviation} (PARAMS names)
    bounds:  {parameter name: (low, high)}: flat prior support; proposals
             outside are rejected without evaluation
    chi2_fn: optional replacement scorer, f(list of K sky models) -> [K]
             chi^2 (by default one batched call on `rime`)
    delta:   score each proposal as a change of the moved sources (those
             with a non-zero step) against the chain's residual D - V held on
             the GPU (rime_chains_*), instead of the whole sky model
    """

    def __init__(self, rime, sources: dict, nchains: int, steps: dict, seed: int, bounds: dict | None = None,
                 chi2_fn=None, delta: bool = False):
        self.rime = rime
        self.K = int(nchains)
        self.base = {k: np.array(v, dtype=np.float64) for k, v in sources.items() if v is not None}
        self.nsrc = int(self.base["alpha"].shape[0])
        self.steps = {p: np.broadcast_to(np.asarray(s, dtype=np.float64), (self.nsrc,)) for p, s in steps.items()}
        for p in self.steps:
            if p not in PARAMS:
                raise ValueError(f"unknown parameter {p!r}")
            if PARAMS[p][0] not in self.base:
                raise ValueError(f"parameter {p!r} needs {PARAMS[p][0]!r} in the sky model")
        self.bounds = dict(bounds or {})
        self.rng = np.random.default_rng(seed)
        self.chi2_fn = chi2_fn or self._batched_chi2
        self.theta = {p: np.tile(self._get(self.base, p), (self.K, 1)) for p in self.steps}
        self.delta = bool(delta)
        if self.delta:
            if rime is None or chi2_fn is not None:
                raise ValueError("delta scoring needs the GPU context and no replacement scorer")
            # the sources a proposal moves: those with a non-zero step
            self.moved = np.flatnonzero(np.any([self.steps[p] != 0 for p in self.steps], axis=0))
            rime.set_sources(self.base)
            chi0 = rime.chi2()
            rime.chains_init(self.K)
            self.chi2 = np.full(self.K, chi0)
        else:
            self.chi2 = np.asarray(self.chi2_fn([self._model(i, self.theta) for i in range(self.K)]),
                                   dtype=np.float64)
        self.naccept = np.zeros(self.K, dtype=np.int64)
        self.nstep = 0

    @staticmethod
    def _get(model, p):
        key, col = PARAMS[p]
        return model[key] if col is None else model[key][:, col]

    def _model(self, i: int, theta: dict) -> dict:
        """Chain i's sky model under parameters theta."""
        m = {k: v.copy() for k, v in self.base.items()}
        for p, vals in theta.items():
            key, col = PARAMS[p]
            if col is None:
                m[key] = vals[i].copy()
            else:
                m[key][:, col] = vals[i]
        return m

    def _batched_chi2(self, models: list) -> np.ndarray:
        offsets = np.arange(len(models) + 1, dtype=np.int32) * self.nsrc
        cat = {k: np.concatenate([m[k] for m in models]) for k in models[0]}
        out = self.rime.chi2_batched(offsets, cat)
        self.rime.sync()
        return out.cpu().numpy()

    def _in_bounds(self, theta: dict) -> np.ndarray:
        ok = np.ones(self.K, dtype=bool)
        for p, (lo, hi) in self.bounds.items():
            if p in theta:
                ok &= np.all((theta[p] >= lo) & (theta[p] <= hi), axis=1)
        if "l" in theta or "m" in theta:   # direction cosines inside the unit circle
            l = theta.get("l", np.tile(self.base["lm"][:, 0], (self.K, 1)))
            m = theta.get("m", np.tile(self.base["lm"][:, 1], (self.K, 1)))
            ok &= np.all(l * l + m * m < 1.0, axis=1)
        return ok

    def _moved_rows(self, theta: dict) -> dict:
        """The moved sources of every chain under theta, chain-major
        ([K * m] rows), as a sky-model dict."""
        out = {}
        for key, v in self.base.items():
            rows = np.repeat(v[self.moved][None], self.K, axis=0)   # [K, m, ...]
            out[key] = rows
        for p, vals in theta.items():
            key, col = PARAMS[p]
            if col is None:
                out[key][:, :] = vals[:, self.moved]
            else:
                out[key][:, :, col] = vals[:, self.moved]
        return {k: np.ascontiguousarray(v.reshape((-1,) + v.shape[2:])) for k, v in out.items()}

    def _delta_chi2(self, prop: dict, ok: np.ndarray) -> np.ndarray:
        # chains whose proposal left the prior's support propose no change
        safe = {p: np.where(ok[:, None], prop[p], self.theta[p]) for p in prop}
        out = self.rime.chains_propose(len(self.moved), self._moved_rows(safe), self._moved_rows(self.theta))
        self.rime.sync()
        return out.cpu().numpy()

    def step(self) -> np.ndarray:
        """One Metropolis step of every chain; returns which chains accepted."""
        prop = {p: self.theta[p] + self.steps[p] * self.rng.standard_normal((self.K, self.nsrc))
                for p in self.steps}
        log_u = np.log(self.rng.uniform(size=self.K))
        ok = self._in_bounds(prop)
        chi2p = np.full(self.K, np.inf)
        idx = np.flatnonzero(ok)
        if self.delta:
            if idx.size:
                chi2p[idx] = self._delta_chi2(prop, ok)[idx]
        elif idx.size:
            chi2p[idx] = self.chi2_fn([self._model(i, prop) for i in idx])
        accept = ok & (log_u < -0.5 * (chi2p - self.chi2))
        if self.delta and accept.any():
            self.rime.chains_accept(accept.astype(np.int32))
        for p in self.steps:
            self.theta[p][accept] = prop[p][accept]
        self.chi2[accept] = chi2p[accept]
        self.naccept += accept
        self.nstep += 1
        return accept

    def adapt(self, nsteps: int, target: float = 0.3, gain: float = 1.0) -> np.ndarray:
        """Burn-in steps that rescale every proposal standard deviation by one
        common factor after each step, log f = gain (a - target) / sqrt(i + 1)
        with a the fraction of chains that accepted at step i (a stochastic
        approximation to the scale whose acceptance rate is `target`). The
        chains are not Markov while this runs: use it before sampling.
        Returns the cumulative scale after each step."""
        total, hist = 1.0, []
        for i in range(nsteps):
            a = float(self.step().mean())
            f = float(np.exp(gain * (a - target) / np.sqrt(i + 1.0)))
            self.steps = {p: s * f for p, s in self.steps.items()}
            total *= f
            hist.append(total)
        return np.array(hist)

    def run(self, nsteps: int, thin: int = 1) -> dict:
        """nsteps steps; returns the chi^2 trace [nsteps, K], the accept trace
        and every `thin`-th state of the moved parameters."""
        chi2s, accs, samples = [], [], {p: [] for p in self.steps}
        for i in range(nsteps):
            accs.append(self.step())
            chi2s.append(self.chi2.copy())
            if (i + 1) % thin == 0:
                for p in self.steps:
                    samples[p].append(self.theta[p].copy())
        return {"chi2": np.array(chi2s), "accept": np.array(accs),
                "samples": {p: np.array(v) for p, v in samples.items()}}

    def sources(self, i: int) -> dict:
        """Chain i's current sky model."""
        return self._model(i, self.theta)


def fit_map(rime, sources: dict, fit=("lm", "stokes", "alpha"), scales: dict | None = None, max_iter: int = 50):
    """Maximum-likelihood sky model from `sources` by L-BFGS (strong Wolfe line
    search) on chi^2 and its adjoint gradient. The fitted arrays are moved in
    units of `scales` (default: 1e-6 rad for lm, 1e-2 Jy for stokes, 1e-2 for
    alpha, 1e-6 rad for shape), which should be near the posterior widths so
    that the problem is well conditioned. Returns the fitted sky model and the
    chi^2 of every evaluation."""
    import torch
    from .autograd import RimeChi2
    scales = {"lm": 1e-6, "stokes": 1e-2, "alpha": 1e-2, "shape": 1e-6, **(scales or {})}
    dev = "cuda"
    base = {k: torch.tensor(np.asarray(v, dtype=np.float64), device=dev) for k, v in sources.items()
            if v is not None}
    x = {k: torch.zeros_like(base[k], requires_grad=True) for k in fit}
    trace = []

    def model():
        return {k: base[k] + scales[k] * x[k] if k in x else base[k] for k in base}

    opt = torch.optim.LBFGS(list(x.values()), lr=1.0, max_iter=max_iter, line_search_fn="strong_wolfe",
                            tolerance_grad=1e-12, tolerance_change=1e-14, history_size=20)

    def closure():
        opt.zero_grad()
        m = model()
        chi = RimeChi2.apply(rime, m["lm"], m["stokes"], m["alpha"], m.get("shape"))
        chi.backward()
        trace.append(float(chi.item()))
        return chi

    opt.step(closure)
    with torch.no_grad():
        fitted = {k: v.detach().cpu().numpy() for k, v in model().items()}
    return fitted, trace
