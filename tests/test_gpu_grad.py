"""The adjoint gradient (rime_chi2_grad) against the FP64 oracle's analytic
gradient (itself pinned to finite differences in test_oracle_pins.py), a
finite-difference check through the GPU's own chi^2 at a larger size, and the
torch.autograd wrapper."""
import numpy as np
import pytest

import oracle
import rime_synth
from gpu_cases import JINC, gpu_ctx, make_case, rel_err

pytestmark = pytest.mark.gpu

# Error bound per parameter kind, relative to the largest gradient entry of
# that kind, about 2-3 times the largest error measured over these cases and
# the 64-antenna slice below (FP32: l, m 1.5e-3, Stokes 7.2e-3, alpha 1.3e-2,
# shape 8.7e-3, gains 1.4e-3; FP64: 1.4e-10 at most). In FP32 the residual
# V - D (~1e-2 Jy) is formed from visibilities of ~1e2 Jy, so its rounding
# (~1e-5 Jy) limits every gradient, which sums residuals, to ~1e-3 relative;
# sums whose terms cancel lose more (alpha: ln(nu/nu_ref) changes sign across
# the band; Stokes Q, U, V: the correlations' signs).
GTOL = {"f64": dict(lm=4e-10, stokes=1.2e-10, alpha=2e-10, shape=1.2e-10, gains=1.2e-10),
        "f32": dict(lm=3e-3, stokes=1.5e-2, alpha=2.5e-2, shape=1.8e-2, gains=3e-3)}
KINDS = (("lm", [0, 1]), ("stokes", [2, 3, 4, 5]), ("alpha", [6]), ("shape", [7, 8, 9]))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


CASES = {
    "13ant": dict(wl=rime_synth.custom(13, 3, 5, 20, 17, seed_index=51)),
    "70ant-units": dict(wl=rime_synth.custom(70, 2, 3, 6, 5, seed_index=52)),
    "10ant-pointing": dict(wl=rime_synth.custom(10, 2, 4, 5, 5, seed_index=53), pointing_sigma=0.004),
    "9ant-no-gains": dict(wl=rime_synth.custom(9, 2, 3, 4, 4, seed_index=54), gains=False),
    # the Jinc beam's derivative, per antenna and folded
    "10ant-jinc-pointing": dict(wl=rime_synth.custom(10, 2, 4, 5, 5, seed_index=58), pointing_sigma=0.004, **JINC),
    "12ant-jinc": dict(wl=rime_synth.custom(12, 2, 3, 6, 4, seed_index=59), **JINC),
    # exponential disks beside Gaussians: the shape derivatives of both
    "11ant-disks": dict(wl=rime_synth.custom(11, 2, 3, 4, 12, seed_index=60), disk_fraction=0.5),
    "10ant-disks-pointing": dict(wl=rime_synth.custom(10, 2, 3, 3, 9, seed_index=61), disk_fraction=0.6,
                                 pointing_sigma=0.003),
    # 500 sources: the FP32 forward pass folds segments of its source sum
    "36ant-long-list": dict(wl=rime_synth.custom(36, 1, 2, 250, 250, seed_index=62)),
    # 33 sources: the FP32 source pass's second chunk holds one source (one
    # source pair, 256 baseline groups)
    "30ant-33src": dict(wl=rime_synth.custom(30, 2, 2, 17, 16, seed_index=63)),
}


def _scaled_case(case, precision):
    inp = make_case(precision=precision, **CASES[case])
    return inp


def _check(got, want, tol, what):
    scale = np.abs(want).max()
    err = np.abs(got - want).max()
    assert err <= tol * scale, f"{what}: max err {err:.3e} vs scale {scale:.3e}"


@pytest.mark.parametrize("kernel", [None, "tiled"])
@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("case", list(CASES))
def test_gradient_matches_oracle(case, precision, kernel):
    """The forward pass runs in the kernel a plain chi^2 uses (the small-array
    kernel for the small cases), or forced tiled; both against the oracle."""
    inp = _scaled_case(case, precision)
    chi_ref, gs_ref, gg_ref = oracle.Problem(inp, data=inp["data"]).chi2_grad(want_gains=True)
    import paper_1501_07719_gb300 as R
    r = gpu_ctx(inp, precision)
    if kernel == "tiled":
        r.set_kernel(R.RIME_KERNEL_TILED)
    chi, gs, gg = r.chi2_grad(want_gains=True)
    chi_plain = r.chi2()   # the same kernel's plain chi^2
    r.close()
    assert chi == chi_plain
    assert rel_err(chi, chi_ref) <= (1e-10 if precision == "f64" else 1e-4)
    _check_all(gs.cpu().numpy(), gg.cpu().numpy().reshape(gg_ref.shape), gs_ref, gg_ref, precision)


def _check_all(gs, gg, gs_ref, gg_ref, precision):
    tol = GTOL[precision]
    # per parameter kind: l, m | I, Q, U, V | alpha | shape
    for name, cols in KINDS:
        if np.abs(gs_ref[:, cols]).max() == 0:
            assert np.abs(gs[:, cols]).max() == 0
            continue
        _check(gs[:, cols], gs_ref[:, cols], tol[name], name)
    _check(gg, gg_ref, tol["gains"], "gains")


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_gradient_64ant_workload_slice(precision):
    """The 64-antenna gradient workload (2016 baselines, 100 point + 100
    Gaussian sources, gains, weights) on one timestep and four channels, in
    the tiled kernels: chi^2 and every source and gain gradient against the
    oracle's."""
    inp = rime_synth.make_inputs("64ant-100t-64ch-100pt100g-grad", precision=precision)
    sl = dict(inp, ntime=1, nchan=4, freq=inp["freq"][:4], uvw=inp["uvw"][:1], gains=inp["gains"][:1, :, :4],
              weight=inp["weight"][:1, :, :4], noise=inp["noise"][:1, :, :4])
    sl["data"] = rime_synth.observe(oracle.Problem(sl).predict(), sl["noise"], precision)
    chi_ref, gs_ref, gg_ref = oracle.Problem(sl, data=sl["data"]).chi2_grad(want_gains=True)
    r = gpu_ctx(sl, precision)
    chi, gs, gg = r.chi2_grad(want_gains=True)
    r.close()
    assert rel_err(chi, chi_ref) <= (1e-10 if precision == "f64" else 1e-4)
    _check_all(gs.cpu().numpy(), gg.cpu().numpy().reshape(gg_ref.shape), gs_ref, gg_ref, precision)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("case,kernel", [("13ant", None), ("70ant-units", None), ("36ant-long-list", None)])
def test_gradient_is_bit_reproducible(case, precision, kernel):
    """Repeated calls give identical chi^2, source and gains gradients: every
    sum runs in a fixed order (the gains gradient from per-visibility terms,
    the source gradient from per-block partials)."""
    inp = _scaled_case(case, precision)
    r = gpu_ctx(inp, precision)
    runs = [r.chi2_grad(want_gains=True) for _ in range(3)]
    r.close()
    chi0, gs0, gg0 = runs[0][0], runs[0][1].cpu().numpy(), runs[0][2].cpu().numpy()
    assert np.any(gg0 != 0)
    for chi, gs, gg in runs[1:]:
        assert chi == chi0
        np.testing.assert_array_equal(gs.cpu().numpy(), gs0)
        np.testing.assert_array_equal(gg.cpu().numpy(), gg0)


def test_gradient_directional_fd_at_scale():
    """A larger problem than the oracle can take quickly: the gradient's
    directional derivative along a random direction equals the central
    difference of the GPU's FP64 chi^2 (steps 1e-6 and 5e-7 relative to each
    parameter's scale, Richardson-extrapolated to cancel the h^2 term, which
    the phase's curvature makes visible at these steps)."""
    import torch
    inp = make_case(rime_synth.custom(40, 6, 8, 30, 30, seed_index=55), "f64")
    r = gpu_ctx(inp, "f64")
    _, gs, gg = r.chi2_grad(want_gains=False)
    gs = gs.cpu().numpy()
    rng = np.random.default_rng(9)
    src = inp["sources"]
    scales = np.array([1e-2, 1e-2, 1, 1, 1, 1, 1, 1e-4, 1e-4, 1])
    d = rng.normal(size=gs.shape) * scales
    d[:30, 7:] = 0.0                      # points have no shape parameters
    d[:, 3:6] *= 0.05                     # keep |Q,U,V| small relative to I
    pts = [src["lm"][:, 0], src["lm"][:, 1], *src["stokes"].T, src["alpha"], *src["shape"].T]
    theta = np.stack(pts, axis=1)
    def central(h):
        vals = []
        for sgn in (1, -1):
            th = theta + sgn * h * d
            r.set_sources(dict(lm=th[:, :2], stokes=th[:, 2:6], alpha=th[:, 6], shape=th[:, 7:10]))
            vals.append(r.chi2())
        return (vals[0] - vals[1]) / (2 * h)
    f1, f2 = central(1e-6), central(5e-7)
    r.close()
    fd = (4 * f2 - f1) / 3
    an = float((gs * d).sum())
    assert abs(fd - an) <= 1e-7 * abs(an), (fd, an, f1, f2)


def test_autograd_wrapper_matches_chi2_grad():
    import torch
    import paper_1501_07719_gb300 as R
    inp = make_case(rime_synth.custom(8, 2, 3, 3, 3, seed_index=56), "f64")
    r = gpu_ctx(inp, "f64")
    chi, gs, gg = r.chi2_grad(want_gains=True)
    dev = lambda a: torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda", requires_grad=True)
    src = inp["sources"]
    lm, st, al, sh = dev(src["lm"]), dev(src["stokes"]), dev(src["alpha"]), dev(src["shape"])
    g = torch.tensor(inp["gains"], dtype=torch.complex128, device="cuda", requires_grad=True)
    out = R.RimeChi2.apply(r, lm, st, al, sh, g)
    (2.0 * out).backward()
    assert abs(out.item() - chi) <= 1e-12 * chi
    np.testing.assert_allclose(lm.grad.cpu().numpy(), 2 * gs[:, 0:2].cpu().numpy(), rtol=1e-12)
    np.testing.assert_allclose(st.grad.cpu().numpy(), 2 * gs[:, 2:6].cpu().numpy(), rtol=1e-12)
    np.testing.assert_allclose(al.grad.cpu().numpy(), 2 * gs[:, 6].cpu().numpy(), rtol=1e-12)
    np.testing.assert_allclose(g.grad.cpu().numpy(), 2 * gg.cpu().numpy(), rtol=1e-12, atol=1e-300)
    r.close()


def test_gradient_rejects_time_varying_brightness():
    import paper_1501_07719_gb300 as R
    inp = make_case(rime_synth.custom(5, 2, 2, 2, 0, seed_index=57), "f64", time_varying=True)
    r = gpu_ctx(inp, "f64")
    with pytest.raises(R.RimeError) as e:
        r.chi2_grad()
    assert e.value.status == R._abi.RIME_E_INVALID
    r.close()
