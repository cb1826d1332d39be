"""The split-precision tensor-core form of the point-source sum
(rime_set_tensor_mode): visibilities and chi^2 against the FP64 oracle at the
error each split states, its degenerate and error cases, and sampled
visibilities at the 256-antenna, 4096-source size."""
import numpy as np
import pytest

import oracle
import rime_synth
from gpu_cases import JINC, gpu_ctx, make_case, rel_err, vis_err

pytestmark = pytest.mark.gpu

# Error bounds against the FP64 oracle. Visibilities: max |dV| / max |V|.
# A product of split operands keeps hi*hi + hi*lo + lo*hi; the rounding of
# the low parts and the dropped lo*lo term leave a relative error of about
# 2^-16 per product for BF16 pairs (one source alone shows 1.2e-5) and 2^-21
# for TF32 pairs (5e-7), plus the SFU sine/cosine (~2^-21 absolute). The
# tensor core truncates its FP32 accumulation (about one unit in the last
# place per MMA, biased toward zero), so the kernel accumulates at most 24
# MMAs in TMEM before adding into FP32 sums with rounding to nearest, which
# keeps that bias near 1e-6. chi^2 inherits |dV|^2 / |V - D|^2 with V - D at
# the 0.01 Jy noise level: measured up to 6e-5 (BF16) and 1e-5 (TF32) on these
# cases.
# FP16 pairs keep TF32's 11 significant bits (their remainders below 2^-14
# are subnormal: an absolute 2^-25); measured on these cases up to 6.7e-7
# (visibilities) and 7.4e-6 (chi^2).
VTOL = {"bf16": 3e-5, "tf32": 3e-6, "f16": 1e-6}
CTOL = {"bf16": 3e-4, "tf32": 5e-5, "f16": 1.1e-5}
# The 256-antenna, 4096-source workload (|V| ~ 1e2 Jy, residuals at the noise
# level), about 1.5 times the errors measured there with the kernel's earlier
# tile plan (the bench's split form measures the same samples and slice):
# visibilities over the 192 sampled (t, baseline, channel) below, BF16 5.7e-6,
# TF32 1.17e-6, FP16 8.2e-7; chi^2 on timestep 0, channels 0-1 with data = the
# oracle's model + noise, BF16 7.3e-4, TF32 2.6e-5, FP16 2.1e-5 (the direct FP32
# path 1.2e-5). With the group-pair plan, which forms half of the cross-group
# baselines in the other orientation: 5.8e-6, 8.6e-7, 8.7e-7 and 7.7e-4,
# 3.0e-5, 1.7e-5. BF16 does not reach the FP32 chi^2 bound of 1e-4 there; TF32
# and FP16 do.
VTOL_256 = {"bf16": 8.5e-6, "tf32": 1.8e-6, "f16": 1.2e-6}
CTOL_256 = {"bf16": 1.1e-3, "tf32": 4e-5, "f16": 3.1e-5}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _mode(name):
    import paper_1501_07719_gb300 as R
    return {"bf16": R.RIME_TC_SPLIT_BF16, "tf32": R.RIME_TC_SPLIT_TF32, "f16": R.RIME_TC_SPLIT_F16}[name]


CASES = {
    # one tile pair, ragged source count (37 = 4 chunks of 8 + 5)
    "13ant-37src": dict(wl=rime_synth.custom(13, 2, 3, 37, 0, seed_index=71)),
    # two row tiles and three column tiles with ragged edges, pointing errors
    "130ant-pointing": dict(wl=rime_synth.custom(130, 1, 2, 20, 0, seed_index=72), pointing_sigma=0.004),
    # no gains, unit weights, a single channel and source
    "9ant-1src": dict(wl=rime_synth.custom(9, 2, 1, 1, 0, seed_index=73), gains=False, unit_weights=True),
    # time-varying brightness
    "20ant-tv": dict(wl=rime_synth.custom(20, 3, 2, 12, 0, seed_index=74), time_varying=True),
    # the Jinc beam: folded into the Stokes scales, and per antenna
    "13ant-jinc": dict(wl=rime_synth.custom(13, 2, 3, 37, 0, seed_index=80), **JINC),
    "130ant-jinc-pointing": dict(wl=rime_synth.custom(130, 1, 2, 20, 0, seed_index=81), pointing_sigma=0.004, **JINC),
}


@pytest.mark.parametrize("split", ["bf16", "tf32", "f16"])
@pytest.mark.parametrize("case", list(CASES))
def test_split_matches_oracle(case, split):
    inp = make_case(precision="f32", **CASES[case])
    r = gpu_ctx(inp, "f32")
    r.set_tensor_mode(_mode(split))
    V = r.predict().cpu().numpy()
    chi = r.chi2()
    r.close()
    ev = vis_err(V, inp["oracle_vis"])
    ec = rel_err(chi, oracle.Problem(inp, data=inp["data"]).chi2())
    assert ev <= VTOL[split], ev
    assert ec <= CTOL[split], ec


def test_split_mode_switch_restores_the_direct_path():
    import paper_1501_07719_gb300 as R
    inp = make_case(rime_synth.custom(13, 2, 3, 9, 0, seed_index=75), "f32")
    r = gpu_ctx(inp, "f32")
    direct = r.chi2()
    r.set_tensor_mode(R.RIME_TC_SPLIT_TF32)
    split = r.chi2()
    r.set_tensor_mode(R.RIME_TC_OFF)
    again = r.chi2()
    r.close()
    assert again == direct and split != direct


def test_split_is_deterministic():
    inp = make_case(rime_synth.custom(70, 2, 2, 30, 0, seed_index=76), "f32")
    r = gpu_ctx(inp, "f32")
    r.set_tensor_mode(_mode("bf16"))
    a, b = r.chi2(), r.chi2()
    r.close()
    assert a == b


def test_split_without_sources_gives_zero_model():
    inp = make_case(rime_synth.custom(10, 2, 2, 0, 0, seed_index=77), "f32")
    r = gpu_ctx(inp, "f32")
    r.set_tensor_mode(_mode("tf32"))
    V = r.predict().cpu().numpy()
    chi = r.chi2()
    r.close()
    assert np.all(V == 0)
    want = oracle.Problem(inp, data=inp["data"]).chi2()
    assert rel_err(chi, want) <= 1e-6


def test_split_rejects_exponential_disks():
    import paper_1501_07719_gb300 as R
    inp = make_case(rime_synth.custom(8, 2, 2, 3, 4, seed_index=82), "f32", disk_fraction=1.0)
    assert inp["sources"]["kind"].sum() == 4
    r = gpu_ctx(inp, "f32")
    r.set_tensor_mode(R.RIME_TC_SPLIT_TF32)
    with pytest.raises(R.RimeError) as e:
        r.chi2()
    assert e.value.status == R._abi.RIME_E_INVALID and "point sources" in str(e.value)
    r.set_tensor_mode(R.RIME_TC_OFF)
    assert rel_err(r.chi2(), oracle.Problem(inp, data=inp["data"]).chi2()) <= 1e-4
    r.close()


def test_split_rejects_gaussian_sources_and_fp64():
    import paper_1501_07719_gb300 as R
    inp = make_case(rime_synth.custom(8, 2, 2, 3, 2, seed_index=78), "f32")
    r = gpu_ctx(inp, "f32")
    r.set_tensor_mode(R.RIME_TC_SPLIT_BF16)
    out = r.torch.full((2, 28, 2, 4), 3.0 + 1j, dtype=r.cdtype, device="cuda")
    r.predict(out)
    with pytest.raises(R.RimeError) as e:
        r.sync()
    assert e.value.status == R._abi.RIME_E_INVALID and "point sources" in str(e.value)
    assert bool((out == 3.0 + 1j).all())
    r.set_tensor_mode(R.RIME_TC_OFF)       # the direct path takes the same model
    assert rel_err(r.chi2(), oracle.Problem(inp, data=inp["data"]).chi2()) <= 1e-4
    r.close()
    inp64 = make_case(rime_synth.custom(5, 1, 1, 1, 0, seed_index=79), "f64")
    r = gpu_ctx(inp64, "f64")
    with pytest.raises(R.RimeError):
        r.set_tensor_mode(R.RIME_TC_SPLIT_TF32)
    with pytest.raises(R.RimeError):
        r.set_tensor_mode(7)
    r.close()


def test_f16_split_rejects_stokes_beyond_its_range():
    """A source whose scaled Stokes vector exceeds the FP16 split's range
    (6e4 in magnitude) makes the FP16 mode's call return RIME_E_INVALID, its
    output untouched; the BF16 split takes the same model."""
    import paper_1501_07719_gb300 as R
    inp = make_case(rime_synth.custom(9, 2, 2, 3, 0, seed_index=83), "f32")
    inp["sources"]["stokes"][1] = [2e5, 0.0, 0.0, 0.0]   # at the phase centre: E = 1
    inp["sources"]["lm"][1] = [0.0, 0.0]
    want = oracle.Problem(inp, data=inp["data"]).chi2()
    r = gpu_ctx(inp, "f32")
    r.set_tensor_mode(R.RIME_TC_SPLIT_F16)
    out = r.torch.full((1,), 7.0, dtype=r.torch.float64, device="cuda")
    r.chi2_async(out)
    with pytest.raises(R.RimeError) as e:
        r.sync()
    assert e.value.status == R._abi.RIME_E_INVALID and "FP16" in str(e.value)
    assert float(out.item()) == 7.0
    r.set_tensor_mode(R.RIME_TC_SPLIT_BF16)
    assert rel_err(r.chi2(), want) <= CTOL["bf16"]
    r.close()


def test_split_256ant_slice_chi2_against_oracle():
    """The 256-antenna, 4096-point workload on one timestep and two channels
    (267 M source-terms): chi^2 of both splits and of the direct path against
    the FP64 oracle; data = model + noise, so V - D is at the noise level."""
    import paper_1501_07719_gb300 as R
    inp = rime_synth.make_inputs("256ant-20t-128ch-4096pt", precision="f32")
    sl = dict(inp, ntime=1, nchan=2, freq=inp["freq"][:2], uvw=inp["uvw"][:1], gains=inp["gains"][:1, :, :2],
              weight=inp["weight"][:1, :, :2], noise=inp["noise"][:1, :, :2])
    P = oracle.Problem(sl)
    sl["data"] = rime_synth.observe(P.predict(), sl["noise"], "f32")
    want = oracle.Problem(sl, data=sl["data"]).chi2()
    r = gpu_ctx(sl, "f32")
    # 4096 sources make |V| ~ 1e2 Jy against 0.01 Jy of noise. A single FP32
    # sum over all 4096 sources rounds each addition at 2^-24 |V|, which
    # showed in chi^2 at 1.2e-4; the direct kernel sums segments of 240
    # sources in FP32 and adds them into compensated running sums, and meets
    # the FP32 bound. The TF32 split adds short MMA segments into its running
    # sums too. The BF16 split's |dV| (~4e-6 of max |V|) shows at ~1e-3.
    for mode, tol in ((R.RIME_TC_OFF, 1e-4), (R.RIME_TC_SPLIT_BF16, CTOL_256["bf16"]),
                      (R.RIME_TC_SPLIT_TF32, CTOL_256["tf32"]), (R.RIME_TC_SPLIT_F16, CTOL_256["f16"])):
        r.set_tensor_mode(mode)
        got = r.chi2()
        assert rel_err(got, want) <= tol, (mode, got, want)
    r.close()


@pytest.mark.parametrize("split", ["bf16", "tf32", "f16"])
def test_split_full_256ant_sampled(split):
    """The 256-antenna, 20-timestep, 128-channel, 4096-point workload in the
    benchmark's configuration: sampled visibilities against the oracle."""
    import torch
    import paper_1501_07719_gb300 as R
    inp = rime_synth.make_inputs("256ant-20t-128ch-4096pt", precision="f32")
    r = R.Rime(inp, R.RIME_FP32, weight=inp["weight"].astype(np.float32))
    r.set_gains(inp["gains"])
    r.set_sources(inp["sources"])
    r.set_tensor_mode(_mode(split))
    V = r.predict()
    r.close()
    rng = np.random.default_rng(1)
    n = 192
    t = rng.integers(0, 20, n)
    bl = rng.integers(0, 32640, n)
    k = rng.integers(0, 128, n)
    tb, blb, kb = (torch.tensor(a, device="cuda") for a in (t, bl, k))
    got = V[tb, blb, kb].cpu().numpy().astype(np.complex128)
    del V
    torch.cuda.empty_cache()
    p, q = rime_synth.baseline_pairs(256)
    ref = oracle.Problem(inp).vis_list(t, p[bl], q[bl], k)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= VTOL_256[split], err


def test_phase_argument_matches_fp64_reduction():
    """The phase argument of eq. 3 as the FP32 and split kernels form it
    (double-float product, exact reduction) against the FP64 definition
    nu tau - round(nu tau): within 2^-24 + 2^-47 |nu tau| turns over the
    range the workloads reach (|nu tau| up to ~1e2 turns) and beyond."""
    import paper_1501_07719_gb300 as R
    rng = np.random.default_rng(11)
    n = 200000
    nu = rng.uniform(1.0e9, 1.5e9, n)
    # delays |tau| <= 1e-6 s: |nu tau| up to 1.5e3 turns (the workloads: ~1e2)
    tau = rng.uniform(-1e-6, 1e-6, n) * rng.choice([1e-3, 1e-2, 1e-1, 1.0], n)
    got = R.rime_phase_turns(nu, tau).astype(np.float64)
    want = oracle.reduced_phase(nu, tau)
    # the same remainder (near +-1/2 either end is the same phase)
    d = np.abs(got - want)
    d = np.minimum(d, np.abs(d - 1.0))
    bound = 2.0 ** -24 + 2.0 ** -47 * np.abs(nu * tau)
    assert np.all(d <= bound), float((d / bound).max())


@pytest.mark.parametrize("split", ["bf16", "tf32", "f16"])
def test_bounded_wait_gives_up_and_the_next_call_recovers(split):
    """With a 1 ns wait limit, the first wait of the tensor-core pipeline that
    is not already satisfied gives up: the block records the timeout, waits
    for the MMAs it issued, frees its tensor memory and returns, and the call
    reports RIME_E_TIMEOUT. With the default limit the next call returns the
    oracle's chi^2 (the tensor memory was freed, the status cleared)."""
    import paper_1501_07719_gb300 as R
    inp = make_case(**CASES["13ant-37src"], precision="f32")
    want = oracle.Problem(inp, data=inp["data"]).chi2()
    r = gpu_ctx(inp, "f32")
    r.set_tensor_mode(_mode(split))
    r.set_wait_limit(1)
    with pytest.raises(R.RimeError) as e:
        r.chi2()
    assert e.value.status == R._abi.RIME_E_TIMEOUT
    r.set_wait_limit(0)
    for _ in range(2):
        assert rel_err(r.chi2(), want) <= CTOL[split]
    r.close()
