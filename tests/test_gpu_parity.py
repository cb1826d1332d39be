"""Parity of the CUDA predict + chi^2 path with the FP64 oracle, through the
C ABI. Element by element on seeded inputs that span several thread tiles,
source chunks and antenna units with ragged tails; sampled at the full
64-antenna workload; plus the edge cases and the error paths."""
import numpy as np
import pytest

import oracle
import rime_synth
from gpu_cases import JINC, TOL, gpu_ctx, gpu_run, make_case, oracle_chi2, rel_err, vis_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1501_07719_gb300 as R
    R.lib()


CASES = {
    # the 7-antenna workload: 21 baselines, 10 timesteps, 16 channels, 10 points
    "7ant": dict(wl="7ant-10t-16ch-10pt"),
    # ragged tiles and source chunks, Gaussians, pointing errors, time-varying flux
    "13ant-ragged": dict(wl=rime_synth.custom(13, 3, 5, 20, 17, seed_index=21),
                         pointing_sigma=0.003, time_varying=True),
    # several antenna units (64-antenna FP32 units, 32-antenna FP64 units)
    "70ant-units": dict(wl=rime_synth.custom(70, 2, 3, 6, 5, seed_index=22), pointing_sigma=0.002),
    # a single baseline, channel and timestep
    "2ant-min": dict(wl=rime_synth.custom(2, 1, 1, 1, 0, seed_index=23)),
    # narrow kernel shapes: 3 baselines x 70 channels (two channel groups of
    # up to 64), Gaussians and pointing errors
    "3ant-70ch": dict(wl=rime_synth.custom(3, 2, 70, 5, 4, seed_index=31), pointing_sigma=0.002),
    # 23..32 antennas: one channel per block, two pairs per thread; 40 sources
    # span three FP64 chunks (16) and two FP32 chunks (32) with ragged tails
    "27ant-2pairs": dict(wl=rime_synth.custom(27, 2, 3, 22, 18, seed_index=32), time_varying=True),
    "32ant": dict(wl=rime_synth.custom(32, 1, 2, 3, 3, seed_index=33), pointing_sigma=0.001),
    # 33..45 antennas: 512-thread blocks of two pairs each (45: the largest)
    "45ant-max": dict(wl=rime_synth.custom(45, 2, 2, 17, 5, seed_index=35), pointing_sigma=0.001),
    # the Jinc beam model: per-antenna (pointing errors) and folded into the
    # Stokes scale (none), across units and both kernels
    "13ant-jinc-pointing": dict(wl=rime_synth.custom(13, 3, 5, 20, 17, seed_index=36), pointing_sigma=0.003,
                                **JINC),
    "70ant-jinc": dict(wl=rime_synth.custom(70, 2, 3, 6, 5, seed_index=37), **JINC),
    "20ant-jinc": dict(wl=rime_synth.custom(20, 2, 3, 9, 9, seed_index=38), **JINC),
    # exponential disks (source kind 1) beside Gaussians and points; with the
    # Jinc beam and pointing errors too, across antenna units
    "13ant-disks": dict(wl=rime_synth.custom(13, 3, 5, 10, 27, seed_index=39), disk_fraction=0.5,
                        time_varying=True),
    "70ant-disks-jinc": dict(wl=rime_synth.custom(70, 2, 3, 6, 11, seed_index=40), disk_fraction=0.5,
                             pointing_sigma=0.002, **JINC),
    # long source lists: the FP32 tiled kernel's per-block running sums (more
    # than two register segments of 240 sources), across units, pointing
    # errors, and with the general instance (Jinc beam, disks)
    "70ant-long": dict(wl=rime_synth.custom(70, 2, 2, 330, 250, seed_index=41), pointing_sigma=0.002),
    "40ant-long-jinc-disks": dict(wl=rime_synth.custom(40, 2, 2, 300, 300, seed_index=42), disk_fraction=0.5,
                                  **JINC),
}


# the kernels a case runs through: the library's choice, and each direct-sum
# kernel that takes the array (the narrow one up to 45 antennas)
KERNELS = [None, "tiled", "narrow"]


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("case", list(CASES))
def test_predict_and_chi2_match_oracle(case, precision, kernel):
    inp = make_case(precision=precision, **CASES[case])
    if kernel == "narrow" and inp["na"] > 45:
        pytest.skip("the narrow kernel takes arrays of up to 45 antennas")
    V, chi = gpu_run(inp, precision, kernel)
    Vref = inp["oracle_vis"]
    assert V.shape == Vref.shape
    assert vis_err(V, Vref) <= TOL[precision]["vis"], vis_err(V, Vref)
    cref = oracle_chi2(inp)
    assert rel_err(chi, cref) <= TOL[precision]["chi2"], (chi, cref)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_no_sources_gives_zero_model(precision):
    inp = make_case(rime_synth.custom(9, 2, 4, 3, 0, seed_index=24), precision)
    r = gpu_ctx(inp, precision)
    r.set_sources(dict(lm=np.zeros((0, 2)), stokes=np.zeros((0, 4)), alpha=np.zeros(0), shape=None))
    V = r.predict().cpu().numpy()
    assert np.all(V == 0)
    D = inp["data"].astype(np.complex128)
    want = (inp["weight"] * (np.abs(D) ** 2).sum(-1)).sum()
    assert rel_err(r.chi2(), want) <= TOL[precision]["chi2"]
    r.close()


def test_identity_gains_equal_no_gains():
    inp = make_case(rime_synth.custom(10, 2, 3, 4, 2, seed_index=25), "f64")
    inp["gains"] = None
    V0, c0 = gpu_run(inp, "f64")
    inp["gains"] = np.broadcast_to(np.eye(2, dtype=complex), (2, 10, 3, 2, 2)).copy()
    V1, c1 = gpu_run(inp, "f64")
    np.testing.assert_array_equal(V0, V1)
    assert c0 == c1


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_chi2_is_deterministic(precision):
    inp = make_case(rime_synth.custom(20, 3, 4, 8, 8, seed_index=26), precision)
    r = gpu_ctx(inp, precision)
    a, b = r.chi2(), r.chi2()
    assert a == b
    r.close()


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_table4_7ant_full_size(precision):
    # the antenna sweep's smallest array at its full size (100 timesteps, 64
    # channels, 50 point + 50 Gaussian sources), element by element, through
    # the kernel the library picks for it (the narrow one) and the tiled one
    inp = make_case(rime_synth.custom(7, 100, 64, 50, 50, seed_index=207), precision)
    cref = oracle_chi2(inp)
    for kernel in (None, "tiled"):
        V, chi = gpu_run(inp, precision, kernel)
        assert vis_err(V, inp["oracle_vis"]) <= TOL[precision]["vis"], (kernel, vis_err(V, inp["oracle_vis"]))
        assert rel_err(chi, cref) <= TOL[precision]["chi2"], (kernel, chi, cref)


def test_kernel_choice_is_validated():
    import paper_1501_07719_gb300 as R
    inp = make_case(rime_synth.custom(46, 1, 1, 1, 0, seed_index=34), "f64")
    r = gpu_ctx(inp, "f64")
    with pytest.raises(R.RimeError) as e:
        r.set_kernel(R.RIME_KERNEL_NARROW)
    assert "45 antennas" in str(e.value)
    with pytest.raises(R.RimeError):
        r.set_kernel(7)
    r.set_kernel(R.RIME_KERNEL_TILED)
    r.set_kernel(R.RIME_KERNEL_AUTO)
    r.close()


def test_full_64ant_workload_sampled_fp32():
    """The 64-antenna, 100-timestep, 64-channel, 100 point + 100 Gaussian
    workload in the benchmark's launch configuration: sampled visibilities
    against the oracle, and chi^2 against the FP64 sum of w |V - D|^2 over the
    visibilities the same kernel predicts."""
    import torch
    inp = rime_synth.make_inputs("64ant-100t-64ch-100pt100g", precision="f32")
    import paper_1501_07719_gb300 as R
    r = R.Rime(inp, R.RIME_FP32, weight=inp["weight"].astype(np.float32))
    r.set_gains(inp["gains"])
    r.set_sources(inp["sources"])
    V = r.predict()
    D = (V.cpu().numpy().astype(np.complex128) + inp["noise"]).astype(np.complex64)
    r.set_data(D, inp["weight"].astype(np.float32))
    chi = r.chi2()
    Vh = V.cpu().numpy().astype(np.complex128)
    want = (inp["weight"] * (np.abs(Vh - D.astype(np.complex128)) ** 2).sum(-1)).sum()
    assert rel_err(chi, want) <= 1e-5
    rng = np.random.default_rng(0)
    n = 256
    t = rng.integers(0, 100, n)
    bl = rng.integers(0, 2016, n)
    k = rng.integers(0, 64, n)
    p, q = rime_synth.baseline_pairs(64)
    ref = oracle.Problem(inp).vis_list(t, p[bl], q[bl], k)
    got = Vh[t, bl, k]
    assert np.abs(got - ref).max() / np.abs(ref).max() <= TOL["f32"]["vis"]
    r.close()
    del V
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def full_64ant():
    """The benchmark's 64-antenna, 100-timestep, 64-channel, 100 point + 100
    Gaussian workload with data = the oracle's model + the seeded noise, every
    input rounded to FP32 (so that the same values serve the FP32 and the FP64
    runs), and the oracle's chi^2 of it."""
    inp = rime_synth.make_inputs("64ant-100t-64ch-100pt100g", precision="f32")
    V = oracle.Problem(inp).predict()
    inp["data"] = rime_synth.observe(V, inp["noise"], "f32")
    del V
    inp["want_chi2"] = oracle.Problem(inp, data=inp["data"]).chi2()
    return inp


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_full_64ant_chi2_against_oracle(full_64ant, precision):
    """rime_chi2 of the whole benchmark workload, in the benchmark's launch
    configuration, against the FP64 oracle's chi^2 of the same inputs."""
    import paper_1501_07719_gb300 as R
    inp = full_64ant
    prec = R.RIME_FP32 if precision == "f32" else R.RIME_FP64
    cd, rd = (np.complex64, np.float32) if precision == "f32" else (np.complex128, np.float64)
    r = R.Rime(inp, prec, data=inp["data"].astype(cd), weight=inp["weight"].astype(rd))
    r.set_gains(inp["gains"])
    r.set_sources(inp["sources"])
    got = r.chi2()
    r.close()
    assert rel_err(got, inp["want_chi2"]) <= TOL[precision]["chi2"], (got, inp["want_chi2"])


def test_invalid_source_is_reported_and_outputs_untouched():
    import paper_1501_07719_gb300 as R
    inp = make_case(rime_synth.custom(6, 2, 3, 3, 0, seed_index=27), "f64")
    r = gpu_ctx(inp, "f64")
    bad = {k: v.copy() for k, v in inp["sources"].items()}
    bad["lm"][1] = [0.8, 0.7]          # l^2 + m^2 >= 1
    r.set_sources(bad)
    out = r.torch.full((2, 15, 3, 4), 7.0 + 1j, dtype=r.cdtype, device="cuda")
    r.predict(out)
    with pytest.raises(R.RimeError) as e:
        r.sync()
    assert e.value.status == R._abi.RIME_E_INVALID and "sources" in str(e.value)
    assert bool((out == 7.0 + 1j).all())
    with pytest.raises(R.RimeError):
        r.chi2()
    r.set_sources(inp["sources"])       # valid again
    assert rel_err(r.chi2(), oracle_chi2(inp)) <= 1e-10
    r.close()


def test_nonfinite_data_and_negative_weight_are_rejected():
    import paper_1501_07719_gb300 as R
    inp = make_case(rime_synth.custom(5, 2, 2, 2, 0, seed_index=28), "f64")
    d = inp["data"].copy()
    d[1, 3, 0, 2] = np.nan
    with pytest.raises(R.RimeError) as e:
        R.Rime(inp, R.RIME_FP64, data=d, weight=inp["weight"])
    assert e.value.status == R._abi.RIME_E_NONFINITE
    w = inp["weight"].copy()
    w[0, 0, 1] = -1.0
    with pytest.raises(R.RimeError) as e:
        R.Rime(inp, R.RIME_FP64, data=inp["data"], weight=w)
    assert e.value.status == R._abi.RIME_E_INVALID


def test_call_order_errors():
    import paper_1501_07719_gb300 as R
    inp = make_case(rime_synth.custom(5, 2, 2, 2, 0, seed_index=29), "f64", gains=False)
    r = R.Rime(inp, R.RIME_FP64)            # no data
    with pytest.raises(R.RimeError) as e:
        r.chi2()
    assert e.value.status == R._abi.RIME_E_STATE
    r.set_sources(inp["sources"])
    with pytest.raises(R.RimeError) as e:
        r.chi2()
    assert e.value.status == R._abi.RIME_E_STATE
    r.set_data(inp["data"], inp["weight"])
    assert rel_err(r.chi2(), oracle_chi2(inp)) <= 1e-10
    r.close()


def test_ln_norm():
    inp = make_case(rime_synth.custom(6, 2, 3, 2, 0, seed_index=30), "f64")
    r = gpu_ctx(inp, "f64")
    want = oracle.Problem(inp, data=inp["data"]).ln_norm()
    assert rel_err(r.ln_norm(), want) <= 1e-12
    r.close()
