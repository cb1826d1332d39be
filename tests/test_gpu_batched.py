"""Batched chi^2 (rime_chi2_batched): every set's chi^2 against the FP64
oracle, against the plain one-set path, across launch configurations and
under CUDA graph capture, and at the 512-set size on sampled sets."""
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


def set_sources(sets, j):
    o = sets["offsets"]
    return {k: v[o[j]:o[j + 1]] for k, v in sets["sources"].items()}


def with_empty_sets(sets, at):
    """The same sources with empty sets inserted before the given set indices."""
    o = list(sets["offsets"])
    for j in sorted(at, reverse=True):
        o.insert(j, o[j])
    return dict(offsets=np.asarray(o, dtype=np.int32), sources=sets["sources"])


def nsets(sets):
    return len(sets["offsets"]) - 1


CASES = {
    # 13 antennas: one diagonal unit with a ragged head; sets of 1..40 sources
    "13ant": dict(wl=rime_synth.custom(13, 3, 5, 6, 4, seed_index=61, nsets=7, set_nsrc=(1, 40)),
                  empty=[0, 3, 7]),
    # 70 antennas: several units (diagonal and off-diagonal)
    "70ant": dict(wl=rime_synth.custom(70, 2, 3, 3, 2, seed_index=62, nsets=4, set_nsrc=(1, 20)),
                  empty=[2]),
}


def _case(name, precision):
    c = CASES[name]
    inp = make_case(c["wl"], precision)
    inp["sets"] = with_empty_sets(inp["sets"], c["empty"])
    return inp


def _run(r, sets):
    out = r.chi2_batched(sets["offsets"], sets["sources"])
    r.sync()
    return out.cpu().numpy()


def _kernel(r, kernel):
    """None: the library's choice (13 antennas: one small-array launch per
    set); "tiled": the persistent launch of the tiled kernel (FP32)."""
    import paper_1501_07719_gb300 as R
    if kernel == "tiled":
        r.set_kernel(R.RIME_KERNEL_TILED)


@pytest.mark.parametrize("kernel", [None, "tiled"])
@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("case", list(CASES))
def test_batched_matches_oracle(case, precision, kernel):
    inp = _case(case, precision)
    sets = inp["sets"]
    r = gpu_ctx(inp, precision)
    _kernel(r, kernel)
    got = _run(r, sets)
    r.close()
    for j in range(nsets(sets)):
        want = oracle.Problem(inp, sources=set_sources(sets, j), data=inp["data"]).chi2()
        assert rel_err(got[j], want) <= TOL[precision]["chi2"], (j, got[j], want)


@pytest.mark.parametrize("kernel", [None, "tiled"])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_batched_equals_plain_per_set(precision, kernel):
    inp = _case("13ant", precision)
    sets = inp["sets"]
    r = gpu_ctx(inp, precision)
    _kernel(r, kernel)
    got = _run(r, sets)
    for j in range(nsets(sets)):
        r.set_sources(set_sources(sets, j))
        plain = r.chi2()
        if precision == "f64" or kernel is None:
            # one launch per set of the kernel a plain call uses
            assert got[j] == plain, j
        else:
            # the persistent FP32 launch runs the tiled kernel's per-item body:
            # the same FP32 block sums as a plain tiled call, added in another order
            assert abs(got[j] - plain) <= 1e-12 * plain, j
    r.close()


@pytest.mark.parametrize("kernel", [None, "tiled"])
def test_batched_with_exponential_disks(kernel):
    """Sets whose extended sources are partly exponential disks (source kind 1):
    each set against the oracle, and equal to its plain call."""
    inp = _case("13ant", "f32")
    sets = inp["sets"]
    rng = np.random.default_rng(5)
    ext = sets["sources"]["shape"][:, 0] > 0
    sets["sources"]["kind"] = (ext & (rng.uniform(size=ext.size) < 0.5)).astype(np.int32)
    assert sets["sources"]["kind"].sum() > 0
    r = gpu_ctx(inp, "f32")
    _kernel(r, kernel)
    got = _run(r, sets)
    for j in range(nsets(sets)):
        want = oracle.Problem(inp, sources=set_sources(sets, j), data=inp["data"]).chi2()
        assert rel_err(got[j], want) <= TOL["f32"]["chi2"], (j, got[j], want)
        r.set_sources(set_sources(sets, j))
        plain = r.chi2()
        assert abs(got[j] - plain) <= 1e-12 * plain, j
    r.close()


def test_batched_configurations_agree_bitwise():
    inp = _case("13ant", "f32")
    sets = inp["sets"]
    r = gpu_ctx(inp, "f32")
    _kernel(r, "tiled")   # the persistent launch, whose configuration this varies
    ref = _run(r, sets)
    for cpi in (1, 2, 4):
        for bps in (1, 2):
            for order in (0, 1):
                for gs in (1, 3, 64):
                    r.set_batched_config(cpi, bps, order, gs)
                    got = _run(r, sets)
                    cfg = r.batched_config()
                    assert (cfg["channels_per_item"], cfg["order"], cfg["sets_per_item"]) == (cpi, order, gs)
                    assert not cfg["tuned"]
                    np.testing.assert_array_equal(got, ref)
    r.close()


def test_tuner_picks_its_fastest_trial():
    inp = _case("70ant", "f32")
    r = gpu_ctx(inp, "f32")
    _run(r, inp["sets"])
    cfg = r.batched_config()
    r.close()
    assert cfg["tuned"] and len(cfg["trials"]) >= 4
    best = min(cfg["trials"], key=lambda x: x["ms"])
    assert (cfg["channels_per_item"], cfg["blocks_per_sm"], cfg["order"], cfg["sets_per_item"]) == \
        (best["channels_per_item"], best["blocks_per_sm"], best["order"], best["sets_per_item"])
    assert all(t["ms"] > 0 for t in cfg["trials"])


@pytest.mark.parametrize("kernel", [None, "tiled"])
def test_batched_under_cuda_graph_replay(kernel):
    """Captured once; replays re-read the device source arrays updated in place."""
    import torch
    inp = _case("13ant", "f32")
    sets = inp["sets"]
    dev = {k: torch.tensor(np.ascontiguousarray(v), dtype=torch.float64, device="cuda")
           for k, v in sets["sources"].items()}
    r = gpu_ctx(inp, "f32")
    out = torch.zeros(nsets(sets), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    r2 = gpu_ctx(inp, "f32")   # reference context on the default stream
    import paper_1501_07719_gb300 as R
    rc = R.Rime(inp, R.RIME_FP32, data=inp["data"], weight=np.asarray(inp["weight"], np.float32), stream=s)
    rc.set_gains(inp["gains"])
    _kernel(rc, kernel)
    _kernel(r2, kernel)
    rc.chi2_batched(sets["offsets"], dev, out=out)   # first call: buffers and tuning
    rc.sync()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin(capture_error_mode="relaxed")
        rc.chi2_batched(sets["offsets"], dev, out=out)
        g.capture_end()
    for scale in (1.0, 1.25, 0.8):
        with torch.no_grad():
            dev["stokes"].copy_(torch.tensor(sets["sources"]["stokes"] * scale, device="cuda"))
            dev["lm"].copy_(torch.tensor(sets["sources"]["lm"] * scale, device="cuda"))
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            g.replay()
        s.synchronize()
        want = r2.chi2_batched(sets["offsets"], {k: v.cpu().numpy() for k, v in dev.items()})
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), want.cpu().numpy())
    rc.close()
    r.close()
    r2.close()


def test_batched_full_size_sampled_sets():
    """The 512-set workload (64 antennas, 50 timesteps, 32 channels, sets of
    5..500 sources): sampled sets against the plain path, and the two
    smallest against the oracle. Data: noise only (any data serve chi^2)."""
    inp = rime_synth.make_inputs("64ant-50t-32ch-512sets", precision="f32")
    inp["data"] = rime_synth.observe(np.zeros_like(inp["noise"]), inp["noise"], "f32")
    sets = inp["sets"]
    r = gpu_ctx(inp, "f32")
    got = _run(r, sets)
    assert got.shape == (512,) and np.all(np.isfinite(got)) and np.all(got > 0)
    counts = np.diff(sets["offsets"])
    order = np.argsort(counts, kind="stable")
    rng = np.random.default_rng(5)
    sample = sorted(set([int(order[0]), int(order[1]), int(order[-1])] + list(rng.choice(512, 5, replace=False))))
    for j in sample:
        r.set_sources(set_sources(sets, j))
        plain = r.chi2()
        assert abs(got[j] - plain) <= 1e-12 * plain, (j, got[j], plain)
    r.close()
    for j in order[:2]:
        want = oracle.Problem(inp, sources=set_sources(sets, int(j)), data=inp["data"]).chi2()
        assert rel_err(got[j], want) <= TOL["f32"]["chi2"], (j, got[j], want)


def test_batched_512_sets_against_oracle_on_a_slice():
    """All 512 sets of the batched workload (5..500 sources) on its first 4
    timesteps: the smallest, the largest and 6 seeded sets against the FP64
    oracle (chi^2 tolerance of the FP32 path)."""
    inp = rime_synth.make_inputs("64ant-50t-32ch-512sets", precision="f32")
    nt = 4
    sl = dict(inp, ntime=nt, uvw=inp["uvw"][:nt], gains=inp["gains"][:nt], weight=inp["weight"][:nt],
              noise=inp["noise"][:nt])
    sl["data"] = rime_synth.observe(oracle.Problem(sl).predict(), sl["noise"], "f32")
    sets = inp["sets"]
    r = gpu_ctx(sl, "f32")
    got = _run(r, sets)
    r.close()
    counts = np.diff(sets["offsets"])
    rng = np.random.default_rng(11)
    pick = {int(np.argmin(counts)), int(np.argmax(counts))} | {int(j) for j in rng.choice(512, 6, replace=False)}
    for j in sorted(pick):
        want = oracle.Problem(sl, sources=set_sources(sets, j), data=sl["data"]).chi2()
        assert rel_err(got[j], want) <= TOL["f32"]["chi2"], (j, counts[j], got[j], want)


def test_batched_argument_errors():
    import paper_1501_07719_gb300 as R
    inp = _case("13ant", "f64")
    sets = inp["sets"]
    r = gpu_ctx(inp, "f64")
    src = sets["sources"]
    o = sets["offsets"].copy()
    j = int(np.argmax(np.diff(o) > 0))           # a non-empty set
    dec = o.copy()
    dec[j + 1] = o[j] - 1                        # offsets decrease
    bad = [np.concatenate([[1], o[1:]]),          # first offset not 0
           np.concatenate([o[:-1], [o[-1] + 1]]),  # last offset past the sources
           dec]
    for b in bad:
        with pytest.raises(R.RimeError) as e:
            r.chi2_batched(b.astype(np.int32), src)
        assert e.value.status == R._abi.RIME_E_INVALID
    out = r.chi2_batched(np.zeros(1, np.int32), {k: v[:0] for k, v in src.items()})
    assert out.numel() == 0
    with pytest.raises(R.RimeError):
        r.set_batched_config(3, 2, 0)
    with pytest.raises(R.RimeError):
        r.set_batched_config(1, 2, 0, 0)
    r.close()


def test_batched_invalid_source_leaves_output_untouched():
    import torch
    import paper_1501_07719_gb300 as R
    inp = _case("13ant", "f32")
    sets = inp["sets"]
    src = {k: v.copy() for k, v in sets["sources"].items()}
    src["lm"][sets["offsets"][2] + 1, 0] = np.nan
    r = gpu_ctx(inp, "f32")
    out = torch.full((nsets(sets),), -1.0, dtype=torch.float64, device="cuda")
    r.chi2_batched(sets["offsets"], src, out=out)
    with pytest.raises(R.RimeError) as e:
        r.sync()
    assert e.value.status == R._abi.RIME_E_NONFINITE
    assert torch.all(out == -1.0)
    r.close()
