"""rime_chi2_streamed: chi^2 of data and weights held in host memory, copied to
the GPU in time chunks overlapped with the fused kernel (the two-solver time
subdivision of Sec. 4.4). Parity with the oracle and with the resident-data
call, for chunk lengths from one timestep to the whole observation, both
direct-sum kernels and both precisions; chunk-local error reporting."""
import numpy as np
import pytest

import rime_synth
from gpu_cases import TOL, gpu_ctx, make_case, oracle_chi2, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _streamed_case(na, precision, **kw):
    wl = rime_synth.custom(na, 7, 5, 9, 6, seed_index=40 + na)
    return make_case(wl, precision, **kw)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("na,kernel", [(13, None), (13, "tiled"), (70, None)])
def test_streamed_equals_resident_and_oracle(na, kernel, precision):
    import torch
    import paper_1501_07719_gb300 as R
    inp = _streamed_case(na, precision, pointing_sigma=0.002)
    rd = np.float64 if precision == "f64" else np.float32
    w = np.asarray(inp["weight"], dtype=rd)
    r = gpu_ctx(inp, precision)
    if kernel == "tiled":
        r.set_kernel(R.RIME_KERNEL_TILED)
    resident = r.chi2()
    cref = oracle_chi2(inp)
    pinned_d = torch.from_numpy(np.ascontiguousarray(inp["data"])).pin_memory()
    pinned_w = torch.from_numpy(w).pin_memory()
    for chunk in (1, 2, 3, 7, 100, 0):
        got = r.chi2_streamed(pinned_d, pinned_w, chunk)
        # the same block partials, grouped per chunk before the FP64 sum
        assert rel_err(got, resident) <= 1e-13, (chunk, got, resident)
        assert rel_err(got, cref) <= TOL[precision]["chi2"], (chunk, got, cref)
    # pageable numpy arrays and device tensors are accepted too
    assert rel_err(r.chi2_streamed(inp["data"], w, 3), resident) <= 1e-13
    dev_d = pinned_d.cuda()
    assert rel_err(r.chi2_streamed(dev_d, torch.from_numpy(w).cuda(), 4), resident) <= 1e-13
    # the resident-data call still sees its own data afterwards
    assert r.chi2() == resident
    r.close()


def test_streamed_long_source_list_fp32():
    """500 sources in FP32: every chunk kernel folds segments of its source
    sum into per-block running sums, and the two kernel streams' chunks run
    side by side, each with its own scratch."""
    import torch
    inp = make_case(rime_synth.custom(40, 6, 3, 250, 250, seed_index=47), "f32")
    w = np.asarray(inp["weight"], dtype=np.float32)
    r = gpu_ctx(inp, "f32")
    resident = r.chi2()
    cref = oracle_chi2(inp)
    assert rel_err(resident, cref) <= TOL["f32"]["chi2"]
    pinned_d = torch.from_numpy(np.ascontiguousarray(inp["data"])).pin_memory()
    pinned_w = torch.from_numpy(w).pin_memory()
    for chunk in (1, 2, 3, 0):
        got = r.chi2_streamed(pinned_d, pinned_w, chunk)
        assert rel_err(got, resident) <= 1e-13, (chunk, got, resident)
    r.close()


@pytest.mark.parametrize("kernel", [None, "tiled"])
def test_streamed_follows_uploads_queued_before_it(kernel):
    """The chunk copies run ahead of the context's stream (a ring of up to
    four buffers); the chunk kernels still see the gains and sources set just
    before the call, over more chunks than buffers."""
    import copy
    import torch
    import paper_1501_07719_gb300 as R
    inp = _streamed_case(13, "f32")
    r = gpu_ctx(inp, "f32")
    if kernel == "tiled":
        r.set_kernel(R.RIME_KERNEL_TILED)
    w = np.asarray(inp["weight"], dtype=np.float32)
    pinned_d = torch.from_numpy(np.ascontiguousarray(inp["data"])).pin_memory()
    pinned_w = torch.from_numpy(w).pin_memory()
    for step in range(3):
        src = copy.deepcopy(inp["sources"])
        src["stokes"] = src["stokes"] * (1.0 + 0.25 * step)
        r.set_gains(inp["gains"] * (1.0 - 0.1 * step))
        r.set_sources(src)
        got = r.chi2_streamed(pinned_d, pinned_w, 1)
        expect = r.chi2()
        assert rel_err(got, expect) <= 1e-13, (step, got, expect)
    r.close()


def test_streamed_unit_weights_and_context_without_data():
    import paper_1501_07719_gb300 as R
    inp = _streamed_case(9, "f64")
    inp["weight"] = np.ones_like(inp["weight"])
    r = R.Rime(inp, R.RIME_FP64)            # no data on the device at all
    r.set_gains(inp["gains"])
    r.set_sources(inp["sources"])
    got = r.chi2_streamed(inp["data"], None, 2)
    assert rel_err(got, oracle_chi2(inp)) <= TOL["f64"]["chi2"]
    with pytest.raises(R.RimeError):
        r.chi2()                           # the context itself has no data
    r.close()


def test_streamed_chunk_length_choice():
    import paper_1501_07719_gb300 as R
    inp = _streamed_case(70, "f32")
    r = gpu_ctx(inp, "f32")
    n = r.stream_chunk_ntime()
    assert 1 <= n <= inp["ntime"]
    r.close()
    wl = rime_synth.workload("64ant-100t-64ch-100pt100g", ntime=100)
    big = rime_synth.make_inputs(wl, precision="f32", noise=False)
    r = R.Rime(big, R.RIME_FP32)
    n = r.stream_chunk_ntime()
    # about one wave of 2 blocks per SM (64 channels x 1 unit per timestep)
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    assert n == min(100, -(-2 * nsm // 64)), (n, nsm)
    r.close()


def test_streamed_bad_chunk_is_reported_with_its_global_index_and_cleared():
    import paper_1501_07719_gb300 as R
    inp = _streamed_case(9, "f64")
    r = gpu_ctx(inp, "f64")
    good = r.chi2()
    nvis_t = inp["nbl"] * inp["nchan"]
    bad = np.array(inp["data"], copy=True)
    bad[5, 3, 2, 1] = np.nan                # timestep 5: the third chunk of 2
    with pytest.raises(R.RimeError) as e:
        r.chi2_streamed(bad, inp["weight"], 2)
    assert e.value.status == R._abi.RIME_E_NONFINITE
    assert f"element {5 * nvis_t + 3 * inp['nchan'] + 2}" in str(e.value)
    w = np.array(inp["weight"], copy=True)
    w[6, 0, 0] = -1.0
    with pytest.raises(R.RimeError) as e:
        r.chi2_streamed(inp["data"], w, 3)
    assert e.value.status == R._abi.RIME_E_INVALID and "negative weight" in str(e.value)
    # the errors concerned those calls only
    assert r.chi2() == good
    assert rel_err(r.chi2_streamed(inp["data"], inp["weight"], 2), good) <= 1e-13
    r.close()
