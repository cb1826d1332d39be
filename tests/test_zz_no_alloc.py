"""rime_chi2_noalloc: the chi^2 entry point for callers that cannot allocate
device memory (for example code running inside a framework whose memory pool
has reserved the GPU, or a latency-critical loop that cannot afford
cudaMalloc's device synchronisation). It keeps every intermediate in one
fixed-size array inside the library instead of allocating.

Checked through the C ABI against the FP64 oracle's chi^2 and the context
API's rime_chi2 on the same inputs, on two calls in a row (the second call
reuses the array the first one left behind), through both direct kernels
(the small-array kernel at 20 antennas, the tiled kernels at 48 and 64),
without gains, with a long source list (the FP32 running sums), and its
rejections: a NaN in the data (output untouched), host memory, a problem
beyond the fixed array. This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import oracle
import rime_synth
from gpu_cases import TOL, gpu_ctx, make_case, oracle_chi2, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _device_args(inp, precision):
    import torch
    cd = torch.complex128 if precision == "f64" else torch.complex64
    rd = torch.float64 if precision == "f64" else torch.float32
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)
    src = inp["sources"]
    return dict(freq_hz=dev(inp["freq"], torch.float64), uvw=dev(inp["uvw"], torch.float64),
                pointing=None if inp["pointing"] is None else dev(inp["pointing"], torch.float64),
                data=dev(inp["data"], cd), weight=dev(inp["weight"], rd),
                gains=None if inp["gains"] is None else dev(inp["gains"], torch.complex128),
                lm=dev(src["lm"], torch.float64), stokes=dev(src["stokes"], torch.float64),
                alpha=dev(src["alpha"], torch.float64), shape=dev(src["shape"], torch.float64))


def _noalloc(inp, precision, args, out):
    import torch
    import paper_1501_07719_gb300 as R
    prec = R.RIME_FP64 if precision == "f64" else R.RIME_FP32
    R.rime_chi2_noalloc(inp["na"], inp["ntime"], inp["nchan"], prec, chi2_dev=out,
                        stream=torch.cuda.current_stream().cuda_stream,
                        ref_freq_hz=inp["ref_freq_hz"], beam_c=inp["beam_c"], **args)


CASES = {
    # small-array kernel, pointing errors
    "20ant": dict(wl=rime_synth.custom(20, 3, 5, 10, 8, seed_index=40), pointing_sigma=0.002),
    # tiled kernels: FP64 32-antenna units (two row blocks), FP32 one 64-antenna unit
    "48ant": dict(wl=rime_synth.custom(48, 2, 3, 6, 5, seed_index=41)),
    "64ant": dict(wl=rime_synth.custom(64, 2, 3, 6, 5, seed_index=42)),
    # identity gains (gains = NULL)
    "40ant-no-gains": dict(wl=rime_synth.custom(40, 2, 2, 5, 4, seed_index=43), gains=False),
}


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("case", list(CASES))
def test_noalloc_chi2_matches_oracle_on_two_calls(case, precision):
    import torch
    inp = make_case(precision=precision, **CASES[case])
    want = oracle_chi2(inp)
    r = gpu_ctx(inp, precision)
    ctx_chi = r.chi2()
    r.close()
    args = _device_args(inp, precision)
    for call in range(2):
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        _noalloc(inp, precision, args, out)
        got = float(out.item())
        assert rel_err(got, want) <= TOL[precision]["chi2"], (call, got, want)
        assert rel_err(got, ctx_chi) <= TOL[precision]["chi2"], (call, got, ctx_chi)


def test_noalloc_long_source_list_fp32():
    """More sources than one FP32 register segment holds: the tiled kernel's
    running sums live in the fixed array too (as many blocks as fit)."""
    import torch
    inp = make_case(rime_synth.custom(40, 2, 2, 400, 200, seed_index=44), "f32")
    want = oracle_chi2(inp)
    args = _device_args(inp, "f32")
    for call in range(2):
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        _noalloc(inp, "f32", args, out)
        assert rel_err(float(out.item()), want) <= TOL["f32"]["chi2"], call


def test_noalloc_reports_nonfinite_data_and_leaves_output_untouched():
    import torch
    import paper_1501_07719_gb300 as R
    inp = make_case(rime_synth.custom(64, 2, 2, 4, 3, seed_index=45), "f32")
    args = _device_args(inp, "f32")
    args["data"][1, 7, 0, 2] = float("nan")
    out = torch.full((1,), -7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(R.RimeError) as e:
        _noalloc(inp, "f32", args, out)
    assert e.value.status == R._abi.RIME_E_NONFINITE
    assert float(out.item()) == -7.0
    # the next call with valid data succeeds (the status in the array was cleared)
    args["data"] = _device_args(inp, "f32")["data"]
    _noalloc(inp, "f32", args, out)
    assert rel_err(float(out.item()), oracle_chi2(inp)) <= TOL["f32"]["chi2"]


def test_noalloc_rejects_host_memory():
    import torch
    import paper_1501_07719_gb300 as R
    from paper_1501_07719_gb300 import _abi
    inp = make_case(rime_synth.custom(8, 1, 2, 2, 0, seed_index=46), "f64")
    args = _device_args(inp, "f64")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    # the binding refuses a host tensor
    bad = dict(args, uvw=args["uvw"].cpu())
    with pytest.raises(TypeError):
        _noalloc(inp, "f64", bad, out)
    # the library itself refuses a host pointer before any launch
    host_freq = np.ascontiguousarray(inp["freq"], dtype=np.float64)
    k = _abi._Keep()
    dims = _abi.rime_dims(inp["na"], inp["ntime"], inp["nchan"], _abi.RIME_FP64, inp["ref_freq_hz"], inp["beam_c"])
    src = _abi.make_sources(args["lm"], args["stokes"], args["alpha"], args["shape"], k)
    s = _abi.lib().rime_chi2_noalloc(C.byref(dims), host_freq.ctypes.data, args["uvw"].data_ptr(), None,
                                     args["data"].data_ptr(), args["weight"].data_ptr(), args["gains"].data_ptr(),
                                     C.byref(src), out.data_ptr(), None)
    assert s == _abi.RIME_E_INVALID
    assert "freq_hz" in _abi.rime_last_error(None)


def test_noalloc_rejects_problems_beyond_its_fixed_scratch():
    import torch
    import paper_1501_07719_gb300 as R
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    z = lambda *s: torch.zeros(*s, dtype=torch.float64, device="cuda")
    na, nt, nc, ns = 64, 200, 64, 400          # needs far more than 32 MiB
    with pytest.raises(R.RimeError) as e:
        R.rime_chi2_noalloc(na, nt, nc, R.RIME_FP32, z(nc), z(nt, na, 3), None,
                            torch.zeros(1, dtype=torch.complex64, device="cuda"), None, None,
                            z(ns, 2), z(ns, 4), z(ns), None, out)
    assert e.value.status == R._abi.RIME_E_INVALID and "scratch" in str(e.value)
