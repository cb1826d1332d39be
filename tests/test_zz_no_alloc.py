"""rime_chi2_noalloc: the chi^2 entry point for callers that cannot allocate
device memory (for example code running inside a framework whose memory pool
has reserved the GPU, or a latency-critical loop that cannot afford
cudaMalloc's device synchronisation). It keeps every intermediate in one
fixed-size array inside the library instead of allocating.

Checked through the C ABI against the context API's rime_chi2 on the same
inputs, on two calls in a row (the second call reuses the array the first one
left behind). This file is collected last on purpose."""
import numpy as np
import pytest

import rime_synth
from gpu_cases import TOL, gpu_ctx, make_case, rel_err

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
                gains=dev(inp["gains"], torch.complex128),
                lm=dev(src["lm"], torch.float64), stokes=dev(src["stokes"], torch.float64),
                alpha=dev(src["alpha"], torch.float64), shape=dev(src["shape"], torch.float64))


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_noalloc_chi2_matches_context_chi2_on_two_calls(precision):
    import torch
    import paper_1501_07719_gb300 as R
    inp = make_case(rime_synth.custom(20, 3, 5, 10, 8, seed_index=40), precision, pointing_sigma=0.002)
    r = gpu_ctx(inp, precision)
    want = r.chi2()
    r.close()
    args = _device_args(inp, precision)
    prec = R.RIME_FP64 if precision == "f64" else R.RIME_FP32
    for call in range(2):
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        R.rime_chi2_noalloc(inp["na"], inp["ntime"], inp["nchan"], prec, chi2_dev=out,
                            stream=torch.cuda.current_stream().cuda_stream,
                            ref_freq_hz=inp["ref_freq_hz"], beam_c=inp["beam_c"], **args)
        got = float(out.item())
        assert rel_err(got, want) <= TOL[precision]["chi2"], (call, got, want)


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
