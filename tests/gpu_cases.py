"""Shared helpers for the GPU parity tests: seeded cases with data made by
the oracle, and runs of the CUDA path through the C ABI."""
import numpy as np

import oracle
import rime_synth

# tolerances for the two compute precisions (visibilities: max |dV| / max |V|;
# chi^2: relative)
TOL = {"f64": dict(vis=1e-12, chi2=1e-10), "f32": dict(vis=1e-4, chi2=1e-4)}


# the Jinc beam (beam_model 1) with the constant of a 25 m dish, so that the
# seeded sources (|l|, |m| < 0.01) fall in its main lobe, first null and
# first (negative) sidelobe
JINC = dict(beam_model=1, beam_c=262.0)


def make_case(wl, precision="f64", pointing_sigma=0.0, time_varying=False, seed=None,
              gains=True, unit_weights=None, beam_model=0, beam_c=None, disk_fraction=0.0):
    inp = rime_synth.make_inputs(wl, precision=precision, seed=seed,
                                 pointing_sigma=pointing_sigma, time_varying=time_varying,
                                 beam_model=beam_model, beam_c=beam_c, disk_fraction=disk_fraction)
    if not gains:
        inp["gains"] = None
    if unit_weights:
        inp["weight"] = np.ones_like(inp["weight"])
    V = oracle.Problem(inp).predict()
    inp["data"] = rime_synth.observe(V, inp["noise"], precision)
    inp["oracle_vis"] = V
    return inp


def oracle_chi2(inp):
    return oracle.Problem(inp, data=inp["data"]).chi2()


def gpu_ctx(inp, precision):
    import paper_1501_07719_gb300 as R
    prec = R.RIME_FP64 if precision == "f64" else R.RIME_FP32
    rd = np.float64 if precision == "f64" else np.float32
    r = R.Rime(inp, prec, data=inp.get("data"), weight=np.asarray(inp["weight"], dtype=rd))
    if inp.get("gains") is not None:
        r.set_gains(inp["gains"])
    r.set_sources(inp["sources"])
    return r


def gpu_run(inp, precision, kernel=None):
    """Predict and chi^2 on the GPU; kernel: None (the library's choice),
    "tiled" or "narrow"."""
    import paper_1501_07719_gb300 as R
    r = gpu_ctx(inp, precision)
    if kernel is not None:
        r.set_kernel({"tiled": R.RIME_KERNEL_TILED, "narrow": R.RIME_KERNEL_NARROW}[kernel])
    V = r.predict().cpu().numpy()
    chi = r.chi2() if inp.get("data") is not None else None
    r.close()
    return V, chi


def vis_err(V, Vref):
    return np.abs(V - Vref).max() / np.abs(Vref).max()


def rel_err(a, b):
    return abs(a - b) / abs(b)
