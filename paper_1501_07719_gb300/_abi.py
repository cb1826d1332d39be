"""ctypes binding of librime.so (include/rime.h).

Argument marshalling only: every computation runs in the CUDA library. Arrays
may be numpy arrays (host memory) or torch tensors (host or device); they must
be C-contiguous with the dtype the ABI states. Errors raise RimeError.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librime.so")

RIME_OK, RIME_E_INVALID, RIME_E_STATE, RIME_E_OOM, RIME_E_CUDA, RIME_E_TIMEOUT, RIME_E_NONFINITE = range(7)
RIME_FP32, RIME_FP64 = 0, 1
RIME_TC_OFF, RIME_TC_SPLIT_BF16, RIME_TC_SPLIT_TF32, RIME_TC_SPLIT_F16 = 0, 1, 2, 3
RIME_KERNEL_AUTO, RIME_KERNEL_TILED, RIME_KERNEL_NARROW = 0, 1, 2
RIME_BEAM_COS3, RIME_BEAM_JINC = 0, 1
RIME_PIPE_FFMA, RIME_PIPE_FFMA2, RIME_PIPE_DFMA, RIME_PIPE_EX2 = 0, 1, 2, 3


class rime_dims(C.Structure):
    _fields_ = [("na", C.c_int32), ("ntime", C.c_int32), ("nchan", C.c_int32),
                ("precision", C.c_int32), ("ref_freq_hz", C.c_double), ("beam_c", C.c_double)]


class rime_sources(C.Structure):
    _fields_ = [("nsrc", C.c_int32), ("time_varying", C.c_int32), ("lm", C.c_void_p),
                ("stokes", C.c_void_p), ("alpha", C.c_void_p), ("shape", C.c_void_p), ("kind", C.c_void_p)]


class rime_batch_config(C.Structure):
    _fields_ = [("channels_per_item", C.c_int32), ("blocks_per_sm", C.c_int32), ("order", C.c_int32),
                ("sets_per_item", C.c_int32), ("tuned", C.c_int32), ("ntrials", C.c_int32),
                ("trial_cfg", (C.c_int32 * 4) * 40), ("trial_ms", C.c_float * 40)]


class RimeError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        super().__init__(f"{status_string(status)}: {message}")


_lib = None


def lib():
    """The loaded librime.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1501_07719_gb300.build` (nvcc, sm_103a)")
        L = C.CDLL(LIB_PATH)
        vp, ip = C.c_void_p, C.c_int
        L.rime_nbl.argtypes, L.rime_nbl.restype = [C.c_int32], C.c_int64
        L.rime_status_string.argtypes, L.rime_status_string.restype = [ip], C.c_char_p
        L.rime_last_error.argtypes, L.rime_last_error.restype = [vp], C.c_char_p
        L.rime_create.argtypes = [C.POINTER(vp), C.POINTER(rime_dims), vp, vp, vp, vp, vp, vp]
        L.rime_set_uvw.argtypes = [vp, vp, vp]
        L.rime_set_data.argtypes = [vp, vp, vp]
        L.rime_set_gains.argtypes = [vp, vp]
        L.rime_set_sources.argtypes = [vp, C.POINTER(rime_sources)]
        L.rime_predict.argtypes = [vp, vp]
        L.rime_chi2.argtypes = [vp, C.POINTER(C.c_double)]
        L.rime_chi2_async.argtypes = [vp, vp]
        L.rime_chi2_grad.argtypes = [vp, C.POINTER(C.c_double), vp, vp]
        L.rime_ln_norm.argtypes = [vp, C.POINTER(C.c_double)]
        L.rime_sync.argtypes = [vp]
        L.rime_destroy.argtypes, L.rime_destroy.restype = [vp], None
        L.rime_chi2_noalloc.argtypes = [C.POINTER(rime_dims), vp, vp, vp, vp, vp, vp,
                                        C.POINTER(rime_sources), vp, vp]
        L.rime_chi2_noalloc.restype = ip
        L.rime_chi2_batched.argtypes = [vp, C.c_int32, vp, C.POINTER(rime_sources), vp]
        L.rime_batched_config.argtypes = [vp, C.POINTER(rime_batch_config)]
        L.rime_set_batched_config.argtypes = [vp, C.POINTER(rime_batch_config)]
        L.rime_set_tensor_mode.argtypes = [vp, C.c_int32]
        L.rime_split_tiles.argtypes, L.rime_split_tiles.restype = [C.c_int32, vp, C.c_int32], C.c_int32
        L.rime_set_kernel.argtypes = [vp, C.c_int32]
        L.rime_set_wait_limit.argtypes, L.rime_set_wait_limit.restype = [vp, C.c_uint64], ip
        L.rime_set_beam.argtypes = [vp, C.c_int32, C.c_double]
        L.rime_chains_init.argtypes = [vp, C.c_int32]
        L.rime_chains_propose.argtypes = [vp, C.c_int32, C.POINTER(rime_sources), C.POINTER(rime_sources), vp]
        L.rime_chains_accept.argtypes = [vp, vp]
        L.rime_chi2_streamed.argtypes = [vp, vp, vp, C.c_int32, C.POINTER(C.c_double)]
        L.rime_stream_chunk_ntime.argtypes, L.rime_stream_chunk_ntime.restype = [vp], C.c_int32
        L.rime_phase_turns.argtypes, L.rime_phase_turns.restype = [C.c_int64, vp, vp, vp], ip
        L.rime_pipe_rate.argtypes, L.rime_pipe_rate.restype = [C.c_int32, C.POINTER(C.c_double)], ip
        for f in ("rime_chi2_batched", "rime_batched_config", "rime_set_batched_config", "rime_set_tensor_mode",
                  "rime_set_kernel", "rime_chi2_streamed", "rime_set_beam", "rime_chains_init",
                  "rime_chains_propose", "rime_chains_accept"):
            getattr(L, f).restype = ip
        for f in ("rime_create", "rime_set_uvw", "rime_set_data", "rime_set_gains",
                  "rime_set_sources", "rime_predict", "rime_chi2", "rime_chi2_async", "rime_chi2_grad",
                  "rime_ln_norm", "rime_sync"):
            getattr(L, f).restype = ip
        _lib = L
    return _lib


def status_string(s: int) -> str:
    try:
        return lib().rime_status_string(s).decode()
    except RuntimeError:
        return f"status {s}"


def _check(status: int, ctx=None):
    if status != RIME_OK:
        msg = lib().rime_last_error(ctx).decode()
        raise RimeError(status, msg)


# ---------------------------------------------------------------------------
# array marshalling
# ---------------------------------------------------------------------------
_TORCH_DT = {}


def _torch():
    import torch
    if not _TORCH_DT:
        _TORCH_DT.update({np.dtype(np.float32): torch.float32, np.dtype(np.float64): torch.float64,
                          np.dtype(np.complex64): torch.complex64, np.dtype(np.complex128): torch.complex128,
                          np.dtype(np.int32): torch.int32})
    return torch


class _Keep:
    """Keeps host copies alive for the duration of a call."""

    def __init__(self):
        self.refs = []

    def ptr(self, x, dtype, name):
        if x is None:
            return None
        dtype = np.dtype(dtype)
        if isinstance(x, np.ndarray) or np.isscalar(x) or isinstance(x, (list, tuple)):
            a = np.ascontiguousarray(x, dtype=dtype)
            self.refs.append(a)
            return a.ctypes.data
        torch = _torch()
        if isinstance(x, torch.Tensor):
            if x.dtype != _TORCH_DT[dtype]:
                raise TypeError(f"{name}: expected {_TORCH_DT[dtype]}, got {x.dtype}")
            if not x.is_contiguous():
                raise ValueError(f"{name}: tensor must be contiguous")
            return x.data_ptr()
        raise TypeError(f"{name}: unsupported array type {type(x)}")


def _ctype(precision):
    return (np.complex128, np.float64) if precision == RIME_FP64 else (np.complex64, np.float32)


# ---------------------------------------------------------------------------
# the C ABI, one function per entry point
# ---------------------------------------------------------------------------
def rime_nbl(na: int) -> int:
    return lib().rime_nbl(na)


def rime_create(na, ntime, nchan, precision, freq_hz, uvw, pointing=None, data=None,
                weight=None, stream=0, ref_freq_hz=1.4e9, beam_c=65.0):
    """Returns an opaque context handle (int). stream: a cudaStream_t as int."""
    L = lib()
    dims = rime_dims(na, ntime, nchan, precision, ref_freq_hz, beam_c)
    cd, rd = _ctype(precision)
    k = _Keep()
    ctx = C.c_void_p()
    s = L.rime_create(C.byref(ctx), C.byref(dims), k.ptr(freq_hz, np.float64, "freq_hz"),
                      k.ptr(uvw, np.float64, "uvw"), k.ptr(pointing, np.float64, "pointing"),
                      k.ptr(data, cd, "data"), k.ptr(weight, rd, "weight"), stream or None)
    _check(s, None)
    return ctx.value


def rime_set_uvw(ctx, uvw, pointing=None):
    k = _Keep()
    _check(lib().rime_set_uvw(ctx, k.ptr(uvw, np.float64, "uvw"), k.ptr(pointing, np.float64, "pointing")), ctx)


def rime_set_data(ctx, precision, data, weight=None):
    cd, rd = _ctype(precision)
    k = _Keep()
    _check(lib().rime_set_data(ctx, k.ptr(data, cd, "data"), k.ptr(weight, rd, "weight")), ctx)


def rime_set_gains(ctx, gains):
    k = _Keep()
    _check(lib().rime_set_gains(ctx, k.ptr(gains, np.complex128, "gains")), ctx)


def make_sources(lm, stokes, alpha, shape=None, keep: _Keep | None = None, kind=None) -> rime_sources:
    k = keep if keep is not None else _Keep()
    nsrc = int(alpha.shape[0])
    tv = 1 if len(stokes.shape) == 3 else 0
    return rime_sources(nsrc, tv, k.ptr(lm, np.float64, "lm"), k.ptr(stokes, np.float64, "stokes"),
                        k.ptr(alpha, np.float64, "alpha"), k.ptr(shape, np.float64, "shape"),
                        k.ptr(kind, np.int32, "kind"))


def rime_set_sources(ctx, lm, stokes, alpha, shape=None, kind=None):
    """kind: [nsrc] int32 morphology of the sources with a shape (0 Gaussian,
    1 exponential disk) or None."""
    k = _Keep()
    src = make_sources(lm, stokes, alpha, shape, k, kind)
    _check(lib().rime_set_sources(ctx, C.byref(src)), ctx)


def rime_predict(ctx, vis_out):
    """vis_out: a device tensor [ntime][nbl][nchan][4] of the context's complex type."""
    _check(lib().rime_predict(ctx, vis_out.data_ptr()), ctx)


def rime_chi2(ctx) -> float:
    out = C.c_double()
    _check(lib().rime_chi2(ctx, C.byref(out)), ctx)
    return out.value


def rime_chi2_async(ctx, chi2_dev):
    """chi2_dev: a float64 device tensor with at least one element."""
    _check(lib().rime_chi2_async(ctx, chi2_dev.data_ptr()), ctx)


def rime_chi2_grad(ctx, grad_src, grad_gains=None) -> float:
    """grad_src: float64 device tensor [nsrc][10]; grad_gains: complex128 device
    tensor [ntime][na][nchan][2][2] or None. Returns chi^2."""
    out = C.c_double()
    gs = grad_src.data_ptr() if grad_src is not None and grad_src.numel() else None
    gg = grad_gains.data_ptr() if grad_gains is not None else None
    _check(lib().rime_chi2_grad(ctx, C.byref(out), gs, gg), ctx)
    return out.value


def rime_ln_norm(ctx) -> float:
    out = C.c_double()
    _check(lib().rime_ln_norm(ctx, C.byref(out)), ctx)
    return out.value


def rime_sync(ctx):
    _check(lib().rime_sync(ctx), ctx)


def rime_last_error(ctx) -> str:
    return lib().rime_last_error(ctx).decode()


def rime_destroy(ctx):
    if ctx:
        lib().rime_destroy(ctx)


def rime_chi2_noalloc(na, ntime, nchan, precision, freq_hz, uvw, pointing, data, weight, gains,
                      lm, stokes, alpha, shape, chi2_dev, stream=0, ref_freq_hz=1.4e9, beam_c=65.0, kind=None):
    """The chi^2 entry point that allocates no device memory (see include/rime.h).
    Every array argument must be a CUDA tensor on the current device (or None
    where the ABI allows NULL); chi2_dev receives the value."""
    torch = _torch()
    dev = torch.cuda.current_device()
    named = dict(freq_hz=freq_hz, uvw=uvw, pointing=pointing, data=data, weight=weight, gains=gains,
                 lm=lm, stokes=stokes, alpha=alpha, shape=shape, kind=kind, chi2_dev=chi2_dev)
    for name, x in named.items():
        if x is None:
            continue
        if not isinstance(x, torch.Tensor) or not x.is_cuda or x.device.index != dev:
            raise TypeError(f"rime_chi2_noalloc: {name} must be a CUDA tensor on the current device (cuda:{dev})")
    cd, rd = _ctype(precision)
    k = _Keep()
    dims = rime_dims(na, ntime, nchan, precision, ref_freq_hz, beam_c)
    src = make_sources(lm, stokes, alpha, shape, k, kind)
    s = lib().rime_chi2_noalloc(C.byref(dims), k.ptr(freq_hz, np.float64, "freq_hz"),
                                k.ptr(uvw, np.float64, "uvw"), k.ptr(pointing, np.float64, "pointing"),
                                k.ptr(data, cd, "data"), k.ptr(weight, rd, "weight"),
                                k.ptr(gains, np.complex128, "gains"), C.byref(src),
                                chi2_dev.data_ptr(), stream or None)
    _check(s, None)


def rime_chi2_batched(ctx, src_offsets, lm, stokes, alpha, shape, chi2_dev, kind=None):
    """chi^2 of each source set against the context's observation.
    src_offsets: host int32 [nsets + 1]; the source arrays hold the
    concatenated sets; chi2_dev: float64 device tensor [nsets]."""
    off = np.ascontiguousarray(src_offsets, dtype=np.int32)
    nsets = int(off.shape[0]) - 1
    k = _Keep()
    src = make_sources(lm, stokes, alpha, shape, k, kind)
    out = chi2_dev.data_ptr() if chi2_dev is not None and nsets > 0 else None
    _check(lib().rime_chi2_batched(ctx, nsets, off.ctypes.data, C.byref(src), out), ctx)


def rime_batched_config(ctx) -> dict:
    """The batched launch configuration in use and the tuner's trials."""
    c = rime_batch_config()
    _check(lib().rime_batched_config(ctx, C.byref(c)), ctx)
    trials = [dict(channels_per_item=c.trial_cfg[i][0], blocks_per_sm=c.trial_cfg[i][1],
                   order=c.trial_cfg[i][2], sets_per_item=c.trial_cfg[i][3], ms=float(c.trial_ms[i]))
              for i in range(c.ntrials)]
    return dict(channels_per_item=c.channels_per_item, blocks_per_sm=c.blocks_per_sm, order=c.order,
                sets_per_item=c.sets_per_item, tuned=bool(c.tuned), trials=trials)


def rime_set_batched_config(ctx, channels_per_item=None, blocks_per_sm=2, order=0, sets_per_item=1):
    """Fixes the batched configuration; channels_per_item=None returns to tuning."""
    if channels_per_item is None:
        _check(lib().rime_set_batched_config(ctx, None), ctx)
        return
    c = rime_batch_config(channels_per_item, blocks_per_sm, order, sets_per_item)
    _check(lib().rime_set_batched_config(ctx, C.byref(c)), ctx)


def rime_chi2_streamed(ctx, precision, data, weight=None, chunk_ntime: int = 0) -> float:
    """chi^2 of data / weights in host (ideally pinned) or device memory, copied
    to the GPU in chunks of chunk_ntime timesteps overlapped with the kernel
    (0: the library's choice)."""
    cd, rd = _ctype(precision)
    k = _Keep()
    out = C.c_double(0.0)
    _check(lib().rime_chi2_streamed(ctx, k.ptr(data, cd, "data"), k.ptr(weight, rd, "weight"), int(chunk_ntime),
                                    C.byref(out)), ctx)
    return out.value


def rime_stream_chunk_ntime(ctx) -> int:
    return int(lib().rime_stream_chunk_ntime(ctx))


def rime_set_beam(ctx, model: int, beam_c: float):
    """RIME_BEAM_COS3 (eq. 4) or RIME_BEAM_JINC, with the constant C (rad^-1 GHz^-1)."""
    _check(lib().rime_set_beam(ctx, int(model), float(beam_c)), ctx)


def rime_chains_init(ctx, nchains: int):
    """Per-chain residuals N_c = D - V for nchains chains at the context's sky model."""
    _check(lib().rime_chains_init(ctx, int(nchains)), ctx)


def rime_chains_propose(ctx, nmove: int, proposed: dict, current: dict, chi2_dev):
    """chi^2 of each chain's proposal: proposed / current are SoA source dicts of
    nchains * nmove sources (chain c: rows c*nmove .. c*nmove + nmove - 1)."""
    k = _Keep()
    p = make_sources(proposed["lm"], proposed["stokes"], proposed["alpha"], proposed.get("shape"), k,
                     proposed.get("kind"))
    c = make_sources(current["lm"], current["stokes"], current["alpha"], current.get("shape"), k,
                     current.get("kind"))
    _check(lib().rime_chains_propose(ctx, int(nmove), C.byref(p), C.byref(c), chi2_dev.data_ptr()), ctx)


def rime_chains_accept(ctx, accept):
    """accept: [nchains] flags (host); applies the last proposal of those chains."""
    a = np.ascontiguousarray(accept, dtype=np.int32)
    _check(lib().rime_chains_accept(ctx, a.ctypes.data), ctx)


def rime_set_kernel(ctx, kernel: int):
    """RIME_KERNEL_AUTO, RIME_KERNEL_TILED or RIME_KERNEL_NARROW (<= 45 antennas)."""
    _check(lib().rime_set_kernel(ctx, int(kernel)), ctx)


def rime_set_tensor_mode(ctx, mode: int):
    """RIME_TC_OFF, RIME_TC_SPLIT_BF16, RIME_TC_SPLIT_TF32 or RIME_TC_SPLIT_F16 (FP32 contexts)."""
    _check(lib().rime_set_tensor_mode(ctx, int(mode)), ctx)


def rime_split_tiles(na: int) -> np.ndarray:
    """The split modes' tile plan: [ntiles, 5] int32 rows (column group, four row groups, -1 empty)."""
    n = lib().rime_split_tiles(int(na), None, 0)
    if n < 0:
        raise RimeError(RIME_E_INVALID, f"rime_split_tiles: na = {na} out of range")
    out = np.zeros((n, 5), dtype=np.int32)
    lib().rime_split_tiles(int(na), out.ctypes.data_as(C.c_void_p), n)
    return out


def rime_phase_turns(nu_hz, tau_s) -> np.ndarray:
    """The FP32 kernels' reduced phase of eq. 3 (turns) for host arrays nu_hz, tau_s."""
    nu = np.ascontiguousarray(nu_hz, dtype=np.float64)
    tau = np.ascontiguousarray(tau_s, dtype=np.float64)
    if nu.shape != tau.shape:
        raise ValueError("nu_hz and tau_s must have the same shape")
    out = np.zeros(nu.shape, dtype=np.float32)
    _check(lib().rime_phase_turns(int(nu.size), nu.ctypes.data, tau.ctypes.data, out.ctypes.data), None)
    return out


def rime_set_wait_limit(ctx, ns: int):
    """Limit (ns) of the tensor-core kernels' bounded waits; 0: the default (about 2 s)."""
    _check(lib().rime_set_wait_limit(ctx, int(ns)), ctx)


def rime_pipe_rate(pipe: int) -> float:
    """Measured lane operations per second of one arithmetic pipe (RIME_PIPE_*)."""
    out = C.c_double()
    _check(lib().rime_pipe_rate(int(pipe), C.byref(out)), None)
    return out.value
