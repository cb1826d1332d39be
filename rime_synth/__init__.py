"""Seeded synthetic inputs for the RIME predict + chi^2 path.

This module only draws random numbers and lays them out. It holds none of the
RIME's arithmetic: model visibilities are always computed by the caller (the
oracle in tests, the CUDA library in the benchmark) and passed to
``observe`` together with the noise drawn here.

Shapes and value distributions follow the workloads the paper measures
(Table 4: 64 channels, 100 timesteps, 50 point + 50 Gaussian sources, 7-192
antennas) with the distributions fixed for this library:

* uvw ~ U(-1000, 1000) m, i.i.d. per (time, antenna, component)
* l, m ~ U(-0.01, 0.01) rad
* Stokes I log-uniform on [0.1, 10] Jy, Q, U, V ~ U(-0.05 I, 0.05 I)
* spectral index alpha ~ N(-0.7, 0.2)
* Gaussian axes: two draws of U(1e-5, 1e-4) rad, major = larger; pa ~ U(0, pi)
* gains G = I + complex N(0, 0.05) per (time, antenna, channel, entry)
* noise complex N(0, 0.01) per correlation (real and imaginary independent)
* weights U(0.5, 2) (unit weights for the 7-antenna workload)
* channels uniformly spaced over 1.0-1.5 GHz, end points included

Every array has its own PCG64 stream spawned from one seed, in a fixed order,
so adding an array never changes the others.  For single-precision runs every
real input is rounded to float32 here (and handed on as the exactly upcast
float64 value), so that the oracle and the kernels see identical inputs.
"""
from __future__ import annotations

from dataclasses import dataclass, replace
import numpy as np

SEED_BASE = 1501077190
REF_FREQ_HZ = 1.4e9
BEAM_C = 65.0
BAND_HZ = (1.0e9, 1.5e9)

# Stream order is part of the recipe: never reorder, only append.
_STREAMS = ("uvw", "lm", "stokes", "alpha", "shape", "gains", "noise",
            "weights", "sets", "pointing", "kind")


@dataclass(frozen=True)
class Workload:
    name: str
    na: int
    ntime: int
    nchan: int
    npsrc: int = 0          # point sources (listed first)
    ngsrc: int = 0          # Gaussian sources (listed after the points)
    unit_weights: bool = False
    seed_index: int = 0
    # batched sampling: nsets parameter sets, nsrc per set ~ U{lo..hi},
    # each source Gaussian with probability p_gauss
    nsets: int = 0
    set_nsrc: tuple = (5, 500)
    p_gauss: float = 0.5

    @property
    def nbl(self) -> int:
        return self.na * (self.na - 1) // 2

    @property
    def nsrc(self) -> int:
        return self.npsrc + self.ngsrc


WORKLOADS = {
    w.name: w for w in (
        Workload("7ant-10t-16ch-10pt", na=7, ntime=10, nchan=16, npsrc=10,
                 unit_weights=True, seed_index=0),
        Workload("64ant-100t-64ch-100pt100g", na=64, ntime=100, nchan=64,
                 npsrc=100, ngsrc=100, seed_index=1),
        # the gradient workload reuses the 64-antenna observation
        Workload("64ant-100t-64ch-100pt100g-grad", na=64, ntime=100, nchan=64,
                 npsrc=100, ngsrc=100, seed_index=2),
        # shared observation; its data come from a 100-source truth sky
        Workload("64ant-50t-32ch-512sets", na=64, ntime=50, nchan=32,
                 npsrc=50, ngsrc=50, nsets=512, seed_index=3),
        Workload("256ant-20t-128ch-4096pt", na=256, ntime=20, nchan=128,
                 npsrc=4096, seed_index=4),
        # Table 4's smallest array (KAT-7 shape) at the table's sizes
        Workload("7ant-100t-64ch-50pt50g", na=7, ntime=100, nchan=64,
                 npsrc=50, ngsrc=50, seed_index=207),
    )
}


def workload(name: str, **overrides) -> Workload:
    """A named workload, optionally with some fields replaced (same recipe)."""
    return replace(WORKLOADS[name], **overrides)


def custom(na, ntime, nchan, npsrc, ngsrc=0, seed_index=100, **kw) -> Workload:
    name = f"{na}ant-{ntime}t-{nchan}ch-{npsrc}pt{ngsrc}g"
    return Workload(name, na=na, ntime=ntime, nchan=nchan, npsrc=npsrc,
                    ngsrc=ngsrc, seed_index=seed_index, **kw)


def streams(seed: int) -> dict:
    children = np.random.SeedSequence(seed).spawn(len(_STREAMS))
    return {n: np.random.Generator(np.random.PCG64(c))
            for n, c in zip(_STREAMS, children)}


def channel_freqs(nchan: int) -> np.ndarray:
    if nchan == 1:
        return np.array([BAND_HZ[0]])
    return BAND_HZ[0] + np.arange(nchan) * ((BAND_HZ[1] - BAND_HZ[0]) / (nchan - 1))


def _r32(x):
    x = np.asarray(x)
    if np.iscomplexobj(x):
        return (x.real.astype(np.float32).astype(np.float64)
                + 1j * x.imag.astype(np.float32).astype(np.float64))
    return x.astype(np.float32).astype(np.float64)


def draw_sources(rs: dict, n: int, gauss_mask) -> dict:
    """n sources in SoA layout: lm [n,2], stokes [n,4] (I,Q,U,V), alpha [n],
    shape [n,3] (major FWHM, minor FWHM, position angle; zeros for points)."""
    lm = rs["lm"].uniform(-0.01, 0.01, size=(n, 2))
    sI = np.exp(rs["stokes"].uniform(np.log(0.1), np.log(10.0), size=n))
    quv = rs["stokes"].uniform(-0.05, 0.05, size=(n, 3)) * sI[:, None]
    stokes = np.concatenate([sI[:, None], quv], axis=1)
    alpha = rs["alpha"].normal(-0.7, 0.2, size=n)
    ax = rs["shape"].uniform(1e-5, 1e-4, size=(n, 2))
    pa = rs["shape"].uniform(0.0, np.pi, size=n)
    shape = np.stack([ax.max(axis=1), ax.min(axis=1), pa], axis=1)
    shape[~np.asarray(gauss_mask, dtype=bool)] = 0.0
    return dict(lm=lm, stokes=stokes, alpha=alpha, shape=shape)


def make_inputs(wl: Workload | str, precision: str = "f64", seed: int | None = None,
                pointing_sigma: float = 0.0, time_varying: bool = False, noise: bool = True,
                beam_model: int = 0, beam_c: float | None = None, disk_fraction: float = 0.0) -> dict:
    """All inputs of one workload except the observed data (see ``observe``).

    precision "f32" rounds every real input to float32 values. noise=False
    leaves the noise out (None; the other arrays are unchanged, every array
    has its own stream), for timing runs that do not need the data values.
    beam_model: 0 the cos^3 beam of eq. 4, 1 the Jinc beam 2 J1(x)/x, with
    x = beam_c nu_GHz rho (beam_c defaults to BEAM_C).
    disk_fraction: the share of the extended sources drawn as exponential
    disks (sources["kind"] = 1; their shape axes are scale lengths) instead of
    Gaussians; 0 leaves "kind" out.
    """
    if isinstance(wl, str):
        wl = WORKLOADS[wl]
    seed = SEED_BASE + wl.seed_index if seed is None else seed
    rs = streams(seed)
    na, nt, nc = wl.na, wl.ntime, wl.nchan
    nbl = wl.nbl
    uvw = rs["uvw"].uniform(-1000.0, 1000.0, size=(nt, na, 3))
    freq = channel_freqs(nc)
    src = draw_sources(rs, wl.nsrc, np.arange(wl.nsrc) >= wl.npsrc)
    if disk_fraction > 0.0:
        disk = (np.arange(wl.nsrc) >= wl.npsrc) & (rs["kind"].uniform(size=wl.nsrc) < disk_fraction)
        src["kind"] = disk.astype(np.int32)
    if time_varying:
        # brightness per (time, source): the static draw times U(0.5, 1.5)
        scale = rs["stokes"].uniform(0.5, 1.5, size=(nt, wl.nsrc, 1))
        src["stokes"] = src["stokes"][None, :, :] * scale
    gains = np.broadcast_to(np.eye(2), (nt, na, nc, 2, 2)).astype(np.complex128)
    gains = gains + (rs["gains"].normal(0.0, 0.05, size=(nt, na, nc, 2, 2))
                     + 1j * rs["gains"].normal(0.0, 0.05, size=(nt, na, nc, 2, 2)))
    if noise:
        noise = (rs["noise"].normal(0.0, 0.01, size=(nt, nbl, nc, 4))
                 + 1j * rs["noise"].normal(0.0, 0.01, size=(nt, nbl, nc, 4)))
    else:
        noise = None
    if wl.unit_weights:
        weight = np.ones((nt, nbl, nc))
    else:
        weight = rs["weights"].uniform(0.5, 2.0, size=(nt, nbl, nc))
    pointing = None
    if pointing_sigma > 0.0:
        pointing = rs["pointing"].normal(0.0, pointing_sigma, size=(nt, na, 2))
    out = dict(workload=wl, precision=precision, na=na, ntime=nt, nchan=nc,
               nbl=nbl, ref_freq_hz=REF_FREQ_HZ, beam_c=BEAM_C if beam_c is None else float(beam_c),
               beam_model=int(beam_model), uvw=uvw,
               freq=freq, pointing=pointing, sources=src, gains=gains,
               noise=noise, weight=weight)
    if wl.nsets:
        out["sets"] = draw_sets(rs, wl)
    if precision == "f32":
        out = round_f32(out)
    return out


def draw_sets(rs: dict, wl: Workload) -> dict:
    """Parameter sets for batched sampling: set k holds sources
    offsets[k]..offsets[k+1]-1 of the concatenated SoA arrays."""
    lo, hi = wl.set_nsrc
    counts = rs["sets"].integers(lo, hi + 1, size=wl.nsets)
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    total = int(offsets[-1])
    gmask = rs["sets"].uniform(size=total) < wl.p_gauss
    src = draw_sources(rs, total, gmask)
    return dict(offsets=offsets, sources=src)


def round_f32(inp: dict) -> dict:
    out = dict(inp)
    for k in ("uvw", "freq", "gains", "noise", "weight"):
        if inp[k] is not None:
            out[k] = _r32(inp[k])
    out["ref_freq_hz"] = float(_r32(inp["ref_freq_hz"]))
    if inp.get("pointing") is not None:
        out["pointing"] = _r32(inp["pointing"])
    out["sources"] = {k: (v if k == "kind" else _r32(v)) for k, v in inp["sources"].items()}
    if "sets" in inp:
        out["sets"] = dict(offsets=inp["sets"]["offsets"],
                           sources={k: _r32(v) for k, v in inp["sets"]["sources"].items()})
    return out


def observe(model_vis: np.ndarray, noise: np.ndarray, precision: str = "f64") -> np.ndarray:
    """Observed data D = model + noise, stored in the run's complex type
    (complex64 for single precision, complex128 otherwise)."""
    d = np.asarray(model_vis) + np.asarray(noise)
    return d.astype(np.complex64) if precision == "f32" else d.astype(np.complex128)


def baseline_pairs(na: int):
    """Antenna pairs (p, q), p < q, in the canonical row-major upper-triangle order."""
    p, q = np.triu_indices(na, k=1)
    return p.astype(np.int32), q.astype(np.int32)
