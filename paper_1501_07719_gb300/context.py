"""A Python handle around one librime context, using torch for device memory
and streams."""
from __future__ import annotations

import numpy as np

from . import _abi as A


class Rime:
    """One observation on the GPU.

    obs: dict with na, ntime, nchan, freq, uvw, pointing (or None),
         ref_freq_hz, beam_c; data / weight may be given here or later.
    precision: RIME_FP32 or RIME_FP64.
    """

    def __init__(self, obs: dict, precision: int = A.RIME_FP32, data=None, weight=None, stream=None):
        import torch
        self.torch = torch
        self.precision = precision
        self.na, self.ntime, self.nchan = int(obs["na"]), int(obs["ntime"]), int(obs["nchan"])
        self.nbl = self.na * (self.na - 1) // 2
        self.cdtype = torch.complex128 if precision == A.RIME_FP64 else torch.complex64
        self.rdtype = torch.float64 if precision == A.RIME_FP64 else torch.float32
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.nsrc = 0
        self.ctx = A.rime_create(self.na, self.ntime, self.nchan, precision, obs["freq"], obs["uvw"],
                                 obs.get("pointing"), data, weight, self.stream.cuda_stream,
                                 float(obs["ref_freq_hz"]), float(obs["beam_c"]))
        if int(obs.get("beam_model", 0)) != A.RIME_BEAM_COS3:
            self.set_beam(int(obs["beam_model"]), float(obs["beam_c"]))

    # inputs ---------------------------------------------------------------
    def set_uvw(self, uvw, pointing=None):
        A.rime_set_uvw(self.ctx, uvw, pointing)

    def set_data(self, data, weight=None):
        A.rime_set_data(self.ctx, self.precision, data, weight)

    def set_gains(self, gains):
        A.rime_set_gains(self.ctx, gains)

    def set_sources(self, src: dict):
        A.rime_set_sources(self.ctx, src["lm"], src["stokes"], src["alpha"], src.get("shape"), src.get("kind"))
        self.nsrc = int(src["alpha"].shape[0])

    # calls ------------------------------------------------------------------
    def predict(self, out=None):
        if out is None:
            out = self.torch.empty((self.ntime, self.nbl, self.nchan, 4), dtype=self.cdtype,
                                   device="cuda")
        A.rime_predict(self.ctx, out)
        return out

    def chi2(self) -> float:
        return A.rime_chi2(self.ctx)

    def chi2_async(self, out):
        A.rime_chi2_async(self.ctx, out)
        return out

    def chi2_streamed(self, data, weight=None, chunk_ntime: int = 0) -> float:
        """chi^2 of an observation whose data / weights stay in host memory
        (pinned torch tensors overlap the copies with the kernel), streamed
        in chunks of chunk_ntime timesteps (0: the library's choice)."""
        return A.rime_chi2_streamed(self.ctx, self.precision, data, weight, chunk_ntime)

    def stream_chunk_ntime(self) -> int:
        return A.rime_stream_chunk_ntime(self.ctx)

    def chi2_grad(self, want_gains: bool = True):
        """chi^2, d chi^2 / d(source parameters) as a [nsrc, 10] float64 device
        tensor (l, m, I, Q, U, V, alpha, major, minor, pa) and, if requested,
        d chi^2 / dG as a [ntime, na, nchan, 2, 2] complex128 device tensor."""
        nsrc = self.nsrc
        gs = self.torch.zeros((nsrc, 10), dtype=self.torch.float64, device="cuda")
        gg = None
        if want_gains:
            gg = self.torch.zeros((self.ntime, self.na, self.nchan, 2, 2), dtype=self.torch.complex128,
                                  device="cuda")
        chi = A.rime_chi2_grad(self.ctx, gs, gg)
        return chi, gs, gg

    def chi2_batched(self, offsets, sources: dict, out=None):
        """chi^2 of each source set (set j = sources offsets[j]:offsets[j+1])
        as a float64 device tensor [nsets]; does not wait."""
        nsets = len(offsets) - 1
        if out is None:
            out = self.torch.empty(max(nsets, 0), dtype=self.torch.float64, device="cuda")
        A.rime_chi2_batched(self.ctx, offsets, sources["lm"], sources["stokes"], sources["alpha"],
                            sources.get("shape"), out, sources.get("kind"))
        self.nsrc = int(sources["alpha"].shape[0])
        return out

    def set_tensor_mode(self, mode: int):
        """Tensor-core split-precision source sum for point sources
        (RIME_TC_SPLIT_BF16 / RIME_TC_SPLIT_TF32 / RIME_TC_SPLIT_F16) or the direct sum (RIME_TC_OFF)."""
        A.rime_set_tensor_mode(self.ctx, mode)

    def chains_init(self, nchains: int):
        """Per-chain residuals D - V at the current sky model (rime_chains_init)."""
        A.rime_chains_init(self.ctx, nchains)
        self.nchains = int(nchains)

    def chains_propose(self, nmove: int, proposed: dict, current: dict, out=None):
        """chi^2 of each chain's proposal as a float64 device tensor [nchains];
        does not wait."""
        if out is None:
            out = self.torch.empty(self.nchains, dtype=self.torch.float64, device="cuda")
        A.rime_chains_propose(self.ctx, nmove, proposed, current, out)
        return out

    def chains_accept(self, accept):
        A.rime_chains_accept(self.ctx, accept)

    def set_beam(self, model: int, beam_c: float):
        """Beam model of eq. 4's E: RIME_BEAM_COS3 (default) or RIME_BEAM_JINC,
        with its constant C in rad^-1 GHz^-1."""
        A.rime_set_beam(self.ctx, model, beam_c)

    def set_wait_limit(self, ns: int):
        """Limit (ns) of the tensor-core kernels' bounded waits (0: about 2 s)."""
        A.rime_set_wait_limit(self.ctx, ns)

    def set_kernel(self, kernel: int):
        """Direct-sum kernel: RIME_KERNEL_AUTO (default), RIME_KERNEL_TILED or
        RIME_KERNEL_NARROW (arrays of up to 45 antennas)."""
        A.rime_set_kernel(self.ctx, kernel)

    def batched_config(self) -> dict:
        return A.rime_batched_config(self.ctx)

    def set_batched_config(self, channels_per_item=None, blocks_per_sm=2, order=0, sets_per_item=1):
        A.rime_set_batched_config(self.ctx, channels_per_item, blocks_per_sm, order, sets_per_item)

    def ln_norm(self) -> float:
        return A.rime_ln_norm(self.ctx)

    def sync(self):
        A.rime_sync(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            A.rime_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
