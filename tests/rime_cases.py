"""Hand-built small problems for the oracle pins and the GPU edge cases.

Only plain array construction lives here; no RIME arithmetic.
"""
import numpy as np

C_LIGHT = 299792458.0


def problem(uvw, freq, lm, stokes, alpha=None, shape=None, gains=None,
            pointing=None, data=None, weight=None, ref_freq_hz=1.4e9, beam_c=65.0):
    """A problem dict in the layout rime_synth.make_inputs returns.

    uvw [ntime][na][3]; freq [nchan]; lm [nsrc][2]; stokes [nsrc][4] or
    [ntime][nsrc][4]; shape [nsrc][3]; gains [ntime][na][nchan][2][2].
    """
    uvw = np.asarray(uvw, dtype=np.float64)
    ntime, na = uvw.shape[:2]
    freq = np.atleast_1d(np.asarray(freq, dtype=np.float64))
    nchan = freq.shape[0]
    lm = np.asarray(lm, dtype=np.float64).reshape(-1, 2)
    nsrc = lm.shape[0]
    stokes = np.asarray(stokes, dtype=np.float64)
    if stokes.ndim == 1:
        stokes = stokes.reshape(-1, 4)
    alpha = np.zeros(nsrc) if alpha is None else np.asarray(alpha, dtype=np.float64).reshape(nsrc)
    shape = np.zeros((nsrc, 3)) if shape is None else np.asarray(shape, dtype=np.float64).reshape(nsrc, 3)
    nbl = na * (na - 1) // 2
    if weight is None:
        weight = np.ones((ntime, nbl, nchan))
    if gains is not None:
        gains = np.asarray(gains, dtype=np.complex128).reshape(ntime, na, nchan, 2, 2)
    if data is None:
        data = np.zeros((ntime, nbl, nchan, 4), dtype=np.complex128)
    return dict(na=na, ntime=ntime, nchan=nchan, nbl=nbl, ref_freq_hz=ref_freq_hz,
                beam_c=beam_c, uvw=uvw, freq=freq, pointing=pointing,
                sources=dict(lm=lm, stokes=stokes, alpha=alpha, shape=shape),
                gains=gains, weight=np.asarray(weight, dtype=np.float64),
                data=np.asarray(data, dtype=np.complex128),
                noise=np.zeros((ntime, nbl, nchan, 4), dtype=np.complex128))


def load_golden(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    rows = []
    with open(path) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append([float(x) for x in line.split()])
    return np.array(rows)
