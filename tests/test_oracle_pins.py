"""Pins for the FP64 oracle: each test checks it against something other than
itself -- values fixed by the paper's equations, closed forms, invariants, an
image-plane quadrature, a matrix formulation, high-precision arithmetic and
finite differences -- so that a dropped term, a wrong sign or index, or a
transposed operand fails at least one of them.
"""
import numpy as np
import pytest

import oracle
import rime_synth
from rime_cases import C_LIGHT, load_golden, problem

pytestmark = pytest.mark.usefixtures("oracle_lib")


def vis_all(inp, **kw):
    return oracle.Problem(inp, **kw).predict()


# --------------------------------------------------------------------------
# Eq. 2 / eq. 3 / eq. 4 at the phase centre
# --------------------------------------------------------------------------
def test_phase_centre_unit_source_gives_identity():
    """A unit point source at l = m = 0 (K = 1, E = 1, alpha = 0) gives
    V = B = identity on every baseline and channel (eqs. 1-4)."""
    inp = rime_synth.make_inputs(rime_synth.custom(5, 3, 4, 1))
    inp["sources"] = dict(lm=np.zeros((1, 2)), stokes=np.array([[1.0, 0, 0, 0]]),
                          alpha=np.zeros(1), shape=np.zeros((1, 3)))
    inp["gains"] = None
    V = vis_all(inp)
    np.testing.assert_array_equal(V, np.broadcast_to(np.array([1, 0, 0, 1]), V.shape))


def test_phase_centre_stokes_matrix_matches_eq2():
    """Eq. 2's brightness matrix for given (I, Q, U, V), hand-derived."""
    rows = load_golden("stokes_coherency.txt")
    for r in rows:
        inp = problem(uvw=[[[100.0, -50, 3], [-70, 20, 8], [5, 5, 5]]], freq=[1.4e9],
                      lm=[[0.0, 0.0]], stokes=r[:4])
        V = vis_all(inp)
        want = r[4:].reshape(4, 2) @ np.array([1, 1j])
        np.testing.assert_allclose(V.reshape(-1, 4), np.broadcast_to(want, (3, 4)),
                                   rtol=0, atol=1e-15)


def test_spectral_index_closed_form():
    """Eq. 2: B scales with (lambda_ref / lambda)^alpha = (nu / nu_ref)^alpha."""
    freq = np.array([0.7e9, 1.4e9, 2.8e9])
    inp = problem(uvw=np.zeros((1, 2, 3)), freq=freq, lm=[[0.0, 0.0]],
                  stokes=[1.0, 0, 0, 0], alpha=[-0.7], beam_c=0.0)
    V = vis_all(inp)[0, 0, :, 0]
    want = np.array([2.0 ** 0.7, 1.0, 2.0 ** -0.7])  # 0.5^-0.7, 1, 2^-0.7
    np.testing.assert_allclose(V.real, want, rtol=1e-14)
    np.testing.assert_allclose(V.imag, 0, atol=1e-15)


def test_phase_sign_and_scale_u_term():
    """Eq. 3 with eq. 5: V_pq = K_p K_q^*, so for u_p = 0, u_q = u and a
    source at (l, 0): V_00 = exp(-2 pi i u l nu / c) exactly (unit beam)."""
    import mpmath as mp
    mp.mp.dps = 40
    u, l, nu = 100.0, 0.001, 1.5e9
    inp = problem(uvw=[[[0.0, 0, 0], [u, 0, 0]]], freq=[nu], lm=[[l, 0.0]],
                  stokes=[1.0, 0, 0, 0], alpha=[0.0], beam_c=0.0, ref_freq_hz=nu)
    V00 = vis_all(inp)[0, 0, 0, 0]
    ph = -2 * mp.pi * mp.mpf(u) * mp.mpf(l) * mp.mpf(nu) / mp.mpf(C_LIGHT)
    want = complex(mp.cos(ph), mp.sin(ph))
    assert abs(V00 - want) < 1e-14
    # phase advances with v m the same way, and the sign flips for V_qp
    P = oracle.Problem(inp)
    assert abs(P.vis(0, 1, 0, 0)[0] - np.conj(want)) < 1e-14


def test_phase_w_term_uses_n_minus_one():
    """Eq. 3: the w coordinate multiplies n - 1 = sqrt(1 - l^2 - m^2) - 1,
    evaluated here at 50 digits."""
    import mpmath as mp
    mp.mp.dps = 50
    w, l, m, nu = 900.0, 0.3, -0.4, 1.1e9
    inp = problem(uvw=[[[0.0, 0, w], [0.0, 0, 0]]], freq=[nu], lm=[[l, m]],
                  stokes=[1.0, 0, 0, 0], alpha=[0.0], beam_c=0.0, ref_freq_hz=nu)
    V00 = vis_all(inp)[0, 0, 0, 0]
    n1 = mp.sqrt(1 - mp.mpf(l) ** 2 - mp.mpf(m) ** 2) - 1
    ph = 2 * mp.pi * mp.mpf(w) * n1 * mp.mpf(nu) / mp.mpf(C_LIGHT)
    want = complex(mp.cos(ph), mp.sin(ph))
    assert abs(V00 - want) < 1e-12


@pytest.mark.parametrize("row", range(2))
def test_beam_cos3_values(row):
    """Eq. 4 read as cos^3(C nu_GHz rho): hand values at C nu rho = pi/3, pi/4."""
    x_over_pi, E, V00 = load_golden("beam_cos3.txt")[row]
    rho = x_over_pi * np.pi / 65.0
    for lm in ([rho, 0.0], [0.0, -rho], [rho * 0.6, rho * 0.8]):
        inp = problem(uvw=np.zeros((1, 2, 3)), freq=[1e9], lm=[lm],
                      stokes=[1.0, 0, 0, 0], ref_freq_hz=1e9)
        V = vis_all(inp)[0, 0, 0]
        np.testing.assert_allclose(V, [V00, 0, 0, V00], rtol=1e-13, atol=1e-16)


def test_beam_null_clamp_and_pointing():
    """Past the first null (C nu rho >= pi/2) E = 0; a pointing offset equal to
    the source position gives rho = 0 and E = 1 for that antenna only."""
    rho = 0.6 * np.pi / 65.0     # C nu rho = 0.6 pi > pi/2
    inp = problem(uvw=np.zeros((1, 2, 3)), freq=[1e9], lm=[[rho, 0.0]],
                  stokes=[1.0, 0, 0, 0], ref_freq_hz=1e9)
    np.testing.assert_array_equal(vis_all(inp), 0)
    rho = np.pi / 3 / 65.0
    inp = problem(uvw=np.zeros((1, 2, 3)), freq=[1e9], lm=[[rho, 0.0]],
                  stokes=[1.0, 0, 0, 0], ref_freq_hz=1e9,
                  pointing=np.array([[[rho, 0.0], [0.0, 0.0]]]))
    V = vis_all(inp)[0, 0, 0]
    np.testing.assert_allclose(V, [0.125, 0, 0, 0.125], rtol=1e-13)


_J1_ZERO_1 = 3.8317059702075125   # first positive zero of J1 (Abramowitz & Stegun, Table 9.5)


def _jinc_E(x):
    """The Jinc beam from scipy's Bessel J1, independent of the oracle's libm."""
    special = pytest.importorskip("scipy.special")
    x = np.asarray(x, dtype=np.float64)
    return np.where(x == 0, 1.0, 2 * special.j1(x) / np.where(x == 0, 1, x))


def _beam_probe(x_q, beam_c=65.0, nu=1e9):
    """V00 of a unit point source on one baseline with u = v = w = 0 (K = 1),
    antenna p pointed at the source (E_p = 1): V00 = E(x_q), x = C nu_GHz rho."""
    rho = x_q / (beam_c * nu * 1e-9)
    inp = problem(uvw=np.zeros((1, 2, 3)), freq=[nu], lm=[[rho * 0.6, rho * 0.8]],
                  stokes=[1.0, 0, 0, 0], ref_freq_hz=nu, beam_c=beam_c,
                  pointing=np.array([[[rho * 0.6, rho * 0.8], [0.0, 0.0]]]))
    inp["beam_model"] = 1
    return vis_all(inp)[0, 0, 0]


@pytest.mark.parametrize("x", [0.0, 1e-3, 0.0499, 0.0501, 0.7, 2.0, 3.3, 5.0, 7.0155867, 9.2])
def test_beam_jinc_equals_bessel_definition(x):
    """The Jinc beam that Sec. 2.1 names for the VLA, E = 2 J1(x)/x, against
    scipy's J1: main lobe, both sides of the oracle's series/libm switch at
    x = 0.05, the negative first sidelobe and the second (x near 7.0156, the
    first zero of J2, is its extremum)."""
    V = _beam_probe(x)
    want = float(_jinc_E(x))
    np.testing.assert_allclose(V, [want, 0, 0, want], rtol=1e-14, atol=1e-16)


def test_beam_jinc_nulls_and_both_antennas():
    """E vanishes at the first zero of J1; with neither antenna pointed at the
    source V00 = E(x_p) E(x_q), which is negative when one of them sees the
    source in a sidelobe."""
    assert abs(_beam_probe(_J1_ZERO_1)[0]) < 1e-15
    nu, beam_c = 1.4e9, 65.0
    cnu = beam_c * nu * 1e-9
    l = 4.5 / cnu
    inp = problem(uvw=np.zeros((1, 2, 3)), freq=[nu], lm=[[l, 0.0]], stokes=[1.0, 0, 0, 0], ref_freq_hz=nu,
                  beam_c=beam_c, pointing=np.array([[[3.0 / cnu, 0.0], [0.0, 0.0]]]))
    inp["beam_model"] = 1
    V00 = vis_all(inp)[0, 0, 0, 0]
    want = _jinc_E(1.5) * _jinc_E(4.5)
    assert want < 0 and V00 == pytest.approx(want, rel=1e-14)


# --------------------------------------------------------------------------
# Gaussian shape: Fourier transform of the image-plane Gaussian, by quadrature
# --------------------------------------------------------------------------
@pytest.mark.parametrize("pa", [0.0, 0.7, np.pi / 2, 2.5])
def test_gaussian_shape_equals_image_plane_fourier_integral(pa):
    """The shape factor is the normalised 2-D Fourier transform of an
    elliptical Gaussian brightness with FWHM axes (maj, min), major axis at
    position angle pa from +m towards +l. Trapezoid quadrature on a wide grid
    is spectrally accurate for this integrand."""
    maj, mn, nu = 8e-5, 3e-5, 1.2e9
    up, uq = np.array([1500.0, -800.0, 0.0]), np.array([0.0, 0.0, 0.0])
    inp = problem(uvw=[[up, uq]], freq=[nu], lm=[[0.0, 0.0]], stokes=[1.0, 0, 0, 0],
                  shape=[[maj, mn, pa]], ref_freq_hz=nu, beam_c=0.0)
    g = vis_all(inp)[0, 0, 0, 0]
    lam = C_LIGHT / nu
    u, v = (up[0] - uq[0]) / lam, (up[1] - uq[1]) / lam
    L, n = 8 * maj, 1601
    x = np.linspace(-L, L, n)
    ll, mm = np.meshgrid(x, x, indexing="ij")
    xmaj = ll * np.sin(pa) + mm * np.cos(pa)
    xmin = ll * np.cos(pa) - mm * np.sin(pa)
    img = np.exp(-4 * np.log(2) * (xmaj ** 2 / maj ** 2 + xmin ** 2 / mn ** 2))
    ft = (img * np.exp(2j * np.pi * (u * ll + v * mm))).sum() / img.sum()
    assert 0.05 < abs(ft) < 0.95          # the case resolves the source partially
    assert abs(g - ft) < 1e-10


@pytest.mark.parametrize("pa", [0.0, 0.7, 2.5])
def test_exponential_disk_equals_image_plane_fourier_integral(pa):
    """kind 1 is the Sersic profile of index 1: an elliptical exponential disk
    exp(-sqrt((x_maj/major)^2 + (x_min/minor)^2)) with scale lengths (major,
    minor), major axis at pa from +m towards +l. Its shape factor is the
    normalised 2-D Fourier transform, here by a trapezoid sum over +-30 scale
    lengths (the cusp at the centre limits it to ~1e-6)."""
    maj, mn, nu = 2e-5, 0.8e-5, 1.2e9
    up, uq = np.array([1500.0, -800.0, 0.0]), np.array([0.0, 0.0, 0.0])
    inp = problem(uvw=[[up, uq]], freq=[nu], lm=[[0.0, 0.0]], stokes=[1.0, 0, 0, 0],
                  shape=[[maj, mn, pa]], ref_freq_hz=nu, beam_c=0.0)
    inp["sources"]["kind"] = np.array([1], dtype=np.int32)
    g = vis_all(inp)[0, 0, 0, 0]
    lam = C_LIGHT / nu
    u, v = (up[0] - uq[0]) / lam, (up[1] - uq[1]) / lam
    L, n = 30 * maj, 3001
    x = np.linspace(-L, L, n)
    ll, mm = np.meshgrid(x, x, indexing="ij")
    xmaj = ll * np.sin(pa) + mm * np.cos(pa)
    xmin = ll * np.cos(pa) - mm * np.sin(pa)
    img = np.exp(-np.sqrt(xmaj ** 2 / maj ** 2 + xmin ** 2 / mn ** 2))
    ft = (img * np.exp(2j * np.pi * (u * ll + v * mm))).sum() / img.sum()
    assert 0.05 < abs(ft) < 0.95
    assert abs(g - ft) < 5e-6


def test_exponential_disk_degenerate_cases_and_kind_zero():
    """A disk with major = minor = 0 is a point; a circular disk does not depend
    on pa; kind 0 (and no kind array) is the Gaussian."""
    up = np.array([1200.0, 700.0, 0.0])
    base = dict(uvw=[[up, np.zeros(3)]], freq=[1.3e9], lm=[[0.0, 0.0]],
                stokes=[1.0, 0, 0, 0], ref_freq_hz=1.3e9, beam_c=0.0)

    def g(shape, kind):
        inp = problem(shape=[shape], **base)
        if kind is not None:
            inp["sources"]["kind"] = np.array([kind], dtype=np.int32)
        return vis_all(inp)[0, 0, 0, 0]
    assert g([0.0, 0.0, 1.0], 1) == 1.0
    vals = [g([2e-5, 2e-5, pa], 1) for pa in (0.0, 0.4, 1.9)]
    np.testing.assert_allclose(vals, vals[0], rtol=1e-14)
    assert g([5e-5, 2e-5, 0.3], 0) == g([5e-5, 2e-5, 0.3], None) != g([5e-5, 2e-5, 0.3], 1)


def test_gaussian_degenerate_cases():
    """maj = min = 0 is a point; maj = min gives a circular Gaussian whose
    value does not depend on pa."""
    up = np.array([1200.0, 700.0, 0.0])
    base = dict(uvw=[[up, np.zeros(3)]], freq=[1.3e9], lm=[[0.0, 0.0]],
                stokes=[1.0, 0, 0, 0], ref_freq_hz=1.3e9, beam_c=0.0)
    assert vis_all(problem(shape=[[0.0, 0.0, 1.0]], **base))[0, 0, 0, 0] == 1.0
    vals = [vis_all(problem(shape=[[5e-5, 5e-5, pa]], **base))[0, 0, 0, 0]
            for pa in (0.0, 0.4, 1.9)]
    np.testing.assert_allclose(vals, vals[0], rtol=1e-14)


# --------------------------------------------------------------------------
# Gains, Hermitian symmetry, the per-antenna matrix formulation
# --------------------------------------------------------------------------
def _random_small(seed=7, na=5, ntime=2, nchan=3, npsrc=3, ngsrc=2, pointing=0.003):
    wl = rime_synth.custom(na, ntime, nchan, npsrc, ngsrc, seed_index=seed)
    return rime_synth.make_inputs(wl, pointing_sigma=pointing)


def test_gains_apply_as_Gp_S_GqH():
    """Eq. 1: V = G_p S G_q^H, checked against numpy products of the
    gain-free oracle result."""
    inp = _random_small()
    G = inp["gains"]
    V = vis_all(inp)
    inp0 = dict(inp, gains=None)
    S = vis_all(inp0)
    p, q = rime_synth.baseline_pairs(inp["na"])
    S22 = S.reshape(*S.shape[:3], 2, 2)
    Gp = G[:, p]            # [t][bl][k][2][2]
    Gq = G[:, q]
    want = Gp @ S22 @ np.conj(np.swapaxes(Gq, -1, -2))
    np.testing.assert_allclose(V, want.reshape(V.shape), rtol=0, atol=1e-12 * np.abs(V).max())


def test_hermitian_symmetry_vqp_equals_vpq_H():
    """B is Hermitian and the shape factor even in (u, v): V_qp = V_pq^H,
    including gains, pointing and Gaussians."""
    inp = _random_small()
    P = oracle.Problem(inp)
    for (t, p, q, k) in [(0, 0, 1, 0), (1, 2, 4, 2), (0, 3, 1, 1)]:
        a = P.vis(t, p, q, k).reshape(2, 2)
        b = P.vis(t, q, p, k).reshape(2, 2)
        np.testing.assert_allclose(b, a.conj().T, rtol=0, atol=1e-13 * np.abs(a).max())


def test_per_antenna_matrix_form_points():
    """Sec. 2.2: the per-antenna factors A_ps = E K sqrt(f) turn the source
    sum into A diag(x) A^H per (t, channel) and Stokes x; numpy matmuls of
    that factorised form agree with the direct sum (points only)."""
    inp = _random_small(npsrc=6, ngsrc=0, pointing=0.002)
    inp["gains"] = None
    V = vis_all(inp)
    src = inp["sources"]
    l, m = src["lm"][:, 0], src["lm"][:, 1]
    n1 = np.sqrt(1 - l ** 2 - m ** 2) - 1
    p, q = rime_synth.baseline_pairs(inp["na"])
    for t in range(inp["ntime"]):
        for k, nu in enumerate(inp["freq"]):
            uvw = inp["uvw"][t]
            ph = 2 * np.pi * nu / C_LIGHT * (np.outer(uvw[:, 0], l) + np.outer(uvw[:, 1], m)
                                             + np.outer(uvw[:, 2], n1))
            dl = src["lm"][None, :, :] - inp["pointing"][t][:, None, :]
            rho = np.sqrt((dl ** 2).sum(-1))
            E = np.cos(65.0 * nu * 1e-9 * rho) ** 3
            f = (nu / inp["ref_freq_hz"]) ** src["alpha"]
            A = E * np.exp(1j * ph) * np.sqrt(f)[None, :]
            M = {x: A @ np.diag(src["stokes"][:, i]) @ A.conj().T
                 for i, x in enumerate("IQUV")}
            S = np.stack([M["I"] + M["Q"], M["U"] + 1j * M["V"],
                          M["U"] - 1j * M["V"], M["I"] - M["Q"]], axis=-1)
            np.testing.assert_allclose(V[t, :, k], S[p, q], rtol=0,
                                       atol=1e-12 * np.abs(S).max())


def test_time_varying_brightness():
    """Table 2 lists brightness per (time, source): with every time equal to
    the static value the result is unchanged; a source at the phase centre
    scales with its own timestep's flux."""
    inp = _random_small()
    V = vis_all(inp)
    tv = dict(inp)
    tv["sources"] = dict(inp["sources"], stokes=np.broadcast_to(
        inp["sources"]["stokes"], (inp["ntime"],) + inp["sources"]["stokes"].shape).copy())
    np.testing.assert_array_equal(vis_all(tv), V)
    c = problem(uvw=np.zeros((3, 2, 3)), freq=[1.4e9], lm=[[0.0, 0.0]],
                stokes=np.array([[[1.0, 0, 0, 0]], [[2.0, 0, 0, 0]], [[0.5, 0.1, 0, 0]]]))
    Vc = vis_all(c)[:, 0, 0]
    np.testing.assert_allclose(Vc, [[1, 0, 0, 1], [2, 0, 0, 2], [0.6, 0, 0, 0.4]], atol=1e-15)


# --------------------------------------------------------------------------
# chi^2 (eq. 7)
# --------------------------------------------------------------------------
def test_chi2_hand_example():
    row = load_golden("chi2_hand.txt")[0]
    w, D, want = row[0], row[1:9].reshape(4, 2) @ np.array([1, 1j]), row[9]
    inp = problem(uvw=np.zeros((1, 2, 3)), freq=[1.4e9], lm=[[0.0, 0.0]],
                  stokes=[1.0, 0, 0, 0], weight=[[[w]]], data=D.reshape(1, 1, 1, 4))
    assert oracle.Problem(inp).chi2() == pytest.approx(want, rel=1e-15)


def test_chi2_zero_when_data_equal_model():
    inp = _random_small()
    V = vis_all(inp)
    assert oracle.Problem(inp, data=V).chi2() == 0.0


def test_chi2_zero_data_and_linear_in_weight():
    inp = _random_small()
    V = vis_all(inp)
    zero = np.zeros_like(V)
    c0 = oracle.Problem(inp, data=zero).chi2()
    want = (inp["weight"] * (np.abs(V) ** 2).sum(-1)).sum()
    assert c0 == pytest.approx(want, rel=1e-13)
    D = V + 0.01 * (np.cos(np.arange(V.size)).reshape(V.shape) + 0.5j)
    c1 = oracle.Problem(inp, data=D).chi2()
    inp3 = dict(inp, weight=3.0 * inp["weight"])
    assert oracle.Problem(inp3, data=D).chi2() == pytest.approx(3 * c1, rel=1e-14)
    # chi^2 over a time range is additive
    P = oracle.Problem(inp, data=D)
    assert P.chi2(0, 1) + P.chi2(1, 2) == pytest.approx(c1, rel=1e-14)


def test_ln_norm_unit_weights():
    """Eq. 7's constant with w = 1: one ln(2 pi) per weight."""
    inp = _random_small()
    inp["weight"] = np.ones_like(inp["weight"])
    P = oracle.Problem(inp, data=np.zeros((2, 10, 3, 4), complex))
    assert P.ln_norm() == pytest.approx(inp["weight"].size * np.log(2 * np.pi), rel=1e-14)


def test_direct_sum_high_precision():
    """Rounding of the FP64 oracle: one visibility of a random problem agrees
    with a 40-digit evaluation of eqs. 1-4 to ~1e-13 of its magnitude."""
    import mpmath as mp
    mp.mp.dps = 40
    inp = _random_small(seed=11, na=3, ntime=1, nchan=2, npsrc=3, ngsrc=2)
    t, p, q, k = 0, 0, 2, 1
    P = oracle.Problem(inp)
    got = P.vis(t, p, q, k)
    src = inp["sources"]
    nu = mp.mpf(inp["freq"][k])
    lam = mp.mpf(C_LIGHT) / nu
    lam_ref = mp.mpf(C_LIGHT) / mp.mpf(inp["ref_freq_hz"])
    S = [mp.mpc(0)] * 4
    for s in range(len(src["alpha"])):
        l, m = (mp.mpf(x) for x in src["lm"][s])
        n1 = mp.sqrt(1 - l * l - m * m) - 1
        A = []
        for a in (p, q):
            u, v, w = (mp.mpf(x) for x in inp["uvw"][t, a])
            dl, dm = (mp.mpf(x) for x in inp["pointing"][t, a])
            x = mp.mpf(65) * nu / mp.mpf(10) ** 9 * mp.sqrt((l - dl) ** 2 + (m - dm) ** 2)
            E = mp.cos(x) ** 3
            A.append(E * mp.expjpi(2 * (u * l + v * m + w * n1) / lam))
        f = (lam_ref / lam) ** mp.mpf(src["alpha"][s])
        maj, mn, pa = (mp.mpf(x) for x in src["shape"][s])
        du = (mp.mpf(inp["uvw"][t, p, 0]) - mp.mpf(inp["uvw"][t, q, 0])) / lam
        dv = (mp.mpf(inp["uvw"][t, p, 1]) - mp.mpf(inp["uvw"][t, q, 1])) / lam
        umaj = du * mp.sin(pa) + dv * mp.cos(pa)
        umin = du * mp.cos(pa) - dv * mp.sin(pa)
        g = mp.exp(-mp.pi ** 2 * (maj ** 2 * umaj ** 2 + mn ** 2 * umin ** 2) / (4 * mp.log(2)))
        sI, sQ, sU, sV = (mp.mpf(x) for x in src["stokes"][s])
        B = [sI + sQ, sU + 1j * sV, sU - 1j * sV, sI - sQ]
        z = A[0] * mp.conj(A[1]) * f * g
        S = [S[c] + z * B[c] for c in range(4)]
    G = inp["gains"][t]
    Gp = mp.matrix([[mp.mpc(x) for x in row] for row in G[p, k]])
    Gq = mp.matrix([[mp.mpc(x) for x in row] for row in G[q, k]])
    Sm = mp.matrix([[S[0], S[1]], [S[2], S[3]]])
    Vm = Gp * Sm * Gq.transpose_conj()
    want = np.array([complex(Vm[0, 0]), complex(Vm[0, 1]), complex(Vm[1, 0]), complex(Vm[1, 1])])
    assert np.abs(got - want).max() < 1e-13 * np.abs(want).max()


# --------------------------------------------------------------------------
# Gradient: central finite differences of the oracle's own chi^2
# --------------------------------------------------------------------------
_SCALES = np.array([1e-2, 1e-2, 1.0, 1.0, 1.0, 1.0, 1.0, 1e-4, 1e-4, 1.0])


def _set_param(inp, s, j, val):
    src = {k: v.copy() for k, v in inp["sources"].items()}
    if j < 2:
        src["lm"][s, j] = val
    elif j < 6:
        src["stokes"][s, j - 2] = val
    elif j == 6:
        src["alpha"][s] = val
    else:
        src["shape"][s, j - 7] = val
    return dict(inp, sources=src)


def _get_param(inp, s, j):
    src = inp["sources"]
    if j < 2:
        return src["lm"][s, j]
    if j < 6:
        return src["stokes"][s, j - 2]
    if j == 6:
        return src["alpha"][s]
    return src["shape"][s, j - 7]


def _fd_problem(beam_model=0, disks=False):
    inp = _random_small(seed=5, na=4, ntime=2, nchan=3, npsrc=1, ngsrc=2, pointing=0.004)
    if disks:
        # the extended sources as exponential disks with scale lengths of the same size
        inp["sources"]["kind"] = np.array([0, 1, 1], dtype=np.int32)
    # larger offsets so the beam derivative matters; data = model + noise
    inp["sources"]["lm"] *= 0.8
    if beam_model == 1:
        # the Jinc beam with x = C nu rho reaching its first sidelobe
        inp["beam_model"], inp["beam_c"] = 1, 400.0
    V = vis_all(inp)
    inp["data"] = V + inp["noise"] * 30
    return inp


@pytest.mark.parametrize("beam_model,disks", [(0, False), (1, False), (0, True)])
def test_gradient_matches_central_differences_sources(beam_model, disks):
    inp = _fd_problem(beam_model, disks)
    chi, gs, _ = oracle.Problem(inp).chi2_grad(want_gains=False)
    assert chi == pytest.approx(oracle.Problem(inp).chi2(), rel=1e-13)
    nsrc = gs.shape[0]
    for s in range(nsrc):
        for j in range(10):
            if j >= 7 and inp["sources"]["shape"][s, 0] == 0.0:
                continue   # points: shape derivatives are zero, checked below
            x0 = _get_param(inp, s, j)
            h = 1e-6 * max(abs(x0), _SCALES[j])
            cp = oracle.Problem(_set_param(inp, s, j, x0 + h)).chi2()
            cm = oracle.Problem(_set_param(inp, s, j, x0 - h)).chi2()
            fd = (cp - cm) / (2 * h)
            tol = 2e-6 * max(abs(fd), 1e-3 * np.abs(gs).max())
            assert abs(gs[s, j] - fd) < tol, (s, j, gs[s, j], fd)
    assert np.all(gs[0, 7:] == 0.0)


def test_gradient_jinc_beam_near_its_centre():
    """The Jinc beam's derivative on its power-series branch (x < 0.05): a
    source 1e-4 rad from the pointing centre, central differences in l, m."""
    inp = _random_small(seed=9, na=3, ntime=1, nchan=2, npsrc=1, ngsrc=0, pointing=0.0)
    inp["sources"]["lm"][:] = [[1e-4, -2e-4]]
    inp["uvw"][:] = 0.0      # K = 1: chi^2 depends on (l, m) through the beam alone
    inp["beam_model"] = 1
    inp["data"] = vis_all(inp) + inp["noise"] * 30
    _, gs, _ = oracle.Problem(inp).chi2_grad(want_gains=False)
    cnu = inp["beam_c"] * inp["freq"].max() * 1e-9
    assert cnu * np.hypot(1e-4, 2e-4) < 0.05
    for j in (0, 1):
        x0 = _get_param(inp, 0, j)
        h = 1e-6   # chi^2 is smooth here; a smaller step drowns the difference in rounding
        fd = (oracle.Problem(_set_param(inp, 0, j, x0 + h)).chi2()
              - oracle.Problem(_set_param(inp, 0, j, x0 - h)).chi2()) / (2 * h)
        assert abs(gs[0, j] - fd) < 1e-6 * abs(fd), (j, gs[0, j], fd)


@pytest.mark.parametrize("beam_model", [0, 1])
def test_gradient_matches_central_differences_gains(beam_model):
    inp = _fd_problem(beam_model)
    _, _, gg = oracle.Problem(inp).chi2_grad(want_gains=True)
    rng = np.random.default_rng(3)
    picks = [(rng.integers(2), rng.integers(4), rng.integers(3), rng.integers(4))
             for _ in range(12)]
    for (t, a, k, e) in picks:
        i, j = divmod(int(e), 2)
        fd = []
        for d in (1.0, 1j):
            h = 1e-6
            gp = inp["gains"].copy(); gp[t, a, k, i, j] += h * d
            gm = inp["gains"].copy(); gm[t, a, k, i, j] -= h * d
            fd.append((oracle.Problem(dict(inp, gains=gp)).chi2()
                       - oracle.Problem(dict(inp, gains=gm)).chi2()) / (2 * h))
        want = fd[0] + 1j * fd[1]
        got = gg[t, a, k, e]
        assert abs(got - want) < 1e-6 * max(abs(want), 1e-3 * np.abs(gg).max()), (t, a, k, e)


def test_gradient_stokes_closed_form_linear():
    """chi^2 is quadratic in each Stokes parameter: the gradient at x equals
    (chi2(x + h) - chi2(x - h)) / 2h exactly for any h."""
    inp = _fd_problem()
    _, gs, _ = oracle.Problem(inp).chi2_grad(want_gains=False)
    for j in range(2, 6):
        x0 = _get_param(inp, 1, j)
        h = 0.37
        fd = (oracle.Problem(_set_param(inp, 1, j, x0 + h)).chi2()
              - oracle.Problem(_set_param(inp, 1, j, x0 - h)).chi2()) / (2 * h)
        assert gs[1, j] == pytest.approx(fd, rel=1e-9, abs=1e-12)


def test_reduced_phase_exact_binary_fractions():
    """nu tau - round(nu tau) for nu = 2^30 Hz and tau = (k + f) 2^-30 s, whose
    product is exactly k + f: the remainder is f, with its sign, for large k
    (rounding to the nearest integer, not down or toward zero)."""
    nu = np.full(12, 2.0 ** 30)
    k = np.array([0, 1, 17, 123456, -5, -77, 3, 9, 250, -250, 1000, 40])
    f = np.array([0.25, -0.375, 0.125, 0.4375, -0.25, 0.375, -0.125, 0.0, 0.3125, -0.3125, 0.0625, -0.0625])
    tau = (k + f) * 2.0 ** -30
    np.testing.assert_array_equal(oracle.reduced_phase(nu, tau), f)


def test_reduced_phase_range_ties_and_phase_factor():
    """The remainder lies in [-1/2, 1/2] (halves go to the even integer), and
    exp(2 pi i r) equals exp(2 pi i nu tau) (eq. 3's factor), checked with
    Python's own cos and sin at moderate arguments."""
    import math
    nu = np.full(4, 2.0 ** 30)
    tau = np.array([2.5, 3.5, -2.5, -3.5]) * 2.0 ** -30
    np.testing.assert_array_equal(oracle.reduced_phase(nu, tau), [0.5, -0.5, -0.5, 0.5])
    rng = np.random.default_rng(5)
    nu = rng.uniform(1e9, 1.5e9, 200)
    tau = rng.uniform(-1e-7, 1e-7, 200)
    r = oracle.reduced_phase(nu, tau)
    assert np.all(np.abs(r) <= 0.5)
    for a, b, x in zip(nu, tau, r):
        ph = 2 * math.pi * a * b
        assert abs(math.cos(2 * math.pi * x) - math.cos(ph)) < 1e-12
        assert abs(math.sin(2 * math.pi * x) - math.sin(ph)) < 1e-12
