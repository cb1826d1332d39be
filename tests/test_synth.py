"""The seeded input generator: deterministic, right shapes and distributions."""
import numpy as np

import rime_synth as rs


def test_deterministic_and_independent_streams():
    a = rs.make_inputs("7ant-10t-16ch-10pt")
    b = rs.make_inputs("7ant-10t-16ch-10pt")
    for k in ("uvw", "gains", "noise", "weight"):
        np.testing.assert_array_equal(a[k], b[k])
    c = rs.make_inputs("7ant-10t-16ch-10pt", seed=rs.SEED_BASE + 99)
    assert not np.array_equal(a["uvw"], c["uvw"])


def test_shapes_and_ranges():
    inp = rs.make_inputs("64ant-100t-64ch-100pt100g")
    assert inp["uvw"].shape == (100, 64, 3) and np.abs(inp["uvw"]).max() <= 1000
    assert inp["noise"].shape == (100, 2016, 64, 4)
    assert inp["gains"].shape == (100, 64, 64, 2, 2)
    s = inp["sources"]
    assert s["lm"].shape == (200, 2) and np.abs(s["lm"]).max() <= 0.01
    assert (s["stokes"][:, 0] >= 0.1).all() and (s["stokes"][:, 0] <= 10).all()
    assert (np.abs(s["stokes"][:, 1:]) <= 0.05 * s["stokes"][:, :1]).all()
    assert (s["shape"][:100] == 0).all()
    g = s["shape"][100:]
    assert (g[:, 0] >= g[:, 1]).all() and (g[:, 1] >= 1e-5).all() and (g[:, 0] <= 1e-4).all()
    assert (inp["weight"] >= 0.5).all() and (inp["weight"] <= 2).all()
    np.testing.assert_allclose(inp["freq"][[0, -1]], [1.0e9, 1.5e9])


def test_f32_rounding_is_exact_upcast():
    inp = rs.make_inputs("7ant-10t-16ch-10pt", precision="f32")
    for x in (inp["uvw"], inp["sources"]["lm"], inp["weight"]):
        np.testing.assert_array_equal(x, x.astype(np.float32).astype(np.float64))
    d = rs.observe(np.zeros_like(inp["noise"]), inp["noise"], "f32")
    assert d.dtype == np.complex64


def test_batched_sets():
    inp = rs.make_inputs("64ant-50t-32ch-512sets")
    off = inp["sets"]["offsets"]
    counts = np.diff(off)
    assert len(counts) == 512 and counts.min() >= 5 and counts.max() <= 500
    frac_g = (inp["sets"]["sources"]["shape"][:, 0] > 0).mean()
    assert 0.45 < frac_g < 0.55


def test_baseline_order():
    p, q = rs.baseline_pairs(4)
    assert list(zip(p, q)) == [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
