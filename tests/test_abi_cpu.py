"""The C-ABI library without a GPU: it loads, exports every entry point that
include/*.h declares, and rejects bad arguments before any CUDA call."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    import paper_1501_07719_gb300 as R
    if not os.path.exists(R._abi.LIB_PATH):
        from paper_1501_07719_gb300 import build
        build.build()
    return R._abi.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(rime_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_entry_points():
    names = declared_functions()
    for want in ("rime_create", "rime_set_sources", "rime_predict", "rime_chi2", "rime_destroy"):
        assert want in names


def test_every_declared_symbol_is_exported(L):
    for name in declared_functions():
        assert hasattr(L, name), name


def test_nbl_and_status_strings(L):
    import paper_1501_07719_gb300 as R
    assert R.rime_nbl(64) == 2016 and R.rime_nbl(7) == 21 and R.rime_nbl(1) == 0
    assert L.rime_status_string(1) == b"RIME_E_INVALID"


def _split_pair_counts(na, tiles):
    """How often each baseline p < q is formed by the split kernel's tiles,
    with its epilogue's rule: within one group p < q only, across groups
    every (row, column) pair (the tile holds one orientation of the pair)."""
    cnt = np.zeros((na, na), dtype=np.int64)
    for c, *rows in tiles:
        cols = np.arange(32 * c, min(32 * c + 32, na))
        for r in rows:
            if r < 0:
                continue
            for p in range(32 * r, min(32 * r + 32, na)):
                q = cols[cols > p] if r == c else cols
                lo, hi = np.minimum(p, q), np.maximum(p, q)
                np.add.at(cnt, (lo, hi), 1)
    return cnt


@pytest.mark.parametrize("na", [2, 3, 31, 32, 33, 64, 95, 129, 200, 256, 257, 300])
def test_split_tile_plan_forms_every_baseline_once(L, na):
    import paper_1501_07719_gb300 as R
    tiles = R.rime_split_tiles(na)
    G = (na + 31) // 32
    assert tiles.shape[1] == 5 and np.all((tiles >= -1) & (tiles < G))
    assert np.all(tiles[:, 1] >= 0)                      # slot 0 always holds a group
    cnt = _split_pair_counts(na, tiles)
    iu = np.triu_indices(na, 1)
    assert np.all(cnt[iu] == 1)
    assert cnt[np.tril_indices(na)].sum() == 0


def test_split_tile_plan_counts_and_range(L):
    import paper_1501_07719_gb300 as R
    # at least ceil(G (G + 1) / 8) tiles for G groups (G (G - 1) / 2 group pairs plus G own
    # groups, four per tile) and at least G (each group's own baselines need a tile of its
    # own column group); the plan reaches that bound
    for na in list(range(2, 4097, 7)) + [4096]:
        G = (na + 31) // 32
        n = len(R.rime_split_tiles(na))
        assert n == max(G, -(-G * (G + 1) // 8)), na
    assert len(R.rime_split_tiles(256)) == 9
    assert len(R.rime_split_tiles(128)) == 4
    for bad in (1, 0, 4097):
        assert L.rime_split_tiles(bad, None, 0) == -1
    assert L.rime_split_tiles(64, None, -1) == -1
    assert L.rime_split_tiles(64, None, 2) == -1          # out NULL with cap > 0
    assert L.rime_split_tiles(64, None, 0) == 2


@pytest.mark.parametrize("kw,msg", [
    (dict(na=1), "na"),
    (dict(na=5000), "na"),
    (dict(ntime=0), "ntime"),
    (dict(nchan=0), "nchan"),
    (dict(precision=7), "precision"),
    (dict(ref_freq_hz=0.0), "ref_freq"),
    (dict(ref_freq_hz=float("nan")), "ref_freq"),
    (dict(beam_c=-1.0), "beam_c"),
    (dict(freq=None), "freq"),
    (dict(uvw=None), "uvw"),
])
def test_create_rejects_bad_arguments_without_cuda(L, kw, msg):
    import paper_1501_07719_gb300 as R
    args = dict(na=4, ntime=2, nchan=3, precision=R.RIME_FP64, freq=np.linspace(1e9, 1.5e9, 3),
                uvw=np.zeros((2, 4, 3)), ref_freq_hz=1.4e9, beam_c=65.0)
    args.update(kw)
    with pytest.raises(R.RimeError) as e:
        R.rime_create(args["na"], args["ntime"], args["nchan"], args["precision"], args["freq"],
                      args["uvw"], ref_freq_hz=args["ref_freq_hz"], beam_c=args["beam_c"])
    assert e.value.status == R._abi.RIME_E_INVALID
    assert msg in str(e.value)


def test_null_context_calls_are_rejected(L):
    assert L.rime_predict(None, None) == 1
    assert L.rime_chi2(None, None) == 1
    assert L.rime_sync(None) == 1
    assert L.rime_chi2_batched(None, 0, None, None, None) == 1
    assert L.rime_batched_config(None, None) == 1
    assert L.rime_set_batched_config(None, None) == 1
    assert L.rime_set_kernel(None, 0) == 1
    assert L.rime_set_beam(None, 0, 65.0) == 1
    assert L.rime_chains_init(None, 4) == 1
    assert L.rime_chains_propose(None, 1, None, None, None) == 1
    assert L.rime_chains_accept(None, None) == 1
    assert L.rime_chi2_streamed(None, None, None, 0, None) == 1
    assert L.rime_stream_chunk_ntime(None) == 0
    assert L.rime_set_tensor_mode(None, 0) == 1
    L.rime_destroy(None)   # ignored


def test_binding_fails_loudly_when_library_missing(monkeypatch, tmp_path):
    import paper_1501_07719_gb300._abi as A
    monkeypatch.setattr(A, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(A, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        A.lib()
