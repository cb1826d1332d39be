"""Time sharding over ranks (paper_1501_07719_gb300.shard) on the CPU: the
chunking, the observation slices, and a two-rank gloo run whose summed
per-rank chi^2 (each rank's slice evaluated by the FP64 oracle) equals the
oracle's chi^2 of the whole observation."""
import os
import socket

import numpy as np
import pytest

import oracle
import rime_synth
from paper_1501_07719_gb300 import shard


def _case(time_varying=False):
    inp = rime_synth.make_inputs(rime_synth.custom(6, 7, 3, 4, 2, seed_index=81), precision="f64",
                                 time_varying=time_varying, pointing_sigma=0.003)
    inp["data"] = rime_synth.observe(oracle.Problem(inp).predict(), inp["noise"], "f64")
    return inp


@pytest.mark.parametrize("ntime,world", [(7, 2), (7, 3), (2, 4), (100, 8), (1, 1)])
def test_time_chunks_are_contiguous_balanced_and_complete(ntime, world):
    chunks = [shard.time_chunk(ntime, r, world) for r in range(world)]
    assert chunks[0][0] == 0 and chunks[-1][1] == ntime
    for (a0, a1), (b0, b1) in zip(chunks, chunks[1:]):
        assert a1 == b0
    sizes = [b - a for a, b in chunks]
    assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 0
    with pytest.raises(ValueError):
        shard.time_chunk(ntime, world, world)


@pytest.mark.parametrize("time_varying", [False, True])
def test_slices_add_up_to_the_whole(time_varying):
    inp = _case(time_varying)
    whole = oracle.Problem(inp, data=inp["data"]).chi2()
    parts = 0.0
    for r in range(3):
        t0, t1 = shard.time_chunk(inp["ntime"], r, 3)
        sl = shard.slice_observation(inp, t0, t1)
        assert sl["ntime"] == t1 - t0 and sl["uvw"].shape[0] == t1 - t0
        parts += oracle.Problem(sl, data=sl["data"]).chi2()
    assert abs(parts - whole) <= 1e-12 * whole


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_path, time_varying):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    inp = _case(time_varying)
    t0, t1 = shard.time_chunk(inp["ntime"], rank, world)
    sl = shard.slice_observation(inp, t0, t1)
    part = oracle.Problem(sl, data=sl["data"]).chi2()
    total = shard.reduce_sum(part)
    slowest = shard.reduce_max(float(rank + 1))
    if rank == 0:
        np.save(out_path, np.array([total, slowest]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("time_varying", [False, True])
def test_two_rank_gloo_sum_equals_whole_chi2(tmp_path, time_varying):
    import torch.multiprocessing as mp
    out = str(tmp_path / "result.npy")
    mp.start_processes(_rank_main, args=(2, _free_port(), out, time_varying), nprocs=2, join=True,
                       start_method="spawn")
    total, slowest = np.load(out)
    inp = _case(time_varying)
    whole = oracle.Problem(inp, data=inp["data"]).chi2()
    assert abs(total - whole) <= 1e-12 * whole
    assert slowest == 2.0


def test_reduce_without_a_process_group_is_identity():
    assert shard.reduce_sum(3.5) == 3.5 and shard.reduce_max(-1.0) == -1.0
