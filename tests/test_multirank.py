"""The multi-rank host path on CPU ranks (gloo, world size 2).

Replicas only: blocks are independent (Sec. 2.2), so ranks share no data
path.  What the ranks do exchange is checked here without a GPU:
  * the field's global range (min/max all-reduce), so every rank thresholds
    with the same t;
  * per-rank streams of z-slabs, joined on rank 0 by cz_stream_concat (the
    exclusive scan of per-rank sizes rebases the offsets) -- the result must
    equal the whole field's stream byte for byte;
  * the benchmark's timing reduction (maximum over ranks) and its whole-job
    throughput.
The per-rank streams come from the CPU oracle (no GPU here); the library's
host-side join is what is under test.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, B, dtype_name, kind, group, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import oracle as O
    import bench
    from paper_1903_07761_gb300 import cz, inputs
    dtype = np.dtype(dtype_name)
    nz = world * 2 * B
    f = inputs.field(inputs.P, (nz, 2 * B, 3 * B), dtype, seed=77, nbubbles=5)
    slab = np.ascontiguousarray(f[rank * 2 * B:(rank + 1) * 2 * B])
    # global range by all-reduce of the slab extrema
    mm = torch.tensor([-float(slab.min()), float(slab.max())], dtype=torch.float64)
    dist.all_reduce(mm, op=dist.ReduceOp.MAX)
    rng = float(mm[1]) - (-float(mm[0]))
    s = O.compress(slab, B, kind, 1e-3, O.EPS_REL, True, range_=rng, group=group)
    got = [None] * world
    dist.all_gather_object(got, s)
    # timing reduction of the benchmark: the slowest rank counts
    times = bench.rank_max([10.0 + rank, 5.0 * (1 - rank)], "cpu")
    if rank == 0:
        joined = cz.stream_concat(got)
        whole = O.compress(f, B, kind, 1e-3, O.EPS_REL, True, range_=rng, group=group)
        ok = joined == whole
        rec = O.decompress(joined)
        np.save(os.path.join(out_dir, "result.npy"),
                np.array([ok, np.array_equal(rec.view(np.uint8), O.decompress(whole).view(np.uint8)),
                          times == [10.0 + world - 1, 5.0],
                          bench.replica_throughput(world, 1e9, 1000.0) == world * 1.0]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("B,dtype_name,kind,group", [(16, "float32", 2, 1), (8, "float64", 0, 1),
                                                     (16, "float32", 1, 4)])
def test_two_ranks_slab_streams_join_to_the_whole_field_stream(tmp_path, B, dtype_name, kind, group):
    """(group 4: aggregate chunks; each slab's 12 blocks are three whole groups)"""
    from paper_1903_07761_gb300 import cz
    cz.lib()  # build once in the parent
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), B, dtype_name, kind, group, str(tmp_path)), nprocs=world,
             join=True)
    res = np.load(tmp_path / "result.npy")
    assert res.tolist() == [True, True, True, True]


def test_concat_refuses_slabs_that_disagree():
    import oracle as O
    from paper_1903_07761_gb300 import cz
    rng = np.random.default_rng(1)
    a = rng.standard_normal((16, 16, 16)).astype(np.float32)
    s1 = O.compress(a, 16, O.W4, 1e-3, O.EPS_REL, True, range_=10.0)
    s2 = O.compress(a, 16, O.W4, 1e-3, O.EPS_REL, True, range_=11.0)  # another threshold
    with pytest.raises(cz.CzError) as e:
        cz.stream_concat([s1, s2])
    assert e.value.code == cz.ERR_ARG
    s3 = O.compress(a, 16, O.W3AI, 1e-3, O.EPS_REL, True, range_=10.0)  # another kind
    with pytest.raises(cz.CzError):
        cz.stream_concat([s1, s3])
    assert cz.stream_concat([s1]) == s1


def test_concat_of_group_streams_needs_whole_groups_but_in_the_last_slab():
    import oracle as O
    from paper_1903_07761_gb300 import cz
    rng = np.random.default_rng(2)
    a = rng.standard_normal((48, 32, 48)).astype(np.float32)  # 3 x 2 x 3 = 18 blocks of 16^3

    def comp(x):
        return O.compress(np.ascontiguousarray(x), 16, O.W3AI, 1e-3, O.EPS_REL, True, range_=9.0, group=4)

    # slabs of 6 blocks: the first one ends in a partial group
    with pytest.raises(cz.CzError) as e:
        cz.stream_concat([comp(a[:16]), comp(a[16:32])])
    assert e.value.code == cz.ERR_ARG
    # 12 blocks (three whole groups), then a last slab of 6 blocks (a partial
    # last group): the whole field's stream
    assert cz.stream_concat([comp(a[:32]), comp(a[32:])]) == comp(a)
