"""Multi-rank path on the CPU: two gloo ranks, each solving its own block of
instances with the FP64 oracle. Instances are independent, so the gathered
shards equal the unsharded result exactly and no data-path exchange exists;
the only collective is the max over ranks of the elapsed time."""

import os
import socket

import numpy as np
import pytest

from paper_1404_0424_gb300 import shard

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("n,world", [(0, 1), (7, 1), (7, 2), (8, 3), (1200, 4), (3, 5)])
def test_instance_range_partitions_exactly(n, world):
    seen = []
    sizes = []
    for r in range(world):
        a, b = shard.instance_range(n, r, world)
        seen.extend(range(a, b))
        sizes.append(b - a)
    assert seen == list(range(n))
    assert max(sizes) - min(sizes) <= 1


def test_instance_range_rejects_bad_arguments():
    for args in [(5, 2, 2), (5, -1, 2), (5, 0, 0), (-1, 0, 1)]:
        with pytest.raises(ValueError):
            shard.instance_range(*args)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import oracle
    from paper_1404_0424_gb300 import workload as wl
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        d = wl.uplink(16, 4, 4, n=9, R=2, snr_db=10.0, seed=5)
        a, b = shard.instance_range(9, rank, world)
        ref = oracle.cg_detect(d["H"][a:b], d["Y"][a:b], d["N0"], d["Es"], 3, 4)
        np.save(os.path.join(out_dir, f"x{rank}.npy"), ref["x_hat"])
        np.save(os.path.join(out_dir, f"l{rank}.npy"), ref["llr"])
        m = shard.max_over_ranks(float(rank + 1), dist)
        np.save(os.path.join(out_dir, f"m{rank}.npy"), np.array([m]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_without_exchange(tmp_path):
    import torch.multiprocessing as mp

    import oracle
    from paper_1404_0424_gb300 import workload as wl
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    d = wl.uplink(16, 4, 4, n=9, R=2, snr_db=10.0, seed=5)
    full = oracle.cg_detect(d["H"], d["Y"], d["N0"], d["Es"], 3, 4)
    x = np.concatenate([np.load(tmp_path / f"x{r}.npy") for r in range(world)])
    llr = np.concatenate([np.load(tmp_path / f"l{r}.npy") for r in range(world)])
    assert np.array_equal(x, full["x_hat"])
    assert np.array_equal(llr, full["llr"])
    for r in range(world):
        assert float(np.load(tmp_path / f"m{r}.npy")[0]) == float(world)
