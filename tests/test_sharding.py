"""Multi-rank path on CPU: world_size-2 gloo ranks shard instances, run them
(the CPU oracle stands in for the GPU batch of each rank) and gather the
per-instance results, which must equal a single-process run."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1501_05630_gb300 import sharding


def test_instance_ranges_are_disjoint_and_cover():
    ids = [sharding.instance_range(r, 4, 250) for r in range(4)]
    allv = np.concatenate(ids)
    assert len(np.unique(allv)) == 1000 and allv.min() == 0 and allv.max() == 999
    for n in (0, 1, 7, 1000):
        parts = [sharding.split_instances(n, r, 3) for r in range(3)]
        assert np.array_equal(np.concatenate(parts), np.arange(n))
        assert max(map(len, parts)) - min(map(len, parts)) <= 1
    with pytest.raises(ValueError):
        sharding.instance_range(2, 2, 10)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path):
    import torch.distributed as dist
    from oracle import oracle as O
    from paper_1501_05630_gb300 import inputs as I
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = O.Geometry(O.SQUARE2D, 4)
    T = I.ladder(0.4, 1.5, 4)
    ids = sharding.instance_range(rank, world, 3)
    rows = []
    for i in ids:
        J = I.couplings(g.Nb, I.PM_J, 9, [int(i)])[0].astype(np.float64)
        s0 = I.initial_spins(g.N, 8, 9, [int(i)])[0]
        inst = O.Instance(g, J, T, s0, pm=True, T_icm=1.0, seed=9, inst=int(i))
        inst.run(50)
        rows.append(np.concatenate([inst.E, inst.acc_d.astype(np.float64)]))
    all_ids, all_rows = sharding.gather_rows(np.array(rows), ids)
    if rank == 0:
        np.savez(out_path, ids=all_ids, rows=all_rows)
    dist.destroy_process_group()


def test_two_rank_gloo_gather_matches_single_process(tmp_path):
    from oracle import oracle as O
    from paper_1501_05630_gb300 import inputs as I
    out = str(tmp_path / "g.npz")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    got = np.load(out)
    g = O.Geometry(O.SQUARE2D, 4)
    T = I.ladder(0.4, 1.5, 4)
    want = []
    for i in range(6):
        J = I.couplings(g.Nb, I.PM_J, 9, [i])[0].astype(np.float64)
        s0 = I.initial_spins(g.N, 8, 9, [i])[0]
        inst = O.Instance(g, J, T, s0, pm=True, T_icm=1.0, seed=9, inst=i)
        inst.run(50)
        want.append(np.concatenate([inst.E, inst.acc_d.astype(np.float64)]))
    assert np.array_equal(got["ids"], np.arange(6))
    assert np.array_equal(got["rows"], np.array(want))
