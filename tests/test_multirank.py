"""Multi-rank path on CPU (gloo, world size 2): each rank simulates its own photon-id
range, as bench.py does with one rank per GPU, and the ranks' results sum to a single run
over the union of the ranges.  The ranks run the FP64 oracle (no GPU here); the sharding
arithmetic and the composition property are what is under test."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n_per_rank, out_dir):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch
    import oracle
    import workloads
    from paper_1711_03244_gb300 import photon_range
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = workloads.c2(n_photons=n_per_rank)
    off, n = photon_range(rank, world, n_per_rank)
    r = oracle.run(wl, n_photons=n, photon_offset=off, n_threads=1)
    energy = torch.from_numpy(r.energy.copy())
    tally = torch.tensor([r.tally[k] for k in oracle.TALLY_NAMES], dtype=torch.float64)
    det_n = torch.tensor([r.det_n], dtype=torch.int64)
    for t in (energy, tally, det_n):
        dist.all_reduce(t)
    if rank == 0:
        np.save(os.path.join(out_dir, "energy.npy"), energy.numpy())
        np.save(os.path.join(out_dir, "tally.npy"), tally.numpy())
        np.save(os.path.join(out_dir, "det_n.npy"), det_n.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_photon_ranges_shard_across_two_ranks(tmp_path, orc):
    import workloads
    world, n = 2, 300
    mp.start_processes(_rank_main, args=(world, _free_port(), n, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    energy = np.load(tmp_path / "energy.npy")
    tally = np.load(tmp_path / "tally.npy")
    det_n = int(np.load(tmp_path / "det_n.npy")[0])
    full = orc.run(workloads.c2(n_photons=world * n))
    assert np.allclose(energy, full.energy, rtol=1e-12, atol=1e-15)
    assert np.allclose(tally, [full.tally[k] for k in orc.TALLY_NAMES], rtol=1e-12)
    assert det_n == full.det_n


def test_photon_range_arithmetic():
    from paper_1711_03244_gb300 import photon_range
    assert photon_range(0, 4, 10) == (0, 10)
    assert photon_range(3, 4, 10) == (30, 10)
    with pytest.raises(ValueError):
        photon_range(4, 4, 10)
