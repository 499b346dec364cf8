"""The replica (multi-GPU) path on CPU: two gloo ranks each solve a disjoint
packet-id range and sum their tallies; the sum equals the unsplit solve
(integer tallies exactly, FP64 peel-off tallies to summation order).  The
ranks run the oracle, since no GPU is present; the partition and the
reduction are the product's (paper_1409_4480_gb300/replicas.py)."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1409_4480_gb300 import replicas
from paper_1409_4480_gb300 import synth as S


def _spec(diffuse=False):
    return S.RunSpec(n_packets=1001, seed=77, albedo=0.32, spec_units=1, spec_lo=-400, spec_hi=400, spec_nbins=40,
                     cameras=S.axis_cameras(4), cam_lo=-400, cam_hi=400, cam_nbins=20, source=int(diffuse))


def _grid(diffuse=False):
    g = S.sphere(10, 1e4, 1e4, v_max_kms=60.0, tau_dust=0.8)
    if diffuse:
        # diffuse emission in proportion to n^2 (recombination-like)
        g.lum = np.asarray(g.n_HI, np.float64) ** 2 + 1e-3
    return g


def _rank_main(rank, world, port, outdir, diffuse=False):
    import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    spec = _spec(diffuse)
    first, n = replicas.packet_range(spec.n_packets, rank, world)
    spec.n_packets, spec.pid_offset = n, first
    r = O.run(_grid(diffuse), spec, images=True)
    tot = replicas.allreduce_tallies(r)
    if rank == 0:
        np.savez(os.path.join(outdir, "sum.npz"), **{k: np.asarray(tot[k]) for k in
                                                      replicas.INT_KEYS + replicas.FLOAT_KEYS if k in tot})
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_packet_range_partitions():
    for n in (0, 1, 7, 1000, 1001):
        for w in (1, 2, 3, 8):
            parts = [replicas.packet_range(n, r, w) for r in range(w)]
            assert sum(c for _, c in parts) == n
            assert all(parts[i][0] + parts[i][1] == parts[i + 1][0] for i in range(w - 1))
            assert max(c for _, c in parts) - min(c for _, c in parts) <= 1
    with pytest.raises(ValueError):
        replicas.packet_range(10, 2, 2)


@pytest.mark.parametrize("diffuse", [False, True])
def test_two_gloo_replicas_sum_to_the_whole(O, tmp_path, diffuse):
    mp.start_processes(_rank_main, args=(2, _free_port(), str(tmp_path), diffuse), nprocs=2, join=True,
                       start_method="spawn")
    got = np.load(tmp_path / "sum.npz")
    whole = O.run(_grid(diffuse), _spec(diffuse), images=True)
    for k in replicas.INT_KEYS:
        assert np.array_equal(got[k], np.asarray(whole[k])), k
    for k in replicas.FLOAT_KEYS:
        assert np.allclose(got[k], whole[k], rtol=1e-12, atol=1e-300), k
    assert int(got["n_emitted"]) == 1001
