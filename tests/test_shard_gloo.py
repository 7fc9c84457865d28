"""The host-side logic of the aux-sharded Fock build on two gloo ranks (CPU):
each rank holds the rows aux_ranges(Naux, 2)[rank] of the oracle's B for
(H2O)_2, forms its partial J and K with the oracle's contraction of those
rows, and shard.allreduce_jk sums them; every rank must then hold the full
oracle J and K.  (The device side, bqc_df_build with an aux range and
bqc_jk's partials, is tested on the GPU in test_gpu_shard.py.)"""
import os
import socket

import numpy as np


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import oracle
    import workload
    from paper_2502_17963_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mol = workload.water_cluster(2)
    I = oracle.system_integrals(mol)
    B, _ = oracle.df_tensor(I["aux"], I["orb"])
    rng = np.random.default_rng(9)
    C = rng.standard_normal((B.shape[1], mol.nocc)) * 0.3
    p0, p1 = shard.aux_ranges(B.shape[0], world)[rank]
    Jl, Kl = oracle.jk_df(B[p0:p1], C)
    J, K = torch.tensor(Jl), torch.tensor(Kl)
    shard.allreduce_jk(J, K)
    Jf, Kf = oracle.jk_df(B, C)
    q.put((rank, float(np.abs(J.numpy() - Jf).max()), float(np.abs(K.numpy() - Kf).max()),
           (p0, p1)))
    dist.destroy_process_group()


def test_sharded_partials_sum_to_full_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=180) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, dj, dk, rng in out:
        assert dj < 1e-12 and dk < 1e-12, (rank, dj, dk)
    assert out[0][3][0] == 0 and out[0][3][1] == out[1][3][0]


def test_aux_ranges_cover_once():
    from paper_2502_17963_gb300 import shard
    for naux, world in ((150, 2), (4800, 8), (7, 7), (10, 3)):
        r = shard.aux_ranges(naux, world)
        assert r[0][0] == 0 and r[-1][1] == naux
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        sizes = [q - p for p, q in r]
        assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
