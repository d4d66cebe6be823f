"""World-size-2 gloo ranks on the CPU.

* The DF Fock build is additive over the auxiliary index P (J = sum_P B_P (B_P . D),
  K = sum_P X_P X_P^T), which is what lets it shard across GPUs: each rank builds partial
  J and K from its slice of P with the oracle and an all_reduce sums them; the result
  must equal the unsliced build.
* bench.py's rank aggregation (maximum step time over ranks) under gloo."""
import os
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import gen
    import oracle
    from oracle import scf as oscf
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mol = gen.make_molecule(6, 4.0, 3)
    sysm = oscf.build_system(mol)
    C, _ = oscf.core_guess(sysm)
    D = 2 * C @ C.T
    sl = np.array_split(np.arange(mol.naux), world)[rank]
    Jp = oracle.df_j(np.ascontiguousarray(sysm.B[sl]), mol.nao, D)
    Kp = oracle.df_k(np.ascontiguousarray(sysm.B[sl]), mol.nao, C)
    t = torch.tensor(np.stack([Jp, Kp]))
    dist.all_reduce(t)
    J, K = t[0].numpy(), t[1].numpy()
    Jf = oracle.df_j(sysm.B, mol.nao, D)
    Kf = oracle.df_k(sysm.B, mol.nao, C)
    step_ms = 10.0 + rank
    mx = bench.max_over_ranks(step_ms, device="cpu")
    out.put((rank, float(np.max(np.abs(J - Jf)) / np.max(np.abs(Jf))),
             float(np.max(np.abs(K - Kf)) / np.max(np.abs(Kf))), mx))
    dist.destroy_process_group()


def test_p_sharded_jk_reduction_and_rank_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ej, ek, mx in res:
        assert ej <= 1e-12 and ek <= 1e-12
        assert mx == 11.0
