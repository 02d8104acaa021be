"""Multi-rank path on CPU: two gloo ranks each transport a disjoint packet-id
range (frozen temperatures) and sum their outputs with the package's
all-reduce; the result equals one process transporting every packet.  The
per-rank transport here is the FP64 CPU reference (no GPU on this host); the
code under test is the sharding and reduction logic, on a uniform grid and
on a grid with one level of refinement."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _model(kind):
    m = W.random_grid(n=(5, 4, 6), ns=2, seed=8, tau_scale=2.0)
    if kind == "refined":
        mask = np.random.default_rng(2).random(m.rho.shape[1:]) < 0.4
        m = W.refine_cubes(m, mask, r=2, jitter=0.4, seed=2)
    return m


def _rank(rank, world, port, N, q, kind="uniform"):
    import torch.distributed as dist
    from oracle import oracle as O
    from paper_1203_2941_gb300.shard import allreduce_mean, allreduce_sum, packet_range
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m = _model(kind)
    T0 = np.full((2, m.ncell), 180.0)
    b, e = packet_range(N, rank, world)
    r = O.transport(m, N, seed=3, mode=O.MODE_FROZEN_T, T_prev=T0, pid_begin=b, pid_end=e)
    E = torch.tensor(r["E_abs"])
    cnt = torch.tensor(r["count"].astype(np.int64))
    sed = torch.tensor(r["sed_esc"])
    allreduce_sum([E, cnt, sed])
    rep = torch.tensor([float(rank + 1)])
    allreduce_mean([rep])
    if rank == 0:
        q.put((E.numpy(), cnt.numpy(), sed.numpy(), float(rep.item())))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["uniform", "refined"])
def test_two_rank_packet_sharding_equals_single_run(O, kind):
    from paper_1203_2941_gb300.shard import packet_range
    assert packet_range(10, 0, 3) == (0, 3) and packet_range(10, 2, 3) == (6, 10)
    N = 3000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, N, q, kind)) for r in range(2)]
    for p in procs:
        p.start()
    E, cnt, sed, rep = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    m = _model(kind)
    full = O.transport(m, N, seed=3, mode=O.MODE_FROZEN_T, T_prev=np.full((2, m.ncell), 180.0))
    np.testing.assert_array_equal(cnt, full["count"].astype(np.int64))
    np.testing.assert_allclose(E, full["E_abs"], rtol=1e-12, atol=0)
    np.testing.assert_allclose(sed, full["sed_esc"], rtol=1e-12, atol=0)
    assert rep == pytest.approx(1.5)
