"""The multi-GPU drivers of paper_1203_2941_gb300.shard on CPU: two gloo ranks
run the iterative scheme sharded by packet id (transport of each rank's
packet range, one sum of the accumulators per iteration, Eq. 4
temperatures), gather the scattering events, trace the cameras sharded
round robin and sum the adjoint's density gradients.  The result equals the
same drivers run by one process.  The per-rank operations come from a small
backend around the FP64 CPU oracle (no GPU on this host); the code under
test is the drivers' partitioning, collectives and reassembly, on a uniform
grid and on a grid with one level of refinement."""
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
    m = W.random_grid(n=(5, 4, 6), ns=2, seed=8, tau_scale=2.0, albedo=(0.3, 0.7))
    if kind == "refined":
        mask = np.random.default_rng(2).random(m.rho.shape[1:]) < 0.4
        m = W.refine_cubes(m, mask, r=2, jitter=0.4, seed=2)
    return m


CAMS = [W.Camera(0.5, 0.2, 9, 1e18), W.Camera(1.2, -0.7, 9, 1e18), W.Camera(2.4, 1.9, 9, 1e18)]
FIDX = [1, 4, 6]


class OracleBackend:
    """One rank's operations by the FP64 CPU oracle, on torch CPU tensors;
    events travel as the library's 20-byte records."""

    def __init__(self, m):
        from oracle import oracle as O
        from paper_1203_2941_gb300 import rtgb as R
        self.O, self.R, self.m = O, R, m
        self.device = torch.device("cpu")
        self.xi = None
        self._ev = None

    def transport(self, T_prev, pid_begin, pid_end, n_packets, seed):
        O = self.O
        r = O.transport(self.m, n_packets, seed=seed, mode=O.MODE_FROZEN_T, T_prev=T_prev.numpy(),
                        pid_begin=pid_begin, pid_end=pid_end, record_events=True,
                        event_cap=50 * n_packets)
        self.xi = r["xi"]
        ev = r["events"]
        rec = np.zeros(len(ev), self.R.EVENT_DTYPE)
        rec["cell"], rec["nu"], rec["species"] = ev["cell"], ev["nu"], ev["species"]
        rec["k"] = ev["k"]
        self._ev = torch.from_numpy(rec.view(np.uint8).copy()) if len(ev) else None
        st = np.array([r["stats"][k] for k in O.STAT_NAMES], dtype=np.int64)
        return {"E_abs": torch.tensor(r["E_abs"]), "count": torch.tensor(r["count"].astype(np.int64)),
                "esq": torch.tensor(r["esq"]), "sed_esc": torch.tensor(r["sed_esc"]),
                "sed_cnt": torch.tensor(r["sed_cnt"].astype(np.int64)), "stats": torch.tensor(st)}

    def temperatures(self, E_abs):
        return torch.tensor(self.O.temperatures(self.m, E_abs.numpy()))

    def events(self):
        return self._ev

    def _oracle_events(self, events):
        if events is None:
            return None
        rec = events.numpy().view(self.R.EVENT_DTYPE)
        ev = np.zeros(len(rec), self.O.EVENT_DTYPE)
        ev["cell"], ev["nu"], ev["species"] = rec["cell"], rec["nu"], rec["species"]
        ev["k"] = rec["k"]
        return ev

    def image_shape(self, n_cams):
        return (n_cams, len(FIDX), CAMS[0].npix, CAMS[0].npix)

    def sed_shape(self, n_cams):
        return (n_cams, len(FIDX))

    def raytrace(self, T, events, cams):
        img, sed = self.O.raytrace(self.m, T.numpy(), self._oracle_events(events), self.xi, cams, FIDX)
        return torch.tensor(img, dtype=torch.float32), torch.tensor(sed)

    def raytrace_backward(self, T, events, cams, dimg, dsed):
        drho, ds = self.O.raytrace_backward(self.m, T.numpy(), self._oracle_events(events), self.xi,
                                            cams, FIDX, dimg.numpy().astype(np.float64), dsed.numpy())
        return torch.tensor(drho, dtype=torch.float32), torch.tensor([ds], dtype=torch.float64)

    def zero_gradient(self):
        return torch.zeros((self.m.ns, self.m.ncell), dtype=torch.float32), torch.zeros(1, dtype=torch.float64)


def _solve(kind, rank, world, N):
    from paper_1203_2941_gb300 import shard
    m = _model(kind)
    be = OracleBackend(m)
    T0 = torch.full((m.ns, m.ncell), 180.0, dtype=torch.float64)
    T, out, ev = shard.frozen_t_iterations(be, T0, 2, N, seed=3, rank=rank, world=world)
    events = shard.gather_events(ev, world)
    img, sed = shard.raytrace_views(be, T, events, CAMS, rank, world)
    g = torch.Generator().manual_seed(4)
    dimg = torch.randn(be.image_shape(len(CAMS)), generator=g)
    dsed = torch.randn(be.sed_shape(len(CAMS)), generator=g, dtype=torch.float64)
    drho, dscale = shard.raytrace_views_backward(be, T, events, CAMS, dimg, dsed, rank, world)
    return {"T": T.numpy(), "E": out["E_abs"].numpy(), "cnt": out["count"].numpy(),
            "sed_esc": out["sed_esc"].numpy(), "stats": out["stats"].numpy(),
            "events": None if events is None else events.numpy(), "img": img.numpy(),
            "sed": sed.numpy(), "drho": drho.numpy(), "dscale": dscale.numpy()}


def _rank(rank, world, port, N, q, kind):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = _solve(kind, rank, world, N)
    if rank == 0:
        q.put(res)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["uniform", "refined"])
def test_two_rank_sharded_solve_equals_single_process(O, kind):
    from paper_1203_2941_gb300.shard import cameras_of, packet_range
    assert packet_range(10, 0, 3) == (0, 3) and packet_range(10, 2, 3) == (6, 10)
    assert cameras_of(5, 1, 2) == [1, 3] and cameras_of(1, 1, 2) == []
    N = 2000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, N, q, kind)) for r in range(2)]
    for p in procs:
        p.start()
    two = q.get(timeout=600)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    one = _solve(kind, 0, 1, N)
    np.testing.assert_array_equal(two["cnt"], one["cnt"])
    np.testing.assert_array_equal(two["stats"], one["stats"])
    np.testing.assert_array_equal(two["events"], one["events"])       # rank order = packet order
    for k in ("E", "sed_esc", "T"):
        np.testing.assert_allclose(two[k], one[k], rtol=1e-12, atol=0)
    np.testing.assert_allclose(two["img"], one["img"], rtol=1e-6, atol=0)
    np.testing.assert_allclose(two["sed"], one["sed"], rtol=1e-10, atol=0)
    np.testing.assert_allclose(two["drho"], one["drho"], rtol=1e-5, atol=1e-6 * np.abs(one["drho"]).max())
    np.testing.assert_allclose(two["dscale"], one["dscale"], rtol=1e-9)
    assert one["events"] is not None and np.abs(one["img"]).max() > 0
