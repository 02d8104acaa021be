"""Schedule autotuner: candidate grid and selection logic (CPU, with a fake
timer), and one tuning run on the GPU."""
import numpy as np
import pytest

import workloads as W
from paper_1203_2941_gb300 import autotune as AT


@pytest.fixture(scope="module")
def rt():
    import __graft_entry__ as g
    g.build()
    import paper_1203_2941_gb300 as rt
    return rt


def test_candidates_cover_the_grid_in_fixed_order():
    c = AT.candidates({"march_min_active": (8, 16), "threads_per_block": (256,), "blocks_per_sm": (0, 2)})
    assert len(c) == 4
    assert c[0] == {"blocks_per_sm": 0, "march_min_active": 8, "threads_per_block": 256}
    assert c[-1] == {"blocks_per_sm": 2, "march_min_active": 16, "threads_per_block": 256}
    assert len(AT.candidates()) == len(AT.DEFAULT_GRID["march_min_active"]) * 2 * 1 == 16


def test_select_takes_the_smallest_median_and_first_of_ties():
    cands = AT.candidates({"march_min_active": (8, 12, 16, 20), "threads_per_block": (256,),
                           "blocks_per_sm": (0,)})
    noise = iter(np.random.default_rng(0).normal(0, 1e-4, size=100))
    cost = {8: 3.0, 12: 1.0, 16: 1.0, 20: 2.0}
    r = AT.select(cands, lambda c: cost[c["march_min_active"]] + abs(next(noise)) * 0, repeats=3)
    assert r.params["march_min_active"] == 12 and r.seconds == 1.0
    assert [t for _, t in r.table] == [3.0, 1.0, 1.0, 2.0]
    # the median resists one slow outlier per candidate
    calls = {}

    def t(c):
        k = c["march_min_active"]
        calls[k] = calls.get(k, 0) + 1
        return 100.0 if calls[k] == 1 else cost[k]
    r = AT.select(cands, t, repeats=3)
    assert r.params["march_min_active"] == 12
    with pytest.raises(ValueError):
        AT.select([], lambda c: 0.0)


@pytest.mark.gpu
def test_tune_transport_and_batch_on_gpu(rt):
    import torch
    ctx = rt.Context(0)
    m = W.r2_shell(n=24, tau_1um=10.0, nf=32)
    grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
    g = {"march_min_active": (8, 16), "threads_per_block": (256, 128), "blocks_per_sm": (0,)}
    r = AT.tune_transport(ctx, grid, opac, srcs, 200000, sample=50000, grid_values=g, repeats=2)
    assert r.params in AT.candidates(g) and len(r.table) == 4 and r.seconds > 0
    out = rt.transport(ctx, grid, opac, srcs, 50000, **r.params)
    torch.cuda.synchronize()
    assert abs(out.stats_dict()["escaped"] - 50000) == 0
    assert abs(out.numpy()["sed_esc"].sum() / m.luminosity - 1) < 1e-9
    models = [W.clumpy_torus(n=n, n_clump=k, seed=s, nf=24, with_pah=False)
              for n, k, s in ((8, 20, 1), (16, 60, 2))]
    op2 = ctx.opacity(models[0])
    rb = AT.tune_batch(ctx, op2, models, [20000, 20000], sample=5000,
                       grid_values={"march_min_active": (8, 16), "threads_per_block": (256,),
                                    "blocks_per_sm": (0,)})
    assert rb.params in AT.candidates({"march_min_active": (8, 16), "threads_per_block": (256,),
                                       "blocks_per_sm": (0,)})
