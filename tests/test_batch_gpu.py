"""Multi-channel batch (one persistent tensor-core launch per step, replayed
from a CUDA graph) against the same contexts stepped one by one, and against
the oracle."""
import json

import numpy as np
import pytest

from paper_2609_23057_b300 import workloads as W
from _util import abs_err_dop, oracle_problem, rel_err_I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def _channels():
    ws = W.channels(count=9, seed=5, steps=7)
    # vary sizes below the workload's range too: ragged tiles, tiny lattices,
    # a channel whose sites mix two phase classes inside tiles
    ws[0] = W.random_medium(37, 5, 2, 4, seed=1, n_phase=1, steps=7)
    ws[1] = W.random_medium(130, 3, 4, 4, seed=2, n_phase=2, steps=7)          # mixed-class tiles
    ws[2] = W.random_medium(64, 4, 4, 8, seed=3, n_phase=1, steps=7, bc=(1, 1, 1, 1))
    return ws


def _mixed_n_channels():
    """Lattices at n = 8 (only one converter group has staging work for
    them), then n = 16 and n = 32: 313 tiles at n = 8 (odd), 154 at n = 16,
    153 at n = 32, about four items per CTA, so CTA slices straddle both
    direction-count changes; some lattices are ragged."""
    ws = []
    for k, (nx, nz, nzen, naz) in enumerate([(1024, 37, 2, 4), (64, 3, 2, 4), (320, 6, 2, 4), (1200, 16, 4, 4),
                                             (130, 3, 4, 4), (596, 32, 4, 8), (100, 5, 4, 8)]):
        ws.append(W.random_medium(nx, nz, nzen, naz, seed=200 + k, n_phase=1, steps=6))
    return ws


@pytest.mark.parametrize("stages,tile_cost", [(2, 4), (4, 4), (6, 4), (8, 4), (4, 0), (2, 16), (8, 64)])
def test_batch_mixed_direction_counts_every_depth(torch_cuda, stages, tile_cost):
    """Bitwise equality with single stepping at every pipeline depth and at
    several work balances (other CTA item ranges) on a batch whose CTA slices
    mix n = 8, 16 and 32."""
    from paper_2609_23057_b300.solver import Batch, solver_for
    ws = _mixed_n_channels()
    states = [W.random_state(w.nz, w.nx, w.n, seed=300 + k, dtype=np.float32) for k, w in enumerate(ws)]
    bs, single = [], []
    for w, S0 in zip(ws, states):
        for lst in (bs, single):
            s = solver_for(w, "bf16")
            s.set_state(torch_cuda.from_numpy(S0).cuda())
            lst.append(s)
    b = Batch(bs)
    b.configure(stages)
    b.balance(tile_cost)
    b.step(6)
    b.check()
    for s in single:
        s.step(6)
        s.total_intensity()
    for k, (sb, ss) in enumerate(zip(bs, single)):
        assert np.array_equal(sb.get_state().cpu().numpy(), ss.get_state().cpu().numpy()), k
    b.close()
    for s in bs + single:
        s.close()


def test_batch_rejects_odd_depth(torch_cuda):
    from paper_2609_23057_b300 import _lib
    from paper_2609_23057_b300.solver import Batch, solver_for
    ss = [solver_for(w, "bf16") for w in _channels()[:2]]
    b = Batch(ss)
    for st in (1, 3, 5, 10):
        with pytest.raises(_lib.RtlbError) as ei:
            b.configure(st)
        assert ei.value.status == 3
    for cost in (-1, 65):
        with pytest.raises(_lib.RtlbError) as ei:
            b.balance(cost)
        assert ei.value.status == 3
    b.close()
    for s in ss:
        s.close()


@pytest.mark.parametrize("prec", ["bf16", "bf16x2"])
def test_batch_equals_individual_steps(torch_cuda, orc, prec):
    from paper_2609_23057_b300.solver import Batch, solver_for
    ws = _channels()
    states = [W.random_state(w.nz, w.nx, w.n, seed=100 + k, dtype=np.float32) for k, w in enumerate(ws)]
    batch_solvers, single = [], []
    for w, S0 in zip(ws, states):
        for lst in (batch_solvers, single):
            s = solver_for(w, prec)
            s.set_state(torch_cuda.from_numpy(S0).cuda())
            lst.append(s)
    b = Batch(batch_solvers)
    b.step(7)                      # 3 graph replays (2 steps each) + 1 direct launch
    b.check()
    for s in single:
        s.step(7)
        s.total_intensity()
    for k, (sb, ss) in enumerate(zip(batch_solvers, single)):
        gb = sb.get_state().cpu().numpy()
        gs = ss.get_state().cpu().numpy()
        assert np.array_equal(gb, gs), k
        assert sb.steps_done == 7
    # two channels against the oracle (bf16 tolerance, 7 steps)
    for k in (0, 4):
        w = ws[k]
        ref = oracle_problem(orc, w).run(states[k].astype(np.float64), 7)
        got = batch_solvers[k].get_state().cpu().numpy().astype(np.float64)
        assert rel_err_I(got, ref) < 2e-2 and abs_err_dop(got, ref) < 2e-2
    b.close()
    for s in batch_solvers + single:
        s.close()


def test_batch_rejects_desynchronized_channels(torch_cuda):
    from paper_2609_23057_b300 import _lib
    from paper_2609_23057_b300.solver import Batch, solver_for
    ws = _channels()[:3]
    ss = [solver_for(w, "bf16") for w in ws]
    b = Batch(ss)
    b.step(2)
    ss[0].step(1)
    with pytest.raises(_lib.RtlbError) as ei:
        b.step(1)
    assert ei.value.status == 5
    b.close()
    for s in ss:
        s.close()


def test_autotune_picks_and_caches(torch_cuda, tmp_path):
    from paper_2609_23057_b300.solver import Batch, autotune_batch, solver_for
    ws = W.channels(count=6, seed=8, steps=4)
    ss = [solver_for(w, "bf16") for w in ws]
    b = Batch(ss)
    cache = tmp_path / "tune.json"
    st = autotune_batch(b, candidates=(2, 4, 8), costs=(4, 0, 16), trial_steps=2, cache_path=str(cache))
    assert st in (2, 4, 8) and b.tile_cost in (4, 0, 16)
    data = json.loads(cache.read_text())
    assert list(data.values())[0]["stages"] == st and list(data.values())[0]["tile_cost"] == b.tile_cost
    assert autotune_batch(b, cache_path=str(cache)) == st      # served from the cache
    b.check()
    b.close()
    for s in ss:
        s.close()
