"""The per-sweep cost history (qf_options.cost_history) against the oracle's.

Alg. 1 tests its stopping rules on the cost after every sweep (Sec. III-A2);
the history returns exactly those costs: entry 0 for the initial circuit,
entry i after sweep i, NaN after a start's last sweep.  The oracle's
Qfactor keeps the same list ("history").  Complex128 runs agree to the
spec cost tolerance (1e-10); a complex64 bulk phase to the complex64
noise (1e-5), its last entry being the reported FP64 cost.
"""
import numpy as np
import pytest
import torch

import oracle as orc
import qf_inputs as qi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qf():
    import paper_2306_08152_gb300 as qf

    qf._native.load()
    return qf


def _check_rows(hist, ref_hists, tol, max_sweeps):
    for s, ref in enumerate(ref_hists):
        k = len(ref)
        assert hist.shape[-1] == max_sweeps + 1
        np.testing.assert_allclose(hist[s][:k], ref, rtol=0, atol=tol)
        assert np.all(np.isnan(hist[s][k:])), s


@pytest.mark.parametrize("n,layers,reachable,reset", [(4, 4, True, 40), (6, 6, False, 4)])
def test_instantiate_ex_history_matches_oracle(qf, n, layers, reachable, reset):
    locs = qi.brickwork_locations(n, layers)
    inst = qi.make_problem(n, locs, 3, seed=13000 + n)
    V = orc.circuit_unitary(inst.target_gates, locs, n) if reachable else \
        qi.haar_unitary(2**n, qi.rng(13100 + n))
    max_sweeps = 12
    r = qf.instantiate_ex(torch.from_numpy(V).cuda(), locs, torch.from_numpy(inst.starts).cuda(),
                          dist_tol=1e-10, max_sweeps=max_sweeps, reset_iter=reset, history=True)
    ref = orc.qfactor_multistart(V, inst.starts, locs, n,
                                 orc.QFactorOptions(dist_tol=1e-10, max_iter=max_sweeps, reset_iter=reset))
    assert r["sweeps"] == ref["sweeps"]
    _check_rows(r["history"], ref["histories"], 1e-10, max_sweeps)
    # the last entry is the reported cost
    for s in range(3):
        assert r["history"][s][r["sweeps"]] == r["costs"][s]


def test_history_of_a_converging_mixed_precision_run(qf):
    n = 4
    locs = qi.brickwork_locations(n, 4)
    inst = qi.make_problem(n, locs, 2, seed=8)
    V = orc.circuit_unitary(inst.target_gates, locs, n)
    max_sweeps = 200
    r = qf.instantiate_ex(torch.from_numpy(V).cuda(), locs, torch.from_numpy(inst.starts).cuda(),
                          dist_tol=1e-10, max_sweeps=max_sweeps, precision=qf.QF_C64_REFINE64,
                          history=True)
    h = r["history"]
    k = r["sweeps"]
    assert r["best_cost"] <= 1e-10
    ref = orc.qfactor_multistart(V, inst.starts, locs, n,
                                 orc.QFactorOptions(dist_tol=1e-10, max_iter=max_sweeps))
    for s in range(2):
        m = min(k, len(ref["histories"][s]) - 1)
        assert np.all(np.abs(h[s][:m + 1] - np.asarray(ref["histories"][s][:m + 1])) <= 1e-5), s
        assert np.all(np.isnan(h[s][k + 1:]))
        assert h[s][k] == r["costs"][s]
    print(f"mixed precision history: {k} sweeps ({r['c64_sweeps']} in c64), best {r['best_cost']:.2e}")


def test_batched_history_matches_oracle(qf):
    """One start per instance: a batched problem is then a plain Qfactor."""
    g = qi.rng(13200)
    insts, refs = [], []
    max_sweeps = 15
    for n, p in [(3, 6), (4, 9), (5, 12), (3, 11)]:
        locs = qi.random_adjacent_locations(n, p, g)
        inst = qi.make_problem(n, locs, 1, seed=int(g.integers(1 << 30)))
        V = qi.haar_unitary(2**n, g) if n == 5 else orc.circuit_unitary(inst.target_gates, locs, n)
        insts.append((V, locs, inst.starts))
        refs.append(orc.qfactor(V, inst.starts[0], locs, n,
                                orc.QFactorOptions(dist_tol=1e-10, max_iter=max_sweeps, reset_iter=6)))
    res = qf.instantiate_batched(insts, dist_tol=1e-10, max_sweeps=max_sweeps, reset_iter=6,
                                 precision=qf.QF_C128, history=True)
    for i, ref in enumerate(refs):
        assert res["sweeps"][i, 0] == ref["sweeps"]
        _check_rows(res["history"][i], [ref["history"]], 1e-10, max_sweeps)
