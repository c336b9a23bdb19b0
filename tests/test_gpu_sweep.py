"""GPU parity of whole sweeps, instantiations and environments against the
FP64 oracle (Alg. 1 TwoSidedSweep and Qfactor; Sec. III environments).

Targets (spec tolerances): costs within 1e-10 and environment entries
within 1e-9 relative, complex128, after 1 and 5 sweeps from the same seeded
initial gates.  Gates are compared too at these short horizons (the paths
only differ by rounding order).  Complex64 results are compared against the
FP64 oracle and their error is printed per result.
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


STRUCTS = {
    "n2_single": (2, np.array([[0, 1], [1, 0], [0, 1]], dtype=np.int32)),
    "n3_alternating": (3, np.array([[0, 1], [1, 2]] * 3, dtype=np.int32)),
    "n4_mixed": (4, np.array([[0, 1], [2, 3], [1, 2], [3, 0], [2, 1], [0, 2]], dtype=np.int32)),
    "n6_brickwork": (6, qi.brickwork_locations(6, 12)),
}


def _oracle_sweeps(V, gates, locs, n, k, reset_iter=0):
    T = orc.init_circuit_tensor(V, gates, locs, n)
    g = gates
    costs = []
    for it in range(1, k + 1):
        T, g = orc.two_sided_sweep(T, g, locs, n)
        if reset_iter and it % reset_iter == 0:
            T = orc.init_circuit_tensor(V, g, locs, n)
        costs.append(orc.trace_cost(T, n))
    return np.array(costs), g


@pytest.mark.parametrize("name", list(STRUCTS))
@pytest.mark.parametrize("reachable", [True, False])
def test_sweeps_match_oracle_c128(qf, name, reachable):
    n, locs = STRUCTS[name]
    inst = qi.make_problem(n, locs, 3, seed=11)
    V = orc.circuit_unitary(inst.target_gates, locs, n) if reachable else qi.haar_unitary(2**n, qi.rng(12))
    plan = qf.Plan(n, locs, inst.n_starts, qf.QF_C128)
    plan.load(torch.from_numpy(V).cuda(), torch.from_numpy(inst.starts).cuda())
    gpu = []
    for it in range(5):
        plan.sweep(1, reset_iter=0)
        gpu.append(plan.costs())
        if it in (0, 4):
            G = plan.gates().numpy()
            for s in range(inst.n_starts):
                ref_c, ref_g = _oracle_sweeps(V, inst.starts[s], locs, n, it + 1)
                assert abs(gpu[-1][s] - ref_c[-1]) <= 1e-10, (it, s)
                assert np.max(np.abs(G[s] - ref_g)) <= 1e-9, (it, s)
    assert plan.status() == 0
    plan.close()


def test_reset_iter_matches_oracle(qf):
    n, locs = STRUCTS["n4_mixed"]
    inst = qi.make_problem(n, locs, 2, seed=21)
    V = orc.circuit_unitary(inst.target_gates, locs, n)
    plan = qf.Plan(n, locs, inst.n_starts, qf.QF_C128)
    plan.load(torch.from_numpy(V).cuda(), torch.from_numpy(inst.starts).cuda())
    plan.sweep(6, reset_iter=2)
    c = plan.costs()
    G = plan.gates().numpy()
    for s in range(inst.n_starts):
        ref_c, ref_g = _oracle_sweeps(V, inst.starts[s], locs, n, 6, reset_iter=2)
        assert abs(c[s] - ref_c[-1]) <= 1e-10
        assert np.max(np.abs(G[s] - ref_g)) <= 1e-9


def test_c64_sweeps_track_the_fp64_oracle(qf):
    n, locs = STRUCTS["n6_brickwork"]
    inst = qi.make_problem(n, locs, 2, seed=31)
    V = orc.circuit_unitary(inst.target_gates, locs, n)
    plan = qf.Plan(n, locs, inst.n_starts, qf.QF_C64)
    plan.load(torch.from_numpy(V).cuda(), torch.from_numpy(inst.starts).cuda())
    plan.sweep(1, reset_iter=0)
    c = plan.costs()
    for s in range(inst.n_starts):
        ref_c, _ = _oracle_sweeps(V, inst.starts[s], locs, n, 1)
        err = abs(c[s] - ref_c[-1])
        print(f"c64 one-sweep cost error start {s}: {err:.2e} (cost {ref_c[-1]:.4e})")
        assert err <= 1e-5


@pytest.mark.parametrize("n,layers,sets", [(3, 4, 3), (5, 6, 4), (8, 16, 32)])
def test_cost_and_env_matches_oracle(qf, n, layers, sets):
    locs = qi.brickwork_locations(n, layers)
    g = qi.rng(40 + n)
    gates = np.stack([qi.haar_gates(len(locs), g) for _ in range(sets)])
    V = qi.haar_unitary(2**n, g)
    costs, envs, trs = qf.cost_and_env(torch.from_numpy(V).cuda(), locs, torch.from_numpy(gates).cuda())
    envs = envs.cpu().numpy()
    check_sets = range(sets) if n < 8 else (0, sets - 1)
    for s in check_sets:
        c_ref, e_ref, t_ref = orc.cost_and_env(V, gates[s], locs, n)
        assert abs(costs[s] - c_ref) <= 1e-10
        assert abs(trs[s] - t_ref) <= 1e-10 * 2**n
        scale = np.max(np.abs(e_ref))
        assert np.max(np.abs(envs[s] - e_ref)) <= 1e-9 * scale, s


def test_instantiate_matches_oracle_multistart(qf):
    n = 4
    locs = qi.brickwork_locations(n, 4)
    inst = qi.make_problem(n, locs, 3, seed=8)
    V = orc.circuit_unitary(inst.target_gates, locs, n)
    ref = orc.qfactor_multistart(V, inst.starts, locs, n, orc.QFactorOptions(dist_tol=1e-10, max_iter=300))
    res = qf.instantiate_ex(torch.from_numpy(V).cuda(), locs, torch.from_numpy(inst.starts).cuda(),
                            dist_tol=1e-10, max_sweeps=300)
    assert res["reason"] == ref["reason"] == "converged"
    assert res["sweeps"] == ref["sweeps"]
    assert res["best_cost"] <= 1e-10
    np.testing.assert_allclose(res["costs"], ref["costs"], atol=1e-10)


def test_instantiate_single_start_host_buffers(qf):
    n = 4
    locs = qi.brickwork_locations(n, 4)
    inst = qi.make_problem(n, locs, 1, seed=8)
    V = orc.circuit_unitary(inst.target_gates, locs, n)
    # host tensors: the library copies in and out itself
    gates, cost, sweeps = qf.instantiate(torch.from_numpy(V), locs, torch.from_numpy(inst.starts[0]),
                                         tol=1e-10, max_sweeps=300)
    ref = orc.qfactor(V, inst.starts[0], locs, n, orc.QFactorOptions(dist_tol=1e-10, max_iter=300))
    assert sweeps == ref["sweeps"]
    assert abs(cost - ref["cost"]) <= 1e-10
    assert gates.device.type == "cpu"


def test_plateau_and_beta_match_oracle(qf):
    n = 3
    locs = np.array([[0, 1], [1, 2]], dtype=np.int32)
    V = qi.haar_unitary(8, qi.rng(150))
    starts = np.stack([qi.haar_gates(2, qi.rng(151 + s)) for s in range(2)])
    o = orc.QFactorOptions(diff_tol_r=1e-5, max_iter=200, beta=0.2)
    ref = orc.qfactor_multistart(V, starts, locs, n, o)
    res = qf.instantiate_ex(torch.from_numpy(V).cuda(), locs, torch.from_numpy(starts).cuda(),
                            diff_tol_r=1e-5, max_sweeps=200, beta=0.2)
    assert res["reason"] == ref["reason"] == "plateau"
    assert res["sweeps"] == ref["sweeps"]
    np.testing.assert_allclose(res["costs"], ref["costs"], atol=1e-10)


def test_mixed_precision_reaches_fp64_tolerance(qf):
    n = 6
    locs = qi.brickwork_locations(n, 6)
    inst = qi.make_problem(n, locs, 4, seed=5)
    V = orc.circuit_unitary(inst.target_gates, locs, n)
    res = qf.instantiate_ex(torch.from_numpy(V).cuda(), locs, torch.from_numpy(inst.starts).cuda(),
                            dist_tol=1e-10, max_sweeps=500, precision=qf.QF_C64_REFINE64)
    print(f"mixed precision: {res['reason']} after {res['sweeps']} sweeps "
          f"({res['c64_sweeps']} in c64), best cost {res['best_cost']:.2e}")
    assert res["c64_sweeps"] >= 1
    best = res["best"]
    # the FP64 oracle agrees on the returned gates' cost
    c_ref, _, _ = orc.cost_and_env(V, res["gates"][best].cpu().numpy(), locs, n)
    assert abs(c_ref - res["best_cost"]) <= 1e-10
    if res["reason"] == "converged":
        assert res["best_cost"] <= 1e-10


def test_nonfinite_target_is_rejected(qf):
    from paper_2306_08152_gb300 import QFactorError

    n = 3
    V = np.eye(8, dtype=np.complex128)
    V[2, 3] = np.nan
    locs = np.array([[0, 1]], dtype=np.int32)
    with pytest.raises(QFactorError) as ei:
        qf.instantiate(torch.from_numpy(V), locs, torch.from_numpy(np.eye(4, dtype=np.complex128)[None]))
    assert ei.value.code == -4
