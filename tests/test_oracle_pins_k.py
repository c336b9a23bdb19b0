"""Pins of the k-qubit oracle (oracle/kqubit.py) against constructions
other than itself: explicit basis-loop operators and partial traces,
finite differences, the trace identity, closed-form single-gate fits,
local optimality and monotonicity (Sec. III, Alg. 1, Eq. opt_u).  Gates of
1, 2, 3 and 4 qubits, in every qubit order."""
import numpy as np
import pytest

import oracle as orc
import oracle.kqubit as ok
import qf_inputs as qi
from tests import dense_ref as dr


def _mixed_structure(n, p, g, ks=(1, 2, 3)):
    locs, gates = [], []
    for _ in range(p):
        k = int(g.choice([kk for kk in ks if kk <= n]))
        q = tuple(int(x) for x in g.choice(n, k, replace=False))
        locs.append(q)
        gates.append(qi.haar_unitary(2**k, g))
    return gates, locs


def test_dense_helper_k_matches_kron_for_adjacent_qubits():
    g = qi.rng(9000)
    u = qi.haar_unitary(8, g)
    G = dr.full_operator_k(u, (1, 2, 3), 5)
    np.testing.assert_allclose(G, np.kron(np.kron(np.eye(2), u), np.eye(2)), atol=1e-15)


@pytest.mark.parametrize("n", [3, 4, 5])
def test_apply_right_left_k_match_dense(n):
    g = qi.rng(9100 + n)
    T = qi.haar_unitary(2**n, g) + 0.3 * qi.haar_unitary(2**n, g)
    for k in (1, 2, 3, 4):
        if k > n:
            continue
        for _ in range(4):
            q = tuple(int(x) for x in g.choice(n, k, replace=False))
            u = qi.haar_unitary(2**k, g)
            G = dr.full_operator_k(u, q, n)
            np.testing.assert_allclose(ok.apply_right_k(T, u, q, n), T @ G, atol=1e-13)
            np.testing.assert_allclose(ok.apply_left_k(T, u, q, n), G @ T, atol=1e-13)


@pytest.mark.parametrize("n", [3, 4, 5])
def test_partial_trace_k_matches_dense(n):
    g = qi.rng(9200 + n)
    M = g.standard_normal((2**n, 2**n)) + 1j * g.standard_normal((2**n, 2**n))
    for k in (1, 2, 3, 4):
        if k > n:
            continue
        for _ in range(3):
            q = tuple(int(x) for x in g.choice(n, k, replace=False))
            np.testing.assert_allclose(ok.calc_env_mat_k(M, q, n), dr.dense_partial_trace_k(M, q, n),
                                       atol=1e-12)


def test_two_qubit_case_agrees_with_the_two_qubit_oracle():
    n = 4
    g = qi.rng(9300)
    T = g.standard_normal((16, 16)) + 1j * g.standard_normal((16, 16))
    u = qi.haar_unitary(4, g)
    for a, b in [(0, 1), (3, 1), (2, 0)]:
        np.testing.assert_allclose(ok.apply_right_k(T, u, (a, b), n), orc.apply_right(T, u, a, b, n), atol=1e-13)
        np.testing.assert_allclose(ok.apply_left_k(T, u, (a, b), n), orc.apply_left(T, u, a, b, n), atol=1e-13)
        np.testing.assert_allclose(ok.calc_env_mat_k(T, (a, b), n), orc.calc_env_mat(T, a, b, n), atol=1e-13)


@pytest.mark.parametrize("n", [3, 4])
def test_environments_k_match_dense_and_trace_identity(n):
    g = qi.rng(9400 + n)
    gates, locs = _mixed_structure(n, 6, g)
    V = qi.haar_unitary(2**n, g)
    cost, envs, t = ok.cost_and_env_k(V, gates, locs, n)
    C = dr.dense_circuit_k(gates, locs, n)
    assert abs(t - np.trace(V.conj().T @ C)) <= 1e-12
    for k in range(len(gates)):
        np.testing.assert_allclose(envs[k], dr.dense_environment_k(V, gates, locs, n, k), atol=1e-12)
        assert abs(np.trace(envs[k] @ gates[k]) - t) <= 1e-12
    assert abs(cost - (1 - abs(t) / 2**n)) <= 1e-15


@pytest.mark.parametrize("n,ks", [(4, (2, 3)), (5, (2, 4))])
def test_environment_k_is_the_gradient_of_the_trace(n, ks):
    """Tr(V^dagger C) is linear in each gate, so a central difference in
    entry (i, j) of u_k equals E_k[j, i] up to rounding."""
    g = qi.rng(9500 + n)
    gates, locs = _mixed_structure(n, 5, g, ks=ks)
    V = qi.haar_unitary(2**n, g)
    _, envs, _ = ok.cost_and_env_k(V, gates, locs, n)
    h = 1e-6
    for k in range(len(gates)):
        d = gates[k].shape[0]
        for (i, j) in [(0, 0), (d - 1, 1), (2, d - 1)]:
            for step in (h, 1j * h):
                gp = [x.copy() for x in gates]
                gm = [x.copy() for x in gates]
                gp[k][i, j] += step
                gm[k][i, j] -= step
                tp = np.trace(V.conj().T @ dr.dense_circuit_k(gp, locs, n))
                tm = np.trace(V.conj().T @ dr.dense_circuit_k(gm, locs, n))
                fd = (tp - tm) / (2 * step)
                assert abs(fd - envs[k][j, i]) <= 1e-8, (k, i, j)


@pytest.mark.parametrize("n,orders", [(3, [(0, 1, 2), (2, 0, 1)]), (4, [(0, 1, 2, 3), (3, 1, 0, 2)])])
def test_single_gate_on_every_qubit_fits_its_target_in_one_update(n, orders):
    """One gate on all n qubits: the environment of u from T = V^dagger u
    after removal is V^dagger, and the update returns u' = V, cost 0."""
    g = qi.rng(9600 + n)
    V = qi.haar_unitary(2**n, g)
    for q in orders:
        u0 = qi.haar_unitary(2**n, g)
        T = ok.init_circuit_tensor_k(V, [u0], [q], n)
        T, gates = ok.two_sided_sweep_k(T, [u0], [q], n)
        # the gate on permuted qubits equals V in the permuted local basis
        np.testing.assert_allclose(dr.full_operator_k(gates[0], q, n), V, atol=1e-12)
        assert ok.trace_cost(T, n) <= 1e-14


@pytest.mark.parametrize("k", [3, 4])
def test_product_target_closed_form_cost(k):
    """n = k + 1, one gate on qubits 0..k-1 and V = w (x) h with h on qubit
    k: the update reaches w up to a phase and the cost 1 - |Tr h| / 2."""
    g = qi.rng(9700 + k)
    d = 2**k
    w = qi.haar_unitary(d, g)
    h = qi.haar_unitary(2, g)
    V = np.kron(w, h)
    q = tuple(range(k))
    u0 = qi.haar_unitary(d, g)
    T = ok.init_circuit_tensor_k(V, [u0], [q], k + 1)
    T, gates = ok.two_sided_sweep_k(T, [u0], [q], k + 1)
    assert abs(ok.trace_cost(T, k + 1) - (1 - abs(np.trace(h)) / 2)) <= 1e-13
    ph = np.trace(w.conj().T @ gates[0]) / d
    np.testing.assert_allclose(gates[0], ph * w, atol=1e-12)
    assert abs(abs(ph) - 1) <= 1e-12


def test_update_k_is_locally_optimal_and_unitary():
    g = qi.rng(9800)
    for d in (2, 8, 16):
        E = g.standard_normal((d, d)) + 1j * g.standard_normal((d, d))
        u, s = ok.optimize_gate_k(E)
        assert abs(np.trace(E @ u) - s) <= 1e-12
        np.testing.assert_allclose(u.conj().T @ u, np.eye(d), atol=1e-13)
        for _ in range(200):
            w = qi.haar_unitary(d, g)
            assert abs(np.trace(E @ w)) <= s + 1e-12


def test_cost_never_increases_after_a_k_update():
    n = 4
    g = qi.rng(9900)
    gates, locs = _mixed_structure(n, 6, g, ks=(2, 3))
    V = qi.haar_unitary(16, g)
    T = ok.init_circuit_tensor_k(V, gates, locs, n)
    prev = ok.trace_cost(T, n)
    for _ in range(3):
        costs = []
        T, gates = ok.two_sided_sweep_k(T, gates, locs, n, update_costs=costs)
        for c in costs:
            assert c <= prev + 1e-14
            prev = c
    # the sweep's tensor is V^dagger C of its gates
    np.testing.assert_allclose(T, ok.init_circuit_tensor_k(V, gates, locs, n), atol=1e-11)


def test_reachable_three_qubit_gate_circuit_converges():
    """A target built from the same structure (3-qubit gates on (0,1,2) and
    (1,2,3), 2-qubit gates between) is fitted to cost < 1e-12 by one of a few
    starts."""
    n = 4
    locs = [(0, 1, 2), (2, 3), (1, 2, 3), (0, 1)]
    g = qi.rng(9950)
    tgt = [qi.haar_unitary(2 ** len(q), g) for q in locs]
    V = ok.circuit_unitary_k(tgt, locs, n)
    starts = [[qi.haar_unitary(2 ** len(q), qi.rng(9951 + s * 10 + i)) for i, q in enumerate(locs)]
              for s in range(4)]
    res = ok.qfactor_multistart_k(V, starts, locs, n, dist_tol=1e-12, max_iter=300)
    assert res["costs"].min() <= 1e-12, res["costs"]
    C = ok.circuit_unitary_k(res["gates"][res["best"]], locs, n)
    ph = np.trace(V.conj().T @ C) / 16
    np.testing.assert_allclose(C, ph * V, atol=1e-5)


def test_reachable_four_qubit_gate_circuit_converges():
    """Four-qubit gates on (0,1,2,3) and (1,2,3,4) with two-qubit gates
    between, target reachable from the same structure: some start reaches
    cost < 1e-12 and its circuit equals V up to a global phase."""
    n = 5
    locs = [(0, 1, 2, 3), (3, 4), (1, 2, 3, 4), (0, 1)]
    g = qi.rng(9960)
    tgt = [qi.haar_unitary(2 ** len(q), g) for q in locs]
    V = ok.circuit_unitary_k(tgt, locs, n)
    starts = [[qi.haar_unitary(2 ** len(q), qi.rng(9961 + s * 10 + i)) for i, q in enumerate(locs)]
              for s in range(4)]
    res = ok.qfactor_multistart_k(V, starts, locs, n, dist_tol=1e-12, max_iter=300)
    assert res["costs"].min() <= 1e-12, res["costs"]
    C = ok.circuit_unitary_k(res["gates"][res["best"]], locs, n)
    ph = np.trace(V.conj().T @ C) / 32
    np.testing.assert_allclose(C, ph * V, atol=1e-5)
