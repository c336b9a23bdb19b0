"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test ties an oracle function to something other than itself: explicit
dense basis-loop constructions (tests/dense_ref.py), central finite
differences, the Frobenius identity of Sec. III (Eq. cost), the optimality
argument of Sec. III-A1 (Eq. opt_u), the monotonicity of Sec. III-A,
hand-derived closed forms (tests/golden/closed_form_cases.json) and exact
fits of reachable targets.
"""
import json
import os

import numpy as np
import pytest

import oracle as orc
import qf_inputs as qi
from tests import dense_ref as dr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_form_cases.json")

CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=np.complex128)


def _cplx(a):
    a = np.asarray(a, dtype=np.float64)
    return a[..., 0] + 1j * a[..., 1]


def _pairs(n):
    return [(a, b) for a in range(n) for b in range(n) if a != b]


# ---------------------------------------------------------------- dense helper


def test_dense_helper_matches_kron_for_adjacent_pairs():
    """The basis-loop operator equals I_{2^a} (x) u (x) I for b = a + 1
    (qubit 0 most significant), which fixes the bit order of the pins."""
    g = qi.rng(1)
    for n in (2, 3, 4):
        for a in range(n - 1):
            u = qi.haar_unitary(4, g)
            ref = np.kron(np.kron(np.eye(2**a), u), np.eye(2 ** (n - a - 2)))
            np.testing.assert_allclose(dr.full_operator(u, a, a + 1, n), ref, atol=0)


def test_dense_helper_reversed_pair_is_swap_conjugation():
    """Location (b, a) is SWAP u SWAP on location (a, b)."""
    g = qi.rng(2)
    u = qi.haar_unitary(4, g)
    swap = np.eye(4)[[0, 2, 1, 3]]
    for n in (2, 3):
        for a, b in _pairs(n):
            np.testing.assert_allclose(dr.full_operator(u, b, a, n),
                                       dr.full_operator(swap @ u @ swap, a, b, n), atol=0)


# ---------------------------------------------------------------- P1 dense


@pytest.mark.parametrize("n", [2, 3, 4])
def test_apply_right_left_match_dense_products(n):
    g = qi.rng(10 + n)
    N = 2**n
    T = g.standard_normal((N, N)) + 1j * g.standard_normal((N, N))
    for a, b in _pairs(n):
        u = qi.haar_unitary(4, g) * (1.3 - 0.2j)  # non-unitary scale: linear maps
        G = dr.full_operator(u, a, b, n)
        np.testing.assert_allclose(orc.apply_right(T, u, a, b, n), T @ G, atol=1e-13)
        np.testing.assert_allclose(orc.apply_left(T, u, a, b, n), G @ T, atol=1e-13)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_partial_trace_matches_dense_loops(n):
    g = qi.rng(20 + n)
    N = 2**n
    T = g.standard_normal((N, N)) + 1j * g.standard_normal((N, N))
    for a, b in _pairs(n):
        np.testing.assert_allclose(orc.calc_env_mat(T, a, b, n),
                                   dr.dense_partial_trace(T, a, b, n), atol=1e-12)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_init_circuit_tensor_is_vdagger_times_circuit(n):
    g = qi.rng(30 + n)
    locs = qi.random_adjacent_locations(n, 7, g) if n > 2 else np.array([[0, 1], [1, 0], [0, 1]])
    gates = qi.haar_gates(len(locs), g)
    V = qi.haar_unitary(2**n, g)
    C = dr.dense_circuit(gates, locs, n)
    T = orc.init_circuit_tensor(V, gates, locs, n)
    np.testing.assert_allclose(T, V.conj().T @ C, atol=1e-13)
    np.testing.assert_allclose(orc.circuit_unitary(gates, locs, n), C, atol=1e-13)
    assert abs(orc.trace_cost(T, n) - (1 - abs(np.trace(V.conj().T @ C)) / 2**n)) < 1e-14


@pytest.mark.parametrize("n", [3, 4])
def test_cost_and_env_matches_dense_environments(n):
    g = qi.rng(40 + n)
    locs = np.array([[0, 1], [1, 2], [2, 0], [1, 2], [0, 2]] if n == 3 else
                    [[0, 1], [2, 3], [1, 2], [3, 0], [0, 1], [2, 3]], dtype=np.int32)
    gates = qi.haar_gates(len(locs), g)
    V = qi.haar_unitary(2**n, g)
    cost, envs, t = orc.cost_and_env(V, gates, locs, n)
    C = dr.dense_circuit(gates, locs, n)
    t_ref = np.trace(V.conj().T @ C)
    assert abs(t - t_ref) < 1e-12
    assert abs(cost - (1 - abs(t_ref) / 2**n)) < 1e-14
    for k in range(len(locs)):
        np.testing.assert_allclose(envs[k], dr.dense_environment(V, gates, locs, n, k), atol=1e-12)


@pytest.mark.parametrize("n", [3, 4])
def test_half_sweep_tensor_forms(n):
    """After the backward half T = C' V^dagger; after the forward half
    T = V^dagger C'' (the circuit-tensor forms of Sec. III), with C', C'' the
    dense products of the gates the oracle returns."""
    g = qi.rng(50 + n)
    locs = qi.brickwork_locations(n, 3)
    gates = qi.haar_gates(len(locs), g)
    V = qi.haar_unitary(2**n, g)
    T = orc.init_circuit_tensor(V, gates, locs, n)
    # Backward half only: run a sweep on a copy and recover the backward
    # gates by sweeping a circuit whose forward half is checked separately.
    T1, g1 = orc.two_sided_sweep(T, gates, locs, n)
    np.testing.assert_allclose(T1, V.conj().T @ dr.dense_circuit(g1, locs, n), atol=1e-12)
    # Backward half by hand from the oracle's primitives, checked densely.
    Tb = T.copy()
    gb = gates.copy()
    for k in range(len(locs) - 1, -1, -1):
        a, b = locs[k]
        Tb = orc.apply_right(Tb, gb[k].conj().T, a, b, n)
        gb[k], _ = orc.optimize_gate(orc.calc_env_mat(Tb, a, b, n))
        Tb = orc.apply_left(Tb, gb[k], a, b, n)
    np.testing.assert_allclose(Tb, dr.dense_circuit(gb, locs, n) @ V.conj().T, atol=1e-12)


# ---------------------------------------------------------------- P2 / P3


def test_environment_is_the_gradient_of_the_trace():
    """t = Tr(V^dagger C) is linear in each u_k; central differences (step
    1e-6, complex128) give dt/d Re(u_k)_ij = (E_k)_ji and dt/d Im = i (E_k)_ji."""
    n = 3
    g = qi.rng(60)
    locs = np.array([[0, 1], [1, 2], [0, 2], [2, 1]], dtype=np.int32)
    gates = qi.haar_gates(len(locs), g)
    V = qi.haar_unitary(8, g)
    _, envs, _ = orc.cost_and_env(V, gates, locs, n)

    def t_of(gs):
        C = dr.dense_circuit(gs, locs, n)
        return np.trace(V.conj().T @ C)

    h = 1e-6
    for k in range(len(locs)):
        for i in range(4):
            for j in range(4):
                for direction, factor in ((1.0, 1.0), (1j, 1j)):
                    gp = gates.copy()
                    gm = gates.copy()
                    gp[k, i, j] += h * direction
                    gm[k, i, j] -= h * direction
                    fd = (t_of(gp) - t_of(gm)) / (2 * h)
                    assert abs(fd - factor * envs[k, j, i]) <= 1e-9 * max(1.0, abs(envs[k, j, i]))


@pytest.mark.parametrize("n", [3, 5, 6])
def test_trace_identity_for_every_gate(n):
    g = qi.rng(70 + n)
    locs = qi.brickwork_locations(n, 4)
    gates = qi.haar_gates(len(locs), g)
    V = qi.haar_unitary(2**n, g)
    _, envs, t = orc.cost_and_env(V, gates, locs, n)
    for k in range(len(locs)):
        assert abs(np.trace(envs[k] @ gates[k]) - t) < 1e-11


# ---------------------------------------------------------------- P4


@pytest.mark.parametrize("n", [2, 4, 6])
def test_frobenius_identity(n):
    """||C - V||^2 = 2^{n+1} (1 - Re Tr(V^dagger C) / 2^n) (Sec. III, Eq. cost)."""
    g = qi.rng(80 + n)
    locs = qi.brickwork_locations(n, 5)
    gates = qi.haar_gates(len(locs), g)
    V = qi.haar_unitary(2**n, g)
    C = orc.circuit_unitary(gates, locs, n)
    lhs = orc.frobenius_distance(C, V) ** 2
    rhs = 2 ** (n + 1) * (1 - np.real(np.trace(V.conj().T @ C)) / 2**n)
    assert abs(lhs - rhs) < 1e-10 * max(1.0, lhs)
    np.testing.assert_allclose(C.conj().T @ C, np.eye(2**n), atol=1e-13)


# ---------------------------------------------------------------- P5


def test_optimize_gate_local_optimality():
    g = qi.rng(90)
    for trial in range(20):
        E = g.standard_normal((4, 4)) + 1j * g.standard_normal((4, 4))
        u, s = orc.optimize_gate(E)
        val = np.trace(E @ u)
        assert abs(val.imag) < 1e-12 and abs(val.real - s) < 1e-12
        np.testing.assert_allclose(u.conj().T @ u, np.eye(4), atol=1e-14)
        # closed-form polar factor of E^dagger: E^dagger (E E^dagger)^{-1/2}
        w, Q = np.linalg.eigh(E @ E.conj().T)
        inv_sqrt = Q @ np.diag(1 / np.sqrt(w)) @ Q.conj().T
        np.testing.assert_allclose(u, E.conj().T @ inv_sqrt, atol=1e-12)
        for _ in range(50):
            wq = qi.haar_unitary(4, g)
            assert np.real(np.trace(E @ wq)) <= s + 1e-12
            assert abs(np.trace(E @ wq)) <= s + 1e-12


def test_optimize_gate_golden_cases():
    with open(GOLDEN) as f:
        gold = json.load(f)
    for case in gold["optimize_gate"]:
        E = np.diag(_cplx(case["E_diag"]))
        u, s = orc.optimize_gate(E)
        np.testing.assert_allclose(u, np.diag(_cplx(case["u_diag"])), atol=1e-15, err_msg=case["name"])
        assert abs(s - case["sigma_sum"]) < 1e-14
    for case in gold["optimize_gate_dense"]:
        E = _cplx(case["E"])
        u_old = _cplx(case["u_old"]) if "u_old" in case else None
        u, s = orc.optimize_gate(E, u_old, case["beta"])
        np.testing.assert_allclose(u, _cplx(case["u"]), atol=1e-14, err_msg=case["name"])
        assert abs(s - case["sigma_sum"]) < 1e-13


def test_beta_update_maximises_the_damped_objective():
    """With beta the update maximises Re Tr(((1-beta) E + beta u_old^dagger) u)."""
    g = qi.rng(91)
    E = g.standard_normal((4, 4)) + 1j * g.standard_normal((4, 4))
    u_old = qi.haar_unitary(4, g)
    beta = 0.3
    u, s = orc.optimize_gate(E, u_old, beta)
    A = (1 - beta) * E + beta * u_old.conj().T
    assert abs(np.trace(A @ u) - s) < 1e-12
    for _ in range(200):
        w = qi.haar_unitary(4, g)
        assert np.real(np.trace(A @ w)) <= s + 1e-12


# ---------------------------------------------------------------- P6


def test_cost_never_increases_after_an_update():
    n = 4
    inst = qi.make_problem(n, qi.brickwork_locations(n, 4), 1, seed=100)
    V = qi.haar_unitary(2**n, qi.rng(101))
    T = orc.init_circuit_tensor(V, inst.starts[0], inst.locs, n)
    costs = [orc.trace_cost(T, n)]
    gates = inst.starts[0]
    for _ in range(4):
        T, gates = orc.two_sided_sweep(T, gates, inst.locs, n, update_costs=costs)
    assert all(c2 <= c1 + 1e-14 for c1, c2 in zip(costs, costs[1:]))
    assert costs[-1] < costs[0]


# ---------------------------------------------------------------- P7


def _golden_V(name):
    if name == "cnot01":
        return CNOT
    if name == "cnot_kron_diag1i":
        return np.kron(CNOT, np.diag([1, 1j]))
    raise KeyError(name)


def test_one_sweep_closed_forms():
    with open(GOLDEN) as f:
        gold = json.load(f)
    for case in gold["one_sweep"]:
        n = case["n"]
        locs = np.array(case["locs"], dtype=np.int32)
        V = _golden_V(case["V"])
        start = np.eye(4, dtype=np.complex128)[None]
        res = orc.qfactor(V, start, locs, n, orc.QFactorOptions(max_iter=1, dist_tol=-1))
        assert abs(res["cost"] - case["cost"]) < 1e-14, case["name"]
        if case.get("u") == "cnot_local":
            want = CNOT
        elif "u_phase_times_cnot" in case:
            ph = complex(*case["u_phase_times_cnot"])
            want = ph * CNOT
        else:
            want = _cplx(case["u"])
        np.testing.assert_allclose(res["gates"][0], want, atol=1e-14, err_msg=case["name"])


def test_product_target_gives_closed_form_cost():
    """n = 3, gate on (0,1), V = g (x) w: one update gives u = e^{i phi} g and
    cost 1 - |Tr w| / 2, for random g and w."""
    gen = qi.rng(110)
    for _ in range(5):
        gg = qi.haar_unitary(4, gen)
        w = qi.haar_unitary(2, gen)
        V = np.kron(gg, w)
        start = qi.haar_unitary(4, gen)[None]
        res = orc.qfactor(V, start, np.array([[0, 1]]), 3, orc.QFactorOptions(max_iter=1, dist_tol=-1))
        assert abs(res["cost"] - (1 - abs(np.trace(w)) / 2)) < 1e-13
        u = res["gates"][0]
        ratio = u @ gg.conj().T
        np.testing.assert_allclose(ratio, ratio[0, 0] * np.eye(4), atol=1e-12)
        assert abs(abs(ratio[0, 0]) - 1) < 1e-12


# ---------------------------------------------------------------- P8


def test_exact_fit_of_reachable_target():
    """Reachable 4-qubit brickwork target (6 U(4) gates, 4 layers): the
    target comes from the same structure, so a start reaches cost below
    1e-12 and C equals V up to a global phase."""
    n = 4
    locs = qi.brickwork_locations(n, 4)
    inst = qi.make_problem(n, locs, 4, seed=8)
    V = orc.circuit_unitary(inst.target_gates, locs, n)
    best = None
    for s in range(inst.n_starts):
        res = orc.qfactor(V, inst.starts[s], locs, n, orc.QFactorOptions(dist_tol=1e-13, max_iter=300))
        if best is None or res["cost"] < best["cost"]:
            best = res
        if best["cost"] < 1e-12:
            break
    assert best["cost"] < 1e-12
    C = orc.circuit_unitary(best["gates"], locs, n)
    phase = np.trace(V.conj().T @ C) / 2**n
    np.testing.assert_allclose(C, phase * V, atol=1e-6)


def test_three_qubit_alternating_circuit_descends():
    """Plain QFactor, 3 qubits: 6 U(4) gates alternating on (0,1),(1,2),
    reachable target.  The structure is over-parameterised and QFactor
    descends slowly on it; the cost still falls by orders of magnitude."""
    n = 3
    locs = np.array([[0, 1], [1, 2]] * 3, dtype=np.int32)
    inst = qi.make_problem(n, locs, 1, seed=7)
    V = orc.circuit_unitary(inst.target_gates, locs, n)
    res = orc.qfactor(V, inst.starts[0], locs, n, orc.QFactorOptions(max_iter=200))
    h = res["history"]
    assert all(b <= a + 1e-14 for a, b in zip(h, h[1:]))
    assert h[-1] < 1e-2 * h[1]


# ---------------------------------------------------------------- P9


def test_gauge_invariance_of_cost():
    """Inserting W W^dagger between two gates on the same location leaves C,
    the cost and the trace unchanged."""
    n = 3
    g = qi.rng(120)
    locs = np.array([[0, 1], [0, 1], [1, 2]], dtype=np.int32)
    gates = qi.haar_gates(3, g)
    V = qi.haar_unitary(8, g)
    W = qi.haar_unitary(4, g)
    g2 = gates.copy()
    g2[0] = gates[0] @ W
    g2[1] = W.conj().T @ gates[1]
    c1, e1, t1 = orc.cost_and_env(V, gates, locs, n)
    c2, e2, t2 = orc.cost_and_env(V, g2, locs, n)
    assert abs(t1 - t2) < 1e-13 and abs(c1 - c2) < 1e-14
    # environments move with the gauge: E_0' = W^dagger ... so Tr(E_0' u_0') = t
    assert abs(np.trace(e2[0] @ g2[0]) - t1) < 1e-12


# ---------------------------------------------------------------- P10


def test_reset_drift_is_small():
    """The maintained circuit tensor after 40 sweeps equals the tensor
    rebuilt from V and the current gates (Sec. III-A2, reset_iter)."""
    n = 4
    locs = qi.brickwork_locations(n, 4)
    inst = qi.make_problem(n, locs, 1, seed=130)
    V = orc.circuit_unitary(inst.target_gates, locs, n)
    T = orc.init_circuit_tensor(V, inst.starts[0], locs, n)
    gates = inst.starts[0]
    for _ in range(40):
        T, gates = orc.two_sided_sweep(T, gates, locs, n)
    T_rebuilt = orc.init_circuit_tensor(V, gates, locs, n)
    assert np.max(np.abs(T - T_rebuilt)) < 1e-12


# ---------------------------------------------------------------- stopping


def test_qfactor_history_and_reset_match_manual_loop():
    n = 3
    locs = np.array([[0, 1], [1, 2]] * 2, dtype=np.int32)
    inst = qi.make_problem(n, locs, 1, seed=140)
    V = qi.haar_unitary(8, qi.rng(141))  # unreachable: runs to max_iter
    o = orc.QFactorOptions(dist_tol=0.0, max_iter=7, reset_iter=3)
    res = orc.qfactor(V, inst.starts[0], locs, n, o)
    assert res["reason"] == "max_iter" and res["sweeps"] == 7 and len(res["history"]) == 8
    T = orc.init_circuit_tensor(V, inst.starts[0], locs, n)
    gates = inst.starts[0]
    for it in range(1, 8):
        T, gates = orc.two_sided_sweep(T, gates, locs, n)
        if it % 3 == 0:
            T = orc.init_circuit_tensor(V, gates, locs, n)
        assert abs(orc.trace_cost(T, n) - res["history"][it]) < 1e-15
    np.testing.assert_allclose(res["gates"], gates, atol=0)


def test_plateau_rules_fire_on_unreachable_target():
    n = 3
    locs = np.array([[0, 1]], dtype=np.int32)
    V = qi.haar_unitary(8, qi.rng(150))
    start = qi.haar_gates(1, qi.rng(151))
    res = orc.qfactor(V, start, locs, n, orc.QFactorOptions(diff_tol_r=1e-5, max_iter=50))
    assert res["reason"] == "plateau" and res["sweeps"] < 50
    # One gate reaches its optimum in the first sweep, so c_1 = c_2 = ...;
    # c_0 - c_5 is large, c_1 - c_6 = 0: the long rule fires at sweep 6.
    res = orc.qfactor(V, start, locs, n, orc.QFactorOptions(long_diff_count=5, long_diff_r=0.1, max_iter=50))
    assert res["reason"] == "plateau" and res["sweeps"] == 6


def test_multistart_lockstep_stops_when_any_start_converges():
    n = 4
    locs = qi.brickwork_locations(n, 4)
    inst = qi.make_problem(n, locs, 3, seed=8)
    V = orc.circuit_unitary(inst.target_gates, locs, n)
    o = orc.QFactorOptions(dist_tol=1e-10, max_iter=300)
    ms = orc.qfactor_multistart(V, inst.starts, locs, n, o)
    singles = [orc.qfactor(V, inst.starts[s], locs, n, o) for s in range(3)]
    first = min(r["sweeps"] for r in singles if r["reason"] == "converged")
    assert ms["reason"] == "converged" and ms["sweeps"] == first
    assert ms["costs"][ms["best"]] <= 1e-10
    for s in range(3):
        # every start followed its own single-start trajectory up to the stop
        assert ms["histories"][s] == singles[s]["history"][: first + 1]
