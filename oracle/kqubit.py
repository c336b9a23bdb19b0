"""QFactor oracle for k-qubit gates: plain FP64 NumPy (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this module.  It restates Alg. 1 (InitCircuitTensor,
TwoSidedSweep, CalcEnvMat, OptimizeGate) for gates on any number k of
qubits: the paper presents the method for two-qubit gates and states that it
extends to k-qubit unitaries, whose environment is then 2^k x 2^k
(Sec. III; conclusion).  Every step is the definition written out with
NumPy library primitives.

Conventions (identical to the two-qubit oracle for k = 2):
  * a location is a tuple of k distinct qubits (q_0, ..., q_{k-1}); the
    gate's local basis index is sum_i bit(q_i) * 2^(k-1-i), so q_0 is the
    most significant local bit;
  * gates are 2^k x 2^k complex matrices; C = G_0 G_1 ... G_{p-1};
  * T starts as V^dagger and every gate is applied on its right
    (T = V^dagger C after InitCircuitTensor);
  * E_k = partial trace over the other qubits of
    R_k = G_{k+1} ... G_{p-1} V^dagger G_0 ... G_{k-1}, so Tr(V^dagger C) =
    Tr(E_k u_k); the update is u' = Y X^dagger from E = X D Y^dagger (Eq. opt_u).

Parity pins (tests/test_oracle_pins_k.py): dense basis-loop operators for
n <= 5 with 1-, 2-, 3- and 4-qubit gates, agreement with the two-qubit oracle at
k = 2, finite differences of Tr(V^dagger C), the identity Tr(E_k u_k) =
Tr(V^dagger C), the closed-form single-gate fits (n = k: one update reaches
cost 0; n = k + 1 with a product target: cost 1 - |Tr g|/2), local
optimality of the update and per-update monotonicity.
"""
from __future__ import annotations

import string

import numpy as np

__all__ = [
    "apply_right_k",
    "apply_left_k",
    "calc_env_mat_k",
    "optimize_gate_k",
    "init_circuit_tensor_k",
    "circuit_unitary_k",
    "two_sided_sweep_k",
    "qfactor_multistart_k",
    "cost_and_env_k",
    "trace_cost",
]


def _legs(T, n):
    return np.asarray(T, dtype=np.complex128).reshape((2,) * (2 * n))


def _gate(u, k):
    u = np.asarray(u, dtype=np.complex128)
    assert u.shape == (2**k, 2**k)
    return u.reshape((2,) * (2 * k))  # legs: k output (row) bits, then k input (column) bits


def apply_right_k(T, u, qubits, n):
    """T <- T (u on qubits): contract the column legs of the qubits with the
    gate's row legs (the gate sits to the right of T)."""
    k = len(qubits)
    t = _legs(T, n)
    r = np.tensordot(t, _gate(u, k), axes=([n + q for q in qubits], list(range(k))))
    # tensordot puts the gate's k column legs last; move them to the columns
    r = np.moveaxis(r, list(range(2 * n - k, 2 * n)), [n + q for q in qubits])
    return np.ascontiguousarray(r).reshape(2**n, 2**n)


def apply_left_k(T, u, qubits, n):
    """T <- (u on qubits) T: contract the gate's column legs with the row legs
    of the qubits."""
    k = len(qubits)
    t = _legs(T, n)
    r = np.tensordot(_gate(u, k), t, axes=(list(range(k, 2 * k)), list(qubits)))
    r = np.moveaxis(r, list(range(k)), list(qubits))
    return np.ascontiguousarray(r).reshape(2**n, 2**n)


def calc_env_mat_k(T, qubits, n):
    """CalcEnvMat: P[x][y] = sum over the other qubits' common index r of
    T[(x, r), (y, r)], x and y the local indices of the qubits."""
    k = len(qubits)
    letters = string.ascii_letters
    row_loc = letters[:k]
    col_loc = letters[k:2 * k]
    free = iter(letters[2 * k:])
    rows, cols = [], []
    for q in range(n):
        if q in qubits:
            i = list(qubits).index(q)
            rows.append(row_loc[i])
            cols.append(col_loc[i])
        else:
            c = next(free)
            rows.append(c)
            cols.append(c)
    spec = "".join(rows) + "".join(cols) + "->" + row_loc + col_loc
    return np.einsum(spec, _legs(T, n)).reshape(2**k, 2**k)


def optimize_gate_k(E, u_old=None, beta=0.0):
    """OptimizeGate (Sec. III-A1, Eq. opt_u) for any size: with the SVD
    A = X D Y^dagger of A = (1 - beta) E + beta u_old^dagger, u = Y X^dagger
    maximises Re Tr(A u) and the maximum is sum(D)."""
    A = np.asarray(E, dtype=np.complex128)
    if beta != 0.0:
        A = (1.0 - beta) * A + beta * np.asarray(u_old).conj().T
    X, s, Yh = np.linalg.svd(A)
    return Yh.conj().T @ X.conj().T, float(s.sum())


def init_circuit_tensor_k(V, gates, locs, n):
    """InitCircuitTensor: T <- V^dagger, then every gate on the right in list order."""
    T = np.asarray(V, dtype=np.complex128).conj().T.copy()
    for u, q in zip(gates, locs):
        T = apply_right_k(T, u, tuple(int(x) for x in q), n)
    return T


def circuit_unitary_k(gates, locs, n):
    """C = G_0 ... G_{p-1}."""
    return init_circuit_tensor_k(np.eye(2**n, dtype=np.complex128), gates, locs, n)


def trace_cost(T, n):
    """Delta = 1 - |Tr T| / N (Sec. II)."""
    return 1.0 - abs(np.trace(T)) / 2**n


def two_sided_sweep_k(T, gates, locs, n, beta=0.0, update_costs=None):
    """TwoSidedSweep of Alg. 1 for gates of any size: backward k = p-1..0
    (remove on the right, environment, update, apply on the left), then
    forward k = 0..p-1 (remove on the left, environment, update, apply on
    the right).  ``gates`` is a list of 2^k x 2^k arrays."""
    gates = [np.array(g, dtype=np.complex128, copy=True) for g in gates]
    p = len(gates)
    N = 2**n
    for k in range(p - 1, -1, -1):
        q = tuple(int(x) for x in locs[k])
        T = apply_right_k(T, gates[k].conj().T, q, n)
        u, _ = optimize_gate_k(calc_env_mat_k(T, q, n), gates[k], beta)
        gates[k] = u
        T = apply_left_k(T, u, q, n)
        if update_costs is not None:
            update_costs.append(1.0 - abs(np.trace(T)) / N)
    for k in range(p):
        q = tuple(int(x) for x in locs[k])
        T = apply_left_k(T, gates[k].conj().T, q, n)
        u, _ = optimize_gate_k(calc_env_mat_k(T, q, n), gates[k], beta)
        gates[k] = u
        T = apply_right_k(T, u, q, n)
        if update_costs is not None:
            update_costs.append(1.0 - abs(np.trace(T)) / N)
    return T, gates


def qfactor_multistart_k(V, starts, locs, n, dist_tol=1e-10, max_iter=500, reset_iter=40):
    """Lock-step multistart (Sec. IV-A) with the tolerance and sweep-count
    stopping rules; the tensor is rebuilt after every reset_iter-th sweep.
    Returns per-start gates and costs, the best start and the sweep count."""
    S = len(starts)
    gates = [[np.array(g, dtype=np.complex128) for g in st] for st in starts]
    Ts = [init_circuit_tensor_k(V, g, locs, n) for g in gates]
    costs = [trace_cost(T, n) for T in Ts]
    it = 0
    for it in range(1, max_iter + 1):
        for s in range(S):
            Ts[s], gates[s] = two_sided_sweep_k(Ts[s], gates[s], locs, n)
            if reset_iter > 0 and it % reset_iter == 0:
                Ts[s] = init_circuit_tensor_k(V, gates[s], locs, n)
            costs[s] = trace_cost(Ts[s], n)
        if min(costs) <= dist_tol:
            break
    return {"gates": gates, "costs": np.array(costs), "best": int(np.argmin(costs)), "sweeps": it}


def cost_and_env_k(V, gates, locs, n):
    """Cost, every environment E_k (by its definition: the partial trace of
    R_k = G_{k+1}..G_{p-1} V^dagger G_0..G_{k-1}) and t = Tr(V^dagger C)."""
    p = len(gates)
    Vd = np.asarray(V, dtype=np.complex128).conj().T
    envs = []
    for k in range(p):
        R = Vd.copy()
        for j in range(k):
            R = apply_right_k(R, gates[j], tuple(locs[j]), n)
        for j in range(p - 1, k, -1):
            R = apply_left_k(R, gates[j], tuple(locs[j]), n)
        envs.append(calc_env_mat_k(R, tuple(locs[k]), n))
    C = circuit_unitary_k(gates, locs, n)
    t = complex(np.sum(Vd.T * C))
    return 1.0 - abs(t) / 2**n, envs, t
