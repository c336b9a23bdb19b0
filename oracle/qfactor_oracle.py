"""QFactor oracle: plain FP64 NumPy implementation (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this module.  It is deliberately unoptimised: every step is the
paper's definition or algorithm step written out with NumPy library primitives
(tensordot, einsum, SVD), so that a reader can check it against the paper.

Paper: A. Kukliansky, E. Younis, L. Cincio, C. Iancu, "QFactor: A
Domain-Specific Optimizer for Quantum Circuit Instantiation", arXiv 2306.08152.

Conventions (the paper leaves them open; the CUDA path uses the same ones):
  * N = 2**n.  Qubit 0 is the most significant bit of a basis index.
  * A gate u (4x4) on location (a, b) acts on the local index 2*bit(a)+bit(b);
    G = u on (a, b) tensored with identity on every other qubit.
  * Gate lists are in product order: C = G_0 G_1 ... G_{p-1}; list index 0 is
    the paper's u_1 (Sec. III, U = u_1 ... u_p).
  * The circuit tensor starts as V^dagger and every gate is applied on its
    right, so T = V^dagger C after InitCircuitTensor (Alg. 1).
  * Environment of gate k: E_k = partial trace over every qubit except (a, b)
    of R_k = G_{k+1} ... G_{p-1} V^dagger G_0 ... G_{k-1}, so that
    Tr(V^dagger C) = Tr(E_k u_k) (Sec. III, environment matrix; Fig. 3).
  * Cost: Delta = 1 - |Tr(V^dagger C)| / N (Sec. II, cost function Delta).

Parity pins (tests/test_oracle_pins.py) fix every public function against
dense Kronecker-product constructions, finite differences, closed-form cases,
the Frobenius identity (Sec. III, Eq. cost), the optimality argument of
Sec. III-A1 and the monotonicity property of Sec. III-A.  The multistart and
plateau stopping rules (``qfactor_multistart``, diff/long-diff tests) follow a
reading of garbled text and are "parity unpinned" beyond their stated
properties.
"""
from __future__ import annotations

import string

import numpy as np

__all__ = [
    "apply_right",
    "apply_left",
    "calc_env_mat",
    "optimize_gate",
    "init_circuit_tensor",
    "circuit_unitary",
    "trace_cost",
    "two_sided_sweep",
    "QFactorOptions",
    "qfactor",
    "qfactor_multistart",
    "cost_and_env",
    "frobenius_distance",
]


def _as_tensor(T, n):
    return np.asarray(T, dtype=np.complex128).reshape((2,) * (2 * n))


def apply_right(T, u, a, b, n):
    """T <- T . (u on (a, b))  -- ApplyRight of Alg. 1.

    Contracts the column legs (a, b) of the circuit tensor with the input legs
    of the gate tensor (Fig. 3(a): applying a gate is a tensor contraction)."""
    N = 2**n
    t = _as_tensor(T, n)
    r = np.tensordot(t, np.asarray(u).reshape(2, 2, 2, 2), axes=([n + a, n + b], [0, 1]))
    r = np.moveaxis(r, [2 * n - 2, 2 * n - 1], [n + a, n + b])
    return np.ascontiguousarray(r).reshape(N, N)


def apply_left(T, u, a, b, n):
    """T <- (u on (a, b)) . T  -- ApplyLeft of Alg. 1 (contract row legs)."""
    N = 2**n
    t = _as_tensor(T, n)
    r = np.tensordot(np.asarray(u).reshape(2, 2, 2, 2), t, axes=([2, 3], [a, b]))
    r = np.moveaxis(r, [0, 1], [a, b])
    return np.ascontiguousarray(r).reshape(N, N)


def calc_env_mat(T, a, b, n):
    """CalcEnvMat of Alg. 1: partial trace of T over every qubit except
    (a, b).  Returns P with P[x, y] = sum_r T[(x, r), (y, r)]; when T has had
    gate k removed this P is E_k (Sec. III, Fig. 3(c))."""
    letters = string.ascii_letters
    rows = []
    cols = []
    free = iter(letters[4:])
    for q in range(n):
        if q == a:
            rows.append("w")
            cols.append("y")
        elif q == b:
            rows.append("x")
            cols.append("z")
        else:
            c = next(free)
            rows.append(c)
            cols.append(c)
    spec = "".join(rows) + "".join(cols) + "->wxyz"
    return np.einsum(spec, _as_tensor(T, n)).reshape(4, 4)


def optimize_gate(E, u_old=None, beta=0.0):
    """OptimizeGate (Sec. III-A1, Eq. opt_u): with the SVD E = X D Y^dagger
    the unitary maximising Re Tr(E u) is u_new = Y X^dagger, and the maximum
    is sum(D).  With beta != 0 the SVD is taken of (1-beta) E + beta u_old^dagger
    (Sec. III-A2, hyperparameter Beta).  Returns (u_new, sum of singular
    values of the decomposed matrix)."""
    A = np.asarray(E, dtype=np.complex128)
    if beta != 0.0:
        A = (1.0 - beta) * A + beta * np.asarray(u_old).conj().T
    X, s, Yh = np.linalg.svd(A)
    u_new = Yh.conj().T @ X.conj().T
    return u_new, float(s.sum())


def init_circuit_tensor(V, gates, locs, n):
    """InitCircuitTensor of Alg. 1: T <- V^dagger, then ApplyRight of every
    gate in list order, giving T = V^dagger C."""
    T = np.asarray(V, dtype=np.complex128).conj().T.copy()
    for u, (a, b) in zip(gates, locs):
        T = apply_right(T, u, int(a), int(b), n)
    return T


def circuit_unitary(gates, locs, n):
    """C = G_0 G_1 ... G_{p-1}: InitCircuitTensor with the identity target."""
    return init_circuit_tensor(np.eye(2**n, dtype=np.complex128), gates, locs, n)


def trace_cost(T, n):
    """Delta = 1 - |Tr T| / N for T = V^dagger C (Sec. II)."""
    return 1.0 - abs(np.trace(T)) / 2**n


def frobenius_distance(C, V):
    """||C - V||_F (the distance of Sec. III-A2's dist_tol)."""
    return float(np.linalg.norm(np.asarray(C) - np.asarray(V)))


def two_sided_sweep(T, gates, locs, n, beta=0.0, update_costs=None):
    """TwoSidedSweep of Alg. 1.

    Backward half, for k = p-1 .. 0: ApplyRight(u_k^dagger) removes the gate,
    CalcEnvMat gives E_k, OptimizeGate gives u_k', ApplyLeft(u_k') puts it
    back on the other side.  Forward half, for k = 0 .. p-1: ApplyLeft(u_k^dagger),
    CalcEnvMat, OptimizeGate, ApplyRight(u_k').  If ``update_costs`` is a list,
    the cost 1 - |Tr T|/N after every single update is appended to it."""
    gates = np.array(gates, dtype=np.complex128, copy=True)
    p = len(gates)
    N = 2**n
    for k in range(p - 1, -1, -1):
        a, b = int(locs[k][0]), int(locs[k][1])
        T = apply_right(T, gates[k].conj().T, a, b, n)
        E = calc_env_mat(T, a, b, n)
        u, _ = optimize_gate(E, gates[k], beta)
        gates[k] = u
        T = apply_left(T, u, a, b, n)
        if update_costs is not None:
            update_costs.append(1.0 - abs(np.trace(T)) / N)
    for k in range(p):
        a, b = int(locs[k][0]), int(locs[k][1])
        T = apply_left(T, gates[k].conj().T, a, b, n)
        E = calc_env_mat(T, a, b, n)
        u, _ = optimize_gate(E, gates[k], beta)
        gates[k] = u
        T = apply_right(T, u, a, b, n)
        if update_costs is not None:
            update_costs.append(1.0 - abs(np.trace(T)) / N)
    return T, gates


class QFactorOptions:
    """Termination and update hyperparameters (Sec. III-A2).

    Defaults follow the instantiation workloads used here: dist_tol 1e-10,
    max_iter 500, reset_iter 40 (the paper's value), beta 0; both plateau
    rules are off unless their tolerances are set (diff rule: diff_tol_a or
    diff_tol_r > 0; long rule: long_diff_count > 0).  Readings of the garbled
    plateau text: the short rule stops when c_{i-1} - c_i <= diff_tol_a +
    diff_tol_r * c_i; the long rule stops when c_{i-L} - c_i < long_diff_r *
    c_{i-L} with L = long_diff_count."""

    def __init__(self, dist_tol=1e-10, max_iter=500, min_iter=0, reset_iter=40,
                 diff_tol_a=0.0, diff_tol_r=0.0, long_diff_count=0,
                 long_diff_r=0.1, beta=0.0):
        self.dist_tol = float(dist_tol)
        self.max_iter = int(max_iter)
        self.min_iter = int(min_iter)
        self.reset_iter = int(reset_iter)
        self.diff_tol_a = float(diff_tol_a)
        self.diff_tol_r = float(diff_tol_r)
        self.long_diff_count = int(long_diff_count)
        self.long_diff_r = float(long_diff_r)
        self.beta = float(beta)


def _plateau(hist, it, o):
    """Plateau tests after iteration ``it`` on cost history ``hist``
    (hist[0] is the cost before the first sweep)."""
    c = hist[-1]
    if (o.diff_tol_a > 0.0 or o.diff_tol_r > 0.0) and len(hist) >= 2:
        if hist[-2] - c <= o.diff_tol_a + o.diff_tol_r * c:
            return True
    L = o.long_diff_count
    if L > 0 and it >= L:
        old = hist[-1 - L]
        if old - c < o.long_diff_r * old:
            return True
    return False


def qfactor(V, gates0, locs, n, opts=None):
    """Qfactor of Alg. 1 for one start.

    Repeats TwoSidedSweep; after each sweep the circuit tensor is rebuilt
    from V and the current gates when the sweep count is a multiple of
    reset_iter (Sec. III-A2, reset_iter), then the cost is taken and the
    termination conditions are tested.  Returns a dict with gates, cost,
    sweeps, history (costs after 0, 1, ... sweeps) and reason
    ('converged' | 'plateau' | 'max_iter')."""
    o = opts or QFactorOptions()
    gates = np.array(gates0, dtype=np.complex128, copy=True)
    T = init_circuit_tensor(V, gates, locs, n)
    hist = [trace_cost(T, n)]
    reason = "max_iter"
    it = 0
    for it in range(1, o.max_iter + 1):
        T, gates = two_sided_sweep(T, gates, locs, n, o.beta)
        if o.reset_iter > 0 and it % o.reset_iter == 0:
            T = init_circuit_tensor(V, gates, locs, n)
        hist.append(trace_cost(T, n))
        if it >= o.min_iter:
            if hist[-1] <= o.dist_tol:
                reason = "converged"
                break
            if _plateau(hist, it, o):
                reason = "plateau"
                break
    return {"gates": gates, "cost": hist[-1], "sweeps": it, "history": hist,
            "reason": reason, "T": T}


def qfactor_multistart(V, starts, locs, n, opts=None):
    """Lock-step multistart (Sec. IV-A): all starts sweep together; the run
    stops after the first sweep in which any start reaches dist_tol, or once
    every start has (at some sweep) met a plateau test, or at max_iter.
    Returns per-start gates/costs, the best start index, sweeps and reason."""
    o = opts or QFactorOptions()
    S = len(starts)
    gates = [np.array(g, dtype=np.complex128, copy=True) for g in starts]
    Ts = [init_circuit_tensor(V, g, locs, n) for g in gates]
    hists = [[trace_cost(T, n)] for T in Ts]
    plateaued = [False] * S
    reason = "max_iter"
    it = 0
    for it in range(1, o.max_iter + 1):
        for s in range(S):
            Ts[s], gates[s] = two_sided_sweep(Ts[s], gates[s], locs, n, o.beta)
            if o.reset_iter > 0 and it % o.reset_iter == 0:
                Ts[s] = init_circuit_tensor(V, gates[s], locs, n)
            hists[s].append(trace_cost(Ts[s], n))
        if it >= o.min_iter:
            if any(h[-1] <= o.dist_tol for h in hists):
                reason = "converged"
                break
            for s in range(S):
                if _plateau(hists[s], it, o):
                    plateaued[s] = True
            if all(plateaued):
                reason = "plateau"
                break
    costs = np.array([h[-1] for h in hists])
    return {"gates": np.stack(gates), "costs": costs, "best": int(np.argmin(costs)),
            "sweeps": it, "reason": reason, "histories": hists}


def cost_and_env(V, gates, locs, n):
    """Cost and every environment matrix, by definition (Sec. III, Fig. 3).

    t = Tr(V^dagger C); for each k, R_k = G_{k+1}..G_{p-1} V^dagger G_0..G_{k-1}
    is built from V^dagger by right-applying gates 0..k-1 and left-applying
    gates p-1 down to k+1, and E_k is its partial trace over the other qubits.
    Returns (cost, envs of shape (p, 4, 4), t)."""
    gates = np.asarray(gates, dtype=np.complex128)
    p = len(gates)
    Vd = np.asarray(V, dtype=np.complex128).conj().T
    envs = np.empty((p, 4, 4), dtype=np.complex128)
    for k in range(p):
        R = Vd.copy()
        for j in range(k):
            R = apply_right(R, gates[j], int(locs[j][0]), int(locs[j][1]), n)
        for j in range(p - 1, k, -1):
            R = apply_left(R, gates[j], int(locs[j][0]), int(locs[j][1]), n)
        envs[k] = calc_env_mat(R, int(locs[k][0]), int(locs[k][1]), n)
    C = circuit_unitary(gates, locs, n)
    t = complex(np.sum(Vd.T * C))  # Tr(V^dagger C) = sum_ij (V^dagger)_ij C_ji
    return 1.0 - abs(t) / 2**n, envs, t
