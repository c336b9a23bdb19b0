"""Three-qubit gates (and circuits mixing 2- and 3-qubit gates) on the GPU
against the k-qubit FP64 oracle (oracle/kqubit.py).

Steps: the fused 8x8 pass, the 8x8 partial trace, the 8x8 FP64 polar, and
InitCircuitTensor; sweeps of mixed circuits through a resident plan; a full
instantiation.  Tolerances as for two-qubit gates: complex128 steps to 1e-12
of the largest entry, sweeps to cost 1e-10 and gates 1e-9; complex64 passes
to 4e-6 (two 8-term FP32 products) and partial traces to 1e-6 of the sum of
magnitudes they add.
"""
import numpy as np
import pytest
import torch

import oracle.kqubit as ok
import qf_inputs as qi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qf():
    import paper_2306_08152_gb300 as qf

    qf._native.load()
    return qf


def _rand_T(S, n, g):
    N = 2**n
    return (g.standard_normal((S, N, N)) + 1j * g.standard_normal((S, N, N))) / np.sqrt(2)


def _relerr(x, ref):
    return float(np.max(np.abs(np.asarray(x) - ref)) / max(np.max(np.abs(ref)), 1e-300))


def _triples(n, g, count):
    fixed = [(0, 1, 2), (n - 1, n - 2, n - 3), (2, 0, n - 1), (n - 3, n - 1, 1)]
    out = [q for q in fixed if len(set(q)) == 3 and max(q) < n]
    while len(out) < len(fixed) + count:
        out.append(tuple(int(x) for x in g.choice(n, 3, replace=False)))
    return out


@pytest.mark.parametrize("n,dtype", [(3, torch.complex128), (4, torch.complex128), (6, torch.complex128),
                                     (9, torch.complex128), (3, torch.complex64), (4, torch.complex64),
                                     (6, torch.complex64), (7, torch.complex64), (10, torch.complex64),
                                     (11, torch.complex64)])
def test_apply_gate_k3_matches_oracle(qf, n, dtype):
    """Complex64 covers both pass kernels: gates whose bits are all >= 2 (the
    coalesced kernel; n = 7 is its smallest case, one 16-column group per
    rest row) and the rest (n = 3: a single block, so most of a warp's
    eight-block group is empty)."""
    g = qi.rng(10000 + n)
    S = 2
    T0 = _rand_T(S, n, g)
    tol = 1e-12 if dtype == torch.complex128 else 4e-6
    worst = 0.0
    for q in _triples(n, g, 3):
        L = np.stack([qi.haar_unitary(8, g) for _ in range(S)])
        R = np.stack([qi.haar_unitary(8, g) for _ in range(S)])
        for mode in ("L", "R", "LR"):
            Tg = torch.from_numpy(T0).to(dtype).cuda()
            qf.apply_gate_k(Tg, q, torch.from_numpy(L).cuda() if "L" in mode else None,
                            torch.from_numpy(R).cuda() if "R" in mode else None)
            out = Tg.cpu().numpy()
            for s in range(S):
                ref = T0[s]
                if "R" in mode:
                    ref = ok.apply_right_k(ref, R[s], q, n)
                if "L" in mode:
                    ref = ok.apply_left_k(ref, L[s], q, n)
                e = _relerr(out[s], ref)
                worst = max(worst, e)
                assert e <= tol, (q, mode, s, e)
    print(f"apply_gate_k3 n={n} {dtype}: max rel err {worst:.2e}")


@pytest.mark.parametrize("n,dtype", [(3, torch.complex128), (5, torch.complex128), (8, torch.complex128),
                                     (11, torch.complex128), (7, torch.complex64), (10, torch.complex64)])
def test_partial_trace_k3_matches_oracle(qf, n, dtype):
    g = qi.rng(10100 + n)
    S = 2
    T0 = _rand_T(S, n, g)
    Tg = torch.from_numpy(T0).to(dtype).cuda()
    Tc = Tg.cpu().numpy().astype(np.complex128)
    for q in _triples(n, g, 2):
        P = qf.partial_trace_k(Tg, q).cpu().numpy()
        for s in range(S):
            ref = ok.calc_env_mat_k(Tc[s], q, n)
            if dtype == torch.complex128:
                assert _relerr(P[s], ref) <= 1e-12, (q, s)
            else:
                bound = 1e-6 * ok.calc_env_mat_k(np.abs(Tc[s]).astype(np.complex128), q, n).real
                assert np.all(np.abs(P[s] - ref) <= bound), (q, s)


def test_optimize_gates_8x8_matches_oracle(qf):
    g = qi.rng(10200)
    count = 64
    E = g.standard_normal((count, 8, 8)) + 1j * g.standard_normal((count, 8, 8))
    U, sig = qf.optimize_gates_k(torch.from_numpy(E).cuda())
    U, sig = U.cpu().numpy(), sig.cpu().numpy()
    for i in range(count):
        u_ref, s_ref = ok.optimize_gate_k(E[i])
        assert abs(sig[i] - s_ref) <= 1e-12 * s_ref, i
        assert np.max(np.abs(U[i] - u_ref)) <= 1e-10, i
        assert np.max(np.abs(U[i].conj().T @ U[i] - np.eye(8))) <= 1e-13


def test_optimize_gates_8x8_rank_deficient_and_beta(qf):
    """Rank-deficient E: every completion of X is optimal, so compare the
    objective Re Tr(E u) = sum of singular values and unitarity, not u."""
    g = qi.rng(10300)
    Es = []
    for r in (7, 5, 2, 1):
        A = g.standard_normal((8, r)) + 1j * g.standard_normal((8, r))
        B = g.standard_normal((r, 8)) + 1j * g.standard_normal((r, 8))
        Es.append(A @ B)
    Es.append(np.zeros((8, 8), dtype=np.complex128))
    Es = np.stack(Es)
    U, sig = qf.optimize_gates_k(torch.from_numpy(Es).cuda())
    U, sig = U.cpu().numpy(), sig.cpu().numpy()
    for i in range(len(Es)):
        _, s_ref = ok.optimize_gate_k(Es[i])
        assert abs(sig[i] - s_ref) <= 1e-11 * max(s_ref, 1.0), i
        assert abs(np.trace(Es[i] @ U[i]).real - s_ref) <= 1e-11 * max(s_ref, 1.0), i
        assert np.max(np.abs(U[i].conj().T @ U[i] - np.eye(8))) <= 1e-13, i
    E = g.standard_normal((8, 8, 8)) + 1j * g.standard_normal((8, 8, 8))
    u_old = np.stack([qi.haar_unitary(8, g) for _ in range(8)])
    U, _ = qf.optimize_gates_k(torch.from_numpy(E).cuda(), torch.from_numpy(u_old).cuda(), 0.3)
    for i in range(8):
        u_ref, _ = ok.optimize_gate_k(E[i], u_old[i], 0.3)
        assert np.max(np.abs(U[i].cpu().numpy() - u_ref)) <= 1e-10


def _mixed(n, p, g):
    locs, gates = [], []
    for i in range(p):
        k = 3 if (i % 3 == 0 and n >= 3) else 2
        locs.append(tuple(int(x) for x in g.choice(n, k, replace=False)))
        gates.append(qi.haar_unitary(2**k, g))
    return locs, gates


@pytest.mark.parametrize("n", [3, 5, 8])
def test_init_tensor_k_and_circuit_unitary(qf, n):
    g = qi.rng(10400 + n)
    locs, gates = _mixed(n, 7, g)
    V = qi.haar_unitary(2**n, g)
    T = qf.init_tensor_k(torch.from_numpy(V).cuda(), locs, [gates]).cpu().numpy()[0]
    assert _relerr(T, ok.init_circuit_tensor_k(V, gates, locs, n)) <= 1e-12
    C = qf.circuit_unitary_k(n, locs, gates).cpu().numpy()
    assert _relerr(C, ok.circuit_unitary_k(gates, locs, n)) <= 1e-12


@pytest.mark.parametrize("n,S,prec", [(4, 2, "c128"), (6, 3, "c128"), (9, 2, "c128"), (7, 2, "c64")])
def test_mixed_sweeps_match_oracle(qf, n, S, prec):
    g = qi.rng(10500 + n)
    locs, _ = _mixed(n, 8, g)
    V = qi.haar_unitary(2**n, g)
    starts = [[qi.haar_unitary(2 ** len(q), g) for q in locs] for _ in range(S)]
    plan = qf.Plan(n, locs, S, qf.QF_C128 if prec == "c128" else qf.QF_C64)
    plan.load(torch.from_numpy(V).cuda(), qf.flatten_gates(starts).cuda())
    plan.sweep(3, reset_iter=2)
    costs = plan.costs()
    gates = qf.unflatten_gates(plan.gates(), locs)
    plan.close()
    for s in range(S):
        T = ok.init_circuit_tensor_k(V, starts[s], locs, n)
        gref = starts[s]
        for it in range(1, 4):
            T, gref = ok.two_sided_sweep_k(T, gref, locs, n)
            if it % 2 == 0:
                T = ok.init_circuit_tensor_k(V, gref, locs, n)
        c_ref = ok.trace_cost(T, n)
        if prec == "c128":
            assert abs(costs[s] - c_ref) <= 1e-10, (s, costs[s], c_ref)
            for a, b in zip(gates[s], gref):
                assert np.max(np.abs(a - b)) <= 1e-9
        else:
            assert abs(costs[s] - c_ref) <= 1e-5, (s, costs[s], c_ref)


@pytest.mark.parametrize("precision", ["c128", "c64refine"])
def test_instantiate_k_reaches_tolerance(qf, precision):
    n = 4
    locs = [(0, 1, 2), (2, 3), (1, 2, 3), (0, 1)]
    g = qi.rng(9950)
    tgt = [qi.haar_unitary(2 ** len(q), g) for q in locs]
    V = ok.circuit_unitary_k(tgt, locs, n)
    starts = [[qi.haar_unitary(2 ** len(q), qi.rng(9951 + s * 10 + i)) for i, q in enumerate(locs)]
              for s in range(4)]
    prec = qf.QF_C128 if precision == "c128" else qf.QF_C64_REFINE64
    res = qf.instantiate_k(torch.from_numpy(V).cuda(), locs, starts, dist_tol=1e-10, max_sweeps=300,
                           precision=prec)
    assert res["best_cost"] <= 1e-10, res["costs"]
    c_ref, _, _ = ok.cost_and_env_k(V, res["gates"][res["best"]], locs, n)
    assert c_ref <= 2e-10 and abs(c_ref - res["best_cost"]) <= 1e-10


def test_invalid_k_locations_are_rejected(qf):
    from paper_2306_08152_gb300 import QFactorError

    V = torch.eye(16, dtype=torch.complex128).cuda()
    with pytest.raises(QFactorError):
        qf.instantiate_k(V, [(0, 1, 1)], [[np.eye(8)]])
    with pytest.raises(QFactorError):
        qf.instantiate_k(V, [(0, 1, 4)], [[np.eye(8)]])
    with pytest.raises(ValueError):
        qf.instantiate_k(V, [(0, 1, 2, 3, 4)], [[np.eye(32)]])
