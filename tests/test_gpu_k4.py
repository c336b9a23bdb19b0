"""Four-qubit gates (a 16 x 16 unitary as one variable, Sec. III and VI) on
the GPU against the k-qubit FP64 oracle (oracle/kqubit.py).

Steps: the fused 16x16 pass, the 16x16 partial trace (one and several CTAs
per start), the 16x16 FP64 polar on one CTA, InitCircuitTensor; sweeps of
circuits mixing 2-, 3- and 4-qubit gates through a resident plan (two start
groups, the second sweep a graph replay); reachable instantiations.
Tolerances as for smaller gates: complex128 and double-FP32 steps to 1e-12
of the largest entry, sweeps to cost 1e-10 and gates 1e-9; complex64 passes
to 8e-6 (two 16-term FP32 products) and partial traces to 1e-6 of the sum of
magnitudes they add; updates within the polar-factor perturbation bound of
tests/test_gpu_polar_edge.py.
"""
import numpy as np
import pytest
import torch

import oracle.kqubit as ok
import qf_inputs as qi

pytestmark = pytest.mark.gpu

EPS = 2.0**-52


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


def _quads(n, g, count):
    fixed = [(0, 1, 2, 3), (n - 1, n - 2, n - 3, n - 4), (3, 0, n - 1, 1), (n - 4, 2, n - 1, 0)]
    out = [q for q in fixed if len(set(q)) == 4 and max(q) < n]
    while len(out) < len(fixed) + count:
        out.append(tuple(int(x) for x in g.choice(n, 4, replace=False)))
    return out


def _to_dtype(qf, T128, dtype):
    if dtype == "df64":
        return qf.convert_tensor(torch.from_numpy(T128).cuda(), qf.QF_DF64)
    return torch.from_numpy(T128).to(dtype).cuda()


def _back(qf, T, dtype):
    if dtype == "df64":
        return qf.convert_tensor(T, qf.QF_C128).cpu().numpy()
    return T.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("n,dtype", [(4, torch.complex128), (5, torch.complex128), (7, torch.complex128),
                                     (4, torch.complex64), (6, torch.complex64), (9, torch.complex64),
                                     (11, torch.complex64), (6, "df64")])
def test_apply_gate_k4_matches_oracle(qf, n, dtype):
    g = qi.rng(14000 + n)
    S = 2
    for q in _quads(n, g, 2):
        T0 = _rand_T(S, n, g)
        L = np.stack([qi.haar_unitary(16, g) for _ in range(S)])
        R = np.stack([qi.haar_unitary(16, g) for _ in range(S)])
        T = _to_dtype(qf, T0, dtype)
        qf.apply_gate_k(T, q, torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda())
        out = _back(qf, T, dtype)
        tol = 8e-6 if dtype == torch.complex64 else 1e-12
        worst = 0.0
        for s in range(S):
            ref = ok.apply_left_k(ok.apply_right_k(T0[s], R[s], q, n), L[s], q, n)
            if dtype == torch.complex64:  # the input was rounded to FP32 too
                Tin = T0[s].astype(np.complex64).astype(np.complex128)
                ref = ok.apply_left_k(ok.apply_right_k(Tin, R[s], q, n), L[s], q, n)
            worst = max(worst, _relerr(out[s], ref))
        assert worst <= tol, (q, worst)
        # right-only (InitCircuitTensor's form)
        T = _to_dtype(qf, T0, dtype)
        qf.apply_gate_k(T, q, None, torch.from_numpy(R).cuda())
        out = _back(qf, T, dtype)
        for s in range(S):
            Tin = T0[s].astype(np.complex64).astype(np.complex128) if dtype == torch.complex64 else T0[s]
            assert _relerr(out[s], ok.apply_right_k(Tin, R[s], q, n)) <= tol
    print(f"apply_gate_k4 n={n} {dtype}: max rel err {worst:.2e}")


@pytest.mark.parametrize("n,dtype,S", [(4, torch.complex128, 2), (6, torch.complex128, 3),
                                       (11, torch.complex128, 2), (12, torch.complex128, 1),
                                       (6, torch.complex64, 2), (12, torch.complex64, 2),
                                       (7, "df64", 2)])
def test_partial_trace_k4_matches_oracle(qf, n, dtype, S):
    g = qi.rng(14100 + n)
    T0 = _rand_T(S, n, g)
    T = _to_dtype(qf, T0, dtype)
    for q in _quads(n, g, 1):
        P = qf.partial_trace_k(T, q).cpu().numpy()
        for s in range(S):
            Ts = T0[s].astype(np.complex64).astype(np.complex128) if dtype == torch.complex64 else T0[s]
            ref = ok.calc_env_mat_k(Ts, q, n)
            if dtype == torch.complex64:
                bound = 1e-6 * ok.calc_env_mat_k(np.abs(Ts).astype(np.complex128), q, n).real
                assert np.all(np.abs(P[s] - ref) <= bound), (q, s)
            else:
                assert _relerr(P[s], ref) <= 1e-12, (q, s)


def _bound(sig):
    sig = np.asarray(sig, dtype=float)
    return max(100.0 * EPS * sig.max() / sig.min(), 1e-11)


def test_optimize_gates_16x16_matches_oracle(qf):
    g = qi.rng(14200)
    Es, sigs = [], []
    for _ in range(12):  # Gaussian environments
        E = g.standard_normal((16, 16)) + 1j * g.standard_normal((16, 16))
        Es.append(E)
        sigs.append(np.linalg.svd(E, compute_uv=False))
    for r in (1e-3, 1e-6, 1e-9, 1e-12):  # graded spectra
        sig = r ** (np.arange(16) / 15)
        X, Y = qi.haar_unitary(16, g), qi.haar_unitary(16, g)
        for scale in (1.0, 1e-150):
            Es.append(scale * (X * sig[None, :]) @ Y.conj().T)
            sigs.append(scale * sig)
    Es.append(np.eye(16) * 3.0 * np.exp(0.7j))  # degenerate
    sigs.append(np.full(16, 3.0))
    Es = np.stack(Es)
    U, S = qf.optimize_gates_k(torch.from_numpy(Es).cuda())
    U, S = U.cpu().numpy(), S.cpu().numpy()
    worst = 0.0
    for i, E in enumerate(Es):
        u_ref, s_ref = ok.optimize_gate_k(E)
        s_true = float(np.sum(sigs[i]))
        assert np.max(np.abs(U[i].conj().T @ U[i] - np.eye(16))) <= 1e-13, i
        assert abs(np.trace(E @ U[i]).real - s_true) <= 1e-12 * s_true, i
        assert abs(S[i] - s_true) <= 1e-12 * s_true, i
        err = float(np.max(np.abs(U[i] - u_ref)))
        worst = max(worst, err / _bound(sigs[i]))
        assert err <= _bound(sigs[i]), (i, err)
    print(f"16x16 polar: worst |u - u_oracle| / bound = {worst:.3f}")


def test_optimize_gates_16x16_rank_deficient_and_beta(qf):
    g = qi.rng(14300)
    cases = [np.zeros((16, 16), complex)]
    for r in (1, 5, 15):
        A = g.standard_normal((16, r)) + 1j * g.standard_normal((16, r))
        B = g.standard_normal((r, 16)) + 1j * g.standard_normal((r, 16))
        cases.append(A @ B)
    U, S = qf.optimize_gates_k(torch.from_numpy(np.stack(cases)).cuda())
    U = U.cpu().numpy()
    for i, E in enumerate(cases):
        s_ref = np.linalg.svd(E, compute_uv=False).sum()
        assert abs(S[i].item() - s_ref) <= 1e-12 * max(1, s_ref)
        assert np.max(np.abs(U[i].conj().T @ U[i] - np.eye(16))) <= 1e-13
        assert abs(np.trace(E @ U[i]) - s_ref) <= 1e-12 * max(1, s_ref)
    E = np.stack([g.standard_normal((16, 16)) + 1j * g.standard_normal((16, 16)) for _ in range(3)])
    u_old = np.stack([qi.haar_unitary(16, g) for _ in range(3)])
    for beta in (0.3, 1.0):
        U, S = qf.optimize_gates_k(torch.from_numpy(E).cuda(), torch.from_numpy(u_old).cuda(), beta)
        U = U.cpu().numpy()
        for i in range(3):
            u_ref, s_ref = ok.optimize_gate_k(E[i], u_old[i], beta)
            assert np.max(np.abs(U[i] - u_ref)) <= 1e-10
            assert abs(S[i].item() - s_ref) <= 1e-12 * max(1, s_ref)


@pytest.mark.parametrize("n", [4, 6])
def test_init_tensor_k4_and_circuit_unitary(qf, n):
    g = qi.rng(14400 + n)
    locs = [(0, 1, 2, 3), (n - 1, 1), (1, n - 1, 2, 0), (n - 2, n - 1, 0)]
    gates = [qi.haar_unitary(2 ** len(q), g) for q in locs]
    V = qi.haar_unitary(2**n, g)
    T = qf.init_tensor_k(torch.from_numpy(V).cuda(), locs, [gates]).cpu().numpy()[0]
    assert _relerr(T, ok.init_circuit_tensor_k(V, gates, locs, n)) <= 1e-12
    C = qf.circuit_unitary_k(n, locs, gates).cpu().numpy()
    assert _relerr(C, ok.circuit_unitary_k(gates, locs, n)) <= 1e-12


def _mixed4(n, p, g):
    locs = []
    for i in range(p):
        k = (4, 2, 3)[i % 3]
        locs.append(tuple(int(x) for x in g.choice(n, k, replace=False)))
    return locs


@pytest.mark.parametrize("n,S,prec,sweeps", [(5, 2, "c128", 3), (7, 3, "c128", 3), (11, 2, "c128", 2),
                                             (8, 2, "c64", 2), (6, 2, "df64", 2)])
def test_mixed_k4_sweeps_match_oracle(qf, n, S, prec, sweeps):
    g = qi.rng(14500 + n)
    locs = _mixed4(n, 7, g)
    V = qi.haar_unitary(2**n, g)
    starts = [[qi.haar_unitary(2 ** len(q), g) for q in locs] for _ in range(S)]
    qprec = {"c128": qf.QF_C128, "c64": qf.QF_C64, "df64": qf.QF_DF64}[prec]
    plan = qf.Plan(n, locs, S, qprec)
    plan.load(torch.from_numpy(V).cuda(), qf.flatten_gates(starts).cuda())
    plan.sweep(sweeps, reset_iter=2)
    costs = plan.costs()
    gates = qf.unflatten_gates(plan.gates(), locs)
    assert plan.status() == 0
    plan.close()
    for s in range(S):
        T = ok.init_circuit_tensor_k(V, starts[s], locs, n)
        gref = starts[s]
        for it in range(1, sweeps + 1):
            T, gref = ok.two_sided_sweep_k(T, gref, locs, n)
            if it % 2 == 0:
                T = ok.init_circuit_tensor_k(V, gref, locs, n)
        c_ref = ok.trace_cost(T, n)
        print(f"k4 mixed n={n} {prec} start {s}: |dcost| {abs(costs[s] - c_ref):.2e}")
        if prec == "c64":
            assert abs(costs[s] - c_ref) <= 1e-5, (s, costs[s], c_ref)
        else:
            assert abs(costs[s] - c_ref) <= 1e-10, (s, costs[s], c_ref)
            for a, b in zip(gates[s], gref):
                assert np.max(np.abs(a - b)) <= 1e-9, s


@pytest.mark.parametrize("precision", ["c128", "c64refine"])
def test_instantiate_k4_reaches_tolerance(qf, precision):
    n = 5
    locs = [(0, 1, 2, 3), (3, 4), (1, 2, 3, 4), (0, 1)]
    g = qi.rng(9960)  # the oracle's pin fits this target to < 1e-12
    tgt = [qi.haar_unitary(2 ** len(q), g) for q in locs]
    V = ok.circuit_unitary_k(tgt, locs, n)
    starts = [[qi.haar_unitary(2 ** len(q), qi.rng(9961 + s * 10 + i)) for i, q in enumerate(locs)]
              for s in range(4)]
    prec = qf.QF_C128 if precision == "c128" else qf.QF_C64_REFINE64
    res = qf.instantiate_k(torch.from_numpy(V).cuda(), locs, starts, dist_tol=1e-10, max_sweeps=300,
                           precision=prec)
    assert res["best_cost"] <= 1e-10, res["costs"]
    c_ref, _, _ = ok.cost_and_env_k(V, res["gates"][res["best"]], locs, n)
    assert c_ref <= 2e-10 and abs(c_ref - res["best_cost"]) <= 1e-10


def test_invalid_k4_locations_are_rejected(qf):
    from paper_2306_08152_gb300 import QFactorError

    V = torch.eye(16, dtype=torch.complex128).cuda()
    with pytest.raises(QFactorError):
        qf.instantiate_k(V, [(0, 1, 2, 2)], [[np.eye(16)]])
    with pytest.raises(QFactorError):
        qf.instantiate_k(V, [(0, 1, 2, 4)], [[np.eye(16)]])
    V3 = torch.eye(8, dtype=torch.complex128).cuda()
    with pytest.raises(QFactorError):  # k > n_qubits
        qf.instantiate_k(V3, [(0, 1, 2, 3)], [[np.eye(16)]])
