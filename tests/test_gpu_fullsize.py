"""Full-size parity: 12 qubits, linear brickwork of 12 layers (66 U(4)
gates), 8 starts -- the launch configuration the benchmark times.

The oracle cannot run whole 12-qubit sweeps in test time, so the full-size
checks are (a) every single step of one gate update, on a sampled start,
compared element by element with the oracle, in the 8-start launch
configuration, and (b) properties that hold at any size for whole sweeps:
the cost never increases (Sec. III-A), the gates stay unitary, and after a
sweep Tr(T) is real and non-negative (it equals the last update's sum of
singular values, Sec. III-A1).
"""
import numpy as np
import pytest
import torch

import oracle as orc
import qf_inputs as qi

pytestmark = pytest.mark.gpu

N_QUBITS = 12
LAYERS = 12
STARTS = 8


@pytest.fixture(scope="module")
def qf():
    import paper_2306_08152_gb300 as qf

    qf._native.load()
    return qf


@pytest.fixture(scope="module")
def problem():
    locs = qi.brickwork_locations(N_QUBITS, LAYERS)
    assert len(locs) == 66
    inst = qi.make_problem(N_QUBITS, locs, STARTS, seed=2024)
    V = orc.circuit_unitary(inst.target_gates, locs, N_QUBITS)
    return inst, V


def _relerr(x, ref):
    return float(np.max(np.abs(x - ref)) / np.max(np.abs(ref)))


@pytest.mark.parametrize("dtype,S,tol", [(torch.complex64, STARTS, 2e-5), (torch.complex128, 1, 1e-12)])
def test_one_update_at_full_size(qf, problem, dtype, S, tol):
    inst, V = problem
    n, locs = N_QUBITS, inst.locs
    p = len(locs)
    Vg = torch.from_numpy(V).cuda()
    starts = torch.from_numpy(inst.starts[:S]).cuda()
    T = qf.init_tensor(Vg, locs, starts, dtype=dtype)
    # sampled start: the last one of the launch
    s = S - 1
    T_ref = orc.init_circuit_tensor(V, inst.starts[s], locs, n)
    e_init = _relerr(T[s].cpu().numpy(), T_ref)
    print(f"{dtype} init rel err {e_init:.2e}")
    assert e_init <= tol * 10  # 66 chained passes
    # first backward update of gate p-1, step by step
    k = p - 1
    a, b = int(locs[k][0]), int(locs[k][1])
    u = inst.starts[:, k][:S]
    P = qf.partial_trace(T, a, b).cpu().numpy()
    Tc = T[s].cpu().numpy().astype(np.complex128)
    P_ref = orc.calc_env_mat(Tc, a, b, n)
    if dtype == torch.complex128:
        assert _relerr(P[s], P_ref) <= 1e-11
    else:  # FP32 band sums (see test_partial_trace_matches_oracle)
        bound = 1e-6 * orc.calc_env_mat(np.abs(Tc).astype(np.complex128), a, b, n).real
        assert np.all(np.abs(P[s] - P_ref) <= bound)
    E = np.einsum("sij,skj->sik", P, u.conj())  # E = P u^dagger
    U, sig = qf.optimize_gates(torch.from_numpy(E).cuda())
    U = U.cpu().numpy()
    T_rem = orc.apply_right(Tc, u[s].conj().T, a, b, n)
    u_ref, s_ref = orc.optimize_gate(orc.calc_env_mat(T_rem, a, b, n))
    # complex64: the environment carries the FP32 band-sum error above
    assert np.max(np.abs(U[s] - u_ref)) <= (1e-9 if dtype == torch.complex128 else 1e-5)
    qf.apply_pair(T, a, b, torch.from_numpy(U).cuda(), torch.from_numpy(u.conj().transpose(0, 2, 1).copy()).cuda())
    T_new_ref = orc.apply_left(T_rem, U[s], a, b, n)
    e_upd = _relerr(T[s].cpu().numpy(), T_new_ref)
    print(f"{dtype} one update rel err {e_upd:.2e}")
    assert e_upd <= tol
    tr = qf.trace(T).cpu().numpy()[s]
    assert abs(tr - np.trace(T[s].cpu().numpy().astype(np.complex128))) <= 1e-9 * 2**n


def test_full_size_sweeps_keep_invariants(qf, problem):
    inst, V = problem
    n, locs = N_QUBITS, inst.locs
    plan = qf.Plan(n, locs, STARTS, qf.QF_C64)
    plan.load(torch.from_numpy(V).cuda(), torch.from_numpy(inst.starts).cuda())
    c0 = plan.costs()
    prev = c0
    for _ in range(3):
        plan.sweep(1)
        c = plan.costs()
        assert np.all(c <= prev + 1e-5), (prev, c)  # FP32 tensor: 1e-5 noise
        prev = c
    assert np.all(prev < c0)
    assert plan.status() == 0
    G = plan.gates().numpy()
    eye = np.eye(4)
    assert max(np.max(np.abs(g.conj().T @ g - eye)) for g in G.reshape(-1, 4, 4)) <= 1e-12
    plan.close()
