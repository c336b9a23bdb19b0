"""The tensor-core 16x16 pass: every complex64 four-qubit pass with both
operators at 7 qubits and above runs on the fifth-generation tensor cores
(tcgen05 MMAs in 3xTF32 form, qf_k4.cu).  Checked against the FP64 oracle's
ApplyRight / ApplyLeft (Alg. 1) element by element:

- gate positions with and without bit 0, consecutive and scattered bits,
  unsorted qubit orders (the kernel permutes the operators to ascending-bit
  order); 7 qubits (8 tiles per start, fewer than the CTAs) up to 13; three
  starts per launch, so CTAs whose tiles cross into the next start re-embed
  the operators;
- the benchmark's launch (12 qubits, 4 starts per launch) at every
  consecutive quadruple, and every set of four qubits at 8 qubits;
- a whole 12-qubit sweep of 15 four-qubit gates through the plan (two start
  groups, the second sweep a CUDA-graph replay) against the oracle's
  TwoSidedSweep;
- the bounded completion waits: with a limit of 0 polls every wait runs out
  at once; the pass leaves NaN, a plan reports QF_ETIMEOUT, and the context
  stays usable.

Tolerance: 8e-6 of the largest entry, as for the FP32 kernels (two 16-term
complex products; the 3xTF32 products keep about 2^-21 of each term).
"""
import numpy as np
import pytest
import torch

import oracle.kqubit as ok
import qf_inputs as qi

pytestmark = pytest.mark.gpu

TOL = 8e-6


@pytest.fixture(scope="module")
def qf():
    import paper_2306_08152_gb300 as qf

    qf._native.load()
    return qf


def _rand_T(S, n, g):
    N = 2**n
    return (g.standard_normal((S, N, N)) + 1j * g.standard_normal((S, N, N))) / np.sqrt(2 * N)


def _relerr(x, ref):
    return float(np.max(np.abs(x - ref)) / np.max(np.abs(ref)))


def _check_pass(qf, n, S, quads, seed):
    g = qi.rng(seed)
    worst = 0.0
    for q in quads:
        T0 = _rand_T(S, n, g).astype(np.complex64)
        L = np.stack([qi.haar_unitary(16, g) for _ in range(S)])
        R = np.stack([qi.haar_unitary(16, g) for _ in range(S)])
        T = torch.from_numpy(T0).cuda()
        qf.apply_gate_k(T, q, torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda())
        out = T.cpu().numpy().astype(np.complex128)
        for s in range(S):
            ref = ok.apply_left_k(ok.apply_right_k(T0[s].astype(np.complex128), R[s], q, n), L[s], q, n)
            err = _relerr(out[s], ref)
            worst = max(worst, err)
            assert err <= TOL, (n, q, s, err)
    return worst


@pytest.mark.parametrize("n", [7, 8, 10, 13])
def test_tc_pass_matches_oracle(qf, n):
    S = 3 if n < 13 else 1
    g = qi.rng(15000 + n)
    quads = [(0, 1, 2, 3), (n - 1, n - 2, n - 3, n - 4), (3, 0, n - 1, 1), (n - 4, 2, n - 1, 0),
             (n - 1, 0, n // 2, 2)]
    quads += [tuple(int(x) for x in g.choice(n, 4, replace=False)) for _ in range(3)]
    quads = [q for q in quads if len(set(q)) == 4]
    worst = _check_pass(qf, n, S, quads, 15100 + n)
    print(f"tensor-core 16x16 pass n={n} S={S}: max rel err {worst:.2e}")


def test_tc_pass_benchmark_launch(qf):
    """12 qubits, 4 starts per launch, every consecutive quadruple."""
    n = 12
    quads = [(q, q + 1, q + 2, q + 3) for q in range(n - 3)]
    worst = 0.0
    for i in range(0, len(quads), 3):
        worst = max(worst, _check_pass(qf, n, 4 if i == 0 else 2, quads[i:i + 3], 15200 + i))
    print(f"tensor-core 16x16 pass n=12 (benchmark launch): max rel err {worst:.2e}")


def test_tc_sweep_12q_tracks_oracle(qf):
    """One sweep of the four-qubit benchmark circuit (two start groups; the
    plan's second sweep is a graph replay, checked against the first on the
    oracle's trajectory)."""
    n, S = 12, 2
    locs = []
    for layer in range(6):
        o = 0 if layer % 2 == 0 else 2
        locs += [(q, q + 1, q + 2, q + 3) for q in range(o, n - 3, 4)]
    g = qi.rng(15300)
    tgt = [qi.haar_unitary(16, g) for _ in locs]
    V = ok.circuit_unitary_k(tgt, locs, n)
    starts = [[qi.haar_unitary(16, g) for _ in locs] for _ in range(S)]
    plan = qf.Plan(n, locs, S, qf.QF_C64)
    plan.load(torch.from_numpy(V).cuda(), qf.flatten_gates(starts).cuda())
    got = []
    for _ in range(2):
        plan.sweep(1, reset_iter=0)
        got.append((plan.costs(), qf.unflatten_gates(plan.gates(), locs)))
    assert plan.status() == 0
    plan.close()
    T = ok.init_circuit_tensor_k(V, starts[0], locs, n)
    gref = starts[0]
    for it in range(2):
        T, gref = ok.two_sided_sweep_k(T, gref, locs, n)
        c_ref = ok.trace_cost(T, n)
        costs, gates = got[it]
        dg = max(float(np.max(np.abs(a - b))) for a, b in zip(gates[0], gref))
        print(f"k4 tensor-core sweep {it + 1}: cost {costs[0]:.10e} |dcost| {abs(costs[0] - c_ref):.2e} "
              f"max|dgate| {dg:.2e}")
        assert abs(costs[0] - c_ref) <= 1e-6, (it, costs[0], c_ref)
        assert dg <= 1e-4, (it, dg)


def test_tc_wait_limit_reports_timeout(qf):
    n, S = 8, 2
    q = (0, 3, 5, 7)
    g = qi.rng(15400)
    L = torch.from_numpy(np.stack([qi.haar_unitary(16, g) for _ in range(S)])).cuda()
    R = torch.from_numpy(np.stack([qi.haar_unitary(16, g) for _ in range(S)])).cuda()
    T0 = _rand_T(S, n, g).astype(np.complex64)
    old = qf.set_tc_wait_limit(0)
    try:
        assert qf.set_tc_wait_limit(-1) == 0
        T = torch.from_numpy(T0).cuda()
        qf.apply_gate_k(T, q, L, R)
        assert torch.isnan(T).all().item()  # every tile either ran out or was filled
        locs = [q, (1, 2, 4, 6), (0, 1)]
        V = qi.haar_unitary(2**n, g)
        st = [[qi.haar_unitary(2 ** len(x), g) for x in locs] for _ in range(S)]
        plan = qf.Plan(n, locs, S, qf.QF_C64)
        plan.load(torch.from_numpy(V).cuda(), qf.flatten_gates(st).cuda())
        plan.sweep(1, reset_iter=0)
        assert plan.status() == qf._native.QF_ETIMEOUT
        plan.close()
    finally:
        qf.set_tc_wait_limit(old)
    assert qf.set_tc_wait_limit(-1) == old > 0
    # the context is still usable: the same pass is correct again
    T = torch.from_numpy(T0).cuda()
    qf.apply_gate_k(T, q, L, R)
    out = T.cpu().numpy().astype(np.complex128)
    for s in range(S):
        ref = ok.apply_left_k(ok.apply_right_k(T0[s].astype(np.complex128), R[s].cpu().numpy(), q, n),
                              L[s].cpu().numpy(), q, n)
        assert _relerr(out[s], ref) <= TOL


def test_tc_pass_every_gate_position_8q(qf):
    """Every set of four qubits at 8 qubits (70 sets, each in a shuffled
    local order): the tile's column set, the operator permutation to
    ascending-bit order and the bank layout all depend on where the gate
    bits fall."""
    import itertools

    n, S = 8, 2
    g = qi.rng(15500)
    worst = 0.0
    for subset in itertools.combinations(range(n), 4):
        q = tuple(int(x) for x in g.permutation(np.array(subset)))
        T0 = _rand_T(S, n, g).astype(np.complex64)
        L = np.stack([qi.haar_unitary(16, g) for _ in range(S)])
        R = np.stack([qi.haar_unitary(16, g) for _ in range(S)])
        T = torch.from_numpy(T0).cuda()
        qf.apply_gate_k(T, q, torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda())
        out = T.cpu().numpy().astype(np.complex128)
        for s in range(S):
            ref = ok.apply_left_k(ok.apply_right_k(T0[s].astype(np.complex128), R[s], q, n), L[s], q, n)
            err = _relerr(out[s], ref)
            worst = max(worst, err)
            assert err <= TOL, (q, s, err)
    print(f"tensor-core 16x16 pass, all 70 four-qubit sets at n=8: max rel err {worst:.2e}")
