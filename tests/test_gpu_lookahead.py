"""Look-ahead windows (two consecutive updates on disjoint pairs, one pass)
against the FP64 oracle.

Step level: qf_apply_two_pairs is the composition of two ApplyLeft/
ApplyRight steps of Alg. 1 on four distinct qubits, and qf_partial_trace_after
is CalcEnvMat of the tensor after a pending update, computed without applying
it.  Sweep level: a look-ahead sweep visits the gates in the order of Alg. 1
and every environment is the same quantity as in the one-update sweep, so
costs and gates follow the oracle's TwoSidedSweep to complex64 rounding.

Tolerances (complex64): the pair pass rounds two 4-term complex products
per side, so entries agree to 4e-6 of the largest entry; the look-ahead
partial trace sums 16N weighted FP32 products per start, bounded by
2e-6 x sum |M_ji| |T_entry| (M = R1 L1) entrywise.
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


def _rand_T(S, n, g):
    N = 2**n
    return (g.standard_normal((S, N, N)) + 1j * g.standard_normal((S, N, N))) / np.sqrt(2)


def _relerr(x, ref):
    return float(np.max(np.abs(np.asarray(x) - ref)) / max(np.max(np.abs(ref)), 1e-300))


def _quads(n, g, count):
    """Fixed quadruples (adjacent brickwork neighbours, a layer boundary,
    lowest and highest bit positions, reversed qubit order) plus random ones."""
    fixed = [(0, 1, 2, 3), (n - 2, n - 1, n - 4, n - 3), (1, 2, n - 2, n - 1),
             (n - 1, 0, 3, 2), (4, 2, 7, 5), (n - 1, n - 2, n - 3, n - 4)]
    out = [q for q in fixed if len(set(q)) == 4 and max(q) < n]
    while len(out) < len(fixed) + count:
        out.append(tuple(int(x) for x in g.choice(n, 4, replace=False)))
    return out


@pytest.mark.parametrize("n,dtype", [(8, torch.complex64), (9, torch.complex64),
                                     (10, torch.complex64), (11, torch.complex64),
                                     (6, torch.complex64), (9, torch.complex128)])
def test_apply_two_pairs_matches_oracle(qf, n, dtype):
    g = qi.rng(7100 + n)
    S = 2
    T0 = _rand_T(S, n, g)
    tol = 4e-6 if dtype == torch.complex64 else 1e-12
    worst = 0.0
    for a1, b1, a2, b2 in _quads(n, g, 4):
        ops = [np.stack([qi.haar_unitary(4, g) for _ in range(S)]) for _ in range(4)]
        Tg = torch.from_numpy(T0).to(dtype).cuda()
        qf.apply_two_pairs(Tg, a1, b1, torch.from_numpy(ops[0]).cuda(), torch.from_numpy(ops[1]).cuda(),
                           a2, b2, torch.from_numpy(ops[2]).cuda(), torch.from_numpy(ops[3]).cuda())
        out = Tg.cpu().numpy()
        for s in range(S):
            ref = orc.apply_right(T0[s], ops[1][s], a1, b1, n)
            ref = orc.apply_left(ref, ops[0][s], a1, b1, n)
            ref = orc.apply_right(ref, ops[3][s], a2, b2, n)
            ref = orc.apply_left(ref, ops[2][s], a2, b2, n)
            e = _relerr(out[s], ref)
            worst = max(worst, e)
            assert e <= tol, ((a1, b1, a2, b2), s, e)
    print(f"apply_two_pairs n={n} {dtype}: max rel err {worst:.2e}")


def test_apply_two_pairs_rejects_shared_qubit(qf):
    from paper_2306_08152_gb300 import QFactorError

    T = torch.zeros((1, 512, 512), dtype=torch.complex64, device="cuda")
    I = torch.eye(4, dtype=torch.complex128, device="cuda").reshape(1, 4, 4)
    with pytest.raises(QFactorError):
        qf.apply_two_pairs(T, 0, 1, I, I, 1, 2, I, I)


def _bound_after(T, a1, b1, M, a, b, n):
    """sum_rest sum_{i,j} |M[j][i]| |T[(rest,i,x),(rest,j,y)]| by explicit
    index loops (the magnitude analogue of the look-ahead partial trace)."""
    pos = lambda q: n - 1 - q
    others = [q for q in range(n) if q not in (a1, b1, a, b)]
    A = np.abs(T)
    out = np.zeros((4, 4))
    for r in range(2 ** len(others)):
        base = 0
        for t, q in enumerate(others):
            base |= ((r >> t) & 1) << pos(q)
        for i in range(4):
            oi = ((i >> 1) << pos(a1)) | ((i & 1) << pos(b1))
            for j in range(4):
                oj = ((j >> 1) << pos(a1)) | ((j & 1) << pos(b1))
                for x in range(4):
                    ox = ((x >> 1) << pos(a)) | ((x & 1) << pos(b))
                    for y in range(4):
                        oy = ((y >> 1) << pos(a)) | ((y & 1) << pos(b))
                        out[x, y] += abs(M[j, i]) * A[base | oi | ox, base | oj | oy]
    return out


@pytest.mark.parametrize("n,dtype", [(4, torch.complex128), (7, torch.complex128),
                                     (7, torch.complex64), (10, torch.complex64)])
def test_partial_trace_after_matches_oracle(qf, n, dtype):
    g = qi.rng(7200 + n)
    S = 2
    T0 = _rand_T(S, n, g)
    Tg = torch.from_numpy(T0).to(dtype).cuda()
    Tc = Tg.cpu().numpy().astype(np.complex128)
    worst = 0.0
    quads = _quads(n, g, 3) if n > 4 else [(0, 1, 2, 3), (3, 1, 0, 2), (2, 0, 3, 1)]
    for a1, b1, a, b in quads:
        L1 = np.stack([qi.haar_unitary(4, g) for _ in range(S)])
        R1 = np.stack([qi.haar_unitary(4, g) for _ in range(S)])
        P = qf.partial_trace_after(Tg, a1, b1, torch.from_numpy(L1).cuda(), torch.from_numpy(R1).cuda(),
                                   a, b).cpu().numpy()
        for s in range(S):
            Tp = orc.apply_left(orc.apply_right(Tc[s], R1[s], a1, b1, n), L1[s], a1, b1, n)
            ref = orc.calc_env_mat(Tp, a, b, n)
            if dtype == torch.complex128:
                assert _relerr(P[s], ref) <= 1e-12, ((a1, b1, a, b), s)
            else:
                bound = 2e-6 * _bound_after(Tc[s], a1, b1, R1[s] @ L1[s], a, b, n)
                err = np.abs(P[s] - ref)
                worst = max(worst, float(np.max(err / bound)))
                assert np.all(err <= bound), ((a1, b1, a, b), s, float(np.max(err / bound)))
    if dtype == torch.complex64:
        print(f"partial_trace_after c64 n={n}: worst error / bound = {worst:.3f}")


def _oracle_sweeps(V, gates, locs, n, k):
    T = orc.init_circuit_tensor(V, gates, locs, n)
    g = gates
    for _ in range(k):
        T, g = orc.two_sided_sweep(T, g, locs, n)
    return orc.trace_cost(T, n), g


@pytest.mark.parametrize("structure,S,n", [("brickwork", 4, 9), ("brickwork", 1, 9), ("random", 2, 9),
                                           ("brickwork", 3, 8)])
def test_lookahead_sweeps_match_oracle(qf, structure, S, n):
    g = qi.rng(7300)
    locs = qi.brickwork_locations(n, 4) if structure == "brickwork" else \
        qi.random_adjacent_locations(n, 16, g)
    assert len(locs) % 2 == 0
    inst = qi.make_problem(n, locs, S, seed=7301)
    # an unreachable Haar target: every update moves the gates
    V = qi.haar_unitary(2**n, g)
    Vt = torch.from_numpy(V).cuda()
    starts = torch.from_numpy(inst.starts).cuda()
    plan = qf.Plan(n, locs, S, qf.QF_C64)
    windows = plan.set_lookahead(True)
    if structure == "brickwork":
        assert windows == len(locs)  # every consecutive pair is disjoint: p/2 per half
    else:
        assert 0 < windows <= len(locs)
    ref_plan = qf.Plan(n, locs, S, qf.QF_C64)
    plan.load(Vt, starts)
    ref_plan.load(Vt, starts)
    plan.sweep(2, reset_iter=0)
    ref_plan.sweep(2, reset_iter=0)
    c_look, g_look = plan.costs(), plan.gates().numpy()
    c_one, g_one = ref_plan.costs(), ref_plan.gates().numpy()
    plan.close()
    ref_plan.close()
    for s in range(S):
        c_ref, g_ref = _oracle_sweeps(V, inst.starts[s], locs, n, 2)
        assert abs(c_look[s] - c_ref) <= 1e-5, (s, c_look[s], c_ref)
        assert abs(c_look[s] - c_one[s]) <= 1e-5
        assert np.max(np.abs(g_look[s] - g_ref)) <= 1e-3, s
    print(f"look-ahead {structure} S={S}: {windows} pair windows/sweep, costs {c_look}")


def test_lookahead_timed_and_graph_paths_agree(qf):
    """Live launches (pass timing on) and the replayed graph run the same
    windows; the pass count halves for brickwork."""
    n = 10
    locs = qi.brickwork_locations(n, 4)
    inst = qi.make_problem(n, locs, 4, seed=7400)
    V = torch.from_numpy(orc.circuit_unitary(inst.target_gates, locs, n)).cuda()
    starts = torch.from_numpy(inst.starts).cuda()
    res = []
    for timing in (True, False):
        plan = qf.Plan(n, locs, 4, qf.QF_C64)
        plan.set_lookahead(True)
        plan.enable_pass_timing(timing)
        plan.load(V, starts)
        plan.pass_stats()
        plan.sweep(3, reset_iter=0)
        ms, passes, launches, _ = plan.pass_stats()
        res.append((plan.costs(), plan.gates().numpy(), passes))
        plan.close()
    (c0, g0, p0), (c1, g1, p1) = res
    p = len(locs)
    assert p0 == p1 == 3 * 2 * (p // 2) * 2  # sweeps x halves x windows x start groups
    np.testing.assert_allclose(c0, c1, atol=1e-12)
    assert np.max(np.abs(g0 - g1)) <= 1e-12


def test_lookahead_is_ignored_for_complex128(qf):
    n = 9
    locs = qi.brickwork_locations(n, 2)
    plan = qf.Plan(n, locs, 1, qf.QF_C128)
    assert plan.set_lookahead(True) == 0
    plan.close()
