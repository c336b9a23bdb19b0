"""The double-FP32 (df64) tensor precision against the FP64 oracle.

A df64 entry holds each real part as hi + lo (two floats, about 48
significant bits), and the pass works in FP32 error-free arithmetic
(TwoProd by FMA, TwoSum).  Each step therefore matches the oracle to a few
units of 2^-48 of the entries it sums, far inside the complex128 tolerances
used for the sweeps (cost 1e-10, gates 1e-9): the step tolerances below are
1e-12 relative to the largest entry, as for complex128.
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


def _to_df(qf, T128):
    return qf.convert_tensor(torch.from_numpy(T128).cuda(), qf.QF_DF64)


def _from_df(qf, Tdf):
    return qf.convert_tensor(Tdf, qf.QF_C128).cpu().numpy()


def test_conversion_round_trip(qf):
    g = qi.rng(8100)
    T = _rand_T(3, 6, g) * np.exp(g.uniform(-20, 20, (3, 64, 64)))  # wide exponents
    Tdf = _to_df(qf, T)
    assert Tdf.dtype == torch.float32 and tuple(Tdf.shape) == (3, 64, 64, 4)
    back = _from_df(qf, Tdf)
    # hi = float(x), lo = float(x - hi): the pair keeps x to 2^-48 relative
    assert np.all(np.abs(back.real - T.real) <= 2.0**-47 * np.abs(T.real))
    assert np.all(np.abs(back.imag - T.imag) <= 2.0**-47 * np.abs(T.imag))
    hi = Tdf[..., 0].cpu().numpy()
    np.testing.assert_array_equal(hi, T.real.astype(np.float32))
    # df64 -> df64 and complex64 -> df64 are exact
    again = qf.convert_tensor(Tdf, qf.QF_DF64)
    assert torch.equal(again, Tdf)
    T64 = torch.from_numpy(T).to(torch.complex64).cuda()
    np.testing.assert_array_equal(_from_df(qf, qf.convert_tensor(T64, qf.QF_DF64)),
                                  T64.cpu().numpy().astype(np.complex128))


def test_conversion_rejects_overlap(qf):
    from paper_2306_08152_gb300 import QFactorError

    buf = torch.zeros(64, dtype=torch.complex128, device="cuda")
    with pytest.raises(QFactorError):
        qf._native.check(qf._native.load().qf_convert_tensor(
            buf.data_ptr(), qf.QF_C128, buf.data_ptr() + 16, qf.QF_DF64, 32, None))


@pytest.mark.parametrize("n", [2, 3, 5, 7])
def test_apply_pair_df64_matches_oracle(qf, n):
    g = qi.rng(8200 + n)
    S = 2
    T0 = _rand_T(S, n, g)
    worst = 0.0
    pairs = [(a, b) for a in range(n) for b in range(n) if a != b]
    for a, b in pairs:
        L = np.stack([qi.haar_unitary(4, g) for _ in range(S)])
        R = np.stack([qi.haar_unitary(4, g) for _ in range(S)])
        for mode in ("L", "R", "LR"):
            Tg = _to_df(qf, T0)
            qf.apply_pair(Tg, a, b, torch.from_numpy(L).cuda() if "L" in mode else None,
                          torch.from_numpy(R).cuda() if "R" in mode else None)
            out = _from_df(qf, Tg)
            for s in range(S):
                ref = T0[s]
                if "R" in mode:
                    ref = orc.apply_right(ref, R[s], a, b, n)
                if "L" in mode:
                    ref = orc.apply_left(ref, L[s], a, b, n)
                e = _relerr(out[s], ref)
                worst = max(worst, e)
                assert e <= 1e-12, (a, b, mode, s, e)
    print(f"apply_pair df64 n={n}: max rel err {worst:.2e}")


@pytest.mark.parametrize("n", [3, 6, 10])
def test_partial_trace_and_trace_df64(qf, n):
    g = qi.rng(8300 + n)
    S = 2
    T0 = _rand_T(S, n, g)
    Tg = _to_df(qf, T0)
    tr = qf.trace(Tg).cpu().numpy()
    for s in range(S):
        assert abs(tr[s] - np.trace(T0[s])) <= 1e-12 * np.sum(np.abs(np.diag(T0[s])))
    for a, b in [(0, 1), (n - 1, 0), (1, n - 1)]:
        P = qf.partial_trace(Tg, a, b).cpu().numpy()
        for s in range(S):
            assert _relerr(P[s], orc.calc_env_mat(T0[s], a, b, n)) <= 1e-12, (a, b, s)


def test_init_tensor_df64(qf):
    n = 6
    locs = qi.brickwork_locations(n, 4)
    inst = qi.make_problem(n, locs, 2, seed=8400)
    V = qi.haar_unitary(2**n, qi.rng(8401))
    Tg = qf.init_tensor(torch.from_numpy(V).cuda(), locs, torch.from_numpy(inst.starts).cuda(),
                        dtype="df64")
    out = _from_df(qf, Tg)
    for s in range(2):
        ref = orc.init_circuit_tensor(V, inst.starts[s], locs, n)
        assert _relerr(out[s], ref) <= 1e-12


@pytest.mark.parametrize("n,layers,S", [(4, 4, 2), (7, 6, 3), (10, 4, 2)])
def test_df64_sweeps_match_oracle(qf, n, layers, S):
    locs = qi.brickwork_locations(n, layers)
    inst = qi.make_problem(n, locs, S, seed=8500 + n)
    V = qi.haar_unitary(2**n, qi.rng(8600 + n))
    plan = qf.Plan(n, locs, S, qf.QF_DF64)
    plan.load(torch.from_numpy(V).cuda(), torch.from_numpy(inst.starts).cuda())
    plan.sweep(3, reset_iter=2)
    costs, gates = plan.costs(), plan.gates().numpy()
    plan.close()
    for s in range(S):
        T = orc.init_circuit_tensor(V, inst.starts[s], locs, n)
        gref = inst.starts[s]
        for it in range(1, 4):
            T, gref = orc.two_sided_sweep(T, gref, locs, n)
            if it % 2 == 0:
                T = orc.init_circuit_tensor(V, gref, locs, n)
        c_ref = orc.trace_cost(T, n)
        assert abs(costs[s] - c_ref) <= 1e-10, (s, costs[s], c_ref)
        assert np.max(np.abs(gates[s] - gref)) <= 1e-9, s


@pytest.mark.parametrize("precision", ["df64", "c64_refine_df"])
def test_df64_instantiation_reaches_tolerance(qf, precision):
    n = 4
    locs = qi.brickwork_locations(n, 4)
    inst = qi.make_problem(n, locs, 4, seed=8)
    V = orc.circuit_unitary(inst.target_gates, locs, n)
    prec = qf.QF_DF64 if precision == "df64" else qf.QF_C64_REFINE_DF
    res = qf.instantiate_ex(torch.from_numpy(V).cuda(), locs, torch.from_numpy(inst.starts).cuda(),
                            dist_tol=1e-10, max_sweeps=300, precision=prec)
    assert res["best_cost"] <= 1e-10, res
    b = res["best"]
    c_ref, _, _ = orc.cost_and_env(V, res["gates"][b].cpu().numpy(), locs, n)
    assert c_ref <= 2e-10 and abs(c_ref - res["best_cost"]) <= 1e-10


def test_batched_rejects_df64(qf):
    from paper_2306_08152_gb300 import QFactorError

    V = np.eye(8, dtype=np.complex128)
    G = np.tile(np.eye(4, dtype=np.complex128), (1, 1, 1, 1))
    with pytest.raises(QFactorError):
        qf.instantiate_batched([(V, np.array([[0, 1]]), G)], precision=qf.QF_DF64)
