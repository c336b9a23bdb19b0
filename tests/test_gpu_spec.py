"""Specialised gate sets (Sec. III-A, "Specializing gate sets") on the GPU
against the FP64 oracle (oracle/specialised.py): sweeps of circuits that mix
Rz, GPI and Moelmer-Soerensen gates with general 2- and 3-qubit unitaries,
their parameters, resets, and the single-gate closed form.  Tolerances as
for general gates: complex128 and double-FP32 sweeps to cost 1e-10 and gate
matrices 1e-9, complex64 to cost 1e-5."""
import numpy as np
import pytest
import torch

import oracle.kqubit as ok
import oracle.specialised as osp
import qf_inputs as qi

pytestmark = pytest.mark.gpu

KIND = {"u4": osp.U, "u8": osp.U, "rz": osp.RZ, "gpi": osp.GPI, "ms": osp.MS}


@pytest.fixture(scope="module")
def qf():
    import paper_2306_08152_gb300 as qf

    qf._native.load()
    return qf


def _circuit(n, g, with_u8):
    kinds = ["gpi", "rz", "ms", "u4", "gpi", "ms", "rz", "gpi"] + (["u8"] if with_u8 else [])
    specs = []
    for k in kinds:
        if k in ("rz", "gpi"):
            q = int(g.integers(n))
            specs.append((k, q) if g.random() < 0.5 else (k, q, int((q + 2) % n) if n > 2 else 1 - q))
        elif k == "u8":
            specs.append((k, *[int(x) for x in g.choice(n, 3, replace=False)]))
        else:
            specs.append((k, *[int(x) for x in g.choice(n, 2, replace=False)]))
    return specs


def _start(specs, g):
    states = []
    for sp in specs:
        k = sp[0]
        if k == "u4":
            states.append(qi.haar_unitary(4, g))
        elif k == "u8":
            states.append(qi.haar_unitary(8, g))
        else:
            states.append(list(g.uniform(-np.pi, np.pi, osp.NPARAM[KIND[k]])))
    return states


def _gpu_inputs(qf, specs, starts, n):
    slots = qf.spec_slots(specs, n)
    S, p = len(starts), len(specs)
    params = np.zeros((S, p, 2))
    mats = []
    for s, st in enumerate(starts):
        row = []
        for i, (sp, x) in enumerate(zip(specs, st)):
            if sp[0] in ("u4", "u8"):
                row.append(np.asarray(x))
            else:
                params[s, i, :len(x)] = x
                row.append(np.zeros((4, 4)))
        mats.append(row)
    return slots, torch.from_numpy(params), qf.flatten_gates(mats)


def _oracle_locs(specs):
    return [(int(sp[1]),) if sp[0] in ("rz", "gpi") else tuple(int(x) for x in sp[1:]) for sp in specs]


# 11 qubits: the environment kernel splits each start's band over 2 CTAs and
# the closed-form updates run in the last CTA's epilogue
@pytest.mark.parametrize("n,S,prec,with_u8", [(3, 2, "c128", False), (4, 3, "c128", True),
                                              (9, 2, "c128", False), (7, 2, "c64", True),
                                              (5, 2, "df64", True), (11, 2, "c128", True)])
def test_spec_sweeps_match_oracle(qf, n, S, prec, with_u8):
    g = qi.rng(13000 + n)
    specs = _circuit(n, g, with_u8)
    kinds = [KIND[sp[0]] for sp in specs]
    olocs = _oracle_locs(specs)
    V = qi.haar_unitary(2**n, g)
    starts = [_start(specs, g) for _ in range(S)]
    slots, params, mats = _gpu_inputs(qf, specs, starts, n)
    plan = qf.Plan(n, specs, S, {"c128": qf.QF_C128, "c64": qf.QF_C64, "df64": qf.QF_DF64}[prec])
    plan.load_params(torch.from_numpy(V).cuda(), params.cuda(), mats.cuda())
    plan.sweep(3, reset_iter=2)
    costs = plan.costs()
    got_p = plan.params().numpy()
    got_g = qf.unflatten_gates(plan.gates(), slots)
    plan.close()
    for s in range(S):
        T = osp.init_circuit_tensor_spec(V, kinds, olocs, starts[s], n)
        st = starts[s]
        for it in range(1, 4):
            T, st = osp.two_sided_sweep_spec(T, kinds, olocs, st, n)
            if it % 2 == 0:
                T = osp.init_circuit_tensor_spec(V, kinds, olocs, st, n)
        c_ref = ok.trace_cost(T, n)
        if prec in ("c128", "df64"):  # df64 meets the complex128 bars
            assert abs(costs[s] - c_ref) <= 1e-10, (s, costs[s], c_ref)
            for i, (sp, ref) in enumerate(zip(specs, st)):
                if sp[0] in ("u4", "u8"):
                    assert np.max(np.abs(got_g[s][i] - ref)) <= 1e-9
                else:
                    m_gpu = osp.gate_matrix(KIND[sp[0]], got_p[s, i])
                    assert np.max(np.abs(m_gpu - osp.gate_matrix(KIND[sp[0]], ref))) <= 1e-9, (sp, s)
                    # the slot matrix is G (x) I (one-qubit kinds) or G itself
                    slot = np.kron(m_gpu, np.eye(2)) if sp[0] in ("rz", "gpi") else m_gpu
                    assert np.max(np.abs(got_g[s][i] - slot)) <= 1e-12
        else:
            assert abs(costs[s] - c_ref) <= 1e-5, (s, costs[s], c_ref)


@pytest.mark.parametrize("kind", ["rz", "gpi", "ms"])
def test_single_gate_recovers_target(qf, kind):
    n = 3
    g = qi.rng(13100 + len(kind))
    spec = (kind, 1) if kind != "ms" else (kind, 2, 0)
    ol = _oracle_locs([spec])
    p0 = list(g.uniform(-np.pi, np.pi, osp.NPARAM[KIND[kind]]))
    V = osp.circuit_unitary_spec([KIND[kind]], ol, [p0], n)
    start = np.zeros((2, 1, 2))
    start[:, 0, :len(p0)] = g.uniform(-np.pi, np.pi, (2, len(p0)))
    plan = qf.Plan(n, [spec], 2, qf.QF_C128)
    plan.load_params(torch.from_numpy(V).cuda(), torch.from_numpy(start).cuda())
    plan.sweep(1, reset_iter=0)
    costs = plan.costs()
    got = plan.params().numpy()
    plan.close()
    assert np.all(costs <= 1e-14), costs
    for s in range(2):
        np.testing.assert_allclose(osp.gate_matrix(KIND[kind], got[s, 0]),
                                   osp.gate_matrix(KIND[kind], p0), atol=1e-13)


def test_lookahead_flag_is_ignored_and_invalid_specs_rejected(qf):
    from paper_2306_08152_gb300 import QFactorError

    n = 8
    g = qi.rng(13200)
    specs = [("gpi", q) for q in range(n)] + [("ms", q, q + 1) for q in range(0, n - 1, 2)]
    V = qi.haar_unitary(2**n, g)
    params = torch.from_numpy(g.uniform(-np.pi, np.pi, (2, len(specs), 2)))
    out = []
    for look in (False, True):
        plan = qf.Plan(n, specs, 2, qf.QF_C64)
        plan.set_lookahead(look)
        plan.load_params(torch.from_numpy(V).cuda(), params.cuda())
        plan.sweep(2)
        out.append((plan.costs(), plan.params().numpy()))
        plan.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    for bad in ([("rz", 1, 1)], [("ms", 0, 0)], [("xx", 0)], [("gpi", 5)], [("u8", 0, 1, 2)]):
        with pytest.raises((QFactorError, ValueError)):
            qf.Plan(2, bad, 1, qf.QF_C128)
    plan = qf.Plan(3, [("rz", 0), ("u4", 1, 2)], 1, qf.QF_C128)
    with pytest.raises(QFactorError):  # general gates need their matrices
        plan.load_params(torch.eye(8, dtype=torch.complex128).cuda(),
                         torch.zeros((1, 2, 2), dtype=torch.float64).cuda())
    plan.close()


@pytest.mark.parametrize("precision", ["c128", "c64refine"])
def test_instantiate_spec_reaches_tolerance(qf, precision):
    """A reachable circuit of GPI, MS, Rz and one general gate, from starts
    near the target's angles (the angle landscape has local optima): the
    run converges to 1e-10, and the oracle's cost of the returned angles and
    gate agrees."""
    n = 3
    specs = [("gpi", 0), ("gpi", 1), ("ms", 0, 1), ("rz", 2), ("ms", 1, 2), ("u4", 0, 2), ("gpi", 2, 0)]
    kinds = [KIND[sp[0]] for sp in specs]
    olocs = _oracle_locs(specs)
    g = qi.rng(13300)
    tgt = _start(specs, g)
    V = osp.circuit_unitary_spec(kinds, olocs, tgt, n)
    S = 4
    params = np.zeros((S, len(specs), 2))
    mats = []
    for s in range(S):
        row = []
        for i, (sp, x) in enumerate(zip(specs, tgt)):
            if sp[0] == "u4":
                row.append(qi.haar_unitary(4, qi.rng(13310 + s)))
            else:
                params[s, i, :len(x)] = np.asarray(x) + 0.3 * qi.rng(13320 + s).standard_normal(len(x))
                row.append(np.zeros((4, 4)))
        mats.append(row)
    prec = qf.QF_C128 if precision == "c128" else qf.QF_C64_REFINE64
    res = qf.instantiate_spec(torch.from_numpy(V).cuda(), specs, torch.from_numpy(params).cuda(),
                              qf.flatten_gates(mats).cuda(), dist_tol=1e-10, max_sweeps=400, precision=prec)
    assert res["best_cost"] <= 1e-10, res["costs"]
    b = res["best"]
    slots = qf.spec_slots(specs, n)
    gates = qf.unflatten_gates(res["flat"], slots)[b]
    pb = res["params"][b].cpu().numpy()
    st = [gates[i] if sp[0] == "u4" else list(pb[i, :osp.NPARAM[KIND[sp[0]]]]) for i, sp in enumerate(specs)]
    C = osp.circuit_unitary_spec(kinds, olocs, st, n)
    c_ref = 1.0 - abs(np.trace(V.conj().T @ C)) / 2**n
    assert c_ref <= 2e-10 and abs(c_ref - res["best_cost"]) <= 1e-10
