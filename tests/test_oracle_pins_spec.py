"""Pins of the specialised-gate oracle (oracle/specialised.py, Sec. III-A
"Specializing gate sets") against constructions other than itself: gate
identities (GPI as a conjugated X, MS as a matrix exponential through
scipy), brute-force maximisation of Re Tr(E G(theta)) over the parameters,
single-gate fits, and the monotone increase of Re Tr over a sweep."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.optimize as so

import oracle.kqubit as ok
import oracle.specialised as osp
import qf_inputs as qi

X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Z = np.diag([1.0, -1.0]).astype(np.complex128)


def test_gate_identities():
    g = qi.rng(12000)
    np.testing.assert_allclose(osp.rz(np.pi), Z, atol=1e-15)
    np.testing.assert_allclose(osp.gpi(0.0), X, atol=1e-15)
    for _ in range(5):
        phi, phi0, phi1, th = g.uniform(-np.pi, np.pi, 4)
        np.testing.assert_allclose(osp.gpi(phi), osp.rz(phi) @ X @ osp.rz(-phi), atol=1e-15)
        S = np.kron(osp.gpi(phi0), osp.gpi(phi1))
        np.testing.assert_allclose(osp.ms(phi0, phi1), sla.expm(-0.25j * np.pi * S), atol=1e-14)
        for m in (osp.rz(th), osp.gpi(phi), osp.ms(phi0, phi1)):
            np.testing.assert_allclose(m.conj().T @ m, np.eye(len(m)), atol=1e-15)
    # MS(0, 0) = (I - i X (x) X) / sqrt 2
    np.testing.assert_allclose(osp.ms(0.0, 0.0), (np.eye(4) - 1j * np.kron(X, X)) / np.sqrt(2), atol=1e-15)


def _brute_max(kind, A):
    """Maximum of Re Tr(A G) over the parameters: a grid, then a local
    polish of the best grid points with scipy."""
    f = lambda p: -osp.objective(kind, A, p)
    if osp.NPARAM[kind] == 1:
        grid = np.linspace(-np.pi, np.pi, 2049)
        vals = [f([t]) for t in grid]
        t0 = grid[int(np.argmin(vals))]
        r = so.minimize_scalar(lambda t: f([t]), bounds=(t0 - 0.01, t0 + 0.01), method="bounded",
                               options={"xatol": 1e-12})
        return -r.fun
    grid = np.linspace(-np.pi, np.pi, 129)
    best = min(((f([a, b]), a, b) for a in grid for b in grid))
    r = so.minimize(lambda p: f(p), [best[1], best[2]], method="Nelder-Mead",
                    options={"xatol": 1e-12, "fatol": 1e-14, "maxiter": 4000})
    return -r.fun


@pytest.mark.parametrize("kind", [osp.RZ, osp.GPI, osp.MS])
def test_argmax_matches_brute_force(kind):
    g = qi.rng(12100 + len(kind))
    d = 2 ** osp.NQUBITS[kind]
    for _ in range(6):
        A = g.standard_normal((d, d)) + 1j * g.standard_normal((d, d))
        old = list(g.uniform(-np.pi, np.pi, osp.NPARAM[kind]))
        new, best = osp.optimize_param(kind, A, old)
        assert abs(osp.objective(kind, A, new) - best) <= 1e-12 * max(1.0, abs(best))
        bf = _brute_max(kind, A)
        assert best >= bf - 1e-9, (best, bf)
        assert abs(best - bf) <= 1e-8 * max(1.0, abs(bf)), (best, bf)


def test_degenerate_modulus_keeps_the_old_angle():
    A = np.zeros((2, 2), dtype=np.complex128)
    A[0, 0] = 1.0
    new, best = osp.optimize_param(osp.RZ, A, [0.7])
    assert new == [0.7] and best == 1.0
    new, _ = osp.optimize_param(osp.GPI, A, [0.3])
    assert new == [0.3]


@pytest.mark.parametrize("kind,n,q", [(osp.RZ, 1, (0,)), (osp.GPI, 2, (1,)), (osp.MS, 2, (0, 1)),
                                      (osp.MS, 3, (2, 0))])
def test_single_gate_fit_recovers_the_target(kind, n, q):
    """n qubits, one gate: the target is the gate itself (times the identity
    elsewhere), so after removing the gate the environment is the target's
    own block and one update returns the target's gate."""
    g = qi.rng(12200 + n)
    p0 = list(g.uniform(-np.pi, np.pi, osp.NPARAM[kind]))
    V = osp.circuit_unitary_spec([kind], [q], [p0], n)
    start = list(g.uniform(-np.pi, np.pi, osp.NPARAM[kind]))
    T = osp.init_circuit_tensor_spec(V, [kind], [q], [start], n)
    T, st = osp.two_sided_sweep_spec(T, [kind], [q], [start], n)
    np.testing.assert_allclose(osp.gate_matrix(kind, st[0]), osp.gate_matrix(kind, p0), atol=1e-13)
    assert ok.trace_cost(T, n) <= 1e-14


def _circuit(n, g):
    kinds = [osp.GPI, osp.RZ, osp.MS, osp.U, osp.GPI, osp.MS, osp.RZ]
    locs, states = [], []
    for k in kinds:
        if k == osp.U:
            q = tuple(int(x) for x in g.choice(n, 2, replace=False))
            states.append(qi.haar_unitary(4, g))
        else:
            q = tuple(int(x) for x in g.choice(n, osp.NQUBITS[k], replace=False))
            states.append(list(g.uniform(-np.pi, np.pi, osp.NPARAM[k])))
        locs.append(q)
    return kinds, locs, states


@pytest.mark.parametrize("n", [3, 4])
def test_sweep_increases_re_trace_and_matches_dense(n):
    g = qi.rng(12300 + n)
    kinds, locs, states = _circuit(n, g)
    V = qi.haar_unitary(2**n, g)
    T = osp.init_circuit_tensor_spec(V, kinds, locs, states, n)
    C = osp.circuit_unitary_spec(kinds, locs, states, n)
    np.testing.assert_allclose(T, V.conj().T @ C, atol=1e-13)
    retr = [float(np.trace(T).real)]
    for _ in range(3):
        T, states = osp.two_sided_sweep_spec(T, kinds, locs, states, n, retr=retr)
    assert all(b >= a - 1e-12 for a, b in zip(retr, retr[1:]))
    # the incrementally updated tensor is V^dagger C of the final gates
    C = osp.circuit_unitary_spec(kinds, locs, states, n)
    np.testing.assert_allclose(T, V.conj().T @ C, atol=1e-12)


def test_beta_damping_maximises_the_damped_objective():
    g = qi.rng(12400)
    E = g.standard_normal((4, 4)) + 1j * g.standard_normal((4, 4))
    old = [0.4, -1.1]
    beta = 0.3
    A = (1 - beta) * E + beta * osp.ms(*old).conj().T
    new, best = osp.optimize_param(osp.MS, A, old)
    assert abs(best - _brute_max(osp.MS, A)) <= 1e-8
