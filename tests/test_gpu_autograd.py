"""The differentiable cost (qf_cost_grad, QFactorCost) against the oracle,
torch.autograd.gradcheck and central finite differences.

The gradient of cost = 1 - |t|/N, t = Tr(V^dagger C), with respect to gate k
is -(t/(N|t|)) E_k^dagger in PyTorch's d/dRe + i d/dIm convention, where
dt/d(u_k)_ij = (E_k)_ji (Sec. III: t = Tr(E_k u_k)).
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


def test_gradcheck_small_circuit(qf):
    n = 3
    locs = np.array([[0, 1], [1, 2], [2, 0], [1, 0]], dtype=np.int32)
    g = qi.rng(900)
    gates = torch.from_numpy(np.stack([qi.haar_gates(4, g) for _ in range(2)])).cuda().requires_grad_(True)
    V = torch.from_numpy(qi.haar_unitary(8, g)).cuda()
    f = lambda x: qf.QFactorCost.apply(x, V, locs)
    assert torch.autograd.gradcheck(f, (gates,), eps=1e-6, atol=1e-8, rtol=1e-6)


@pytest.mark.parametrize("n,layers,sets", [(4, 4, 3), (8, 16, 32)])
def test_gradient_matches_oracle_and_finite_differences(qf, n, layers, sets):
    """Differentiable cost, 8 qubits: 56 U(4) gates in linear brickwork,
    batch of 32 seeded gate sets (and a small 4-qubit case)."""
    locs = qi.brickwork_locations(n, layers)
    p = len(locs)
    g = qi.rng(910 + n)
    gates = np.stack([qi.haar_gates(p, g) for _ in range(sets)])
    V = qi.haar_unitary(2**n, g)
    Vt = torch.from_numpy(V).cuda()
    x = torch.from_numpy(gates).cuda().requires_grad_(True)
    c = qf.QFactorCost.apply(x, Vt, locs)
    c.sum().backward()
    grad = x.grad.cpu().numpy()
    for s in (0, sets - 1):
        c_ref, e_ref, t_ref = orc.cost_and_env(V, gates[s], locs, n)
        assert abs(c[s].item() - c_ref) <= 1e-10
        want = -(t_ref / (2**n * abs(t_ref))) * np.conj(np.transpose(e_ref, (0, 2, 1)))
        scale = np.max(np.abs(want))
        assert np.max(np.abs(grad[s] - want)) <= 1e-9 * scale
    # central finite differences of the GPU cost (step 1e-6) on sampled entries
    rs = np.random.default_rng(0)
    h = 1e-6
    for _ in range(6):
        s, k, i, j = rs.integers(sets), rs.integers(p), rs.integers(4), rs.integers(4)
        for direction, part in ((1.0, "re"), (1j, "im")):
            gp = gates[s:s + 1].copy()
            gm = gates[s:s + 1].copy()
            gp[0, k, i, j] += h * direction
            gm[0, k, i, j] -= h * direction
            cp = qf.costs(Vt, locs, torch.from_numpy(gp).cuda())[0]
            cm = qf.costs(Vt, locs, torch.from_numpy(gm).cuda())[0]
            fd = (cp - cm) / (2 * h)
            an = grad[s, k, i, j].real if part == "re" else grad[s, k, i, j].imag
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-9, (s, k, i, j, part, fd, an)


def test_cost_without_grad_is_the_plain_cost(qf):
    n = 5
    locs = qi.brickwork_locations(n, 6)
    g = qi.rng(920)
    gates = np.stack([qi.haar_gates(len(locs), g) for _ in range(2)])
    V = qi.haar_unitary(2**n, g)
    c = qf.QFactorCost.apply(torch.from_numpy(gates).cuda(), torch.from_numpy(V).cuda(), locs)
    for s in range(2):
        c_ref, _, _ = orc.cost_and_env(V, gates[s], locs, n)
        assert abs(c[s].item() - c_ref) <= 1e-10


def _mixed_locs(n, g):
    locs = [(0, 1, 2, 3), (n - 1, 1), (2, n - 1, 0), (1, 3), (n - 4, n - 3, n - 2, n - 1), (0, 2, 4)]
    return [tuple(int(x) for x in q) for q in locs if max(q) < n and len(set(q)) == len(q)]


@pytest.mark.parametrize("n,sets", [(5, 3), (7, 2)])
def test_k_qubit_gradient_matches_oracle(qf, n, sets):
    """Circuits of 2-, 3- and 4-qubit gates (qf_cost_grad_k, QFactorCost on
    the concatenated gate layout): costs, environments and gradients against
    the k-qubit oracle's environments (pinned by finite differences)."""
    import oracle.kqubit as ok

    g = qi.rng(930 + n)
    locs = _mixed_locs(n, g)
    V = qi.haar_unitary(2**n, g)
    sets_l = [[qi.haar_unitary(2 ** len(q), g) for q in locs] for _ in range(sets)]
    flat = qf.flatten_gates(sets_l)
    Vt = torch.from_numpy(V).cuda()
    costs, envs, trs = qf.cost_and_env_k(Vt, locs, flat.cuda())
    envs = qf.unflatten_gates(envs, locs)
    x = flat.cuda().requires_grad_(True)
    c = qf.QFactorCost.apply(x, Vt, locs)
    c.sum().backward()
    grads = qf.unflatten_gates(x.grad, locs)
    for s in range(sets):
        c_ref, e_ref, t_ref = ok.cost_and_env_k(V, sets_l[s], locs, n)
        assert abs(costs[s] - c_ref) <= 1e-10 and abs(c[s].item() - c_ref) <= 1e-10
        assert abs(trs[s] - t_ref) <= 1e-10 * 2**n
        f = -(t_ref / (2**n * abs(t_ref)))
        for k in range(len(locs)):
            scale = np.max(np.abs(e_ref[k]))
            assert np.max(np.abs(envs[s][k] - e_ref[k])) <= 1e-9 * scale, (s, k)
            want = f * e_ref[k].conj().T
            assert np.max(np.abs(grads[s][k] - want)) <= 1e-9 * np.max(np.abs(want)), (s, k)


def test_k_qubit_gradcheck(qf):
    n = 4
    locs = [(0, 1, 2, 3), (1, 2), (3, 0, 2)]
    g = qi.rng(940)
    V = torch.from_numpy(qi.haar_unitary(16, g)).cuda()
    flat = qf.flatten_gates([[qi.haar_unitary(2 ** len(q), g) for q in locs]]).cuda()[0]
    x = flat.clone().requires_grad_(True)
    f = lambda y: qf.QFactorCost.apply(y, V, locs)
    assert torch.autograd.gradcheck(f, (x,), eps=1e-6, atol=1e-8, rtol=1e-6)
