"""The seeded input generators (qf_inputs) that both the oracle and the CUDA
path are fed from: Haar unitaries (QR of a complex Gaussian with R's
diagonal phases divided out, Mezzadri 2007) and the uneven batches of the
batched benchmarks.  Determinism, the stated mixes and ranges, and valid
structures."""
import numpy as np
import pytest

import qf_inputs as qi


def test_haar_unitary_is_unitary_and_seeded():
    a = qi.haar_unitary(8, qi.rng(5))
    b = qi.haar_unitary(8, qi.rng(5))
    assert np.array_equal(a, b)
    assert np.max(np.abs(a.conj().T @ a - np.eye(8))) <= 1e-13
    assert not np.array_equal(a, qi.haar_unitary(8, qi.rng(6)))


def test_haar_unitary_moments():
    """For Haar U(d): E|U_00|^2 = 1/d and E|U_00|^4 = 2/(d(d+1)); the
    phase of U_00 is uniform (E U_00 = 0)."""
    g = qi.rng(11)
    d, m = 4, 4000
    u00 = np.array([qi.haar_unitary(d, g)[0, 0] for _ in range(m)])
    p2 = np.abs(u00) ** 2
    assert abs(p2.mean() - 1 / d) < 0.01
    assert abs((p2**2).mean() - 2 / (d * (d + 1))) < 0.01
    assert abs(u00.mean()) < 0.03


@pytest.mark.parametrize("count", [64, 403])
def test_batched_instances_mix_and_structure(count):
    insts = qi.batched_instances(count, 3, seed=7)
    again = qi.batched_instances(count, 3, seed=7)
    ns = np.array([x.n for x in insts])
    q = count // 4
    assert (ns == 4).sum() == q and (ns == 5).sum() == q and (ns == 3).sum() == count - 2 * q
    for x, y in zip(insts, again):
        assert x.n == y.n and np.array_equal(x.locs, y.locs) and np.array_equal(x.starts, y.starts)
        assert 5 <= x.p <= 40 and x.n_starts == 3
        a, b = x.locs[:, 0], x.locs[:, 1]
        assert np.all(np.abs(a - b) == 1) and a.min() >= 0 and max(a.max(), b.max()) < x.n
        assert np.max(np.abs(np.einsum("pji,pjk->pik", x.target_gates.conj(), x.target_gates) - np.eye(4))) <= 1e-13


def test_batched_instances_k_mix_and_structure():
    count = 400
    insts = qi.batched_instances_k(count, 2, seed=9)
    again = qi.batched_instances_k(count, 2, seed=9)
    ns = np.array([x.n for x in insts])
    assert (ns == 3).sum() == 200 and (ns == 4).sum() == 100 and (ns == 5).sum() == 100
    n3 = n_all = 0
    for x, y in zip(insts, again):
        assert x.locs == y.locs and all(np.array_equal(a, b) for a, b in zip(x.target_gates, y.target_gates))
        assert 4 <= len(x.locs) <= 16 and len(x.starts) == 2
        for q, u in zip(x.locs, x.target_gates):
            assert len(q) in (2, 3) and len(set(q)) == len(q) and min(q) >= 0 and max(q) < x.n
            d = 2 ** len(q)
            assert u.shape == (d, d) and np.max(np.abs(u.conj().T @ u - np.eye(d))) <= 1e-13
            n3 += len(q) == 3
            n_all += 1
        for s in x.starts:
            assert [g.shape[0] for g in s] == [2 ** len(q) for q in x.locs]
    # each gate three-qubit with probability 1/2
    assert abs(n3 / n_all - 0.5) < 0.03, n3 / n_all
