"""Seeded synthetic inputs for QFactor instantiation problems.

This module is shared by the FP64 oracle tests, the CUDA-path tests and the
benchmark.  It draws random numbers and lays out circuit structures only; it
contains none of the method's arithmetic (no circuit products, traces,
environments or gate updates).  A reachable target unitary is therefore
returned as the *gates* that produce it; the caller turns them into a matrix
with whichever implementation it is testing or trusting.

Conventions shared with both implementations:
  * a gate is a 4x4 complex128 matrix stored row-major (16 entries);
  * a location is a pair (a, b) of distinct qubits; the gate's local basis
    index is 2*bit(a) + bit(b);
  * gate lists are in product order: C = G_0 . G_1 ... G_{p-1}.

Random unitaries follow the published recipe of F. Mezzadri, "How to generate
random matrices from the classical compact groups" (Notices AMS, 2007): QR of a
complex Gaussian matrix with the phases of R's diagonal divided out, which is
Haar distributed on U(d).

Workload shapes follow the QFactor paper's instantiation workloads (Sec. V:
3-12 qubit partitions, up to tens of U(4) gates); the paper's benchmark
partitions are not available, so seeded brickwork and random-adjacent circuits
with matched qubit and gate counts stand in for them.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng",
    "haar_unitary",
    "haar_gates",
    "brickwork_locations",
    "random_adjacent_locations",
    "Instance",
    "make_problem",
    "batched_instances",
]


def rng(seed: int) -> np.random.Generator:
    """NumPy PCG64 generator for a given integer seed."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def haar_unitary(dim: int, gen: np.random.Generator) -> np.ndarray:
    """Haar-random dim x dim unitary (Mezzadri 2007): QR of a complex
    Gaussian, columns multiplied by the unit phases of diag(R)."""
    z = (gen.standard_normal((dim, dim)) + 1j * gen.standard_normal((dim, dim))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    ph = d / np.abs(d)
    return np.ascontiguousarray(q * ph[None, :], dtype=np.complex128)


def haar_gates(p: int, gen: np.random.Generator) -> np.ndarray:
    """p Haar-random U(4) gates, shape (p, 4, 4) complex128.  Draws the same
    numbers in the same order as p calls of haar_unitary(4, gen) (real then
    imaginary part of each gate) and factors them in one batched QR."""
    a = gen.standard_normal((p, 2, 4, 4))
    z = (a[:, 0] + 1j * a[:, 1]) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    ph = d / np.abs(d)
    return np.ascontiguousarray(q * ph[:, None, :], dtype=np.complex128)


def brickwork_locations(n: int, layers: int) -> np.ndarray:
    """Linear nearest-neighbour brickwork: even layers hold (0,1),(2,3),...,
    odd layers hold (1,2),(3,4),...; returns an int32 array of shape (p, 2)."""
    locs = []
    for layer in range(layers):
        start = layer % 2
        for q in range(start, n - 1, 2):
            locs.append((q, q + 1))
    return np.asarray(locs, dtype=np.int32).reshape(-1, 2)


def random_adjacent_locations(n: int, p: int, gen: np.random.Generator) -> np.ndarray:
    """p gates on random adjacent pairs (q, q+1), q uniform in [0, n-2]."""
    q = gen.integers(0, n - 1, size=p)
    return np.stack([q, q + 1], axis=1).astype(np.int32)


class Instance:
    """One instantiation problem: structure, target gates and start gates.

    ``target_gates`` produce a reachable target V = C(target_gates) for the
    given structure; ``starts`` holds the initial gates of every start,
    shape (n_starts, p, 4, 4).
    """

    def __init__(self, n, locs, target_gates, starts):
        self.n = int(n)
        self.locs = np.ascontiguousarray(locs, dtype=np.int32)
        self.target_gates = np.ascontiguousarray(target_gates, dtype=np.complex128)
        self.starts = np.ascontiguousarray(starts, dtype=np.complex128)

    @property
    def p(self):
        return int(self.locs.shape[0])

    @property
    def n_starts(self):
        return int(self.starts.shape[0])


def make_problem(n: int, locs: np.ndarray, n_starts: int, seed: int) -> Instance:
    """Reachable problem on a given structure: target gates Haar with seed
    ``seed``; start j's initial gates Haar with seed ``seed + 1 + j``."""
    p = int(np.asarray(locs).shape[0])
    tg = haar_gates(p, rng(seed))
    starts = np.stack([haar_gates(p, rng(seed + 1 + j)) for j in range(n_starts)])
    return Instance(n, locs, tg, starts)


def batched_instances(count: int, n_starts: int, seed: int,
                      qubit_mix=((3, 2), (4, 1), (5, 1)), p_range=(5, 40)):
    """Uneven batch of small reachable instances: qubit counts drawn in the
    ratio given by ``qubit_mix`` (default 3:4:5 qubits = 2:1:1), gate counts
    uniform in ``p_range`` (inclusive), gates on random adjacent pairs."""
    gen = rng(seed)
    sizes = []
    total = sum(w for _, w in qubit_mix)
    for nq, w in qubit_mix:
        sizes += [nq] * (count * w // total)
    while len(sizes) < count:
        sizes.append(qubit_mix[0][0])
    sizes = np.asarray(sizes[:count])
    gen.shuffle(sizes)
    out = []
    for i, nq in enumerate(sizes):
        p = int(gen.integers(p_range[0], p_range[1] + 1))
        locs = random_adjacent_locations(int(nq), p, gen)
        sub = int(gen.integers(0, 2**31 - 1))
        out.append(make_problem(int(nq), locs, n_starts, sub))
    return out


class InstanceK:
    """A reachable problem of 2- and 3-qubit gates: ``locs`` qubit tuples,
    ``target_gates`` and ``starts[j]`` lists of 2^k x 2^k Haar unitaries."""

    def __init__(self, n, locs, target_gates, starts):
        self.n, self.locs, self.target_gates, self.starts = n, locs, target_gates, starts


def batched_instances_k(count: int, n_starts: int, seed: int,
                        qubit_mix=((3, 2), (4, 1), (5, 1)), p_range=(4, 16), frac3=0.5):
    """Uneven batch of small reachable instances mixing 2- and 3-qubit
    gates: qubit counts in the ratio ``qubit_mix``, gate counts uniform in
    ``p_range``, each gate three-qubit with probability ``frac3`` on a random
    set of distinct qubits in random order (two-qubit otherwise); target and
    start gates Haar."""
    gen = rng(seed)
    sizes = []
    total = sum(w for _, w in qubit_mix)
    for nq, w in qubit_mix:
        sizes += [nq] * (count * w // total)
    while len(sizes) < count:
        sizes.append(qubit_mix[0][0])
    sizes = np.asarray(sizes[:count])
    gen.shuffle(sizes)
    out = []
    for nq in sizes:
        nq = int(nq)
        p = int(gen.integers(p_range[0], p_range[1] + 1))
        locs = []
        for _ in range(p):
            k = 3 if (nq >= 3 and gen.random() < frac3) else 2
            locs.append(tuple(int(x) for x in gen.choice(nq, k, replace=False)))
        tg = [haar_unitary(2 ** len(q), gen) for q in locs]
        starts = [[haar_unitary(2 ** len(q), gen) for q in locs] for _ in range(n_starts)]
        out.append(InstanceK(nq, locs, tg, starts))
    return out
