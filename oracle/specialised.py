"""QFactor oracle for specialised (parameterised) gate sets: plain FP64 NumPy.

Test infrastructure only: ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import this module.

Sec. III-A ("Specializing gate sets"): the circuit may use parameterised
gates G(theta) instead of general unitaries.  The SVD update does not apply
to them; the update is theta' = argmax_theta Re Tr(E G(theta)), which for
these gates has a closed form.  The gates (the paper names them for a
trapped-ion target and writes out Rz):

  Rz(theta)     = diag(1, e^{i theta})                     (the paper's definition)
  GPI(phi)      = [[0, e^{-i phi}], [e^{i phi}, 0]]
  MS(phi0, phi1) = (1/sqrt 2) [[1, 0, 0, -i e^{-i(phi0+phi1)}],
                               [0, 1, -i e^{-i(phi0-phi1)}, 0],
                               [0, -i e^{i(phi0-phi1)}, 1, 0],
                               [-i e^{i(phi0+phi1)}, 0, 0, 1]]

(the Moelmer-Soerensen gate; local index 2 bit(q0) + bit(q1) as for every
two-qubit gate here).  The maximisers, derived from the definitions (the
paper's printed Rz maximiser is garbled):

  Rz:  Re Tr(E Rz) = Re E00 + Re(e^{i theta} E11),  theta = -arg E11;
  GPI: Re Tr(E GPI) = Re(e^{i phi} (E01 + conj E10)),  phi = -arg(E01 + conj E10);
  MS:  with a = phi0 + phi1 and b = phi0 - phi1,
       sqrt 2 Re Tr(E MS) = Re Tr E + Re(e^{i a} z_a) + Re(e^{i b} z_b),
       z_a = -i (E03 - conj E30),  z_b = -i (E12 - conj E21),
       a = -arg z_a,  b = -arg z_b,  phi0 = (a + b)/2,  phi1 = (a - b)/2.

Where the modulus that sets an angle is zero every angle is optimal and the
old one is kept.  With beta damping the same maximisers apply to
A = (1 - beta) E + beta u^dagger, as for the SVD update.

The sweep is Alg. 1's TwoSidedSweep with this update for parameterised
gates and the SVD update (oracle/kqubit.py) for general unitaries.  A
one-qubit gate acts on its own qubit here (no partner qubit).

Parity pins (tests/test_oracle_pins_spec.py): GPI(phi) = Rz(phi) X Rz(-phi),
MS(phi0, phi1) = expm(-i pi/4 GPI(phi0) (x) GPI(phi1)) (scipy), Rz(pi) = Z,
brute-force maximisation over the parameters, single-gate fits, and the
monotone increase of Re Tr over the updates of a sweep.
"""
from __future__ import annotations

import numpy as np

from . import kqubit as ok

U = "u"
RZ = "rz"
GPI = "gpi"
MS = "ms"

NPARAM = {RZ: 1, GPI: 1, MS: 2}
NQUBITS = {RZ: 1, GPI: 1, MS: 2}

__all__ = ["U", "RZ", "GPI", "MS", "NPARAM", "NQUBITS", "rz", "gpi", "ms", "gate_matrix",
           "objective", "optimize_param", "init_circuit_tensor_spec", "two_sided_sweep_spec",
           "circuit_unitary_spec"]


def rz(theta):
    return np.array([[1.0, 0.0], [0.0, np.exp(1j * theta)]], dtype=np.complex128)


def gpi(phi):
    return np.array([[0.0, np.exp(-1j * phi)], [np.exp(1j * phi), 0.0]], dtype=np.complex128)


def ms(phi0, phi1):
    a, b = phi0 + phi1, phi0 - phi1
    m = np.eye(4, dtype=np.complex128)
    m[0, 3] = -1j * np.exp(-1j * a)
    m[1, 2] = -1j * np.exp(-1j * b)
    m[2, 1] = -1j * np.exp(1j * b)
    m[3, 0] = -1j * np.exp(1j * a)
    return m / np.sqrt(2.0)


def gate_matrix(kind, params):
    if kind == RZ:
        return rz(params[0])
    if kind == GPI:
        return gpi(params[0])
    if kind == MS:
        return ms(params[0], params[1])
    raise ValueError(kind)


def objective(kind, A, params):
    """Re Tr(A G(params))."""
    return float(np.real(np.trace(np.asarray(A) @ gate_matrix(kind, params))))


def optimize_param(kind, A, old):
    """argmax over the parameters of Re Tr(A G); keeps an old angle whose
    modulus is zero.  Returns (params, maximum)."""
    A = np.asarray(A, dtype=np.complex128)
    new = list(old)
    if kind == RZ:
        z = A[1, 1]
        if z != 0:
            new[0] = -np.angle(z)
        return new, float(A[0, 0].real + abs(z))
    if kind == GPI:
        z = A[0, 1] + np.conj(A[1, 0])
        if z != 0:
            new[0] = -np.angle(z)
        return new, float(abs(z))
    if kind == MS:
        za = -1j * (A[0, 3] - np.conj(A[3, 0]))
        zb = -1j * (A[1, 2] - np.conj(A[2, 1]))
        a, b = old[0] + old[1], old[0] - old[1]
        if za != 0:
            a = -np.angle(za)
        if zb != 0:
            b = -np.angle(zb)
        new = [(a + b) / 2.0, (a - b) / 2.0]
        return new, float((np.trace(A).real + abs(za) + abs(zb)) / np.sqrt(2.0))
    raise ValueError(kind)


def _matrix(kind, state):
    return np.asarray(state, dtype=np.complex128) if kind == U else gate_matrix(kind, state)


def init_circuit_tensor_spec(V, kinds, locs, states, n):
    """InitCircuitTensor: T <- V^dagger, then every gate on the right."""
    return ok.init_circuit_tensor_k(V, [_matrix(k, s) for k, s in zip(kinds, states)], locs, n)


def circuit_unitary_spec(kinds, locs, states, n):
    return ok.circuit_unitary_k([_matrix(k, s) for k, s in zip(kinds, states)], locs, n)


def _update(kind, E, state, beta):
    if kind == U:
        u, _ = ok.optimize_gate_k(E, state, beta)
        return u
    A = np.asarray(E, dtype=np.complex128)
    if beta != 0.0:
        A = (1.0 - beta) * A + beta * _matrix(kind, state).conj().T
    new, _ = optimize_param(kind, A, state)
    return new


def two_sided_sweep_spec(T, kinds, locs, states, n, beta=0.0, retr=None):
    """TwoSidedSweep of Alg. 1 over a circuit of general and parameterised
    gates; ``states`` holds a matrix per general gate and a parameter list
    per parameterised gate.  ``retr`` collects Re Tr(T) after every update."""
    states = [np.array(s, dtype=np.complex128, copy=True) if k == U else list(s)
              for k, s in zip(kinds, states)]
    p = len(kinds)
    for k in range(p - 1, -1, -1):
        q = tuple(int(x) for x in locs[k])
        T = ok.apply_right_k(T, _matrix(kinds[k], states[k]).conj().T, q, n)
        states[k] = _update(kinds[k], ok.calc_env_mat_k(T, q, n), states[k], beta)
        T = ok.apply_left_k(T, _matrix(kinds[k], states[k]), q, n)
        if retr is not None:
            retr.append(float(np.trace(T).real))
    for k in range(p):
        q = tuple(int(x) for x in locs[k])
        T = ok.apply_left_k(T, _matrix(kinds[k], states[k]).conj().T, q, n)
        states[k] = _update(kinds[k], ok.calc_env_mat_k(T, q, n), states[k], beta)
        T = ok.apply_right_k(T, _matrix(kinds[k], states[k]), q, n)
        if retr is not None:
            retr.append(float(np.trace(T).real))
    return T, states
