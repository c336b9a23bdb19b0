"""Independent dense constructions used to pin the oracle (test helper).

Everything here is built from explicit loops over computational-basis indices
(the definition of "a gate on qubits (a, b) tensored with identity" and of a
partial trace), not from the tensor contractions the oracle uses, so that a
wrong leg, a transposed operand or a bit-order slip in either shows up as a
mismatch.  Qubit 0 is the most significant bit; a gate on (a, b) acts on the
local index 2*bit(a) + bit(b).
"""
import numpy as np


def bit(i, q, n):
    return (i >> (n - 1 - q)) & 1


def local_index(i, a, b, n):
    return 2 * bit(i, a, n) + bit(i, b, n)


def rest_bits(i, a, b, n):
    mask = (1 << (n - 1 - a)) | (1 << (n - 1 - b))
    return i & ~mask


def full_operator(u, a, b, n):
    """N x N matrix of u on (a, b): G[i, j] = u[loc(i), loc(j)] if i and j
    agree on every other qubit, else 0."""
    N = 2**n
    G = np.zeros((N, N), dtype=np.complex128)
    for i in range(N):
        for j in range(N):
            if rest_bits(i, a, b, n) == rest_bits(j, a, b, n):
                G[i, j] = u[local_index(i, a, b, n), local_index(j, a, b, n)]
    return G


def dense_circuit(gates, locs, n):
    """C = G_0 G_1 ... G_{p-1} as an explicit matrix product."""
    C = np.eye(2**n, dtype=np.complex128)
    for u, (a, b) in zip(gates, locs):
        C = C @ full_operator(u, int(a), int(b), n)
    return C


def dense_partial_trace(M, a, b, n):
    """P[x, y] = sum over i, j with equal bits outside (a, b), loc(i)=x,
    loc(j)=y, of M[i, j]."""
    N = 2**n
    P = np.zeros((4, 4), dtype=np.complex128)
    for i in range(N):
        for j in range(N):
            if rest_bits(i, a, b, n) == rest_bits(j, a, b, n):
                P[local_index(i, a, b, n), local_index(j, a, b, n)] += M[i, j]
    return P


def dense_environment(V, gates, locs, n, k):
    """E_k = partial trace of R_k = G_{k+1}..G_{p-1} V^dagger G_0..G_{k-1}."""
    N = 2**n
    left = np.eye(N, dtype=np.complex128)
    for j in range(k + 1, len(gates)):
        left = left @ full_operator(gates[j], int(locs[j][0]), int(locs[j][1]), n)
    right = np.eye(N, dtype=np.complex128)
    for j in range(k):
        right = right @ full_operator(gates[j], int(locs[j][0]), int(locs[j][1]), n)
    R = left @ np.asarray(V).conj().T @ right
    return dense_partial_trace(R, int(locs[k][0]), int(locs[k][1]), n)


# ---- gates on any number k of qubits: local index sum_i bit(q_i) 2^(k-1-i)

def local_index_k(i, qubits, n):
    x = 0
    for q in qubits:
        x = 2 * x + bit(i, q, n)
    return x


def rest_bits_k(i, qubits, n):
    mask = 0
    for q in qubits:
        mask |= 1 << (n - 1 - q)
    return i & ~mask


def full_operator_k(u, qubits, n):
    """N x N matrix of u on `qubits`: G[i, j] = u[loc(i), loc(j)] if i and j
    agree on every other qubit, else 0."""
    N = 2**n
    G = np.zeros((N, N), dtype=np.complex128)
    for i in range(N):
        for j in range(N):
            if rest_bits_k(i, qubits, n) == rest_bits_k(j, qubits, n):
                G[i, j] = u[local_index_k(i, qubits, n), local_index_k(j, qubits, n)]
    return G


def dense_circuit_k(gates, locs, n):
    C = np.eye(2**n, dtype=np.complex128)
    for u, q in zip(gates, locs):
        C = C @ full_operator_k(u, tuple(q), n)
    return C


def dense_partial_trace_k(M, qubits, n):
    N = 2**n
    d = 2 ** len(qubits)
    P = np.zeros((d, d), dtype=np.complex128)
    for i in range(N):
        for j in range(N):
            if rest_bits_k(i, qubits, n) == rest_bits_k(j, qubits, n):
                P[local_index_k(i, qubits, n), local_index_k(j, qubits, n)] += M[i, j]
    return P


def dense_environment_k(V, gates, locs, n, k):
    N = 2**n
    left = np.eye(N, dtype=np.complex128)
    for j in range(k + 1, len(gates)):
        left = left @ full_operator_k(gates[j], tuple(locs[j]), n)
    right = np.eye(N, dtype=np.complex128)
    for j in range(k):
        right = right @ full_operator_k(gates[j], tuple(locs[j]), n)
    R = left @ np.asarray(V).conj().T @ right
    return dense_partial_trace_k(R, tuple(locs[k]), n)
