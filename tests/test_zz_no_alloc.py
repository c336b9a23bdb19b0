"""The allocation-free partial trace against the allocating one and the oracle.

qf_partial_trace_noalloc serves callers that cannot allocate device memory
inside the call (code that must not stall the device, embedders whose own
allocator holds all free memory).  It keeps the environment kernel's scratch
(the per-CTA partial sums and the per-start completion counters) in a fixed
static device array.  Through the C ABI, this file checks:
  - on two calls in a row (the second reuses the array the first one left
    behind), that it returns exactly what qf_partial_trace returns: both
    launch the same kernel with the same grid, and the kernel adds the CTA
    partials in a fixed order, so the results are bitwise equal;
  - that both match the oracle's CalcEnvMat (Alg. 1) within the bounds the
    other partial-trace tests use;
  - one CTA per start (10 qubits), 4 CTAs per start (12 qubits) and 16 CTAs
    per start (14 qubits), so the cross-CTA partials and the last-CTA
    reduction run out of the static array;
  - all three tensor precisions (complex128, complex64, double-FP32);
  - a request that fills the array to within 16 bytes of its end (252
    starts at 8 qubits) is accepted and exact, and one start more is refused.

This file is collected last so that a failure here cannot hide another test.
"""
import ctypes as ct

import numpy as np
import pytest
import torch

import oracle as orc
import qf_inputs as qi

pytestmark = pytest.mark.gpu

QF_C128, QF_C64, QF_DF64 = 0, 1, 3


@pytest.fixture(scope="module")
def lib():
    from paper_2306_08152_gb300 import _native

    return _native.load()


def _call(lib, name, T, n, a, b, prec):
    S = T.shape[0]
    P = torch.zeros((S, 4, 4), dtype=torch.complex128, device=T.device)
    rc = getattr(lib, name)(ct.c_void_p(T.data_ptr()), n, S, a, b, ct.c_void_p(P.data_ptr()), prec,
                            ct.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.qf_last_error()
    torch.cuda.synchronize()
    return P.cpu().numpy()


def _tensor(n, S, prec, seed):
    """Seeded tensor on the device in the given precision, and the exact
    complex128 values it holds (host) for the oracle."""
    import paper_2306_08152_gb300 as qf

    g = qi.rng(seed)
    N = 2**n
    if prec == QF_C128:
        host = (g.standard_normal((S, N, N)) + 1j * g.standard_normal((S, N, N))) / np.sqrt(2)
        return torch.from_numpy(host).cuda(), host
    re = g.standard_normal((S, N, N), dtype=np.float32)
    im = g.standard_normal((S, N, N), dtype=np.float32)
    h64 = np.empty((S, N, N), dtype=np.complex64)
    h64.real = re
    h64.imag = im
    T = torch.from_numpy(h64).cuda()
    if prec == QF_DF64:  # complex64 -> double-FP32 is exact
        T = qf.convert_tensor(T, qf.QF_DF64)
    return T, h64


def _check_oracle(P, host, n, a, b, prec):
    for s in range(P.shape[0]):
        Ts = host[s].astype(np.complex128)
        ref = orc.calc_env_mat(Ts, a, b, n)
        if prec == QF_C128:
            assert np.max(np.abs(P[s] - ref)) <= 1e-12 * np.max(np.abs(ref)), s
        else:
            # complex64: FP32 band sums within a CTA, 1e-6 of the sum of
            # magnitudes; double-FP32 holds these values exactly and sums them
            # in FP64, so the complex128 bound applies
            mag = orc.calc_env_mat(np.abs(Ts).astype(np.complex128), a, b, n).real
            rel = 1e-6 if prec == QF_C64 else 1e-12
            assert np.all(np.abs(P[s] - ref) <= rel * mag), s


@pytest.mark.parametrize("n,S,prec", [(10, 3, QF_C128), (10, 3, QF_C64), (10, 3, QF_DF64),
                                      (12, 3, QF_C128), (12, 3, QF_C64), (12, 3, QF_DF64),
                                      (14, 2, QF_C64)])
def test_noalloc_matches_allocating_partial_trace(lib, n, S, prec):
    T, host = _tensor(n, S, prec, 777 + n)
    for call, (a, b) in enumerate([(1, n - 2), (n - 1, 0)]):  # two calls in a row
        ref = _call(lib, "qf_partial_trace", T, n, a, b, prec)
        got = _call(lib, "qf_partial_trace_noalloc", T, n, a, b, prec)
        assert np.array_equal(got, ref), (call, a, b)
        _check_oracle(got, host, n, a, b, prec)


def test_noalloc_accepts_a_full_array(lib):
    from paper_2306_08152_gb300 import _native as nat

    # 8 qubits: one CTA per start; 252 starts take 252 x 256 bytes of partial
    # sums plus 252 four-byte counters = 65520 of the 65536 bytes
    n, S = 8, 252
    assert nat.QF_NOALLOC_SCRATCH_BYTES == 65536
    T, host = _tensor(n, S, QF_C64, 881)
    for a, b in [(3, 4), (7, 0)]:
        ref = _call(lib, "qf_partial_trace", T, n, a, b, QF_C64)
        got = _call(lib, "qf_partial_trace_noalloc", T, n, a, b, QF_C64)
        assert np.array_equal(got, ref), (a, b)
    _check_oracle(got[-2:], host[-2:], n, 7, 0, QF_C64)


def test_noalloc_refuses_requests_beyond_its_array(lib):
    from paper_2306_08152_gb300 import _native as nat

    # one start more than test_noalloc_accepts_a_full_array; and at any qubit
    # count, more starts than the array holds partial-sum blocks.  The tensor
    # is still sized for each request, so even a wrong acceptance stays in
    # bounds.
    for n, S in [(8, 253), (2, nat.QF_NOALLOC_SCRATCH_BYTES // 256 + 1)]:
        T = torch.zeros((S, 2**n, 2**n), dtype=torch.complex64, device="cuda")
        P = torch.zeros((S, 4, 4), dtype=torch.complex128, device="cuda")
        rc = lib.qf_partial_trace_noalloc(ct.c_void_p(T.data_ptr()), n, S, 0, 1,
                                          ct.c_void_p(P.data_ptr()), QF_C64, None)
        torch.cuda.synchronize()
        assert rc == nat.QF_EINVAL, (n, S)
        assert b"QF_NOALLOC_SCRATCH_BYTES" in lib.qf_last_error()
