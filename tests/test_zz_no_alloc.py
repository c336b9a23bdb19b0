"""The allocation-free partial trace against the allocating one.

qf_partial_trace_noalloc serves callers that cannot allocate device memory
inside the call (code that must not stall the device, embedders whose own
allocator holds all free memory).  It keeps the environment kernel's scratch
in a fixed static device array, so this test checks, through the C ABI, that
it returns what qf_partial_trace returns, on two calls in a row (the second
call reuses the array the first one left behind), for both tensor
precisions, and that a request larger than the array is refused.

This file is collected last so that a failure here cannot hide another test.
"""
import ctypes as ct

import numpy as np
import pytest
import torch

import oracle as orc
import qf_inputs as qi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2306_08152_gb300 import _native

    return _native.load()


def _call(lib, name, T, a, b, prec):
    S, N = T.shape[0], T.shape[-1]
    n = int(N).bit_length() - 1
    P = torch.zeros((S, 4, 4), dtype=torch.complex128, device=T.device)
    rc = getattr(lib, name)(ct.c_void_p(T.data_ptr()), n, S, a, b, ct.c_void_p(P.data_ptr()), prec,
                            ct.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.qf_last_error()
    torch.cuda.synchronize()
    return P.cpu().numpy()


@pytest.mark.parametrize("dtype,prec", [(torch.complex128, 0), (torch.complex64, 1)])
def test_noalloc_matches_allocating_partial_trace(lib, dtype, prec):
    g = qi.rng(777)
    n, S = 10, 3
    N = 2**n
    for call, (a, b) in enumerate([(2, 7), (9, 0)]):  # two calls in a row
        T0 = (g.standard_normal((S, N, N)) + 1j * g.standard_normal((S, N, N))) / np.sqrt(2)
        T = torch.from_numpy(T0).to(dtype).cuda()
        ref = _call(lib, "qf_partial_trace", T, a, b, prec)
        got = _call(lib, "qf_partial_trace_noalloc", T, a, b, prec)
        Tc = T.cpu().numpy().astype(np.complex128)
        for s in range(S):
            if prec == 0:
                scale = np.max(np.abs(ref[s]))
                assert np.max(np.abs(got[s] - ref[s])) <= 1e-12 * scale, (call, s)
            else:  # the complex64 FP32-summation bound used by the other tests
                bound = 1e-6 * orc.calc_env_mat(np.abs(Tc[s]).astype(np.complex128), a, b, n).real
                assert np.all(np.abs(got[s] - ref[s]) <= bound), (call, s)


def test_noalloc_refuses_requests_beyond_its_array(lib):
    from paper_2306_08152_gb300 import _native as nat

    # every start needs at least one CTA's 32 partial sums (256 bytes), so
    # this many starts exceeds the array at any qubit count; the tensor is
    # still sized for the request, so even a wrong acceptance stays in bounds
    n = 2
    S = nat.QF_NOALLOC_SCRATCH_BYTES // 256 + 1
    T = torch.zeros((S, 2**n, 2**n), dtype=torch.complex64, device="cuda")
    P = torch.zeros((S, 4, 4), dtype=torch.complex128, device="cuda")
    rc = lib.qf_partial_trace_noalloc(ct.c_void_p(T.data_ptr()), n, S, 0, 1,
                                      ct.c_void_p(P.data_ptr()), 1, None)
    torch.cuda.synchronize()
    assert rc == nat.QF_EINVAL
    assert b"QF_NOALLOC_SCRATCH_BYTES" in lib.qf_last_error()
