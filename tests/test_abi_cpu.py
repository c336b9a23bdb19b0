"""Host-side checks of the C ABI that need no GPU: the library loads, it
exports every function include/qfactor.h declares, option defaults, and
argument validation that returns before any CUDA call."""
import ctypes as ct
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qfactor.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2306_08152_gb300 import _build, _native

    if not os.path.exists(_build.LIB_PATH):
        _build.build()
    return _native.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qf_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("qf_instantiate", "qf_cost_and_env", "qf_instantiate_ex",
                     "qf_last_error", "qf_init_tensor", "qf_apply_pair",
                     "qf_partial_trace", "qf_optimize_gates", "qf_trace"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2306_08152_gb300 import _build

    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB_PATH],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (qf_[a-z0-9_]+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    for f in declared_functions():
        assert hasattr(lib, f)


def test_binding_covers_every_declared_symbol():
    from paper_2306_08152_gb300 import _native

    assert set(declared_functions()) <= set(_native.SIGNATURES)


def test_options_defaults(lib):
    from paper_2306_08152_gb300 import _native as nat

    o = nat.qf_options()
    assert lib.qf_options_default(ct.byref(o)) == 0
    assert o.dist_tol == 1e-10 and o.max_sweeps == 500 and o.reset_iter == 40
    assert o.beta == 0.0 and o.precision == nat.QF_C128
    assert o.cost_history is None
    assert lib.qf_options_default(None) == nat.QF_EINVAL
    assert b"NULL" in lib.qf_last_error()
    assert lib.qf_version() >= 100


def test_struct_layouts_match_header(lib, tmp_path):
    """The ctypes structures have the header's sizes and field offsets (a C
    program built from include/qfactor.h prints them)."""
    import shutil
    import subprocess

    from paper_2306_08152_gb300 import _native as nat

    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    structs = {"qf_options": nat.qf_options, "qf_result": nat.qf_result,
               "qf_batch_stats": nat.qf_batch_stats, "qf_gate_loc": nat.qf_gate_loc,
               "qf_gate_spec": nat.qf_gate_spec}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "qfactor.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, cls in structs.items():
        assert got[(name, "size")] == ct.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)
    assert ct.sizeof(nat.qf_options) == 80 and ct.sizeof(nat.qf_result) == 24


def _call_instantiate(lib, n, p, locs):
    N = 2**n
    V = np.eye(N, dtype=np.complex128)
    g = np.tile(np.eye(4, dtype=np.complex128), (max(p, 1), 1, 1))
    locs = np.ascontiguousarray(np.asarray(locs, dtype=np.int32).reshape(-1, 2))
    out = np.zeros_like(g)
    cost = ct.c_double()
    return lib.qf_instantiate(V.ctypes.data, n, p, locs.ctypes.data, g.ctypes.data, 1e-10, 10,
                              out.ctypes.data, ct.byref(cost), None, None)


def test_invalid_sizes_are_rejected_before_any_cuda_call(lib):
    from paper_2306_08152_gb300 import _native as nat

    assert _call_instantiate(lib, 1, 1, [[0, 1]]) == nat.QF_EINVAL
    assert b"n_qubits" in lib.qf_last_error()
    assert _call_instantiate(lib, 15, 1, [[0, 1]]) == nat.QF_EINVAL
    assert _call_instantiate(lib, 3, 0, [[0, 1]]) == nat.QF_EINVAL
    assert b"n_gates" in lib.qf_last_error()


@pytest.mark.parametrize("bad", [[[0, 0]], [[0, 3]], [[-1, 1]], [[1, 2], [2, 2]]])
def test_invalid_locations_are_rejected(lib, bad):
    from paper_2306_08152_gb300 import _native as nat

    locs = np.ascontiguousarray(np.asarray(bad, dtype=np.int32))
    h = ct.c_void_p()
    rc = lib.qf_plan_create(3, len(bad), locs.ctypes.data, 1, nat.QF_C128, ct.byref(h))
    assert rc == nat.QF_EINVAL
    assert b"location" in lib.qf_last_error()
    assert not h.value


def test_invalid_plan_arguments(lib):
    from paper_2306_08152_gb300 import _native as nat

    locs = np.array([[0, 1]], dtype=np.int32)
    h = ct.c_void_p()
    assert lib.qf_plan_create(3, 1, locs.ctypes.data, 0, nat.QF_C128, ct.byref(h)) == nat.QF_EINVAL
    assert lib.qf_plan_create(3, 1, locs.ctypes.data, 1, 7, ct.byref(h)) == nat.QF_EINVAL
    assert lib.qf_plan_create(3, 1, None, 1, nat.QF_C128, ct.byref(h)) == nat.QF_EINVAL
    assert lib.qf_plan_sweep(None, 1, 40, 0.0) == nat.QF_EINVAL
    assert lib.qf_optimize_gates(None, None, 0.5, 1, None, None, None) == nat.QF_EINVAL
    assert lib.qf_optimize_gates(None, None, 0.0, 0, None, None, None) == 0


def test_invalid_options_are_rejected(lib):
    from paper_2306_08152_gb300 import _native as nat

    o = nat.qf_options()
    lib.qf_options_default(ct.byref(o))
    V = np.eye(8, dtype=np.complex128)
    g = np.eye(4, dtype=np.complex128)[None]
    locs = np.array([[0, 1]], dtype=np.int32)
    out = np.zeros_like(g)
    for field, value in (("beta", 1.5), ("precision", 9), ("max_sweeps", 0)):
        bad = nat.qf_options()
        ct.memmove(ct.byref(bad), ct.byref(o), ct.sizeof(o))
        setattr(bad, field, value)
        rc = lib.qf_instantiate_ex(V.ctypes.data, 3, 1, locs.ctypes.data, 1, g.ctypes.data,
                                   ct.byref(bad), out.ctypes.data, None, None, None)
        assert rc == nat.QF_EINVAL, field


@pytest.mark.parametrize("spec,msg", [((2, 1, 1), b"repeated"), ((4, 0, 0), b"repeated"),
                                      ((7, 0, 1), b"unknown kind"), ((3, 5, -1), b"invalid"),
                                      ((1, 0, 1, 2), b"qubits >")])
def test_invalid_gate_specs_are_rejected(lib, spec, msg):
    """Specialised-gate plans (Sec. III-A): unknown kinds, repeated or
    out-of-range qubits and too-large gates fail before any CUDA call."""
    from paper_2306_08152_gb300 import _native as nat

    arr = (nat.qf_gate_spec * 1)()
    arr[0].kind = spec[0]
    q = list(spec[1:]) + [-1] * (4 - len(spec))
    for j in range(3):
        arr[0].q[j] = q[j]
    h = ct.c_void_p()
    rc = lib.qf_plan_create_spec(2, 1, arr, 1, nat.QF_C128, ct.byref(h))
    assert rc == nat.QF_EINVAL
    assert msg in lib.qf_last_error(), lib.qf_last_error()
    assert not h.value
    assert lib.qf_plan_load_spec(None, None, None, None, None) == nat.QF_EINVAL
    assert lib.qf_plan_get_params(None, None) == nat.QF_EINVAL


def test_spec_helpers_match_the_slot_rule():
    import paper_2306_08152_gb300 as qf
    from paper_2306_08152_gb300 import _native as nat

    specs = [("rz", 2), ("gpi", 0, 3), ("ms", 1, 2), ("u4", 0, 1), ("u8", 0, 1, 2), ("GPI", 1)]
    arr = qf.gate_specs(specs)
    assert [arr[i].kind for i in range(len(specs))] == [nat.QF_GATE_RZ, nat.QF_GATE_GPI, nat.QF_GATE_MS,
                                                        nat.QF_GATE_U4, nat.QF_GATE_U8, nat.QF_GATE_GPI]
    assert list(arr[0].q) == [2, -1, -1] and list(arr[4].q) == [0, 1, 2]
    # automatic partner: the next qubit, or the previous one for the last qubit
    assert qf.spec_slots(specs, 3) == [(2, 1), (0, 3), (1, 2), (0, 1), (0, 1, 2), (1, 2)]
    with pytest.raises(ValueError):
        qf.gate_specs([("cx", 0, 1)])


def _call_batched_k(lib, n, gates, S=1, precision=None, n_instances=1):
    """qf_instantiate_batched_k on one instance of n qubits with the given
    (k, qubits) gates; host arrays, default options."""
    from paper_2306_08152_gb300 import _native as nat

    p = len(gates)
    locs = (nat.qf_gate_loc * max(p, 1))()
    for i, (k, qs) in enumerate(gates):
        locs[i].k = k
        for j, q in enumerate(qs):
            locs[i].q[j] = q
    nq = np.full(max(n_instances, 1), n, dtype=np.int32)
    ng = np.full(max(n_instances, 1), p, dtype=np.int32)
    V = np.eye(2**n, dtype=np.complex128)
    g = np.zeros(S * max(p, 1) * 256, dtype=np.complex128)
    out = np.zeros_like(g)
    costs = np.zeros(S * max(n_instances, 1))
    sweeps = np.zeros(S * max(n_instances, 1), dtype=np.int32)
    best = np.zeros(max(n_instances, 1), dtype=np.int32)
    stats = nat.qf_batch_stats()
    opts = None
    if precision is not None:
        opts = nat.qf_options()
        lib.qf_options_default(ct.byref(opts))
        opts.precision = precision
    return lib.qf_instantiate_batched_k(n_instances, nq.ctypes.data, ng.ctypes.data, locs, V.ctypes.data, S,
                                        g.ctypes.data, ct.byref(opts) if opts is not None else None,
                                        out.ctypes.data, costs.ctypes.data_as(ct.POINTER(ct.c_double)),
                                        sweeps.ctypes.data, best.ctypes.data, ct.byref(stats), None)


@pytest.mark.parametrize("n,gates,msg", [
    (4, [(4, (0, 1, 2, 3))], b"2 or 3 qubits"),
    (3, [(1, (0,))], b"2 or 3 qubits"),
    (3, [(3, (0, 1, 1))], b"repeated qubit"),
    (3, [(2, (2, 2))], b"repeated qubit"),
    (3, [(3, (0, 1, 3))], b"invalid location"),
    (3, [(2, (-1, 0))], b"invalid location"),
    (2, [(3, (0, 1, 2))], b"invalid location"),
    (3, [(2, (0, 1)), (3, (2, 1, 5))], b"invalid location"),
])
def test_batched_k_rejects_invalid_gates_before_any_cuda_call(lib, n, gates, msg):
    from paper_2306_08152_gb300 import _native as nat

    assert _call_batched_k(lib, n, gates) == nat.QF_EINVAL
    assert msg in lib.qf_last_error(), lib.qf_last_error()


def test_batched_k_rejects_invalid_sizes_and_precisions(lib):
    from paper_2306_08152_gb300 import _native as nat

    ok_gates = [(3, (0, 1, 2))]
    assert _call_batched_k(lib, 3, ok_gates, n_instances=0) == nat.QF_EINVAL
    assert b"n_instances" in lib.qf_last_error()
    assert _call_batched_k(lib, 3, ok_gates, S=0) == nat.QF_EINVAL
    assert _call_batched_k(lib, 1, [(2, (0, 1))]) == nat.QF_EINVAL
    assert b"qubit count" in lib.qf_last_error()
    assert _call_batched_k(lib, 3, []) == nat.QF_EINVAL
    assert b"no gates" in lib.qf_last_error()
    for prec in (nat.QF_DF64, nat.QF_C64_REFINE_DF):
        assert _call_batched_k(lib, 3, ok_gates, precision=prec) == nat.QF_EINVAL
        assert b"batched kernel takes" in lib.qf_last_error()
    assert _call_batched_k(lib, 3, ok_gates, precision=9) == nat.QF_EINVAL
    assert b"unknown precision" in lib.qf_last_error()


def _call_instantiate_k(lib, n, gates, S=1):
    from paper_2306_08152_gb300 import _native as nat

    p = len(gates)
    locs = (nat.qf_gate_loc * max(p, 1))()
    for i, (k, qs) in enumerate(gates):
        locs[i].k = k
        for j, q in enumerate(qs):
            locs[i].q[j] = q
    V = np.eye(2**n, dtype=np.complex128)
    g = np.zeros(max(S, 1) * max(p, 1) * 256, dtype=np.complex128)
    out = np.zeros_like(g)
    costs = (ct.c_double * max(S, 1))()
    res = nat.qf_result()
    return lib.qf_instantiate_k(V.ctypes.data, n, p, locs, S, g.ctypes.data, None, out.ctypes.data, costs,
                                ct.byref(res), None)


@pytest.mark.parametrize("n,gates,S,msg", [
    (4, [(5, (0, 1, 2, 3))], 1, b"must be 2, 3 or 4"),
    (4, [(4, (0, 1, 2, 2))], 1, b"repeated qubit"),
    (4, [(4, (0, 1, 2, 4))], 1, b"invalid for 4 qubits"),
    (3, [(4, (0, 1, 2, 3))], 1, b"invalid for 3 qubits"),
    (3, [(2, (0, 0))], 1, b"repeated qubit"),
    (3, [], 1, b"n_gates"),
    (1, [(2, (0, 1))], 1, b"n_qubits"),
    (15, [(2, (0, 1))], 1, b"n_qubits"),
    (3, [(2, (0, 1))], 0, b"n_starts"),
])
def test_instantiate_k_rejects_invalid_arguments_before_any_cuda_call(lib, n, gates, S, msg):
    from paper_2306_08152_gb300 import _native as nat

    assert _call_instantiate_k(lib, n, gates, S) == nat.QF_EINVAL
    assert msg in lib.qf_last_error(), lib.qf_last_error()


def test_valid_call_without_a_gpu_fails_loudly(lib):
    """No CPU fallback: with no CUDA device a valid call returns a CUDA or
    memory error and says why."""
    import torch

    from paper_2306_08152_gb300 import _native as nat

    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    rc = _call_instantiate_k(lib, 3, [(3, (0, 1, 2))])
    assert rc in (nat.QF_ENOMEM, nat.QF_ECUDA), rc
    assert lib.qf_last_error()


def test_every_entry_point_rejects_null_pointers(lib):
    """Every call of the boundary, given NULL for each pointer argument and
    small sizes, returns QF_EINVAL with a message (qf_plan_destroy(NULL) is
    a no-op, like free(NULL)); none dereferences a NULL pointer."""
    from paper_2306_08152_gb300 import _native as nat

    skip = {"qf_last_error", "qf_version", "qf_set_tc_wait_limit", "qf_options_default"}
    checked = 0
    for name in declared_functions():
        if name in skip:
            continue
        fn = getattr(lib, name)
        args = []
        for t in fn.argtypes:
            if t in (ct.c_int, ct.c_int32):
                args.append(3)
            elif t is ct.c_double:
                args.append(0.0)
            elif t is ct.c_int64:
                args.append(8)
            else:
                args.append(None)
        rc = fn(*args)
        if name == "qf_plan_destroy":
            assert rc == 0
            continue
        assert rc == nat.QF_EINVAL, (name, rc, lib.qf_last_error())
        assert lib.qf_last_error(), name
        checked += 1
    assert checked >= 40
