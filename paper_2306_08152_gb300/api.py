"""Python binding of the QFactor C ABI (argument marshalling only).

Tensors are PyTorch tensors: targets complex128 (N, N), gates complex128
(..., 4, 4) in the list order C = G_0 ... G_{p-1}, locations int32 (p, 2).
Host (CPU) tensors are accepted where the C ABI accepts host-or-device
arrays; the single-step functions need CUDA tensors.  Every computation runs
in libqfactor.so on the GPU.
"""
from __future__ import annotations

import ctypes as ct

import numpy as np
import torch

from . import _native as nat
from ._native import check

__all__ = [
    "QF_C128", "QF_C64", "QF_C64_REFINE64", "QF_DF64", "QF_C64_REFINE_DF", "Options", "instantiate",
    "instantiate_ex", "instantiate_batched", "cost_and_env", "cost_grad", "costs", "Plan", "init_tensor", "apply_pair",
    "partial_trace", "partial_trace_noalloc", "apply_two_pairs", "partial_trace_after", "convert_tensor",
    "instantiate_k", "apply_gate_k", "partial_trace_k", "optimize_gates_k", "init_tensor_k",
    "circuit_unitary_k", "flatten_gates", "unflatten_gates", "gate_entries", "optimize_gates", "reunitarize_gates", "trace", "circuit_unitary",
    "gate_specs", "spec_slots", "instantiate_spec", "cost_and_env_k", "cost_grad_k", "set_tc_wait_limit",
    "instantiate_batched_k",
]

QF_C128 = nat.QF_C128
QF_C64 = nat.QF_C64
QF_C64_REFINE64 = nat.QF_C64_REFINE64
QF_DF64 = nat.QF_DF64
QF_C64_REFINE_DF = nat.QF_C64_REFINE_DF


def _lib():
    return nat.load()


def _stream_handle(stream):
    if stream is None:
        if torch.cuda.is_available():
            return ct.c_void_p(torch.cuda.current_stream().cuda_stream)
        return ct.c_void_p(0)
    if isinstance(stream, torch.cuda.Stream):
        return ct.c_void_p(stream.cuda_stream)
    return ct.c_void_p(int(stream))


def _c128(t, name):
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(np.asarray(t, dtype=np.complex128))
    if t.dtype != torch.complex128:
        raise TypeError(f"{name} must be complex128, got {t.dtype}")
    return t.contiguous()


def _locs(locations):
    if isinstance(locations, torch.Tensor):
        t = locations.to(torch.int32).contiguous()
    else:
        t = torch.as_tensor(np.ascontiguousarray(np.asarray(locations, dtype=np.int32)))
    if t.dim() != 2 or t.shape[1] != 2:
        raise ValueError("locations must have shape (p, 2)")
    return t


def _ptr(t):
    return ct.c_void_p(t.data_ptr())


def _is_pairs(locations):
    """True when every location is a qubit pair (the two-qubit entry points)."""
    if isinstance(locations, torch.Tensor) or isinstance(locations, np.ndarray):
        return np.asarray(locations).ndim == 2 and np.asarray(locations).shape[1] == 2
    return all(len(q) == 2 for q in locations)


def _gate_locs(locations):
    """ctypes array of qf_gate_loc from a sequence of qubit tuples (2, 3 or 4)."""
    locs = [tuple(int(x) for x in q) for q in (locations.tolist() if hasattr(locations, "tolist")
                                                else locations)]
    arr = (nat.qf_gate_loc * len(locs))()
    for i, q in enumerate(locs):
        if len(q) not in (2, 3, 4):
            raise ValueError("a location has 2, 3 or 4 qubits")
        arr[i].k = len(q)
        for j, x in enumerate(q):
            arr[i].q[j] = x
    return arr, locs


_SPEC_KINDS = {"u4": nat.QF_GATE_U4, "u8": nat.QF_GATE_U8, "rz": nat.QF_GATE_RZ,
               "gpi": nat.QF_GATE_GPI, "ms": nat.QF_GATE_MS}


def _is_specs(locations):
    """True for a sequence of (kind, qubit, ...) tuples with a string kind."""
    return (not isinstance(locations, (torch.Tensor, np.ndarray)) and len(locations) > 0
            and all(isinstance(g, (tuple, list)) and isinstance(g[0], str) for g in locations))


def gate_specs(specs):
    """ctypes array of qf_gate_spec from (kind, q0[, q1[, q2]]) tuples, kind
    one of "u4", "u8", "rz", "gpi", "ms" (Sec. III-A, specialised gate sets);
    "rz"/"gpi" take an optional partner qubit for their 4x4 slot."""
    arr = (nat.qf_gate_spec * len(specs))()
    for i, g in enumerate(specs):
        kind = g[0].lower()
        if kind not in _SPEC_KINDS:
            raise ValueError(f"unknown gate kind {g[0]!r}")
        arr[i].kind = _SPEC_KINDS[kind]
        q = [int(x) for x in g[1:]] + [-1] * (4 - len(g))
        for j in range(3):
            arr[i].q[j] = q[j]
    return arr


def spec_slots(specs, n_qubits):
    """The qubits of each gate's matrix slot: (a, b) for 4x4 slots (rz/gpi
    with their partner qubit, automatic: q0 + 1, or q0 - 1 for the last
    qubit), (a, b, c) for "u8"."""
    out = []
    for g in specs:
        kind = g[0].lower()
        q = [int(x) for x in g[1:]]
        if kind in ("rz", "gpi"):
            partner = q[1] if len(q) > 1 and q[1] >= 0 else (q[0] + 1 if q[0] + 1 < n_qubits else q[0] - 1)
            out.append((q[0], partner))
        else:
            out.append(tuple(q))
    return out


def gate_entries(locations):
    """Entries of one start's concatenated gate array: sum of 4^k."""
    return sum(4 ** len(tuple(q)) for q in locations)


def flatten_gates(gate_sets):
    """Concatenated layout (S, E) complex128 from S lists of 2^k x 2^k
    arrays (one list per start, gates in circuit order)."""
    rows = [np.concatenate([np.asarray(g, dtype=np.complex128).reshape(-1) for g in gs])
            for gs in gate_sets]
    return torch.from_numpy(np.ascontiguousarray(np.stack(rows)))


def unflatten_gates(flat, locations):
    """S lists of 2^k x 2^k numpy arrays from the concatenated layout."""
    a = flat.detach().cpu().numpy() if isinstance(flat, torch.Tensor) else np.asarray(flat)
    out = []
    for row in a.reshape(a.shape[0], -1):
        gs, off = [], 0
        for q in locations:
            d = 2 ** len(tuple(q))
            gs.append(row[off:off + d * d].reshape(d, d))
            off += d * d
        out.append(gs)
    return out


def _nqubits(target):
    N = target.shape[-1]
    n = int(N).bit_length() - 1
    if target.dim() != 2 or target.shape[0] != N or (1 << n) != N:
        raise ValueError("target must be a 2^n x 2^n matrix")
    return n


class Options:
    """Hyperparameters of Sec. III-A2 (see qf_options in qfactor.h)."""

    def __init__(self, **kw):
        o = nat.qf_options()
        check(_lib().qf_options_default(ct.byref(o)))
        for k, v in kw.items():
            if not hasattr(o, k):
                raise AttributeError(f"unknown option {k}")
            setattr(o, k, v)
        self.c = o

    def __getattr__(self, k):
        return getattr(self.__dict__["c"], k)


def instantiate(target, locations, initial_gates, tol=1e-10, max_sweeps=500, stream=None):
    """One-start Qfactor (qf_instantiate).  Returns (gates, cost, sweeps);
    gates live where ``initial_gates`` lives."""
    target = _c128(target, "target")
    gates = _c128(initial_gates, "initial_gates")
    locs = _locs(locations)
    n = _nqubits(target)
    out = torch.empty_like(gates)
    cost = ct.c_double()
    sweeps = ct.c_int()
    check(_lib().qf_instantiate(_ptr(target), n, locs.shape[0], _ptr(locs), _ptr(gates),
                                float(tol), int(max_sweeps), _ptr(out), ct.byref(cost),
                                ct.byref(sweeps), _stream_handle(stream)))
    return out, cost.value, sweeps.value


def _history_buffer(opts, rows):
    """A host buffer for qf_options.cost_history (rows x (max_sweeps + 1)
    doubles), set in a copy of the options; returns (options, buffer)."""
    o = nat.qf_options.from_buffer_copy(opts.c)
    h = np.empty((rows, int(o.max_sweeps) + 1), dtype=np.float64)
    o.cost_history = h.ctypes.data
    return o, h


def instantiate_ex(target, locations, starts, options=None, stream=None, history=False, **kw):
    """Lock-step multistart Qfactor (qf_instantiate_ex).  ``starts`` has
    shape (S, p, 4, 4).  Returns a dict with gates, costs, best, sweeps,
    c64_sweeps, reason and best_cost; with ``history=True`` also "history",
    the cost of every start after every sweep (S, max_sweeps + 1), NaN after
    the last sweep."""
    target = _c128(target, "target")
    starts = _c128(starts, "starts")
    locs = _locs(locations)
    n = _nqubits(target)
    S, p = starts.shape[0], starts.shape[1]
    if p != locs.shape[0]:
        raise ValueError("starts and locations disagree on the gate count")
    opts = options if options is not None else Options(**kw)
    oc, hist = _history_buffer(opts, S) if history else (opts.c, None)
    out = torch.empty_like(starts)
    costs = (ct.c_double * S)()
    res = nat.qf_result()
    check(_lib().qf_instantiate_ex(_ptr(target), n, p, _ptr(locs), S, _ptr(starts),
                                   ct.byref(oc), _ptr(out), costs, ct.byref(res),
                                   _stream_handle(stream)))
    r = {"gates": out, "costs": np.array(costs[:]), "best": res.best_start,
         "sweeps": res.sweeps, "c64_sweeps": res.c64_sweeps,
         "reason": nat.REASONS.get(res.reason, str(res.reason)), "best_cost": res.best_cost}
    if history:
        r["history"] = hist
    return r


def cost_and_env(target, locations, gates, stream=None):
    """Costs, environments and traces of gate sets (qf_cost_and_env).
    ``gates`` has shape (S, p, 4, 4) or (p, 4, 4).  Returns (costs (S,),
    envs like gates, traces (S,) complex)."""
    target = _c128(target, "target")
    g = _c128(gates, "gates")
    single = g.dim() == 3
    if single:
        g = g.unsqueeze(0)
    locs = _locs(locations)
    n = _nqubits(target)
    S, p = g.shape[0], g.shape[1]
    envs = torch.empty_like(g)
    costs = (ct.c_double * S)()
    trs = np.zeros(S, dtype=np.complex128)
    check(_lib().qf_cost_and_env(_ptr(target), n, p, _ptr(locs), S, _ptr(g), costs, _ptr(envs),
                                 ct.c_void_p(trs.ctypes.data), _stream_handle(stream)))
    c = np.array(costs[:])
    if single:
        return c[0], envs[0], trs[0]
    return c, envs, trs


def instantiate_batched(instances, options=None, stream=None, history=False, **kw):
    """Many small instantiations in one persistent launch
    (qf_instantiate_batched).  ``instances`` is a sequence of
    (target (N,N), locations (p,2), starts (S,p,4,4)) with the same S; arrays
    may be numpy or CPU tensors.  Returns a dict with per-(instance, start)
    costs and sweeps, per-instance best start, the gates and launch stats;
    with ``history=True`` also "history" (I, S, max_sweeps + 1), the cost
    after every sweep, NaN after a start's last sweep."""
    targets, locs, starts, nq, ng = [], [], [], [], []
    S = None
    for V, L, G in instances:
        V = np.ascontiguousarray(np.asarray(V, dtype=np.complex128))
        L = np.ascontiguousarray(np.asarray(L, dtype=np.int32)).reshape(-1, 2)
        G = np.ascontiguousarray(np.asarray(G, dtype=np.complex128))
        if S is None:
            S = G.shape[0]
        if G.shape[0] != S or G.shape[1] != L.shape[0]:
            raise ValueError("every instance needs the same number of starts and p gates per start")
        nq.append(int(V.shape[0]).bit_length() - 1)
        ng.append(L.shape[0])
        targets.append(V.reshape(-1))
        locs.append(L)
        starts.append(G.reshape(-1))
    I = len(nq)
    nq = np.asarray(nq, dtype=np.int32)
    ng = np.asarray(ng, dtype=np.int32)
    tg = np.concatenate(targets)
    lc = np.ascontiguousarray(np.concatenate(locs))
    st = np.concatenate(starts)
    out = np.empty_like(st)
    costs = np.empty(I * S, dtype=np.float64)
    sweeps = np.empty(I * S, dtype=np.int32)
    best = np.empty(I, dtype=np.int32)
    stats = nat.qf_batch_stats()
    opts = options if options is not None else Options(**kw)
    oc, hist = _history_buffer(opts, I * S) if history else (opts.c, None)
    check(_lib().qf_instantiate_batched(
        I, ct.c_void_p(nq.ctypes.data), ct.c_void_p(ng.ctypes.data), ct.c_void_p(lc.ctypes.data),
        ct.c_void_p(tg.ctypes.data), S, ct.c_void_p(st.ctypes.data), ct.byref(oc),
        ct.c_void_p(out.ctypes.data), costs.ctypes.data_as(ct.POINTER(ct.c_double)),
        ct.c_void_p(sweeps.ctypes.data), ct.c_void_p(best.ctypes.data), ct.byref(stats),
        _stream_handle(stream)))
    gates, off = [], 0
    for i in range(I):
        k = S * ng[i] * 16
        gates.append(out[off:off + k].reshape(S, ng[i], 4, 4))
        off += k
    r = {"costs": costs.reshape(I, S), "sweeps": sweeps.reshape(I, S), "best": best,
         "gates": gates, "warps_per_cta": stats.warps_per_cta, "ctas": stats.ctas,
         "kernel_ms": stats.kernel_ms, "total_sweeps": stats.total_sweeps,
         "total_c64_sweeps": stats.total_c64_sweeps}
    if history:
        r["history"] = hist.reshape(I, S, -1)
    return r


def instantiate_batched_k(instances, options=None, stream=None, history=False, **kw):
    """instantiate_batched for circuits of 2- and 3-qubit gates
    (qf_instantiate_batched_k).  ``instances`` is a sequence of (target
    (N,N), locations (sequence of qubit tuples of 2 or 3), starts: S lists
    of 2^k x 2^k gates or an (S, E) concatenated array) with the same S.
    Returns the dict of instantiate_batched with "gates" as S lists of
    gate arrays per instance."""
    targets, locs, starts, nq, ng, lists = [], [], [], [], [], []
    S = None
    for V, L, G in instances:
        V = np.ascontiguousarray(np.asarray(V, dtype=np.complex128))
        arr, lq = _gate_locs(L)
        flat = G if isinstance(G, (np.ndarray, torch.Tensor)) and np.ndim(G) == 2 else flatten_gates(G)
        flat = np.ascontiguousarray(np.asarray(flat, dtype=np.complex128))
        if S is None:
            S = flat.shape[0]
        if flat.shape != (S, gate_entries(lq)):
            raise ValueError("every instance needs the same number of starts and its gate entries per start")
        nq.append(int(V.shape[0]).bit_length() - 1)
        ng.append(len(lq))
        targets.append(V.reshape(-1))
        locs.extend(arr)
        lists.append(lq)
        starts.append(flat.reshape(-1))
    I = len(nq)
    nq = np.asarray(nq, dtype=np.int32)
    ng = np.asarray(ng, dtype=np.int32)
    tg = np.concatenate(targets)
    larr = (nat.qf_gate_loc * len(locs))(*locs)
    st = np.concatenate(starts)
    out = np.empty_like(st)
    costs = np.empty(I * S, dtype=np.float64)
    sweeps = np.empty(I * S, dtype=np.int32)
    best = np.empty(I, dtype=np.int32)
    stats = nat.qf_batch_stats()
    opts = options if options is not None else Options(**kw)
    oc, hist = _history_buffer(opts, I * S) if history else (opts.c, None)
    check(_lib().qf_instantiate_batched_k(
        I, ct.c_void_p(nq.ctypes.data), ct.c_void_p(ng.ctypes.data), larr,
        ct.c_void_p(tg.ctypes.data), S, ct.c_void_p(st.ctypes.data), ct.byref(oc),
        ct.c_void_p(out.ctypes.data), costs.ctypes.data_as(ct.POINTER(ct.c_double)),
        ct.c_void_p(sweeps.ctypes.data), ct.c_void_p(best.ctypes.data), ct.byref(stats),
        _stream_handle(stream)))
    gates, off = [], 0
    for i in range(I):
        k = S * gate_entries(lists[i])
        gates.append(unflatten_gates(out[off:off + k].reshape(S, -1), lists[i]))
        off += k
    r = {"costs": costs.reshape(I, S), "sweeps": sweeps.reshape(I, S), "best": best,
         "gates": gates, "warps_per_cta": stats.warps_per_cta, "ctas": stats.ctas,
         "kernel_ms": stats.kernel_ms, "total_sweeps": stats.total_sweeps,
         "total_c64_sweeps": stats.total_c64_sweeps}
    if history:
        r["history"] = hist.reshape(I, S, -1)
    return r


def cost_grad(target, locations, gates, stream=None):
    """Costs and their gradients with respect to the gates (qf_cost_grad),
    in PyTorch's complex-autograd convention.  ``gates`` (S, p, 4, 4) or
    (p, 4, 4); returns (costs (S,) numpy, grads like gates)."""
    target = _c128(target, "target")
    g = _c128(gates, "gates")
    single = g.dim() == 3
    if single:
        g = g.unsqueeze(0)
    locs = _locs(locations)
    n = _nqubits(target)
    S, p = g.shape[0], g.shape[1]
    grads = torch.empty_like(g)
    costs = (ct.c_double * S)()
    check(_lib().qf_cost_grad(_ptr(target), n, p, _ptr(locs), S, _ptr(g), costs, _ptr(grads),
                              _stream_handle(stream)))
    c = np.array(costs[:])
    if single:
        return c[0], grads[0]
    return c, grads


def _flat_sets(gates, locs):
    """(S, E) complex128 gate sets from a tensor (S, E) / (E,) or S lists."""
    if not isinstance(gates, torch.Tensor):
        gates = flatten_gates(gates)
    g = _c128(gates, "gates")
    single = g.dim() == 1
    if single:
        g = g.unsqueeze(0)
    if g.shape[1] != gate_entries(locs):
        raise ValueError("gates do not match the locations' gate sizes")
    return g.contiguous(), single


def cost_and_env_k(target, locations, gates, stream=None):
    """Costs, environments and traces of gate sets of 2-, 3- and 4-qubit
    gates (qf_cost_and_env_k).  ``gates``: (S, E) concatenated layout, (E,),
    or S lists of arrays.  Returns (costs (S,), envs like the (S, E) gates,
    traces (S,) complex)."""
    target = _c128(target, "target")
    larr, locs = _gate_locs(locations)
    g, single = _flat_sets(gates, locs)
    n = _nqubits(target)
    S = g.shape[0]
    envs = torch.empty_like(g)
    costs = (ct.c_double * S)()
    trs = np.zeros(S, dtype=np.complex128)
    check(_lib().qf_cost_and_env_k(_ptr(target), n, len(locs), larr, S, _ptr(g), costs, _ptr(envs),
                                   ct.c_void_p(trs.ctypes.data), _stream_handle(stream)))
    c = np.array(costs[:])
    if single:
        return c[0], envs[0], trs[0]
    return c, envs, trs


def cost_grad_k(target, locations, gates, stream=None):
    """Costs and gradients for gate sets of 2-, 3- and 4-qubit gates
    (qf_cost_grad_k), in PyTorch's complex-autograd convention; gates and
    gradients in the concatenated layout (S, E) (or (E,))."""
    target = _c128(target, "target")
    larr, locs = _gate_locs(locations)
    g, single = _flat_sets(gates, locs)
    n = _nqubits(target)
    S = g.shape[0]
    grads = torch.empty_like(g)
    costs = (ct.c_double * S)()
    check(_lib().qf_cost_grad_k(_ptr(target), n, len(locs), larr, S, _ptr(g), costs, _ptr(grads),
                                _stream_handle(stream)))
    c = np.array(costs[:])
    if single:
        return c[0], grads[0]
    return c, grads


def costs(target, locations, gates, stream=None):
    """Costs 1 - |Tr(V^dagger C)|/N of gate sets (S, p, 4, 4), without
    environments: InitCircuitTensor plus an FP64 trace on the GPU."""
    g = _c128(gates, "gates")
    if g.dim() == 3:
        g = g.unsqueeze(0)
    target = _c128(target, "target")
    plan = Plan(_nqubits(target), locations, g.shape[0], QF_C128)
    try:
        plan.load(target, g, stream=stream)
        return plan.costs()
    finally:
        plan.close()


class Plan:
    """Device-resident multistart state (qf_plan_*).  ``locations`` holds
    qubit pairs, or tuples of 2 or 3 qubits (qf_plan_create_k; gates then
    use the concatenated layout (S, E), see flatten_gates)."""

    def __init__(self, n_qubits, locations, n_starts, precision=QF_C128):
        self.n = int(n_qubits)
        self.S = int(n_starts)
        h = ct.c_void_p()
        self.spec = _is_specs(locations)
        self.k_path = self.spec or not _is_pairs(locations)
        if self.spec:
            self.specs = [tuple(g) for g in locations]
            self._sarr = gate_specs(self.specs)
            self.p = len(self.specs)
            check(_lib().qf_plan_create_spec(self.n, self.p, self._sarr, self.S, int(precision),
                                             ct.byref(h)))
        elif self.k_path:
            self._larr, self.locations = _gate_locs(locations)
            self.p = len(self.locations)
            check(_lib().qf_plan_create_k(self.n, self.p, self._larr, self.S, int(precision),
                                          ct.byref(h)))
        else:
            self.locs = _locs(locations)
            self.p = int(self.locs.shape[0])
            check(_lib().qf_plan_create(self.n, self.p, _ptr(self.locs), self.S, int(precision),
                                        ct.byref(h)))
        self.h = h
        e = ct.c_int64()
        check(_lib().qf_plan_gate_entries(self.h, ct.byref(e)))
        self.E = e.value

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _lib().qf_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, target, gates, stream=None):
        self._t = _c128(target, "target")
        self._g = _c128(gates, "gates")
        check(_lib().qf_plan_load(self.h, _ptr(self._t), _ptr(self._g), _stream_handle(stream)))

    def load_params(self, target, params, gates=None, stream=None):
        """Specialised-gate plans: load the target, the parameters (S, p, 2)
        float64 and, for circuits with general gates, their matrices in the
        concatenated layout (S, E)."""
        self._t = _c128(target, "target")
        pr = params if isinstance(params, torch.Tensor) else torch.as_tensor(np.asarray(params, dtype=np.float64))
        if pr.dtype != torch.float64:
            raise TypeError("params must be float64")
        self._p = pr.contiguous()
        self._g = _c128(gates, "gates") if gates is not None else None
        check(_lib().qf_plan_load_spec(self.h, _ptr(self._t), _ptr(self._g) if self._g is not None else None,
                                       _ptr(self._p), _stream_handle(stream)))

    def params(self, device="cpu"):
        """Specialised-gate plans: the current parameters, (S, p, 2) float64."""
        out = torch.empty((self.S, self.p, 2), dtype=torch.float64, device=device)
        check(_lib().qf_plan_get_params(self.h, _ptr(out)))
        return out

    def sweep(self, n_sweeps=1, reset_iter=40, beta=0.0):
        check(_lib().qf_plan_sweep(self.h, int(n_sweeps), int(reset_iter), float(beta)))

    def rebuild(self, precision):
        check(_lib().qf_plan_rebuild(self.h, int(precision)))

    def costs(self):
        out = (ct.c_double * self.S)()
        check(_lib().qf_plan_costs(self.h, out, None))
        return np.array(out[:])

    def gates(self, device="cpu"):
        if self.k_path:
            out = torch.empty((self.S, self.E), dtype=torch.complex128, device=device)
        else:
            out = torch.empty((self.S, self.p, 4, 4), dtype=torch.complex128, device=device)
        check(_lib().qf_plan_get_gates(self.h, _ptr(out)))
        return out

    def enable_pass_timing(self, enable=True):
        check(_lib().qf_plan_enable_pass_timing(self.h, int(bool(enable))))

    def set_lookahead(self, enable=True):
        """Two consecutive updates on disjoint pairs per pass (complex64,
        n >= 8); returns the two-update windows per sweep (0 = none)."""
        check(_lib().qf_plan_set_lookahead(self.h, int(bool(enable))))
        w = ct.c_int()
        check(_lib().qf_plan_lookahead_windows(self.h, ct.byref(w)))
        return w.value

    def pass_stats(self):
        """(pass ms, pass launches, all launches, pass algorithmic bytes)
        since the last call."""
        ms = ct.c_double()
        pl = ct.c_int64()
        al = ct.c_int64()
        by = ct.c_double()
        check(_lib().qf_plan_pass_stats(self.h, ct.byref(ms), ct.byref(pl), ct.byref(al),
                                        ct.byref(by)))
        return ms.value, pl.value, al.value, by.value

    def status(self):
        return _lib().qf_plan_status(self.h)


# ------------------------------------------------------------ single steps


def _dev(t, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError(f"{name} must be a CUDA tensor")
    return t.contiguous()


def _is_df(T):
    return T.dtype == torch.float32 and T.dim() >= 3 and T.shape[-1] == 4


def _tensor_prec(T):
    """complex128 -> QF_C128, complex64 -> QF_C64; a float32 tensor whose last
    dimension is 4 holds double-FP32 entries (re.hi, im.hi, re.lo, im.lo) ->
    QF_DF64."""
    if T.dtype == torch.complex128:
        return QF_C128
    if T.dtype == torch.complex64:
        return QF_C64
    if _is_df(T):
        return QF_DF64
    raise TypeError("circuit tensor must be complex64, complex128 or float32 (..., 4) df64")


def _tensor_sn(T):
    """(starts, N) of a circuit tensor of any precision."""
    if _is_df(T):
        return T.shape[0], T.shape[-2]
    return T.shape[0], T.shape[-1]


_PREC_SHAPE = {QF_C128: (torch.complex128, ()), QF_C64: (torch.complex64, ()),
               QF_DF64: (torch.float32, (4,))}


def _empty_tensor(S, N, precision, device):
    dt, tail = _PREC_SHAPE[precision]
    return torch.empty((S, N, N) + tail, dtype=dt, device=device)


def convert_tensor(T, precision, stream=None):
    """A copy of circuit tensor(s) T in `precision` (QF_C128, QF_C64 or
    QF_DF64), converted on the device."""
    T = _dev(T, "T")
    src = _tensor_prec(T)
    S, N = _tensor_sn(T)
    out = _empty_tensor(S, N, precision, T.device)
    check(_lib().qf_convert_tensor(_ptr(T), src, _ptr(out), int(precision), S * N * N,
                                   _stream_handle(stream)))
    return out


def init_tensor(target, locations, gates, dtype=torch.complex128, stream=None):
    """InitCircuitTensor for S starts: gates (S, p, 4, 4) -> T (S, N, N).
    dtype: torch.complex128, torch.complex64, or "df64" for a double-FP32
    tensor (float32, shape (S, N, N, 4))."""
    target = _dev(_c128(target, "target"), "target")
    g = _dev(_c128(gates, "gates"), "gates")
    if g.dim() == 3:
        g = g.unsqueeze(0)
    locs = _locs(locations)
    n = _nqubits(target)
    N = 1 << n
    prec = QF_DF64 if dtype == "df64" else (QF_C128 if dtype == torch.complex128 else QF_C64)
    T = _empty_tensor(g.shape[0], N, prec, target.device)
    check(_lib().qf_init_tensor(_ptr(target), n, g.shape[1], _ptr(locs), g.shape[0], _ptr(g),
                                _ptr(T), _tensor_prec(T), _stream_handle(stream)))
    return T


def apply_pair(T, a, b, L=None, R=None, stream=None):
    """In place: T_s <- (L_s on (a,b)) T_s (R_s on (a,b)); L, R (S, 4, 4)."""
    T = _dev(T, "T")
    S, N = _tensor_sn(T)
    n = int(N).bit_length() - 1
    Lp = _ptr(_dev(_c128(L, "L"), "L")) if L is not None else None
    Rp = _ptr(_dev(_c128(R, "R"), "R")) if R is not None else None
    check(_lib().qf_apply_pair(_ptr(T), n, S, int(a), int(b), Lp, Rp, _tensor_prec(T),
                               _stream_handle(stream)))
    return T


def partial_trace(T, a, b, stream=None):
    T = _dev(T, "T")
    S, N = _tensor_sn(T)
    n = int(N).bit_length() - 1
    P = torch.empty((S, 4, 4), dtype=torch.complex128, device=T.device)
    check(_lib().qf_partial_trace(_ptr(T), n, S, int(a), int(b), _ptr(P), _tensor_prec(T),
                                  _stream_handle(stream)))
    return P


def apply_two_pairs(T, a1, b1, L1, R1, a2, b2, L2, R2, stream=None):
    """In place: T_s <- (L1_s on (a1,b1)) (L2_s on (a2,b2)) T_s
    (R1_s on (a1,b1)) (R2_s on (a2,b2)); four distinct qubits; operators
    (S, 4, 4)."""
    T = _dev(T, "T")
    S, N = _tensor_sn(T)
    n = int(N).bit_length() - 1
    ops = [_dev(_c128(X, nm), nm) for X, nm in ((L1, "L1"), (R1, "R1"), (L2, "L2"), (R2, "R2"))]
    check(_lib().qf_apply_two_pairs(_ptr(T), n, S, int(a1), int(b1), _ptr(ops[0]), _ptr(ops[1]),
                                    int(a2), int(b2), _ptr(ops[2]), _ptr(ops[3]),
                                    _tensor_prec(T), _stream_handle(stream)))
    return T


def partial_trace_after(T, a1, b1, L1, R1, a, b, stream=None):
    """Partial trace over every qubit but (a, b) of (L1 on (a1,b1)) T
    (R1 on (a1,b1)), computed without applying the pending update."""
    T = _dev(T, "T")
    S, N = _tensor_sn(T)
    n = int(N).bit_length() - 1
    L1 = _dev(_c128(L1, "L1"), "L1")
    R1 = _dev(_c128(R1, "R1"), "R1")
    P = torch.empty((S, 4, 4), dtype=torch.complex128, device=T.device)
    check(_lib().qf_partial_trace_after(_ptr(T), n, S, int(a1), int(b1), _ptr(L1), _ptr(R1),
                                        int(a), int(b), _ptr(P), _tensor_prec(T),
                                        _stream_handle(stream)))
    return P


def instantiate_k(target, locations, starts, options=None, stream=None, **kw):
    """Lock-step multistart Qfactor with 2-, 3- and 4-qubit gates
    (qf_instantiate_k).  ``locations``: sequence of qubit tuples; ``starts``:
    (S, E) complex128 in the concatenated layout or S lists of gate arrays.
    Returns the dict of instantiate_ex with ``gates`` as S lists of arrays
    and ``flat`` the (S, E) tensor."""
    target = _c128(target, "target")
    larr, locs = _gate_locs(locations)
    if not isinstance(starts, torch.Tensor):
        starts = flatten_gates(starts)
    starts = _c128(starts, "starts")
    if starts.dim() == 1:
        starts = starts.unsqueeze(0)
    n = _nqubits(target)
    S = starts.shape[0]
    if starts.shape[1] != gate_entries(locs):
        raise ValueError("starts do not match the locations' gate sizes")
    opts = options if options is not None else Options(**kw)
    out = torch.empty_like(starts)
    costs = (ct.c_double * S)()
    res = nat.qf_result()
    check(_lib().qf_instantiate_k(_ptr(target), n, len(locs), larr, S, _ptr(starts),
                                  ct.byref(opts.c), _ptr(out), costs, ct.byref(res),
                                  _stream_handle(stream)))
    return {"gates": unflatten_gates(out, locs), "flat": out, "costs": np.array(costs[:]),
            "best": res.best_start, "sweeps": res.sweeps, "c64_sweeps": res.c64_sweeps,
            "reason": nat.REASONS.get(res.reason, str(res.reason)), "best_cost": res.best_cost}


def instantiate_spec(target, specs, params, gates=None, options=None, stream=None, **kw):
    """Lock-step multistart Qfactor over a circuit of specialised gates
    (rz, gpi, ms) and general unitaries (u4, u8) (qf_instantiate_spec).
    ``params``: (S, p, 2) float64 start angles; ``gates``: (S, E) complex128
    start matrices of the general gates (None if there are none).  Returns
    the dict of instantiate_ex with ``params`` (S, p, 2) and ``flat`` the
    (S, E) slot matrices."""
    target = _c128(target, "target")
    specs = [tuple(g) for g in specs]
    sarr = gate_specs(specs)
    n = _nqubits(target)
    pr = params if isinstance(params, torch.Tensor) else torch.as_tensor(np.asarray(params, dtype=np.float64))
    if pr.dtype != torch.float64 or pr.dim() != 3 or pr.shape[1:] != (len(specs), 2):
        raise ValueError("params must be float64 of shape (S, n_gates, 2)")
    pr = pr.contiguous()
    S = pr.shape[0]
    E = sum(64 if g[0].lower() == "u8" else 16 for g in specs)
    g = _c128(gates, "gates") if gates is not None else None
    if g is not None and tuple(g.shape) != (S, E):
        raise ValueError(f"gates must be (S, {E})")
    opts = options if options is not None else Options(**kw)
    out = torch.empty((S, E), dtype=torch.complex128, device=pr.device)
    out_p = torch.empty_like(pr)
    costs = (ct.c_double * S)()
    res = nat.qf_result()
    check(_lib().qf_instantiate_spec(_ptr(target), n, len(specs), sarr, S,
                                     _ptr(g) if g is not None else None, _ptr(pr), ct.byref(opts.c),
                                     _ptr(out), _ptr(out_p), costs, ct.byref(res), _stream_handle(stream)))
    return {"params": out_p, "flat": out, "costs": np.array(costs[:]), "best": res.best_start,
            "sweeps": res.sweeps, "c64_sweeps": res.c64_sweeps,
            "reason": nat.REASONS.get(res.reason, str(res.reason)), "best_cost": res.best_cost}


def apply_gate_k(T, qubits, L=None, R=None, stream=None):
    """In place: T_s <- (L_s on qubits) T_s (R_s on qubits); L, R (S, d, d)."""
    T = _dev(T, "T")
    S, N = _tensor_sn(T)
    n = int(N).bit_length() - 1
    larr, _ = _gate_locs([qubits])
    Lp = _ptr(_dev(_c128(L, "L"), "L")) if L is not None else None
    Rp = _ptr(_dev(_c128(R, "R"), "R")) if R is not None else None
    check(_lib().qf_apply_gate_k(_ptr(T), n, S, larr, Lp, Rp, _tensor_prec(T), _stream_handle(stream)))
    return T


def set_tc_wait_limit(polls):
    """Polls of each tensor-core completion wait for later launches (0: every
    wait runs out at once); returns the previous limit.  polls < 0 only queries."""
    return int(_lib().qf_set_tc_wait_limit(int(polls)))


def partial_trace_k(T, qubits, stream=None):
    T = _dev(T, "T")
    S, N = _tensor_sn(T)
    n = int(N).bit_length() - 1
    d = 2 ** len(tuple(qubits))
    larr, _ = _gate_locs([qubits])
    P = torch.empty((S, d, d), dtype=torch.complex128, device=T.device)
    check(_lib().qf_partial_trace_k(_ptr(T), n, S, larr, _ptr(P), _tensor_prec(T),
                                    _stream_handle(stream)))
    return P


def optimize_gates_k(E, u_old=None, beta=0.0, stream=None):
    """OptimizeGate on (..., d, d) matrices, d = 4, 8 or 16."""
    E = _dev(_c128(E, "E"), "E")
    d = E.shape[-1]
    count = E.numel() // (d * d)
    U = torch.empty_like(E)
    sig = torch.empty(E.shape[:-2], dtype=torch.float64, device=E.device)
    up = _ptr(_dev(_c128(u_old, "u_old"), "u_old")) if u_old is not None else None
    check(_lib().qf_optimize_gates_k(_ptr(E), int(d), up, float(beta), count, _ptr(U), _ptr(sig),
                                     _stream_handle(stream)))
    return U, sig


def init_tensor_k(target, locations, gates, dtype=torch.complex128, stream=None):
    """InitCircuitTensor with 2- and 3-qubit gates; gates (S, E) or S lists."""
    target = _dev(_c128(target, "target"), "target")
    larr, locs = _gate_locs(locations)
    if not isinstance(gates, torch.Tensor):
        gates = flatten_gates(gates)
    g = _c128(gates, "gates").to(target.device)
    if g.dim() == 1:
        g = g.unsqueeze(0)
    n = _nqubits(target)
    prec = QF_DF64 if dtype == "df64" else (QF_C128 if dtype == torch.complex128 else QF_C64)
    T = _empty_tensor(g.shape[0], 1 << n, prec, target.device)
    check(_lib().qf_init_tensor_k(_ptr(target), n, len(locs), larr, g.shape[0], _ptr(g), _ptr(T), prec,
                                  _stream_handle(stream)))
    return T


def circuit_unitary_k(n_qubits, locations, gates, device="cuda", stream=None):
    """C = G_0 ... G_{p-1} for 2- and 3-qubit gates (gates: E entries or a list)."""
    larr, locs = _gate_locs(locations)
    if not isinstance(gates, torch.Tensor):
        gates = flatten_gates([gates])[0]
    g = _c128(gates, "gates").reshape(-1).to(device)
    N = 1 << int(n_qubits)
    C = torch.empty((N, N), dtype=torch.complex128, device=device)
    check(_lib().qf_circuit_unitary_k(int(n_qubits), len(locs), larr, _ptr(g), _ptr(C),
                                      _stream_handle(stream)))
    return C


def partial_trace_noalloc(T, a, b, P=None, stream=None):
    """Like partial_trace, computed by the allocation-free entry point (the
    library allocates nothing; the caller provides the output P, S x 4 x 4
    complex128 on the device, or it is created here)."""
    T = _dev(T, "T")
    S, N = _tensor_sn(T)
    n = int(N).bit_length() - 1
    if P is None:
        P = torch.empty((S, 4, 4), dtype=torch.complex128, device=T.device)
    check(_lib().qf_partial_trace_noalloc(_ptr(T), n, S, int(a), int(b), _ptr(P),
                                          _tensor_prec(T), _stream_handle(stream)))
    return P


def optimize_gates(E, u_old=None, beta=0.0, stream=None):
    E = _dev(_c128(E, "E"), "E")
    count = E.numel() // 16
    U = torch.empty_like(E)
    sig = torch.empty(E.shape[:-2], dtype=torch.float64, device=E.device)
    up = _ptr(_dev(_c128(u_old, "u_old"), "u_old")) if u_old is not None else None
    check(_lib().qf_optimize_gates(_ptr(E), up, float(beta), count, _ptr(U), _ptr(sig),
                                   _stream_handle(stream)))
    return U, sig


def reunitarize_gates(gates, stream=None):
    """In place: three FP64 Newton-Schulz steps on every 4x4 gate (CUDA)."""
    g = _dev(gates, "gates")
    if g.dtype != torch.complex128 or not g.is_contiguous():
        raise TypeError("gates must be a contiguous complex128 CUDA tensor")
    check(_lib().qf_reunitarize_gates(_ptr(g), g.numel() // 16, _stream_handle(stream)))
    return g


def trace(T, stream=None):
    T = _dev(T, "T")
    S, N = _tensor_sn(T)
    n = int(N).bit_length() - 1
    tr = torch.empty((S,), dtype=torch.complex128, device=T.device)
    check(_lib().qf_trace(_ptr(T), n, S, _ptr(tr), _tensor_prec(T), _stream_handle(stream)))
    return tr


def circuit_unitary(n_qubits, locations, gates, device="cuda", stream=None):
    g = _c128(gates, "gates").to(device)
    locs = _locs(locations)
    N = 1 << int(n_qubits)
    C = torch.empty((N, N), dtype=torch.complex128, device=device)
    check(_lib().qf_circuit_unitary(int(n_qubits), g.shape[0], _ptr(locs), _ptr(g), _ptr(C),
                                    _stream_handle(stream)))
    return C
