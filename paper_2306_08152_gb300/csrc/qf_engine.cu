// Host engine of the QFactor library: argument checks, workspace, the sweep
// driver (Alg. 1: TwoSidedSweep inside the Qfactor loop), the stopping rules
// (Sec. III-A2, Sec. IV-A) and the exported C ABI of include/qfactor.h.
//
// Per gate update the engine enqueues two kernels on the caller's stream:
//   update  environment of the gate from the band of the current tensor plus
//           the FP64 4x4 update (one CTA per start);
//   pass    the fused B <- L B R over every 4x4 block of every start's
//           tensor (one read and one write of T).
// Nothing returns to the host inside a sweep; costs are read once per sweep.

#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "qf_internal.h"
#include "qfactor.h"

namespace {

thread_local std::string g_last_error;

// NVTX range for profilers (nsys, ncu --nvtx): one per sweep and per phase
// of an instantiation; free when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

int set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define QF_CUDA(call)                                                          \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess)                                                     \
      return set_error(e_ == cudaErrorMemoryAllocation ? QF_ENOMEM : QF_ECUDA, \
                       "%s failed: %s", #call, cudaGetErrorString(e_));        \
  } while (0)

#define QF_TRY(expr)         \
  do {                       \
    int r_ = (expr);         \
    if (r_ != QF_OK) return r_; \
  } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int check_sizes(int n, int p) {
  if (n < QF_MIN_QUBITS || n > QF_MAX_QUBITS)
    return set_error(QF_EINVAL, "n_qubits=%d outside [%d, %d]", n, QF_MIN_QUBITS, QF_MAX_QUBITS);
  if (p < 1) return set_error(QF_EINVAL, "n_gates=%d must be >= 1", p);
  return QF_OK;
}

int check_prec(int prec) {
  if (prec != QF_C128 && prec != QF_C64 && prec != QF_DF64)
    return set_error(QF_EINVAL, "precision=%d must be QF_C128, QF_C64 or QF_DF64 here", prec);
  return QF_OK;
}

// Tensor precision -> the kernels' precision code (0 complex128, 1 complex64,
// 2 double-FP32).
int kprec(int prec) { return prec == QF_C128 ? 0 : prec == QF_DF64 ? 2 : 1; }

// Copy locations (host or device) to a host vector and validate them.
int fetch_locations(const qf_loc* locs, int n, int p, std::vector<qf_loc>* out) {
  if (!locs) return set_error(QF_EINVAL, "locations is NULL");
  out->resize(p);
  if (is_device_ptr(locs)) {
    QF_CUDA(cudaMemcpy(out->data(), locs, sizeof(qf_loc) * p, cudaMemcpyDeviceToHost));
  } else {
    memcpy(out->data(), locs, sizeof(qf_loc) * p);
  }
  for (int k = 0; k < p; ++k) {
    const qf_loc& l = (*out)[k];
    if (l.a < 0 || l.a >= n || l.b < 0 || l.b >= n || l.a == l.b)
      return set_error(QF_EINVAL, "location %d = (%d, %d) invalid for %d qubits", k, l.a, l.b, n);
  }
  return QF_OK;
}

// A gate of the circuit: size k (2 or 3), its qubits in local-index order,
// and the offset of its 4^k entries within one start's gate array.
struct GateDesc {
  int k;
  int q[4];
  long long off;
  int kind = qf::kGateGeneral;  // parameterised kinds occupy a 4x4 slot (k = 2)
};

int descs_from_pairs(const std::vector<qf_loc>& locs, std::vector<GateDesc>* out, long long* gsz) {
  out->resize(locs.size());
  for (size_t i = 0; i < locs.size(); ++i) {
    (*out)[i] = GateDesc{2, {locs[i].a, locs[i].b, -1, -1}, (long long)i * 16};
  }
  *gsz = (long long)locs.size() * 16;
  return QF_OK;
}

// Copy gate specifications (host or device) and validate them.  RZ and GPI
// act on q[0]; their 4x4 slot pairs it with q[1] (any other qubit), or, for
// q[1] < 0, with q[0] + 1 (q[0] - 1 for the last qubit).
int fetch_gate_specs(const qf_gate_spec* specs, int n, int p, std::vector<GateDesc>* out,
                     long long* gsz) {
  if (!specs) return set_error(QF_EINVAL, "gate specifications are NULL");
  std::vector<qf_gate_spec> h(p);
  if (is_device_ptr(specs)) {
    QF_CUDA(cudaMemcpy(h.data(), specs, sizeof(qf_gate_spec) * p, cudaMemcpyDeviceToHost));
  } else {
    memcpy(h.data(), specs, sizeof(qf_gate_spec) * p);
  }
  out->resize(p);
  long long off = 0;
  for (int i = 0; i < p; ++i) {
    const qf_gate_spec& g = h[i];
    int k = 2, kind = qf::kGateGeneral, q[3] = {g.q[0], g.q[1], -1};
    switch (g.kind) {
      case QF_GATE_U4: break;
      case QF_GATE_U8: k = 3; q[2] = g.q[2]; break;
      case QF_GATE_MS: kind = qf::kGateMs; break;
      case QF_GATE_RZ:
      case QF_GATE_GPI:
        kind = g.kind == QF_GATE_RZ ? qf::kGateRz : qf::kGateGpi;
        if (q[1] < 0) q[1] = q[0] + 1 < n ? q[0] + 1 : q[0] - 1;
        break;
      default: return set_error(QF_EINVAL, "gate %d: unknown kind %d", i, g.kind);
    }
    if (k > n) return set_error(QF_EINVAL, "gate %d: %d qubits > n_qubits=%d", i, k, n);
    for (int a = 0; a < k; ++a) {
      if (q[a] < 0 || q[a] >= n)
        return set_error(QF_EINVAL, "gate %d: qubit %d invalid for %d qubits", i, q[a], n);
      for (int b = 0; b < a; ++b)
        if (q[a] == q[b]) return set_error(QF_EINVAL, "gate %d: repeated qubit %d", i, q[a]);
    }
    (*out)[i] = GateDesc{k, {q[0], q[1], q[2], -1}, off, kind};
    off += k == 3 ? 64 : 16;
  }
  *gsz = off;
  return QF_OK;
}

// Copy k-qubit locations (host or device) and validate them.
int fetch_gate_locs(const qf_gate_loc* locs, int n, int p, std::vector<GateDesc>* out, long long* gsz) {
  if (!locs) return set_error(QF_EINVAL, "locations is NULL");
  std::vector<qf_gate_loc> h(p);
  if (is_device_ptr(locs)) {
    QF_CUDA(cudaMemcpy(h.data(), locs, sizeof(qf_gate_loc) * p, cudaMemcpyDeviceToHost));
  } else {
    memcpy(h.data(), locs, sizeof(qf_gate_loc) * p);
  }
  out->resize(p);
  long long off = 0;
  for (int i = 0; i < p; ++i) {
    const qf_gate_loc& l = h[i];
    if (l.k < 2 || l.k > 4) return set_error(QF_EINVAL, "gate %d: k=%d must be 2, 3 or 4", i, l.k);
    for (int a = 0; a < l.k; ++a) {
      if (l.q[a] < 0 || l.q[a] >= n)
        return set_error(QF_EINVAL, "gate %d: qubit %d invalid for %d qubits", i, l.q[a], n);
      for (int b = 0; b < a; ++b)
        if (l.q[a] == l.q[b]) return set_error(QF_EINVAL, "gate %d: repeated qubit %d", i, l.q[a]);
    }
    if (l.k > n) return set_error(QF_EINVAL, "gate %d: k=%d > n_qubits=%d", i, l.k, n);
    (*out)[i] = GateDesc{l.k, {l.q[0], l.q[1], l.k >= 3 ? l.q[2] : -1, l.k == 4 ? l.q[3] : -1}, off};
    off += 1ll << (2 * l.k);
  }
  *gsz = off;
  return QF_OK;
}

int check_finite_host(const qf_c128* v, size_t count, const char* what) {
  for (size_t i = 0; i < count; ++i)
    if (!std::isfinite(v[i].re) || !std::isfinite(v[i].im))
      return set_error(QF_ENONFINITE, "%s[%zu] is not finite", what, i);
  return QF_OK;
}

// Device buffer owned for the duration of a call.
struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  int alloc(size_t bytes) {
    if (p) {
      cudaFree(p);
      p = nullptr;
    }
    if (bytes == 0) return QF_OK;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return set_error(QF_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    }
    return QF_OK;
  }
  template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

// Make a device copy of a host-or-device input (or borrow it if already on
// the device).  Host inputs are checked for non-finite values.
int stage_input(const qf_c128* src, size_t count, DevBuf* buf, const double2** dev,
                cudaStream_t st, const char* what) {
  if (!src) return set_error(QF_EINVAL, "%s is NULL", what);
  if (is_device_ptr(src)) {
    *dev = reinterpret_cast<const double2*>(src);
    return QF_OK;
  }
  QF_TRY(check_finite_host(src, count, what));
  QF_TRY(buf->alloc(count * sizeof(double2)));
  QF_CUDA(cudaMemcpyAsync(buf->p, src, count * sizeof(double2), cudaMemcpyHostToDevice, st));
  *dev = buf->as<double2>();
  return QF_OK;
}

int store_output(qf_c128* dst, const double2* dev, size_t count, cudaStream_t st) {
  if (!dst) return set_error(QF_EINVAL, "output pointer is NULL");
  if (reinterpret_cast<const void*>(dst) == reinterpret_cast<const void*>(dev)) return QF_OK;
  QF_CUDA(cudaMemcpyAsync(dst, dev, count * sizeof(double2), cudaMemcpyDefault, st));
  return QF_OK;
}

size_t elem_bytes(int prec) { return prec == QF_C64 ? 8 : 16; }

}  // namespace

int qf_internal_set_error(int code, const char* what, const char* detail) {
  if (detail && detail[0]) return set_error(code, "%s: %s", what, detail);
  return set_error(code, "%s", what);
}

int qf_internal_check_sizes(int n_qubits, int n_gates) { return check_sizes(n_qubits, n_gates); }
int qf_internal_check_prec(int precision) { return check_prec(precision); }
int qf_internal_kernel_prec(int precision) { return kprec(precision); }

// ============================================================ the plan

struct qf_plan {
  int n = 0, p = 0, S = 0, prec = QF_C128;
  size_t N = 0, NN = 0;
  std::vector<qf_loc> locs;  // (q0, q1) of every gate
  std::vector<GateDesc> gd;  // size, qubits and entry offset of every gate
  long long gsz = 0;         // gate entries per start
  bool mixed = false;        // some gate acts on three qubits
  DevBuf T, V, gates, LR, sigma, tr, status, part, counters;
  DevBuf LR8, gdesc;         // three-qubit pass operators (start stride 128); gate table
  bool has16 = false;        // some gate acts on four qubits
  DevBuf LR16;               // four-qubit pass operators (start stride 512)
  // parameterised gates: (kind, entry offset) per gate and 2 parameters per
  // (start, gate), start stride 2p
  bool spec = false;
  DevBuf ptab, params;
  size_t T_capacity = 0;  // bytes
  cudaStream_t stream = nullptr;
  long long sweeps_since_load = 0;
  // pass timing
  bool timing = false;
  std::vector<cudaEvent_t> events;  // pairs
  size_t events_used = 0;
  long long pass_launches = 0, all_launches = 0;
  double pass_bytes = 0.0;  // algorithmic bytes (one read + one write) of timed passes
  // start groups: the environment kernels of one group run on s_env while
  // the other group's pass runs on s_pass (passes stay serialised)
  int G = 1;
  cudaStream_t s_env = nullptr, s_pass = nullptr, s_cap = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join_env = nullptr, ev_join_pass = nullptr;
  cudaEvent_t ev_env[2] = {nullptr, nullptr}, ev_pass[2] = {nullptr, nullptr};
  // one sweep captured as a CUDA graph (used when pass timing is off)
  cudaGraphExec_t graph = nullptr;
  double graph_beta = 0.0;
  int graph_prec = -1;
  bool graph_look = false;
  long long graph_pass_launches = 0, graph_all_launches = 0;  // per replay
  bool use_graph = true;
  long long sweeps_enqueued = 0;  // a plan's first sweep runs live (no capture cost for one-sweep uses)
  // look-ahead: consecutive updates on disjoint pairs share one pass
  bool lookahead = false;
  DevBuf LR2;                      // the second update's pass operators
  std::vector<unsigned char> pair_params;  // launch geometry per pair window
  std::vector<int> win_first;      // per half-sweep order position: 1 = starts a pair
  std::vector<int> geo_index;      // per window start (order position): geometry slot
};

namespace {

int plan_ensure_T(qf_plan* P, int prec) {
  const size_t need = (size_t)P->S * P->NN * elem_bytes(prec);
  if (need > P->T_capacity) {
    QF_TRY(P->T.alloc(need));
    P->T_capacity = need;
  }
  P->prec = prec;
  return QF_OK;
}

// A slice of the starts [s0, s0 + Sg) and the stream its work goes to.
struct Slice {
  int s0, Sg;
  cudaStream_t st;
};

Slice all_starts(qf_plan* P, cudaStream_t st) { return Slice{0, P->S, st}; }
Slice all_starts(qf_plan* P) { return all_starts(P, P->stream); }

// Enqueue one pass launch over the slice's tensors; with pass timing on it is
// bracketed by a pair of events and its algorithmic bytes (one read and one
// write of every entry it covers) are counted.
template <typename Launch>
int timed_pass(qf_plan* P, const Slice& sl, Launch launch) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (P->timing) {
    if (P->events_used + 2 > P->events.size()) {
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        QF_CUDA(cudaEventCreate(&e));
        P->events.push_back(e);
      }
    }
    e0 = P->events[P->events_used];
    e1 = P->events[P->events_used + 1];
    P->events_used += 2;
    QF_CUDA(cudaEventRecord(e0, sl.st));
  }
  void* T = static_cast<char*>(P->T.p) + (size_t)sl.s0 * P->NN * elem_bytes(P->prec);
  QF_CUDA(launch(T));
  if (P->timing) {
    QF_CUDA(cudaEventRecord(e1, sl.st));
    P->pass_bytes += 2.0 * (double)sl.Sg * (double)P->NN * (double)elem_bytes(P->prec);
  }
  P->pass_launches++;
  P->all_launches++;
  return QF_OK;
}

int plan_pass(qf_plan* P, const Slice& sl, int a, int b, const double2* L, long long Ls,
              const double2* R, long long Rs) {
  return timed_pass(P, sl, [&](void* T) {
    return qf::launch_pass(T, P->n, sl.Sg, a, b, L ? L + sl.s0 * Ls : nullptr, Ls,
                           R ? R + sl.s0 * Rs : nullptr, Rs, kprec(P->prec), sl.st);
  });
}

// The pass of a three-qubit gate: T <- (L on q) T (R on q), 8x8 operators.
int plan_pass8(qf_plan* P, const Slice& sl, const int* q, const double2* L, long long Ls,
               const double2* R, long long Rs) {
  return timed_pass(P, sl, [&](void* T) {
    return qf::launch_pass8(T, P->n, sl.Sg, q, L ? L + sl.s0 * Ls : nullptr, Ls,
                            R ? R + sl.s0 * Rs : nullptr, Rs, kprec(P->prec), sl.st);
  });
}

// The pass of a four-qubit gate: T <- (L on q) T (R on q), 16x16 operators.
int plan_pass16(qf_plan* P, const Slice& sl, const int* q, const double2* L, long long Ls,
                const double2* R, long long Rs) {
  return timed_pass(P, sl, [&](void* T) {
    return qf::launch_pass16(T, P->n, sl.Sg, q, L ? L + sl.s0 * Ls : nullptr, Ls,
                             R ? R + sl.s0 * Rs : nullptr, Rs, kprec(P->prec), sl.st,
                             P->status.as<int>());
  });
}

// The fused pass of gate k with the operators its update left in LR / LR8 / LR16.
int plan_gate_pass(qf_plan* P, const Slice& sl, int k) {
  if (P->gd[k].k == 4) {
    const double2* L16 = P->LR16.as<double2>();
    return plan_pass16(P, sl, P->gd[k].q, L16, 512, L16 + 256, 512);
  }
  if (P->gd[k].k == 3) {
    const double2* L8 = P->LR8.as<double2>();
    return plan_pass8(P, sl, P->gd[k].q, L8, 128, L8 + 64, 128);
  }
  const double2* LR = P->LR.as<double2>();
  return plan_pass(P, sl, P->locs[k].a, P->locs[k].b, LR, 32, LR + 16, 32);
}

double2* gate_ptr(qf_plan* P, int s0, int k) {
  return P->gates.as<double2>() + (size_t)s0 * P->gsz + P->gd[k].off;
}

// InitCircuitTensor (Alg. 1) for every start.
int plan_build(qf_plan* P) {
  const int pr = kprec(P->prec);
  QF_CUDA(qf::launch_conj_transpose(P->V.as<double2>(), P->T.p, P->n, P->S, pr, P->stream));
  P->all_launches++;
  if (!P->mixed && qf::build_rows_supported(P->n, P->p, pr)) {
    std::vector<int> pa(P->p), pb(P->p);
    for (int k = 0; k < P->p; ++k) {
      pa[k] = qf::qubit_bit(P->n, P->locs[k].a);
      pb[k] = qf::qubit_bit(P->n, P->locs[k].b);
    }
    QF_CUDA(qf::launch_build_rows(P->T.p, P->n, P->S, P->p, pa.data(), pb.data(),
                                  P->gates.as<double2>(), P->gsz, P->stream));
    P->all_launches++;
    return QF_OK;
  }
  for (int k = 0; k < P->p; ++k) {
    if (P->gd[k].k == 4)
      QF_TRY(plan_pass16(P, all_starts(P), P->gd[k].q, nullptr, 0, gate_ptr(P, 0, k), P->gsz));
    else if (P->gd[k].k == 3)
      QF_TRY(plan_pass8(P, all_starts(P), P->gd[k].q, nullptr, 0, gate_ptr(P, 0, k), P->gsz));
    else
      QF_TRY(plan_pass(P, all_starts(P), P->locs[k].a, P->locs[k].b, nullptr, 0, gate_ptr(P, 0, k),
                       P->gsz));
  }
  return QF_OK;
}

// Kernel nodes captured into a graph do not take the capturing stream's
// priority; give the kernel just captured on st (an environment kernel) that
// priority explicitly, so that a replayed sweep keeps the overlap of one
// group's environment with the other group's pass.
int mark_stream_priority(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  QF_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &nd));
  if (cs != cudaStreamCaptureStatusActive) return QF_OK;
  int prio = 0;
  QF_CUDA(cudaStreamGetPriority(st, &prio));
  cudaLaunchAttributeValue v;
  memset(&v, 0, sizeof(v));
  v.priority = prio;
  for (size_t i = 0; i < nd; ++i) {
    cudaGraphNodeType t;
    QF_CUDA(cudaGraphNodeGetType(deps[i], &t));
    if (t == cudaGraphNodeTypeKernel)
      QF_CUDA(cudaGraphKernelNodeSetAttribute(deps[i], cudaLaunchAttributePriority, &v));
  }
  return QF_OK;
}

int plan_update(qf_plan* P, const Slice& sl, int k, int mode, double beta, double2* env_out,
                long long env_stride) {
  const int pr = kprec(P->prec);
  const int B = qf::env_ctas(P->n);
  const void* T = static_cast<const char*>(P->T.p) + (size_t)sl.s0 * P->NN * elem_bytes(P->prec);
  if (P->gd[k].k == 4) {
    QF_CUDA(qf::launch_update16(
        T, P->n, sl.Sg, P->gd[k].q, gate_ptr(P, sl.s0, k), P->gsz, mode, beta,
        P->LR16.as<double2>() + (size_t)sl.s0 * 512, env_out ? env_out + sl.s0 * env_stride : nullptr,
        env_stride, P->sigma.as<double>() + sl.s0, P->status.as<int>(),
        P->part.as<double>() + (size_t)sl.s0 * B * 512, P->counters.as<unsigned>() + sl.s0, pr,
        sl.st));
    P->all_launches++;
    return mark_stream_priority(sl.st);
  }
  if (P->gd[k].k == 3) {
    QF_CUDA(qf::launch_update8(
        T, P->n, sl.Sg, P->gd[k].q, gate_ptr(P, sl.s0, k), P->gsz, mode, beta,
        P->LR8.as<double2>() + (size_t)sl.s0 * 128, env_out ? env_out + sl.s0 * env_stride : nullptr,
        env_stride, P->sigma.as<double>() + sl.s0, P->status.as<int>(),
        P->part.as<double>() + (size_t)sl.s0 * B * 128, P->counters.as<unsigned>() + sl.s0, pr,
        sl.st));
    P->all_launches++;
    return mark_stream_priority(sl.st);
  }
  const int kind = P->gd[k].kind;
  double* prm = kind == qf::kGateGeneral ? nullptr
                                         : P->params.as<double>() + (size_t)sl.s0 * 2 * P->p + 2 * k;
  QF_CUDA(qf::launch_update(
      T, P->n, sl.Sg, P->locs[k].a, P->locs[k].b, gate_ptr(P, sl.s0, k), P->gsz,
      mode, beta, P->LR.as<double2>() + (size_t)sl.s0 * 32,
      env_out ? env_out + sl.s0 * env_stride : nullptr, env_stride,
      P->sigma.as<double>() + sl.s0, P->status.as<int>(),
      P->part.as<double>() + (size_t)sl.s0 * B * 32, P->counters.as<unsigned>() + sl.s0, pr, sl.st,
      kind, prm, 2LL * P->p));
  P->all_launches++;
  return mark_stream_priority(sl.st);
}

// Look-ahead update of gate k2, whose environment sees the pending update of
// gate k1 (operators in LR) through the light cone; its own operators go to LR2.
int plan_update_look(qf_plan* P, const Slice& sl, int k1, int k2, int mode, double beta) {
  const int pr = kprec(P->prec);
  const int B = qf::env_ctas(P->n);
  const void* T = static_cast<const char*>(P->T.p) + (size_t)sl.s0 * P->NN * elem_bytes(P->prec);
  const double2* LR = P->LR.as<double2>() + (size_t)sl.s0 * 32;
  QF_CUDA(qf::launch_update_lookahead(
      T, P->n, sl.Sg, P->locs[k1].a, P->locs[k1].b, LR, LR + 16, 32, P->locs[k2].a, P->locs[k2].b,
      gate_ptr(P, sl.s0, k2), P->gsz,
      mode, beta, P->LR2.as<double2>() + (size_t)sl.s0 * 32, nullptr, 0,
      P->sigma.as<double>() + sl.s0, P->status.as<int>(),
      P->part.as<double>() + (size_t)sl.s0 * B * 32, P->counters.as<unsigned>() + sl.s0, pr, sl.st));
  P->all_launches++;
  return mark_stream_priority(sl.st);
}

// The pass of a look-ahead window: both updates' operators in one pass.
int plan_pair_pass(qf_plan* P, const Slice& sl, int slot) {
  const double2* LR = P->LR.as<double2>() + (size_t)sl.s0 * 32;
  const double2* LR2 = P->LR2.as<double2>() + (size_t)sl.s0 * 32;
  const void* pp = P->pair_params.data() + (size_t)slot * qf::pair_params_bytes();
  return timed_pass(P, sl, [&](void* T) {
    return qf::launch_pair_pass(T, P->n, sl.Sg, pp, LR, LR + 16, 32, LR2, LR2 + 16, 32, sl.st);
  });
}

// Gate order of half-sweep h (0 = backward k = p-1..0, 1 = forward k = 0..p-1).
int order_gate(const qf_plan* P, int h, int i) { return h == 0 ? P->p - 1 - i : i; }

bool disjoint(const qf_loc& x, const qf_loc& y) {
  return x.a != y.a && x.a != y.b && x.b != y.a && x.b != y.b;
}

// Windows of both half-sweeps: greedily pair position i with i+1 when their
// gates act on disjoint pairs and the tiled pass supports the case, and
// prepare one launch geometry per pair.
int plan_windows(qf_plan* P) {
  if (!P->win_first.empty()) return QF_OK;
  P->win_first.assign(2 * P->p, 0);
  P->geo_index.assign(2 * P->p, -1);
  int slots = 0;
  for (int h = 0; h < 2; ++h)
    for (int i = 0; i + 1 < P->p;) {
      const qf_loc& x = P->locs[order_gate(P, h, i)];
      const qf_loc& y = P->locs[order_gate(P, h, i + 1)];
      if (disjoint(x, y) && qf::pair_pass_supported(P->n, x.a, x.b, y.a, y.b, 1)) {
        P->win_first[h * P->p + i] = 1;
        P->geo_index[h * P->p + i] = slots++;
        i += 2;
      } else {
        i += 1;
      }
    }
  P->pair_params.assign((size_t)slots * qf::pair_params_bytes(), 0);
  for (int h = 0; h < 2; ++h)
    for (int i = 0; i < P->p; ++i) {
      const int slot = P->geo_index[h * P->p + i];
      if (slot < 0) continue;
      const qf_loc& x = P->locs[order_gate(P, h, i)];
      const qf_loc& y = P->locs[order_gate(P, h, i + 1)];
      qf::make_pair_params(P->n, x.a, x.b, y.a, y.b,
                           P->pair_params.data() + (size_t)slot * qf::pair_params_bytes());
    }
  if (!P->LR2.p) QF_TRY(P->LR2.alloc((size_t)P->S * 32 * sizeof(double2)));
  return QF_OK;
}

bool plan_uses_lookahead(const qf_plan* P) {
  return P->lookahead && !P->mixed && !P->spec && P->prec == QF_C64 && P->n >= 8;
}

int plan_streams(qf_plan* P) {
  if (P->s_env) return QF_OK;
  // the environment stream has the higher priority: its CTAs take the SM
  // slots that the running pass's CTAs free, so that a pass that fills every
  // SM does not hold the other group's environment back until it ends
  int lo = 0, hi = 0;
  QF_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
  QF_CUDA(cudaStreamCreateWithPriority(&P->s_env, cudaStreamNonBlocking, hi));
  QF_CUDA(cudaStreamCreateWithPriority(&P->s_pass, cudaStreamNonBlocking, lo));
  QF_CUDA(cudaStreamCreateWithFlags(&P->s_cap, cudaStreamNonBlocking));
  cudaEvent_t* evs[] = {&P->ev_fork, &P->ev_join_env, &P->ev_join_pass, &P->ev_env[0],
                        &P->ev_env[1], &P->ev_pass[0], &P->ev_pass[1]};
  for (cudaEvent_t* e : evs) QF_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  return QF_OK;
}

// TwoSidedSweep (Alg. 1).  Backward half: for k = p-1..0 the environment of
// gate k (still on the tensor's right), its update, and the pass that
// removes u_k from the right and applies u_k' on the left.  Forward half:
// the mirror image, k = 0..p-1.  With two start groups the environment
// kernels go to s_env and the passes to s_pass, so the environment of one
// group overlaps the pass of the other:
//   env_0(u) | pass_0(u) + env_1(u) | pass_1(u) + env_0(u+1) | ...
//
// With look-ahead on, a window of two consecutive updates on disjoint pairs
// runs as: the first gate's environment and update (operators -> LR), the
// second gate's environment through the first's pending update and its
// update (-> LR2), then one pass applying both; the sweep's result is that
// of the single-update order, up to rounding.
int enqueue_window(qf_plan* P, const Slice& env_sl, const Slice& pass_sl, int h, int i,
                   double beta, bool look) {
  const int k = order_gate(P, h, i);
  const int mode = h == 0 ? qf::kBackward : qf::kForward;
  QF_TRY(plan_update(P, env_sl, k, mode, beta, nullptr, 0));
  if (look && P->win_first[h * P->p + i]) {
    const int k2 = order_gate(P, h, i + 1);
    QF_TRY(plan_update_look(P, env_sl, k, k2, mode, beta));
    if (env_sl.st != pass_sl.st) return QF_OK;  // the caller forks to the pass stream
    return plan_pair_pass(P, pass_sl, P->geo_index[h * P->p + i]);
  }
  if (env_sl.st != pass_sl.st) return QF_OK;
  return plan_gate_pass(P, pass_sl, k);
}

int enqueue_window_pass(qf_plan* P, const Slice& pass_sl, int h, int i, bool look) {
  if (look && P->win_first[h * P->p + i]) return plan_pair_pass(P, pass_sl, P->geo_index[h * P->p + i]);
  const int k = order_gate(P, h, i);
  return plan_gate_pass(P, pass_sl, k);
}

int enqueue_sweep(qf_plan* P, double beta, cudaStream_t origin) {
  const bool look = plan_uses_lookahead(P);
  if (look) QF_TRY(plan_windows(P));
  if (look) {
    if (P->G == 1) {
      const Slice sl = all_starts(P, origin);
      for (int h = 0; h < 2; ++h)
        for (int i = 0; i < P->p; i += (P->win_first[h * P->p + i] ? 2 : 1))
          QF_TRY(enqueue_window(P, sl, sl, h, i, beta, true));
      return QF_OK;
    }
    QF_TRY(plan_streams(P));
    const int half = P->S / 2;
    const Slice env_sl[2] = {{0, half, P->s_env}, {half, P->S - half, P->s_env}};
    const Slice pass_sl[2] = {{0, half, P->s_pass}, {half, P->S - half, P->s_pass}};
    QF_CUDA(cudaEventRecord(P->ev_fork, origin));
    QF_CUDA(cudaStreamWaitEvent(P->s_env, P->ev_fork, 0));
    QF_CUDA(cudaStreamWaitEvent(P->s_pass, P->ev_fork, 0));
    bool first = true;
    for (int h = 0; h < 2; ++h)
      for (int i = 0; i < P->p; i += (P->win_first[h * P->p + i] ? 2 : 1)) {
        for (int g = 0; g < 2; ++g) {
          if (!first) QF_CUDA(cudaStreamWaitEvent(P->s_env, P->ev_pass[g], 0));
          QF_TRY(enqueue_window(P, env_sl[g], pass_sl[g], h, i, beta, true));
          QF_CUDA(cudaEventRecord(P->ev_env[g], P->s_env));
          QF_CUDA(cudaStreamWaitEvent(P->s_pass, P->ev_env[g], 0));
          QF_TRY(enqueue_window_pass(P, pass_sl[g], h, i, true));
          QF_CUDA(cudaEventRecord(P->ev_pass[g], P->s_pass));
        }
        first = false;
      }
    QF_CUDA(cudaEventRecord(P->ev_join_env, P->s_env));
    QF_CUDA(cudaEventRecord(P->ev_join_pass, P->s_pass));
    QF_CUDA(cudaStreamWaitEvent(origin, P->ev_join_env, 0));
    QF_CUDA(cudaStreamWaitEvent(origin, P->ev_join_pass, 0));
    return QF_OK;
  }
  if (P->G == 1) {
    const Slice sl = all_starts(P, origin);
    for (int k = P->p - 1; k >= 0; --k) {
      QF_TRY(plan_update(P, sl, k, qf::kBackward, beta, nullptr, 0));
      QF_TRY(plan_gate_pass(P, sl, k));
    }
    for (int k = 0; k < P->p; ++k) {
      QF_TRY(plan_update(P, sl, k, qf::kForward, beta, nullptr, 0));
      QF_TRY(plan_gate_pass(P, sl, k));
    }
    return QF_OK;
  }
  QF_TRY(plan_streams(P));
  const int half = P->S / 2;
  const Slice env_sl[2] = {{0, half, P->s_env}, {half, P->S - half, P->s_env}};
  const Slice pass_sl[2] = {{0, half, P->s_pass}, {half, P->S - half, P->s_pass}};
  QF_CUDA(cudaEventRecord(P->ev_fork, origin));
  QF_CUDA(cudaStreamWaitEvent(P->s_env, P->ev_fork, 0));
  QF_CUDA(cudaStreamWaitEvent(P->s_pass, P->ev_fork, 0));
  for (int u = 0; u < 2 * P->p; ++u) {
    const bool backward = u < P->p;
    const int k = backward ? P->p - 1 - u : u - P->p;
    for (int g = 0; g < 2; ++g) {
      if (u > 0) QF_CUDA(cudaStreamWaitEvent(P->s_env, P->ev_pass[g], 0));
      QF_TRY(plan_update(P, env_sl[g], k, backward ? qf::kBackward : qf::kForward, beta, nullptr, 0));
      QF_CUDA(cudaEventRecord(P->ev_env[g], P->s_env));
      QF_CUDA(cudaStreamWaitEvent(P->s_pass, P->ev_env[g], 0));
      QF_TRY(plan_gate_pass(P, pass_sl[g], k));
      QF_CUDA(cudaEventRecord(P->ev_pass[g], P->s_pass));
    }
  }
  QF_CUDA(cudaEventRecord(P->ev_join_env, P->s_env));
  QF_CUDA(cudaEventRecord(P->ev_join_pass, P->s_pass));
  QF_CUDA(cudaStreamWaitEvent(origin, P->ev_join_env, 0));
  QF_CUDA(cudaStreamWaitEvent(origin, P->ev_join_pass, 0));
  return QF_OK;
}

// One sweep: live launches when pass timing is on (every pass bracketed by
// events), otherwise the sweep is captured once as a CUDA graph per (beta,
// precision) and replayed.
int plan_sweep_once(qf_plan* P, double beta) {
  // the first sweep of a plan runs as live launches: capturing and
  // instantiating the graph costs more than it saves for a single sweep
  if (P->timing || !P->use_graph || P->sweeps_enqueued++ == 0) return enqueue_sweep(P, beta, P->stream);
  const bool look = plan_uses_lookahead(P);
  if (!P->graph || P->graph_beta != beta || P->graph_prec != P->prec || P->graph_look != look) {
    if (P->graph) {
      cudaGraphExecDestroy(P->graph);
      P->graph = nullptr;
    }
    QF_TRY(plan_streams(P));
    if (look) QF_TRY(plan_windows(P));  // allocates: not inside the capture
    // captured on an internal stream (the caller's may be the legacy default
    // stream, which cannot be captured), launched on the caller's stream
    const long long pl = P->pass_launches, al = P->all_launches;
    cudaGraph_t g = nullptr;
    QF_CUDA(cudaStreamBeginCapture(P->s_cap, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue_sweep(P, beta, P->s_cap);
    const cudaError_t e = cudaStreamEndCapture(P->s_cap, &g);
    if (rc != QF_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return set_error(QF_ECUDA, "sweep capture failed: %s", cudaGetErrorString(e));
    // the environment kernels carry a higher node priority (mark_stream_priority)
    const cudaError_t ei = cudaGraphInstantiate(&P->graph, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess)
      return set_error(QF_ECUDA, "sweep graph instantiation failed: %s", cudaGetErrorString(ei));
    P->graph_beta = beta;
    P->graph_prec = P->prec;
    P->graph_look = look;
    P->graph_pass_launches = P->pass_launches - pl;  // what one replay launches
    P->graph_all_launches = P->all_launches - al;
    P->pass_launches = pl;  // capture launches nothing
    P->all_launches = al;
  }
  QF_CUDA(cudaGraphLaunch(P->graph, P->stream));
  P->pass_launches += P->graph_pass_launches;
  P->all_launches += P->graph_all_launches;
  return QF_OK;
}

int plan_costs_impl(qf_plan* P, double* costs, qf_c128* traces) {
  const int pr = kprec(P->prec);
  QF_CUDA(qf::launch_trace(P->T.p, P->n, P->S, P->tr.as<double2>(), pr, P->stream));
  P->all_launches++;
  std::vector<double2> h(P->S);
  QF_CUDA(cudaMemcpyAsync(h.data(), P->tr.p, sizeof(double2) * P->S, cudaMemcpyDeviceToHost,
                          P->stream));
  QF_CUDA(cudaStreamSynchronize(P->stream));
  for (int s = 0; s < P->S; ++s) {
    if (costs) costs[s] = 1.0 - std::hypot(h[s].x, h[s].y) / (double)P->N;
    if (traces) {
      traces[s].re = h[s].x;
      traces[s].im = h[s].y;
    }
  }
  return QF_OK;
}

int plan_create_desc(int n, const std::vector<GateDesc>& gd, long long gsz, int S, int prec,
                     qf_plan** out, bool with_params = false) {
  if (!out) return set_error(QF_EINVAL, "out_plan is NULL");
  *out = nullptr;
  const int p = (int)gd.size();
  QF_TRY(check_sizes(n, p));
  QF_TRY(check_prec(prec));
  if (S < 1) return set_error(QF_EINVAL, "n_starts=%d must be >= 1", S);
  qf_plan* P = new qf_plan();
  P->n = n;
  P->p = p;
  P->S = S;
  P->G = S >= 2 ? 2 : 1;
  P->N = (size_t)1 << n;
  P->NN = P->N * P->N;
  P->gd = gd;
  P->gsz = gsz;
  P->locs.resize(p);
  for (int k = 0; k < p; ++k) {
    P->locs[k] = qf_loc{gd[k].q[0], gd[k].q[1]};
    if (gd[k].k >= 3) P->mixed = true;
    if (gd[k].k == 4) P->has16 = true;
  }
  // partial sums per environment CTA: 16, 64 or 256 complex values
  const int part_per_cta = P->has16 ? 512 : P->mixed ? 128 : 32;
  const int B = qf::env_ctas(n);
  int rc = plan_ensure_T(P, prec);
  if (rc == QF_OK) rc = P->V.alloc(P->NN * sizeof(double2));
  if (rc == QF_OK) rc = P->gates.alloc((size_t)S * gsz * sizeof(double2));
  if (rc == QF_OK) rc = P->LR.alloc((size_t)S * 32 * sizeof(double2));
  if (rc == QF_OK) rc = P->sigma.alloc((size_t)S * sizeof(double));
  if (rc == QF_OK) rc = P->tr.alloc((size_t)S * sizeof(double2));
  if (rc == QF_OK) rc = P->status.alloc(sizeof(int));
  if (rc == QF_OK) rc = P->part.alloc((size_t)S * B * part_per_cta * sizeof(double));
  if (rc == QF_OK) rc = P->counters.alloc((size_t)S * sizeof(unsigned));
  if (rc == QF_OK && P->has16) rc = P->LR16.alloc((size_t)S * 512 * sizeof(double2));
  if (rc == QF_OK && P->mixed) {
    rc = P->LR8.alloc((size_t)S * 128 * sizeof(double2));
    // (k, entry offset) per gate, for the re-unitarisation kernel
    std::vector<int2> tab(p);
    for (int k = 0; k < p; ++k) tab[k] = make_int2(gd[k].k, (int)gd[k].off);
    if (rc == QF_OK) rc = P->gdesc.alloc(sizeof(int2) * p);
    if (rc == QF_OK && cudaMemcpy(P->gdesc.p, tab.data(), sizeof(int2) * p, cudaMemcpyHostToDevice) !=
                           cudaSuccess)
      rc = set_error(QF_ECUDA, "copying the gate table failed");
  }
  P->spec = with_params;
  for (int k = 0; k < p; ++k) P->spec |= gd[k].kind != qf::kGateGeneral;
  if (rc == QF_OK && P->spec) {
    // parameterised gates: (kind, entry offset) per gate, 2 parameters per (start, gate)
    std::vector<int2> tab(p);
    for (int k = 0; k < p; ++k) tab[k] = make_int2(gd[k].kind, (int)gd[k].off);
    rc = P->ptab.alloc(sizeof(int2) * p);
    if (rc == QF_OK) rc = P->params.alloc(sizeof(double) * 2 * p * (size_t)S);
    if (rc == QF_OK &&
        (cudaMemcpy(P->ptab.p, tab.data(), sizeof(int2) * p, cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemset(P->params.p, 0, sizeof(double) * 2 * p * (size_t)S) != cudaSuccess))
      rc = set_error(QF_ECUDA, "copying the gate kinds failed");
  }
  if (rc == QF_OK && (cudaMemset(P->status.p, 0, sizeof(int)) != cudaSuccess ||
                      cudaMemset(P->counters.p, 0, (size_t)S * sizeof(unsigned)) != cudaSuccess))
    rc = set_error(QF_ECUDA, "cudaMemset of the plan's status words failed");
  if (rc != QF_OK) {
    delete P;
    return rc;
  }
  *out = P;
  return QF_OK;
}

int plan_create_impl(int n, int p, const qf_loc* locs, int S, int prec, qf_plan** out) {
  if (!out) return set_error(QF_EINVAL, "out_plan is NULL");
  *out = nullptr;
  QF_TRY(check_sizes(n, p));
  std::vector<qf_loc> l;
  QF_TRY(fetch_locations(locs, n, p, &l));
  std::vector<GateDesc> gd;
  long long gsz = 0;
  QF_TRY(descs_from_pairs(l, &gd, &gsz));
  return plan_create_desc(n, gd, gsz, S, prec, out);
}

int plan_load_impl(qf_plan* P, const qf_c128* target, const qf_c128* gates, cudaStream_t st) {
  P->stream = st;
  if (!target || !gates) return set_error(QF_EINVAL, "target or gates is NULL");
  const size_t gcount = (size_t)P->S * P->gsz;
  QF_CUDA(cudaMemcpyAsync(P->V.p, target, P->NN * sizeof(double2), cudaMemcpyDefault, st));
  QF_CUDA(cudaMemcpyAsync(P->gates.p, gates, gcount * sizeof(double2), cudaMemcpyDefault, st));
  QF_CUDA(cudaMemsetAsync(P->status.p, 0, sizeof(int), st));
  // non-finite inputs raise the status word (read at the next status check)
  QF_CUDA(qf::launch_check_finite(P->V.as<double>(), P->NN * 2, P->status.as<int>(), st));
  QF_CUDA(qf::launch_check_finite(P->gates.as<double>(), gcount * 2, P->status.as<int>(), st));
  P->sweeps_since_load = 0;
  return plan_build(P);
}

// Load for plans with parameterised gates: the general gates' matrices (the
// parameterised slots are ignored; gates may be NULL when every gate is
// parameterised), the parameters, then the parameterised slots built from
// them, then the tensors.
int plan_load_spec_impl(qf_plan* P, const qf_c128* target, const qf_c128* gates, const double* params,
                        cudaStream_t st) {
  if (!target || !params) return set_error(QF_EINVAL, "target or params is NULL");
  bool general = false;
  for (const GateDesc& g : P->gd) general |= g.kind == qf::kGateGeneral;
  if (general && !gates) return set_error(QF_EINVAL, "gates is NULL but the circuit has general gates");
  P->stream = st;
  const size_t gcount = (size_t)P->S * P->gsz;
  const size_t pcount = (size_t)P->S * 2 * P->p;
  QF_CUDA(cudaMemcpyAsync(P->V.p, target, P->NN * sizeof(double2), cudaMemcpyDefault, st));
  if (gates)
    QF_CUDA(cudaMemcpyAsync(P->gates.p, gates, gcount * sizeof(double2), cudaMemcpyDefault, st));
  else
    QF_CUDA(cudaMemsetAsync(P->gates.p, 0, gcount * sizeof(double2), st));
  QF_CUDA(cudaMemcpyAsync(P->params.p, params, pcount * sizeof(double), cudaMemcpyDefault, st));
  QF_CUDA(cudaMemsetAsync(P->status.p, 0, sizeof(int), st));
  QF_CUDA(qf::launch_check_finite(P->params.as<double>(), pcount, P->status.as<int>(), st));
  QF_CUDA(qf::launch_param_gates(P->gates.as<double2>(), P->gsz, P->ptab.as<int2>(), P->params.as<double>(),
                                 2LL * P->p, P->p, P->S, st));
  QF_CUDA(qf::launch_check_finite(P->V.as<double>(), P->NN * 2, P->status.as<int>(), st));
  QF_CUDA(qf::launch_check_finite(P->gates.as<double>(), gcount * 2, P->status.as<int>(), st));
  P->sweeps_since_load = 0;
  return plan_build(P);
}

// The periodic reset (Sec. III-A2, reset_iter): re-unitarise every gate in
// FP64, then rebuild every tensor from V and the gates.
int plan_reset(qf_plan* P) {
  if (P->mixed)
    QF_CUDA(qf::launch_reunitarize_mixed(P->gates.as<double2>(), P->gsz, P->gdesc.as<int2>(), P->p,
                                         P->S, P->stream));
  else
    QF_CUDA(qf::launch_reunitarize(P->gates.as<double2>(), P->S * P->p, P->stream));
  P->all_launches++;
  if (P->has16) {  // the mixed kernel leaves 16x16 gates to this one
    QF_CUDA(qf::launch_reunitarize16(P->gates.as<double2>(), P->gsz, P->gdesc.as<int2>(), P->p, P->S,
                                     P->stream));
    P->all_launches++;
  }
  if (P->spec) {  // parameterised gates: exactly G(theta) again
    QF_CUDA(qf::launch_param_gates(P->gates.as<double2>(), P->gsz, P->ptab.as<int2>(),
                                   P->params.as<double>(), 2LL * P->p, P->p, P->S, P->stream));
    P->all_launches++;
  }
  return plan_build(P);
}

int plan_sweep_impl(qf_plan* P, int n_sweeps, int reset_iter, double beta) {
  for (int i = 0; i < n_sweeps; ++i) {
    NvtxRange r("qf sweep");
    QF_TRY(plan_sweep_once(P, beta));
    P->sweeps_since_load++;
    if (reset_iter > 0 && P->sweeps_since_load % reset_iter == 0) {
      NvtxRange rr("qf reset");
      QF_TRY(plan_reset(P));
    }
  }
  return QF_OK;
}

int plan_status_impl(qf_plan* P) {
  int st = 0;
  QF_CUDA(cudaMemcpyAsync(&st, P->status.p, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
  QF_CUDA(cudaStreamSynchronize(P->stream));
  if (st == QF_ETIMEOUT) return set_error(st, "a tensor-core completion wait ran out in a 16x16 pass");
  if (st != 0) return set_error(st, "an environment or update was not finite");
  return QF_OK;
}

// Plateau tests of Sec. III-A2 (readings documented in qfactor.h).
bool plateau(const std::vector<double>& h, int it, const qf_options& o) {
  const double c = h.back();
  if ((o.diff_tol_a > 0.0 || o.diff_tol_r > 0.0) && h.size() >= 2) {
    if (h[h.size() - 2] - c <= o.diff_tol_a + o.diff_tol_r * c) return true;
  }
  const int L = o.long_diff_count;
  if (L > 0 && it >= L) {
    const double old = h[h.size() - 1 - L];
    if (old - c < o.long_diff_r * old) return true;
  }
  return false;
}

struct PlanGuard {
  qf_plan* p = nullptr;
  ~PlanGuard() {
    if (p) qf_plan_destroy(p);
  }
};

}  // namespace

// ============================================================ C ABI

extern "C" {

const char* qf_last_error(void) { return g_last_error.c_str(); }

int qf_version(void) { return 200; }

int qf_options_default(qf_options* o) {
  if (!o) return set_error(QF_EINVAL, "opts is NULL");
  o->dist_tol = 1e-10;
  o->max_sweeps = 500;
  o->min_sweeps = 0;
  o->reset_iter = 40;
  o->long_diff_count = 0;
  o->diff_tol_a = 0.0;
  o->diff_tol_r = 0.0;
  o->long_diff_r = 0.1;
  o->beta = 0.0;
  o->precision = QF_C128;
  o->max_c64_sweeps = 1000;
  o->switch_tol = 1e-6;
  o->cost_history = nullptr;
  return QF_OK;
}

int qf_plan_create(int n_qubits, int n_gates, const qf_loc* locations, int n_starts,
                   int precision, qf_plan** out_plan) {
  return plan_create_impl(n_qubits, n_gates, locations, n_starts, precision, out_plan);
}

int qf_plan_destroy(qf_plan* plan) {
  if (!plan) return QF_OK;
  if (plan->stream) cudaStreamSynchronize(plan->stream);
  for (cudaEvent_t e : plan->events) cudaEventDestroy(e);
  if (plan->graph) cudaGraphExecDestroy(plan->graph);
  cudaEvent_t evs[] = {plan->ev_fork, plan->ev_join_env, plan->ev_join_pass, plan->ev_env[0],
                       plan->ev_env[1], plan->ev_pass[0], plan->ev_pass[1]};
  for (cudaEvent_t e : evs)
    if (e) cudaEventDestroy(e);
  if (plan->s_env) cudaStreamDestroy(plan->s_env);
  if (plan->s_pass) cudaStreamDestroy(plan->s_pass);
  if (plan->s_cap) cudaStreamDestroy(plan->s_cap);
  delete plan;
  return QF_OK;
}

int qf_plan_load(qf_plan* plan, const qf_c128* target, const qf_c128* gates, void* stream) {
  if (!plan) return set_error(QF_EINVAL, "plan is NULL");
  return plan_load_impl(plan, target, gates, as_stream(stream));
}

int qf_plan_sweep(qf_plan* plan, int n_sweeps, int reset_iter, double beta) {
  if (!plan) return set_error(QF_EINVAL, "plan is NULL");
  if (n_sweeps < 0) return set_error(QF_EINVAL, "n_sweeps=%d < 0", n_sweeps);
  return plan_sweep_impl(plan, n_sweeps, reset_iter, beta);
}

int qf_plan_rebuild(qf_plan* plan, int precision) {
  if (!plan) return set_error(QF_EINVAL, "plan is NULL");
  QF_TRY(check_prec(precision));
  if (precision != plan->prec) {
    QF_CUDA(cudaStreamSynchronize(plan->stream));
    QF_TRY(plan_ensure_T(plan, precision));
  }
  return plan_build(plan);
}

int qf_plan_costs(qf_plan* plan, double* out_costs, qf_c128* out_trace) {
  if (!plan) return set_error(QF_EINVAL, "plan is NULL");
  return plan_costs_impl(plan, out_costs, out_trace);
}

int qf_plan_get_gates(qf_plan* plan, qf_c128* out) {
  if (!plan) return set_error(QF_EINVAL, "plan is NULL");
  QF_TRY(store_output(out, plan->gates.as<double2>(), (size_t)plan->S * plan->gsz, plan->stream));
  QF_CUDA(cudaStreamSynchronize(plan->stream));
  return QF_OK;
}

int qf_plan_set_lookahead(qf_plan* plan, int enable) {
  if (!plan) return set_error(QF_EINVAL, "plan is NULL");
  plan->lookahead = enable != 0;
  if (plan->lookahead) QF_TRY(plan_windows(plan));
  return QF_OK;
}

int qf_plan_lookahead_windows(qf_plan* plan, int* pairs_per_sweep) {
  if (!plan || !pairs_per_sweep) return set_error(QF_EINVAL, "NULL argument");
  *pairs_per_sweep = 0;
  if (!plan_uses_lookahead(plan)) return QF_OK;
  QF_TRY(plan_windows(plan));
  for (int v : plan->win_first) *pairs_per_sweep += v;
  return QF_OK;
}

int qf_plan_enable_pass_timing(qf_plan* plan, int enable) {
  if (!plan) return set_error(QF_EINVAL, "plan is NULL");
  plan->timing = enable != 0;
  return QF_OK;
}

int qf_plan_pass_stats(qf_plan* plan, double* pass_ms, int64_t* pass_launches,
                       int64_t* all_launches, double* pass_bytes) {
  if (!plan) return set_error(QF_EINVAL, "plan is NULL");
  QF_CUDA(cudaStreamSynchronize(plan->stream));
  double ms = 0.0;
  for (size_t i = 0; i + 1 < plan->events_used; i += 2) {
    float t = 0.f;
    QF_CUDA(cudaEventElapsedTime(&t, plan->events[i], plan->events[i + 1]));
    ms += t;
  }
  if (pass_ms) *pass_ms = ms;
  if (pass_launches) *pass_launches = plan->pass_launches;
  if (all_launches) *all_launches = plan->all_launches;
  if (pass_bytes) *pass_bytes = plan->pass_bytes;
  plan->events_used = 0;
  plan->pass_launches = 0;
  plan->all_launches = 0;
  plan->pass_bytes = 0.0;
  return QF_OK;
}

int qf_plan_status(qf_plan* plan) {
  if (!plan) return set_error(QF_EINVAL, "plan is NULL");
  return plan_status_impl(plan);
}

// A complex64 run whose best cost stalls at or below this switches to FP64
// (the complex64 noise floor is ~1e-7); above it the stall is the method's
// own plateau.
constexpr double kStallSwitchCost = 1e-5;

}  // extern "C"

namespace {

int instantiate_core(const qf_c128* target, int n_qubits, const std::vector<GateDesc>& gd,
                     long long gsz, int n_starts, const qf_c128* initial_gates,
                     const qf_options* opts, qf_c128* out_gates, double* out_costs,
                     qf_result* out_result, void* stream, const double* initial_params = nullptr,
                     double* out_params = nullptr) {
  qf_options o;
  qf_options_default(&o);
  if (opts) o = *opts;
  QF_TRY(check_sizes(n_qubits, (int)gd.size()));
  if (n_starts < 1) return set_error(QF_EINVAL, "n_starts=%d must be >= 1", n_starts);
  if (o.max_sweeps < 1) return set_error(QF_EINVAL, "max_sweeps=%d must be >= 1", o.max_sweeps);
  if (o.precision != QF_C128 && o.precision != QF_C64 && o.precision != QF_C64_REFINE64 &&
      o.precision != QF_DF64 && o.precision != QF_C64_REFINE_DF)
    return set_error(QF_EINVAL, "precision=%d unknown", o.precision);
  if (!(o.beta >= 0.0 && o.beta <= 1.0))
    return set_error(QF_EINVAL, "beta=%g outside [0, 1]", o.beta);
  if (!out_gates) return set_error(QF_EINVAL, "out_gates is NULL");
  cudaStream_t st = as_stream(stream);
  const int S = n_starts;

  PlanGuard g;
  const bool refine = o.precision == QF_C64_REFINE64 || o.precision == QF_C64_REFINE_DF;
  // the precision of the final (or only) phase
  const int fine_prec = o.precision == QF_C64_REFINE_DF || o.precision == QF_DF64 ? QF_DF64
                        : o.precision == QF_C64                                   ? QF_C64
                                                                                  : QF_C128;
  const int tensor_prec = refine ? QF_C64 : fine_prec;
  QF_TRY(plan_create_desc(n_qubits, gd, gsz, S, tensor_prec, &g.p));
  qf_plan* P = g.p;
  if (refine) {
    // reserve the 16-byte tensor up front so the switch cannot fail late
    QF_TRY(plan_ensure_T(P, fine_prec));
    P->prec = QF_C64;
  }
  if (P->spec)
    QF_TRY(plan_load_spec_impl(P, target, initial_gates, initial_params, st));
  else
    QF_TRY(plan_load_impl(P, target, initial_gates, st));

  std::vector<std::vector<double>> hist(S);
  std::vector<double> c(S);
  QF_TRY(plan_costs_impl(P, c.data(), nullptr));
  QF_TRY(plan_status_impl(P));  // non-finite target or start gates
  for (int s = 0; s < S; ++s) hist[s].push_back(c[s]);
  std::vector<char> plateaued(S, 0);
  bool c64_phase = refine;
  int reason = QF_STOP_MAX_SWEEPS, it = 0, c64_sweeps = 0;
  nvtxRangePushA(c64_phase ? "qf bulk complex64 phase" : "qf sweeps");
  for (it = 1; it <= o.max_sweeps; ++it) {
    NvtxRange sweep_range("qf sweep");
    QF_TRY(plan_sweep_once(P, o.beta));
    P->sweeps_since_load++;
    if (o.reset_iter > 0 && P->sweeps_since_load % o.reset_iter == 0) QF_TRY(plan_reset(P));
    QF_TRY(plan_costs_impl(P, c.data(), nullptr));
    QF_TRY(plan_status_impl(P));
    if (c64_phase) {
      ++c64_sweeps;
      // leave complex64 once the best cost is below switch_tol, or once ten
      // c64 sweeps have lowered every start's cost by less than the
      // complex64 noise floor (1e-7) while the best cost is near that floor
      // (<= 1e-5; a stall above it is the method's own plateau, which FP64
      // sweeps do not lift)
      double best = c[0];
      bool stalled = hist[0].size() > 10;
      for (int s = 0; s < S; ++s) {
        best = std::min(best, c[s]);
        if (hist[s].size() > 10 && hist[s][hist[s].size() - 10] - c[s] >= 1e-7) stalled = false;
      }
      for (int s = 0; s < S; ++s) hist[s].push_back(c[s]);
      if (best <= o.switch_tol || (stalled && best <= kStallSwitchCost) ||
          c64_sweeps >= o.max_c64_sweeps) {
        // rebuild every tensor in the fine precision from V and the FP64 gates
        nvtxRangePop();
        NvtxRange sw("qf switch to the fine precision");
        nvtxRangePushA("qf refinement phase");
        P->prec = fine_prec;
        QF_TRY(plan_build(P));
        QF_TRY(plan_costs_impl(P, c.data(), nullptr));
        for (int s = 0; s < S; ++s) hist[s].back() = c[s];
        c64_phase = false;
      } else {
        // the plateau rules apply in the complex64 phase too
        if (it >= o.min_sweeps) {
          bool all = true;
          for (int s = 0; s < S; ++s) {
            if (plateau(hist[s], it, o)) plateaued[s] = 1;
            all = all && plateaued[s];
          }
          if (all) {
            reason = QF_STOP_PLATEAU;
            break;
          }
        }
        continue;
      }
    } else {
      for (int s = 0; s < S; ++s) hist[s].push_back(c[s]);
    }
    if (it >= o.min_sweeps) {
      bool conv = false;
      for (int s = 0; s < S; ++s) conv = conv || (c[s] <= o.dist_tol);
      if (conv) {
        reason = QF_STOP_CONVERGED;
        break;
      }
      bool all = true;
      for (int s = 0; s < S; ++s) {
        if (plateau(hist[s], it, o)) plateaued[s] = 1;
        all = all && plateaued[s];
      }
      if (all) {
        reason = QF_STOP_PLATEAU;
        break;
      }
    }
  }
  nvtxRangePop();
  if (it > o.max_sweeps) it = o.max_sweeps;
  if (c64_phase) {  // report FP64 traces of fine tensors: rebuild once
    P->prec = fine_prec;
    QF_TRY(plan_build(P));
    QF_TRY(plan_costs_impl(P, c.data(), nullptr));
  }
  if (o.cost_history) {  // [start][sweep], NaN after a start's last sweep
    const size_t row = (size_t)o.max_sweeps + 1;
    std::vector<double> h((size_t)S * row, std::nan(""));
    for (int s = 0; s < S; ++s)
      for (size_t i = 0; i < hist[s].size() && i < row; ++i) h[s * row + i] = hist[s][i];
    QF_CUDA(cudaMemcpyAsync(o.cost_history, h.data(), h.size() * sizeof(double), cudaMemcpyDefault, st));
    QF_CUDA(cudaStreamSynchronize(st));  // h is released at the end of this block
  }
  int best = 0;
  for (int s = 1; s < S; ++s)
    if (c[s] < c[best]) best = s;
  QF_TRY(store_output(out_gates, P->gates.as<double2>(), (size_t)S * gsz, st));
  if (P->spec && out_params)
    QF_TRY(store_output(reinterpret_cast<qf_c128*>(out_params), P->params.as<double2>(),
                        (size_t)S * P->p, st));
  QF_CUDA(cudaStreamSynchronize(st));
  if (out_costs)
    for (int s = 0; s < S; ++s) out_costs[s] = c[s];
  if (out_result) {
    out_result->best_start = best;
    out_result->sweeps = it;
    out_result->c64_sweeps = c64_sweeps;
    out_result->reason = reason;
    out_result->best_cost = c[best];
  }
  return QF_OK;
}

}  // namespace

extern "C" {

int qf_instantiate_ex(const qf_c128* target, int n_qubits, int n_gates,
                      const qf_loc* locations, int n_starts, const qf_c128* initial_gates,
                      const qf_options* opts, qf_c128* out_gates, double* out_costs,
                      qf_result* out_result, void* stream) {
  QF_TRY(check_sizes(n_qubits, n_gates));
  std::vector<qf_loc> l;
  QF_TRY(fetch_locations(locations, n_qubits, n_gates, &l));
  std::vector<GateDesc> gd;
  long long gsz = 0;
  QF_TRY(descs_from_pairs(l, &gd, &gsz));
  return instantiate_core(target, n_qubits, gd, gsz, n_starts, initial_gates, opts, out_gates,
                          out_costs, out_result, stream);
}

int qf_instantiate_k(const qf_c128* target, int n_qubits, int n_gates,
                     const qf_gate_loc* locations, int n_starts, const qf_c128* initial_gates,
                     const qf_options* opts, qf_c128* out_gates, double* out_costs,
                     qf_result* out_result, void* stream) {
  QF_TRY(check_sizes(n_qubits, n_gates));
  std::vector<GateDesc> gd;
  long long gsz = 0;
  QF_TRY(fetch_gate_locs(locations, n_qubits, n_gates, &gd, &gsz));
  return instantiate_core(target, n_qubits, gd, gsz, n_starts, initial_gates, opts, out_gates,
                          out_costs, out_result, stream);
}

int qf_plan_create_k(int n_qubits, int n_gates, const qf_gate_loc* locations, int n_starts,
                     int precision, qf_plan** out_plan) {
  if (out_plan) *out_plan = nullptr;
  QF_TRY(check_sizes(n_qubits, n_gates));
  std::vector<GateDesc> gd;
  long long gsz = 0;
  QF_TRY(fetch_gate_locs(locations, n_qubits, n_gates, &gd, &gsz));
  return plan_create_desc(n_qubits, gd, gsz, n_starts, precision, out_plan);
}

int qf_instantiate_spec(const qf_c128* target, int n_qubits, int n_gates, const qf_gate_spec* gates,
                        int n_starts, const qf_c128* initial_gates, const double* initial_params,
                        const qf_options* opts, qf_c128* out_gates, double* out_params,
                        double* out_costs, qf_result* out_result, void* stream) {
  QF_TRY(check_sizes(n_qubits, n_gates));
  if (!initial_params || !out_params) return set_error(QF_EINVAL, "initial_params or out_params is NULL");
  std::vector<GateDesc> gd;
  long long gsz = 0;
  QF_TRY(fetch_gate_specs(gates, n_qubits, n_gates, &gd, &gsz));
  bool param = false;
  for (const GateDesc& g : gd) param |= g.kind != qf::kGateGeneral;
  if (!param) {  // all general: the parameters pass through
    QF_TRY(instantiate_core(target, n_qubits, gd, gsz, n_starts, initial_gates, opts, out_gates,
                            out_costs, out_result, stream));
    if (out_params != initial_params)
      QF_CUDA(cudaMemcpy(out_params, initial_params, sizeof(double) * 2 * n_gates * (size_t)n_starts,
                         cudaMemcpyDefault));
    return QF_OK;
  }
  return instantiate_core(target, n_qubits, gd, gsz, n_starts, initial_gates, opts, out_gates, out_costs,
                          out_result, stream, initial_params, out_params);
}

int qf_plan_create_spec(int n_qubits, int n_gates, const qf_gate_spec* gates, int n_starts,
                        int precision, qf_plan** out_plan) {
  if (out_plan) *out_plan = nullptr;
  QF_TRY(check_sizes(n_qubits, n_gates));
  std::vector<GateDesc> gd;
  long long gsz = 0;
  QF_TRY(fetch_gate_specs(gates, n_qubits, n_gates, &gd, &gsz));
  // parameter buffers even for an all-general circuit, so the parameter calls stay valid
  return plan_create_desc(n_qubits, gd, gsz, n_starts, precision, out_plan, true);
}

int qf_plan_load_spec(qf_plan* plan, const qf_c128* target, const qf_c128* gates,
                      const double* params, void* stream) {
  if (!plan) return set_error(QF_EINVAL, "plan is NULL");
  if (!plan->spec) return set_error(QF_EINVAL, "the plan was not made by qf_plan_create_spec");
  return plan_load_spec_impl(plan, target, gates, params, as_stream(stream));
}

int qf_plan_get_params(qf_plan* plan, double* out_params) {
  if (!plan) return set_error(QF_EINVAL, "plan is NULL");
  if (!plan->spec) return set_error(QF_EINVAL, "the plan was not made by qf_plan_create_spec");
  QF_TRY(store_output(reinterpret_cast<qf_c128*>(out_params), plan->params.as<double2>(),
                      (size_t)plan->S * plan->p, plan->stream));
  QF_CUDA(cudaStreamSynchronize(plan->stream));
  return QF_OK;
}

int qf_plan_gate_entries(qf_plan* plan, int64_t* entries_per_start) {
  if (!plan || !entries_per_start) return set_error(QF_EINVAL, "NULL argument");
  *entries_per_start = plan->gsz;
  return QF_OK;
}

int qf_instantiate(const qf_c128* target, int n_qubits, int n_gates, const qf_loc* locations,
                   const qf_c128* initial_gates, double tol, int max_sweeps,
                   qf_c128* out_gates, double* out_cost, int* out_sweeps, void* stream) {
  qf_options o;
  qf_options_default(&o);
  o.dist_tol = tol;
  o.max_sweeps = max_sweeps;
  qf_result r;
  double cost = 0.0;
  QF_TRY(qf_instantiate_ex(target, n_qubits, n_gates, locations, 1, initial_gates, &o, out_gates,
                           &cost, &r, stream));
  if (out_cost) *out_cost = cost;
  if (out_sweeps) *out_sweeps = r.sweeps;
  return QF_OK;
}

namespace {

// The adjoint walk shared by qf_cost_and_env and qf_cost_grad: build every
// tensor, take its trace, then move each gate from the tensor's right to its
// left (one pass, L = u, R = u^dagger), reading its environment on the way.
// With `grad`, the environments are turned into cost gradients on the device.
// The adjoint walk: build T = V^dagger C once, then for k = p-1 .. 0 read the
// environment of gate k (still on T's right: E_k = P u^dagger, kEnvOnly) and
// move the gate to T's left with one pass (L = u, R = u^dagger), so that
// T = G_k..G_{p-1} V^dagger G_0..G_{k-1} when gate k-1 is read.
int adjoint_walk_desc(const qf_c128* target, int n_qubits, const std::vector<GateDesc>& gd,
                      long long gsz, int n_sets, const qf_c128* gates, double* out_cost,
                      qf_c128* out_env, qf_c128* out_trace, bool grad, void* stream) {
  QF_TRY(check_sizes(n_qubits, (int)gd.size()));
  if (n_sets < 1) return set_error(QF_EINVAL, "n_sets=%d must be >= 1", n_sets);
  if (!out_env) return set_error(QF_EINVAL, "output array is NULL");
  cudaStream_t st = as_stream(stream);
  const int S = n_sets, p = (int)gd.size();
  PlanGuard g;
  QF_TRY(plan_create_desc(n_qubits, gd, gsz, S, QF_C128, &g.p));
  qf_plan* P = g.p;
  QF_TRY(plan_load_impl(P, target, gates, st));
  std::vector<double> c(S);
  std::vector<qf_c128> tr(S);
  QF_TRY(plan_costs_impl(P, c.data(), tr.data()));
  // environments land in a device buffer laid out like out_env
  DevBuf envb;
  double2* env_dev = nullptr;
  const size_t ecount = (size_t)S * gsz;
  const bool out_on_device = is_device_ptr(out_env);
  if (out_on_device) {
    env_dev = reinterpret_cast<double2*>(out_env);
  } else {
    QF_TRY(envb.alloc(ecount * sizeof(double2)));
    env_dev = envb.as<double2>();
  }
  for (int k = p - 1; k >= 0; --k) {
    QF_TRY(plan_update(P, all_starts(P), k, qf::kEnvOnly, 0.0, env_dev + gd[k].off, gsz));
    if (k > 0) QF_TRY(plan_gate_pass(P, all_starts(P), k));
  }
  if (grad) {
    if (P->mixed)
      QF_CUDA(qf::launch_grad_from_env_k(env_dev, P->tr.as<double2>(), n_qubits, S, gsz,
                                         P->gdesc.as<int2>(), p, st));
    else
      QF_CUDA(qf::launch_grad_from_env(env_dev, P->tr.as<double2>(), n_qubits, S, p, st));
  }
  if (!out_on_device)
    QF_CUDA(cudaMemcpyAsync(out_env, env_dev, ecount * sizeof(double2), cudaMemcpyDeviceToHost,
                            st));
  QF_CUDA(cudaStreamSynchronize(st));
  if (out_cost)
    for (int s = 0; s < S; ++s) out_cost[s] = c[s];
  if (out_trace)
    for (int s = 0; s < S; ++s) out_trace[s] = tr[s];
  return QF_OK;
}

int adjoint_walk(const qf_c128* target, int n_qubits, int n_gates, const qf_loc* locations,
                 int n_sets, const qf_c128* gates, double* out_cost, qf_c128* out_env,
                 qf_c128* out_trace, bool grad, void* stream) {
  QF_TRY(check_sizes(n_qubits, n_gates));
  std::vector<qf_loc> l;
  QF_TRY(fetch_locations(locations, n_qubits, n_gates, &l));
  std::vector<GateDesc> gd;
  long long gsz = 0;
  QF_TRY(descs_from_pairs(l, &gd, &gsz));
  return adjoint_walk_desc(target, n_qubits, gd, gsz, n_sets, gates, out_cost, out_env, out_trace,
                           grad, stream);
}

int adjoint_walk_k(const qf_c128* target, int n_qubits, int n_gates, const qf_gate_loc* locations,
                   int n_sets, const qf_c128* gates, double* out_cost, qf_c128* out_env,
                   qf_c128* out_trace, bool grad, void* stream) {
  QF_TRY(check_sizes(n_qubits, n_gates));
  std::vector<GateDesc> gd;
  long long gsz = 0;
  QF_TRY(fetch_gate_locs(locations, n_qubits, n_gates, &gd, &gsz));
  return adjoint_walk_desc(target, n_qubits, gd, gsz, n_sets, gates, out_cost, out_env, out_trace,
                           grad, stream);
}

}  // namespace

int qf_cost_and_env(const qf_c128* target, int n_qubits, int n_gates, const qf_loc* locations,
                    int n_sets, const qf_c128* gates, double* out_cost, qf_c128* out_env,
                    qf_c128* out_trace, void* stream) {
  return adjoint_walk(target, n_qubits, n_gates, locations, n_sets, gates, out_cost, out_env,
                      out_trace, false, stream);
}

int qf_cost_grad(const qf_c128* target, int n_qubits, int n_gates, const qf_loc* locations,
                 int n_sets, const qf_c128* gates, double* out_cost, qf_c128* out_grad,
                 void* stream) {
  return adjoint_walk(target, n_qubits, n_gates, locations, n_sets, gates, out_cost, out_grad,
                      nullptr, true, stream);
}

int qf_cost_and_env_k(const qf_c128* target, int n_qubits, int n_gates,
                      const qf_gate_loc* locations, int n_sets, const qf_c128* gates,
                      double* out_cost, qf_c128* out_env, qf_c128* out_trace, void* stream) {
  return adjoint_walk_k(target, n_qubits, n_gates, locations, n_sets, gates, out_cost, out_env,
                        out_trace, false, stream);
}

int qf_cost_grad_k(const qf_c128* target, int n_qubits, int n_gates, const qf_gate_loc* locations,
                   int n_sets, const qf_c128* gates, double* out_cost, qf_c128* out_grad,
                   void* stream) {
  return adjoint_walk_k(target, n_qubits, n_gates, locations, n_sets, gates, out_cost, out_grad,
                        nullptr, true, stream);
}

// ------------------------------------------------------------ single steps

int qf_init_tensor(const qf_c128* target, int n_qubits, int n_gates, const qf_loc* locations,
                   int n_starts, const qf_c128* gates, void* T, int precision, void* stream) {
  QF_TRY(check_sizes(n_qubits, n_gates));
  QF_TRY(check_prec(precision));
  if (n_starts < 1) return set_error(QF_EINVAL, "n_starts=%d must be >= 1", n_starts);
  if (!target || !gates || !T) return set_error(QF_EINVAL, "NULL device pointer");
  std::vector<qf_loc> locs;
  QF_TRY(fetch_locations(locations, n_qubits, n_gates, &locs));
  cudaStream_t st = as_stream(stream);
  const int pr = kprec(precision);
  QF_CUDA(qf::launch_conj_transpose(reinterpret_cast<const double2*>(target), T, n_qubits,
                                    n_starts, pr, st));
  if (qf::build_rows_supported(n_qubits, n_gates, pr)) {
    std::vector<int> pa(n_gates), pb(n_gates);
    for (int k = 0; k < n_gates; ++k) {
      pa[k] = qf::qubit_bit(n_qubits, locs[k].a);
      pb[k] = qf::qubit_bit(n_qubits, locs[k].b);
    }
    QF_CUDA(qf::launch_build_rows(T, n_qubits, n_starts, n_gates, pa.data(), pb.data(),
                                  reinterpret_cast<const double2*>(gates), (long long)n_gates * 16,
                                  st));
    return QF_OK;
  }
  for (int k = 0; k < n_gates; ++k)
    QF_CUDA(qf::launch_pass(T, n_qubits, n_starts, locs[k].a, locs[k].b, nullptr, 0,
                            reinterpret_cast<const double2*>(gates) + (size_t)k * 16,
                            (long long)n_gates * 16, pr, st));
  return QF_OK;
}

int qf_apply_pair(void* T, int n_qubits, int n_starts, int a, int b, const qf_c128* L,
                  const qf_c128* R, int precision, void* stream) {
  QF_TRY(check_sizes(n_qubits, 1));
  QF_TRY(check_prec(precision));
  if (n_starts < 1) return set_error(QF_EINVAL, "n_starts=%d must be >= 1", n_starts);
  if (!T) return set_error(QF_EINVAL, "T is NULL");
  if (a < 0 || a >= n_qubits || b < 0 || b >= n_qubits || a == b)
    return set_error(QF_EINVAL, "location (%d, %d) invalid for %d qubits", a, b, n_qubits);
  QF_CUDA(qf::launch_pass(T, n_qubits, n_starts, a, b, reinterpret_cast<const double2*>(L), 16,
                          reinterpret_cast<const double2*>(R), 16, kprec(precision),
                          as_stream(stream)));
  return QF_OK;
}

int qf_partial_trace(const void* T, int n_qubits, int n_starts, int a, int b, qf_c128* P,
                     int precision, void* stream) {
  QF_TRY(check_sizes(n_qubits, 1));
  QF_TRY(check_prec(precision));
  if (n_starts < 1) return set_error(QF_EINVAL, "n_starts=%d must be >= 1", n_starts);
  if (!T || !P) return set_error(QF_EINVAL, "NULL device pointer");
  if (a < 0 || a >= n_qubits || b < 0 || b >= n_qubits || a == b)
    return set_error(QF_EINVAL, "location (%d, %d) invalid for %d qubits", a, b, n_qubits);
  // stream-ordered scratch for the environment kernel's cross-CTA partials
  cudaStream_t st = as_stream(stream);
  const size_t part_bytes = (size_t)n_starts * qf::env_ctas(n_qubits) * 32 * sizeof(double);
  const size_t cnt_bytes = (size_t)n_starts * sizeof(unsigned);
  void* scratch = nullptr;
  QF_CUDA(cudaMallocAsync(&scratch, part_bytes + cnt_bytes, st));
  unsigned* counters = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(scratch) + part_bytes);
  cudaError_t e = cudaMemsetAsync(counters, 0, cnt_bytes, st);
  if (e == cudaSuccess)
    e = qf::launch_update(T, n_qubits, n_starts, a, b, nullptr, 0, qf::kTraceOnly, 0.0, nullptr,
                          reinterpret_cast<double2*>(P), 16, nullptr, nullptr,
                          reinterpret_cast<double*>(scratch), counters,
                          kprec(precision), st);
  cudaError_t e2 = cudaFreeAsync(scratch, st);
  if (e != cudaSuccess) return set_error(QF_ECUDA, "partial trace launch failed: %s", cudaGetErrorString(e));
  if (e2 != cudaSuccess) return set_error(QF_ECUDA, "cudaFreeAsync failed: %s", cudaGetErrorString(e2));
  return QF_OK;
}

int qf_apply_two_pairs(void* T, int n_qubits, int n_starts, int a1, int b1, const qf_c128* L1,
                       const qf_c128* R1, int a2, int b2, const qf_c128* L2, const qf_c128* R2,
                       int precision, void* stream) {
  QF_TRY(check_sizes(n_qubits, 1));
  QF_TRY(check_prec(precision));
  if (n_starts < 1) return set_error(QF_EINVAL, "n_starts=%d must be >= 1", n_starts);
  if (!T || !L1 || !R1 || !L2 || !R2) return set_error(QF_EINVAL, "NULL device pointer");
  const int q[4] = {a1, b1, a2, b2};
  for (int i = 0; i < 4; ++i) {
    if (q[i] < 0 || q[i] >= n_qubits)
      return set_error(QF_EINVAL, "qubit %d invalid for %d qubits", q[i], n_qubits);
    for (int j = 0; j < i; ++j)
      if (q[i] == q[j]) return set_error(QF_EINVAL, "the two pairs must be four distinct qubits");
  }
  cudaStream_t st = as_stream(stream);
  const int pr = kprec(precision);
  auto d = [](const qf_c128* x) { return reinterpret_cast<const double2*>(x); };
  if (!qf::pair_pass_supported(n_qubits, a1, b1, a2, b2, pr)) {
    // the two single-pair passes in order
    QF_CUDA(qf::launch_pass(T, n_qubits, n_starts, a1, b1, d(L1), 16, d(R1), 16, pr, st));
    QF_CUDA(qf::launch_pass(T, n_qubits, n_starts, a2, b2, d(L2), 16, d(R2), 16, pr, st));
    return QF_OK;
  }
  std::vector<unsigned char> pp(qf::pair_params_bytes());
  qf::make_pair_params(n_qubits, a1, b1, a2, b2, pp.data());
  QF_CUDA(qf::launch_pair_pass(T, n_qubits, n_starts, pp.data(), d(L1), d(R1), 16, d(L2), d(R2), 16,
                               st));
  return QF_OK;
}

int qf_partial_trace_after(const void* T, int n_qubits, int n_starts, int a1, int b1,
                           const qf_c128* L1, const qf_c128* R1, int a, int b, qf_c128* P,
                           int precision, void* stream) {
  QF_TRY(check_sizes(n_qubits, 1));
  QF_TRY(check_prec(precision));
  if (n_qubits < 4) return set_error(QF_EINVAL, "n_qubits=%d: two disjoint pairs need >= 4", n_qubits);
  if (n_starts < 1) return set_error(QF_EINVAL, "n_starts=%d must be >= 1", n_starts);
  if (!T || !L1 || !R1 || !P) return set_error(QF_EINVAL, "NULL device pointer");
  const int q[4] = {a1, b1, a, b};
  for (int i = 0; i < 4; ++i) {
    if (q[i] < 0 || q[i] >= n_qubits)
      return set_error(QF_EINVAL, "qubit %d invalid for %d qubits", q[i], n_qubits);
    for (int j = 0; j < i; ++j)
      if (q[i] == q[j]) return set_error(QF_EINVAL, "the two pairs must be four distinct qubits");
  }
  cudaStream_t st = as_stream(stream);
  const size_t part_bytes = (size_t)n_starts * qf::env_ctas(n_qubits) * 32 * sizeof(double);
  const size_t cnt_bytes = (size_t)n_starts * sizeof(unsigned);
  void* scratch = nullptr;
  QF_CUDA(cudaMallocAsync(&scratch, part_bytes + cnt_bytes, st));
  unsigned* counters = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(scratch) + part_bytes);
  cudaError_t e = cudaMemsetAsync(counters, 0, cnt_bytes, st);
  if (e == cudaSuccess)
    e = qf::launch_update_lookahead(
        T, n_qubits, n_starts, a1, b1, reinterpret_cast<const double2*>(L1),
        reinterpret_cast<const double2*>(R1), 16, a, b, nullptr, 0, qf::kTraceOnly, 0.0, nullptr,
        reinterpret_cast<double2*>(P), 16, nullptr, nullptr, reinterpret_cast<double*>(scratch),
        counters, kprec(precision), st);
  const cudaError_t e2 = cudaFreeAsync(scratch, st);
  if (e != cudaSuccess) return set_error(QF_ECUDA, "partial trace launch failed: %s", cudaGetErrorString(e));
  if (e2 != cudaSuccess) return set_error(QF_ECUDA, "cudaFreeAsync failed: %s", cudaGetErrorString(e2));
  return QF_OK;
}

int qf_optimize_gates(const qf_c128* E, const qf_c128* u_old, double beta, int count,
                      qf_c128* u_out, double* sigma_out, void* stream) {
  if (count < 0) return set_error(QF_EINVAL, "count=%d < 0", count);
  if (count == 0) return QF_OK;
  if (!E || !u_out) return set_error(QF_EINVAL, "NULL device pointer");
  if (beta != 0.0 && !u_old) return set_error(QF_EINVAL, "beta != 0 needs u_old");
  if (!(beta >= 0.0 && beta <= 1.0)) return set_error(QF_EINVAL, "beta=%g outside [0, 1]", beta);
  QF_CUDA(qf::launch_optimize(reinterpret_cast<const double2*>(E),
                              reinterpret_cast<const double2*>(u_old), beta, count,
                              reinterpret_cast<double2*>(u_out), sigma_out, as_stream(stream)));
  return QF_OK;
}

int qf_reunitarize_gates(qf_c128* gates, int count, void* stream) {
  if (count < 0) return set_error(QF_EINVAL, "count=%d < 0", count);
  if (count == 0) return QF_OK;
  if (!gates) return set_error(QF_EINVAL, "gates is NULL");
  QF_CUDA(qf::launch_reunitarize(reinterpret_cast<double2*>(gates), count, as_stream(stream)));
  return QF_OK;
}

int qf_convert_tensor(const void* src, int src_precision, void* dst, int dst_precision,
                      int64_t count, void* stream) {
  QF_TRY(check_prec(src_precision));
  QF_TRY(check_prec(dst_precision));
  if (count < 0) return set_error(QF_EINVAL, "count=%lld < 0", (long long)count);
  if (count == 0) return QF_OK;
  if (!src || !dst) return set_error(QF_EINVAL, "NULL device pointer");
  const char* s0 = static_cast<const char*>(src);
  const char* d0 = static_cast<const char*>(dst);
  const size_t sb = (size_t)count * elem_bytes(src_precision);
  const size_t db = (size_t)count * elem_bytes(dst_precision);
  if (s0 < d0 + db && d0 < s0 + sb && !(s0 == d0 && src_precision == dst_precision))
    return set_error(QF_EINVAL, "src and dst overlap");
  QF_CUDA(qf::launch_convert(src, kprec(src_precision), dst, kprec(dst_precision), (size_t)count,
                             as_stream(stream)));
  return QF_OK;
}

int qf_trace(const void* T, int n_qubits, int n_starts, qf_c128* tr_out, int precision,
             void* stream) {
  QF_TRY(check_sizes(n_qubits, 1));
  QF_TRY(check_prec(precision));
  if (n_starts < 1) return set_error(QF_EINVAL, "n_starts=%d must be >= 1", n_starts);
  if (!T || !tr_out) return set_error(QF_EINVAL, "NULL device pointer");
  QF_CUDA(qf::launch_trace(T, n_qubits, n_starts, reinterpret_cast<double2*>(tr_out),
                           kprec(precision), as_stream(stream)));
  return QF_OK;
}

// ------------------------------------------------------ k-qubit steps

int qf_apply_gate_k(void* T, int n_qubits, int n_starts, const qf_gate_loc* location,
                    const qf_c128* L, const qf_c128* R, int precision, void* stream) {
  QF_TRY(check_sizes(n_qubits, 1));
  QF_TRY(check_prec(precision));
  if (n_starts < 1) return set_error(QF_EINVAL, "n_starts=%d must be >= 1", n_starts);
  if (!T) return set_error(QF_EINVAL, "T is NULL");
  std::vector<GateDesc> gd;
  long long gsz = 0;
  QF_TRY(fetch_gate_locs(location, n_qubits, 1, &gd, &gsz));
  const auto d = [](const qf_c128* x) { return reinterpret_cast<const double2*>(x); };
  if (gd[0].k == 4)
    QF_CUDA(qf::launch_pass16(T, n_qubits, n_starts, gd[0].q, d(L), 256, d(R), 256, kprec(precision),
                              as_stream(stream)));
  else if (gd[0].k == 3)
    QF_CUDA(qf::launch_pass8(T, n_qubits, n_starts, gd[0].q, d(L), 64, d(R), 64, kprec(precision),
                             as_stream(stream)));
  else
    QF_CUDA(qf::launch_pass(T, n_qubits, n_starts, gd[0].q[0], gd[0].q[1], d(L), 16, d(R), 16,
                            kprec(precision), as_stream(stream)));
  return QF_OK;
}

int qf_partial_trace_k(const void* T, int n_qubits, int n_starts, const qf_gate_loc* location,
                       qf_c128* P, int precision, void* stream) {
  QF_TRY(check_sizes(n_qubits, 1));
  QF_TRY(check_prec(precision));
  if (n_starts < 1) return set_error(QF_EINVAL, "n_starts=%d must be >= 1", n_starts);
  if (!T || !P) return set_error(QF_EINVAL, "NULL device pointer");
  std::vector<GateDesc> gd;
  long long gsz = 0;
  QF_TRY(fetch_gate_locs(location, n_qubits, 1, &gd, &gsz));
  if (gd[0].k == 2)
    return qf_partial_trace(T, n_qubits, n_starts, gd[0].q[0], gd[0].q[1], P, precision, stream);
  cudaStream_t st = as_stream(stream);
  const int per_cta = gd[0].k == 4 ? 512 : 128;
  const size_t part_bytes = (size_t)n_starts * qf::env_ctas(n_qubits) * per_cta * sizeof(double);
  const size_t cnt_bytes = (size_t)n_starts * sizeof(unsigned);
  void* scratch = nullptr;
  QF_CUDA(cudaMallocAsync(&scratch, part_bytes + cnt_bytes, st));
  unsigned* counters = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(scratch) + part_bytes);
  cudaError_t e = cudaMemsetAsync(counters, 0, cnt_bytes, st);
  if (e == cudaSuccess && gd[0].k == 4)
    e = qf::launch_update16(T, n_qubits, n_starts, gd[0].q, nullptr, 0, qf::kTraceOnly, 0.0, nullptr,
                            reinterpret_cast<double2*>(P), 256, nullptr, nullptr,
                            reinterpret_cast<double*>(scratch), counters, kprec(precision), st);
  else if (e == cudaSuccess)
    e = qf::launch_update8(T, n_qubits, n_starts, gd[0].q, nullptr, 0, qf::kTraceOnly, 0.0, nullptr,
                           reinterpret_cast<double2*>(P), 64, nullptr, nullptr,
                           reinterpret_cast<double*>(scratch), counters, kprec(precision), st);
  const cudaError_t e2 = cudaFreeAsync(scratch, st);
  if (e != cudaSuccess) return set_error(QF_ECUDA, "partial trace launch failed: %s", cudaGetErrorString(e));
  if (e2 != cudaSuccess) return set_error(QF_ECUDA, "cudaFreeAsync failed: %s", cudaGetErrorString(e2));
  return QF_OK;
}

int qf_optimize_gates_k(const qf_c128* E, int dim, const qf_c128* u_old, double beta, int count,
                        qf_c128* u_out, double* sigma_out, void* stream) {
  if (dim != 4 && dim != 8 && dim != 16) return set_error(QF_EINVAL, "dim=%d must be 4, 8 or 16", dim);
  if (dim == 4) return qf_optimize_gates(E, u_old, beta, count, u_out, sigma_out, stream);
  if (count < 0) return set_error(QF_EINVAL, "count=%d < 0", count);
  if (count == 0) return QF_OK;
  if (!E || !u_out) return set_error(QF_EINVAL, "NULL device pointer");
  if (beta != 0.0 && !u_old) return set_error(QF_EINVAL, "beta != 0 needs u_old");
  if (!(beta >= 0.0 && beta <= 1.0)) return set_error(QF_EINVAL, "beta=%g outside [0, 1]", beta);
  if (dim == 16) {
    QF_CUDA(qf::launch_optimize16(reinterpret_cast<const double2*>(E),
                                  reinterpret_cast<const double2*>(u_old), beta, count,
                                  reinterpret_cast<double2*>(u_out), sigma_out, as_stream(stream)));
    return QF_OK;
  }
  QF_CUDA(qf::launch_optimize8(reinterpret_cast<const double2*>(E),
                               reinterpret_cast<const double2*>(u_old), beta, count,
                               reinterpret_cast<double2*>(u_out), sigma_out, as_stream(stream)));
  return QF_OK;
}

int qf_init_tensor_k(const qf_c128* target, int n_qubits, int n_gates,
                     const qf_gate_loc* locations, int n_starts, const qf_c128* gates, void* T,
                     int precision, void* stream) {
  QF_TRY(check_sizes(n_qubits, n_gates));
  QF_TRY(check_prec(precision));
  if (n_starts < 1) return set_error(QF_EINVAL, "n_starts=%d must be >= 1", n_starts);
  if (!target || !gates || !T) return set_error(QF_EINVAL, "NULL device pointer");
  std::vector<GateDesc> gd;
  long long gsz = 0;
  QF_TRY(fetch_gate_locs(locations, n_qubits, n_gates, &gd, &gsz));
  cudaStream_t st = as_stream(stream);
  const int pr = kprec(precision);
  const double2* g = reinterpret_cast<const double2*>(gates);
  QF_CUDA(qf::launch_conj_transpose(reinterpret_cast<const double2*>(target), T, n_qubits, n_starts,
                                    pr, st));
  for (int k = 0; k < n_gates; ++k) {
    if (gd[k].k == 4)
      QF_CUDA(qf::launch_pass16(T, n_qubits, n_starts, gd[k].q, nullptr, 0, g + gd[k].off, gsz, pr, st));
    else if (gd[k].k == 3)
      QF_CUDA(qf::launch_pass8(T, n_qubits, n_starts, gd[k].q, nullptr, 0, g + gd[k].off, gsz, pr, st));
    else
      QF_CUDA(qf::launch_pass(T, n_qubits, n_starts, gd[k].q[0], gd[k].q[1], nullptr, 0, g + gd[k].off,
                              gsz, pr, st));
  }
  return QF_OK;
}

int qf_circuit_unitary_k(int n_qubits, int n_gates, const qf_gate_loc* locations,
                         const qf_c128* gates, qf_c128* C_out, void* stream) {
  QF_TRY(check_sizes(n_qubits, n_gates));
  if (!gates || !C_out) return set_error(QF_EINVAL, "NULL device pointer");
  const size_t N = (size_t)1 << n_qubits;
  cudaStream_t st = as_stream(stream);
  DevBuf I;
  QF_TRY(I.alloc(N * N * sizeof(double2)));
  QF_CUDA(qf::launch_set_identity(I.as<double2>(), n_qubits, st));
  const int rc = qf_init_tensor_k(reinterpret_cast<const qf_c128*>(I.p), n_qubits, n_gates, locations,
                                  1, gates, C_out, QF_C128, stream);
  QF_CUDA(cudaStreamSynchronize(st));
  return rc;
}

int qf_circuit_unitary(int n_qubits, int n_gates, const qf_loc* locations, const qf_c128* gates,
                       qf_c128* C_out, void* stream) {
  QF_TRY(check_sizes(n_qubits, n_gates));
  if (!gates || !C_out) return set_error(QF_EINVAL, "NULL device pointer");
  std::vector<qf_loc> locs;
  QF_TRY(fetch_locations(locations, n_qubits, n_gates, &locs));
  const size_t N = (size_t)1 << n_qubits;
  cudaStream_t st = as_stream(stream);
  // identity target: V^dagger = I
  DevBuf I;
  QF_TRY(I.alloc(N * N * sizeof(double2)));
  QF_CUDA(qf::launch_set_identity(I.as<double2>(), n_qubits, st));
  int rc = qf_init_tensor(reinterpret_cast<const qf_c128*>(I.p), n_qubits, n_gates, locs.data(),
                          1, gates, C_out, QF_C128, stream);
  QF_CUDA(cudaStreamSynchronize(st));
  return rc;
}

}  // extern "C"
