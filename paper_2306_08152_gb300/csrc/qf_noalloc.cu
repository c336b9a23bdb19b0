// Partial trace without any device allocation.
//
// qf_partial_trace gets the environment kernel's scratch (the per-CTA
// partial sums and the per-start completion counters) from the stream-ordered
// allocator on every call.  Some callers cannot allocate device memory at
// that point:
//   - code that must not synchronise or stall the device while it runs (a
//     latency-critical host loop, where a pool miss turns an allocation into
//     a device-wide synchronisation);
//   - embedders whose device memory is entirely held by their own caching
//     allocator, where a second allocator finds nothing left and fails;
//   - code paths that forbid allocation outright (real-time or certified
//     code that must not fail on resource exhaustion once set up).
// qf_partial_trace_noalloc computes the same result with that scratch in a
// fixed-size array of this library's own device memory instead.

#include <cuda_runtime.h>

#include <mutex>

#include "qf_internal.h"
#include "qfactor.h"

// One array per device that loads the library, held until the process exits.
static __device__ __align__(256) unsigned char qf_noalloc_scratch[QF_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};  // device address of the array, per device

// The array's name is a host-side stand-in in host code; its device address
// has to be looked up once per device, with that device current.
int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess)
    return qf_internal_set_error(QF_ECUDA, "cudaGetDevice failed", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return qf_internal_set_error(QF_EINVAL, "device index outside the supported range", "");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, qf_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return qf_internal_set_error(QF_ECUDA, "cudaGetSymbolAddress of the scratch array failed",
                                   cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return QF_OK;
}

}  // namespace

extern "C" int qf_partial_trace_noalloc(const void* T, int n_qubits, int n_starts, int a, int b,
                                        qf_c128* P, int precision, void* stream) {
  int rc = qf_internal_check_sizes(n_qubits, 1);
  if (rc != QF_OK) return rc;
  rc = qf_internal_check_prec(precision);
  if (rc != QF_OK) return rc;
  if (n_starts < 1) return qf_internal_set_error(QF_EINVAL, "n_starts must be >= 1", "");
  if (!T || !P) return qf_internal_set_error(QF_EINVAL, "NULL device pointer", "");
  if (a < 0 || a >= n_qubits || b < 0 || b >= n_qubits || a == b)
    return qf_internal_set_error(QF_EINVAL, "location invalid for the qubit count", "");
  const size_t part_bytes = (size_t)n_starts * qf::env_ctas(n_qubits) * 32 * sizeof(double);
  const size_t cnt_off = (part_bytes + 255) & ~(size_t)255;
  const size_t need = cnt_off + (size_t)n_starts * sizeof(unsigned);
  if (need > (size_t)QF_NOALLOC_SCRATCH_BYTES)
    return qf_internal_set_error(
        QF_EINVAL,
        "n_starts x CTAs per start needs more scratch than QF_NOALLOC_SCRATCH_BYTES; "
        "use qf_partial_trace or fewer starts per call",
        "");
  void* base = nullptr;
  rc = scratch_address(&base);
  if (rc != QF_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned* counters = reinterpret_cast<unsigned*>(static_cast<char*>(base) + cnt_off);
  // the array keeps the previous call's contents: the completion counters
  // must start at zero; the partial sums are written before they are read
  cudaError_t e = cudaMemsetAsync(counters, 0, (size_t)n_starts * sizeof(unsigned), st);
  if (e != cudaSuccess)
    return qf_internal_set_error(QF_ECUDA, "cudaMemsetAsync of the counters failed",
                                 cudaGetErrorString(e));
  e = qf::launch_update(T, n_qubits, n_starts, a, b, nullptr, 0, qf::kTraceOnly, 0.0, nullptr,
                        reinterpret_cast<double2*>(P), 16, nullptr, nullptr,
                        static_cast<double*>(base), counters, qf_internal_kernel_prec(precision), st);
  if (e != cudaSuccess)
    return qf_internal_set_error(QF_ECUDA, "partial trace launch failed", cudaGetErrorString(e));
  return QF_OK;
}
