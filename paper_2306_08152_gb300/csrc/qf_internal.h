// Internal launch interface between the host engine (qf_engine.cu) and the
// kernels (qf_pass.cu, qf_update.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qf {

// Modes of the environment kernel.
enum UpdateMode {
  kBackward = 0,   // E = P u^dagger; u' = polar; L = u', R = u^dagger
  kForward = 1,    // E = u^dagger P; u' = polar; L = u^dagger, R = u'
  kEnvOnly = 2,    // E = P u^dagger written out; L = u, R = u^dagger
  kTraceOnly = 3,  // P written out
};

// Gate kinds of the 4x4 update (Sec. III-A, "Specializing gate sets").
// kGateGeneral is a general unitary (the SVD update); the others are
// parameterised gates whose update is the closed-form argmax of
// Re Tr(E G(theta)).  A one-qubit kind acts as G (x) I on its qubit and a
// partner qubit (local index 2 bit(qubit) + bit(partner)).
enum GateKind {
  kGateGeneral = 0,
  kGateRz = 2,   // diag(1, e^{i theta})
  kGateGpi = 3,  // [[0, e^{-i phi}], [e^{i phi}, 0]]
  kGateMs = 4,   // Moelmer-Soerensen MS(phi0, phi1)
};

// Bit position of qubit q in an n-bit row or column index (qubit 0 = MSB).
inline int qubit_bit(int n, int q) { return n - 1 - q; }

// T_s <- V^dagger for every start s (prec: 0 = c128, 1 = c64).
cudaError_t launch_conj_transpose(const double2* V, void* T, int n, int S,
                                  int prec, cudaStream_t st);

// T_s <- (L_s on (a,b)) T_s (R_s on (a,b)); L_s = L + s*Lstride (16 FP64
// complex values), likewise R; a NULL operand is the identity.
cudaError_t launch_pass(void* T, int n, int S, int a, int b, const double2* L,
                        long long Lstride, const double2* R, long long Rstride,
                        int prec, cudaStream_t st);

// CTAs per start of the environment kernel.
int env_ctas(int n);

// Environment of gate k from the tensor before its removal, then the FP64
// update.  gates_k = gates + k*16, start stride gstride.  LR (S x 32 FP64)
// receives the pass operators; out (nullable) receives E (or P in
// kTraceOnly mode) with start stride out_stride; sigma_out (nullable, S)
// receives the singular-value sum.  part (S * env_ctas(n) * 32 doubles) and
// counters (S unsigned: zero before the first launch, left zero after each
// launch) are scratch owned by the caller.
// kind selects the update (GateKind); a parameterised kind reads its old
// parameters from and writes the new ones to prm + s * prm_stride (2
// doubles), and sigma_out receives the maximised Re Tr(A G).
cudaError_t launch_update(const void* T, int n, int S, int a, int b,
                          double2* gates_k, long long gstride, int mode,
                          double beta, double2* LR, double2* out,
                          long long out_stride, double* sigma_out, int* status,
                          double* part, unsigned* counters, int prec,
                          cudaStream_t st, int kind = kGateGeneral,
                          double* prm = nullptr, long long prm_stride = 0);

// The 4x4 matrices of the parameterised gates: for every start s and gate
// g with tab[g].x != kGateGeneral, gates[s * gsz + tab[g].y ...] (16
// entries) <- G(params[s * prm_stride + 2 g ...]).  Other gates untouched.
cudaError_t launch_param_gates(double2* gates, long long gsz, const int2* tab,
                               const double* params, long long prm_stride, int p,
                               int S, cudaStream_t st);

// launch_update for a gate on (a, b) whose environment is taken from a tensor
// that still lacks the pending update of the preceding gate on the disjoint
// pair (a1, b1) (look-ahead): L1, R1 (start stride stride1) are that
// update's pass operators.  Needs n >= 4; part and counters as for
// launch_update.
cudaError_t launch_update_lookahead(const void* T, int n, int S, int a1, int b1,
                                    const double2* L1, const double2* R1, long long stride1,
                                    int a, int b, double2* gates_k,
                                    long long gstride, int mode, double beta, double2* LR,
                                    double2* out, long long out_stride, double* sigma_out,
                                    int* status, double* part, unsigned* counters, int prec,
                                    cudaStream_t st);

// Two consecutive updates on disjoint pairs in one pass (complex64 only):
// T_s <- (L1 (x) L2) T_s (R1 (x) R2); L1, R1 have start stride s1, L2, R2
// start stride s2.  pair_pass_supported tells whether the tiled pass
// handles the case (complex64, 8 <= n <= 18, disjoint pairs);
// make_pair_params writes the launch geometry (pair_params_bytes() bytes of
// host memory), which launch_pair_pass passes by value.
bool pair_pass_supported(int n, int a1, int b1, int a2, int b2, int prec);
size_t pair_params_bytes();
void make_pair_params(int n, int a1, int b1, int a2, int b2, void* host_out);
cudaError_t launch_pair_pass(void* T, int n, int S, const void* params, const double2* L1,
                             const double2* R1, long long s1, const double2* L2,
                             const double2* R2, long long s2, cudaStream_t st);

// Three-qubit gates (qf_kq.cu).  q: the gate's three qubits in local-index
// order (q[0] is the most significant local bit).  Operators are 8x8 (64
// FP64 complex values per start); LR has start stride 128 (L, then R); part
// needs S * env_ctas(n) * 128 doubles.  Modes as for launch_update.
cudaError_t launch_pass8(void* T, int n, int S, const int* q, const double2* L, long long Ls,
                         const double2* R, long long Rs, int prec, cudaStream_t st);
cudaError_t launch_update8(const void* T, int n, int S, const int* q, double2* gates_k,
                           long long gstride, int mode, double beta, double2* LR, double2* out,
                           long long out_stride, double* sigma_out, int* status, double* part,
                           unsigned* counters, int prec, cudaStream_t st);
cudaError_t launch_optimize8(const double2* E, const double2* u_old, double beta, int count,
                             double2* u_out, double* sigma_out, cudaStream_t st);
cudaError_t launch_reunitarize8(double2* gates, int count, cudaStream_t st);
// Four-qubit gates (qf_k4.cu): q holds the gate's four qubits in
// local-index order.  Operators are 16x16 (256 FP64 complex values per
// start); LR has start stride 512 (L, then R); part needs
// S * env_ctas(n) * 512 doubles.  Modes as for launch_update; the update
// runs on one CTA of 256 threads per start.
// Complex64 passes with both operators at n >= 7 run on the tensor cores;
// their bounded waits record QF_ETIMEOUT in *status (may be NULL).
cudaError_t launch_pass16(void* T, int n, int S, const int* q, const double2* L, long long Ls,
                          const double2* R, long long Rs, int prec, cudaStream_t st,
                          int* status = nullptr);
cudaError_t launch_update16(const void* T, int n, int S, const int* q, double2* gates_k,
                            long long gstride, int mode, double beta, double2* LR, double2* out,
                            long long out_stride, double* sigma_out, int* status, double* part,
                            unsigned* counters, int prec, cudaStream_t st);
cudaError_t launch_optimize16(const double2* E, const double2* u_old, double beta, int count,
                              double2* u_out, double* sigma_out, cudaStream_t st);
// Three FP64 Newton-Schulz steps on every gate of size 4 in desc (others
// untouched).
cudaError_t launch_reunitarize16(double2* gates, long long gsz, const int2* desc, int p, int S,
                                 cudaStream_t st);
// Re-unitarise a mixed circuit: desc[k] = (size 2, 3 or 4, entry offset) of
// gate k; start s's gates begin at gates + s * gsz.  Gates of size 4 are left
// to launch_reunitarize16.
cudaError_t launch_reunitarize_mixed(double2* gates, long long gsz, const int2* desc, int p, int S,
                                     cudaStream_t st);

// u_i = polar update of E_i (Eq. opt_u) for i < count.
cudaError_t launch_optimize(const double2* E, const double2* u_old, double beta,
                            int count, double2* u_out, double* sigma_out,
                            cudaStream_t st);

// env[s][k] <- -(t_s / (N |t_s|)) env[s][k]^dagger in place (t = tr[s]).
cudaError_t launch_grad_from_env(double2* env, const double2* tr, int n, int S, int p,
                                 cudaStream_t st);
// The same for a circuit of 2-, 3- and 4-qubit gates: desc[k] = (qubits,
// entry offset) of gate k; set s's environments begin at env + s * gsz.
cudaError_t launch_grad_from_env_k(double2* env, const double2* tr, int n, int S, long long gsz,
                                   const int2* desc, int p, cudaStream_t st);

// Two FP64 Newton-Schulz steps on each of `count` gates, in place.
cudaError_t launch_reunitarize(double2* gates, int count, cudaStream_t st);

// *status <- -4 (QF_ENONFINITE) if any of the `count` doubles at x is not
// finite and *status holds no earlier error; otherwise it is left alone.
cudaError_t launch_check_finite(const double* x, size_t count, int* status, cudaStream_t st);

// One-pass InitCircuitTensor after the conjugate transpose: every row of
// each T_s takes T <- T (u_k on (pa[k], pb[k])) for k = 0..p-1 in shared
// memory.  gates + s*gstride holds start s's p gates.  Supported
// (build_rows_supported) for complex64 tensors with n >= 10 whose row and
// gates fit in shared memory; other cases use the per-gate passes.
bool build_rows_supported(int n, int p, int prec);
cudaError_t launch_build_rows(void* T, int n, int S, int p, const int* pa, const int* pb,
                              const double2* gates, long long gstride, cudaStream_t st);

// dst[i] <- src[i] for `count` entries, converting between kernel precision
// codes sp and dp (0 complex128, 1 complex64, 2 df64) through FP64.
cudaError_t launch_convert(const void* src, int sp, void* dst, int dp, size_t count,
                           cudaStream_t st);

// tr_s = Tr T_s (FP64 accumulation).
cudaError_t launch_trace(const void* T, int n, int S, double2* tr, int prec,
                         cudaStream_t st);

// M <- identity (N x N, FP64 complex).
cudaError_t launch_set_identity(double2* M, int n, cudaStream_t st);

// Number of SMs of the current device (cached).
int sm_count();

}  // namespace qf

// Record an error for qf_last_error() from another translation unit and
// return `code`; the message is "<what>: <detail>" (detail may be "").
__attribute__((visibility("hidden"))) int qf_internal_set_error(int code, const char* what,
                                                                const char* detail);

// The argument checks of the exported entry points, for other translation
// units: the qubit count within [QF_MIN_QUBITS, QF_MAX_QUBITS] and n_gates
// >= 1; a tensor precision of QF_C128, QF_C64 or QF_DF64.  Each records a
// message and returns QF_EINVAL on failure, QF_OK otherwise.
__attribute__((visibility("hidden"))) int qf_internal_check_sizes(int n_qubits, int n_gates);
__attribute__((visibility("hidden"))) int qf_internal_check_prec(int precision);
// Tensor precision (QF_C128, QF_C64, QF_DF64) -> the kernels' precision code
// (0 complex128, 1 complex64, 2 double-FP32).
__attribute__((visibility("hidden"))) int qf_internal_kernel_prec(int precision);
