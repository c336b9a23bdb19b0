/*
 * qfactor.h -- C ABI of the GB300 QFactor instantiation engine.
 *
 * QFactor (Kukliansky, Younis, Cincio, Iancu, arXiv 2306.08152) fits the
 * gates of a circuit of general two-qubit unitaries to a target unitary V by
 * sweeping over one 2^n x 2^n complex circuit tensor T (Sec. III, Alg. 1).
 * Every step of the sweep runs in hand-written CUDA kernels for sm_103a.
 *
 * Conventions (shared with the test oracle):
 *   - N = 2^n.  Qubit 0 is the most significant bit of a basis index.
 *   - A gate is 16 qf_c128 values, a 4x4 matrix in row-major order.  A gate on
 *     location (a, b) acts on the local index 2*bit(a) + bit(b), tensored with
 *     the identity on every other qubit; (b, a) is SWAP u SWAP on (a, b).
 *   - Gate lists are in product order: C = G_0 G_1 ... G_{p-1}, where list
 *     index 0 is the paper's u_1 (Sec. III: U = u_1 ... u_p).
 *   - Matrices (targets, circuit tensors) are row-major, entry (r, c) at
 *     r*N + c, interleaved complex (re, im).
 *   - Circuit tensors hold T = V^dagger C after initialisation (Alg. 1,
 *     InitCircuitTensor).  In precision QF_C128 an entry is a qf_c128
 *     (16 bytes); in QF_C64 it is a qf_c64 (8 bytes).  Several starts are
 *     stored back to back: start s begins at entry s*N*N.
 *   - The environment of gate k is E_k = Tr_{other qubits}(G_{k+1}...G_{p-1}
 *     V^dagger G_0...G_{k-1}), so Tr(V^dagger C) = Tr(E_k u_k) (Sec. III,
 *     environment matrix, Fig. 3).  dTr(V^dagger C)/d(u_k)_{ij} = (E_k)_{ji}.
 *   - Cost: 1 - |Tr(V^dagger C)| / N (Sec. II, Delta).
 *
 * Memory: "device" arguments are CUDA device pointers in the current
 * context; "host-or-device" arguments may be either (the library inspects the
 * pointer and copies host data itself).  The caller owns every argument
 * array.  The library allocates its own workspace (circuit tensors) with
 * cudaMalloc and frees it before a call returns, except inside a qf_plan,
 * which owns its workspace until qf_plan_destroy.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Calls that return host values synchronise that stream; the
 * others only enqueue work.
 *
 * Errors: every call returns QF_OK (0) or a negative QF_E* code, and
 * qf_last_error() returns a message for the calling thread's last failure.
 * Output arrays are unspecified after a failure.
 */
#ifndef QFACTOR_H
#define QFACTOR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } qf_c128;   /* same layout as cuDoubleComplex */
typedef struct { float re, im; } qf_c64;     /* same layout as cuFloatComplex  */
typedef struct { int32_t a, b; } qf_loc;     /* gate location: qubits a != b  */

/* Return codes. */
#define QF_OK            0
#define QF_EINVAL       -1   /* bad size, location, NULL pointer or option   */
#define QF_ENOMEM       -2   /* device allocation failed                     */
#define QF_ECUDA        -3   /* a CUDA runtime call failed                   */
#define QF_ENONFINITE   -4   /* NaN/Inf in an input or in an environment     */
#define QF_ETIMEOUT     -5   /* a bounded tensor-core completion wait ran out;
                                the tensor entries it left are NaN          */

/* Circuit-tensor precision. */
#define QF_C128          0   /* complex128 tensor, FP64 arithmetic throughout */
#define QF_C64           1   /* complex64 tensor, FP32 gate application; the
                                partial trace sums in FP32 within each CTA's
                                slice of the band and in FP64 across CTAs;
                                the 4x4 update runs in FP64 */
#define QF_C64_REFINE64  2   /* bulk sweeps in QF_C64, then the tensor is
                                rebuilt in QF_C128 for the final sweeps    */
#define QF_DF64          3   /* double-FP32 complex tensor: each real part is
                                an unevaluated sum hi + lo of two floats
                                (about 48 significant bits), 16 bytes per
                                entry laid out (re.hi, im.hi, re.lo, im.lo);
                                gate application in FP32 error-free
                                arithmetic (TwoSum, TwoProd), partial traces
                                and the 4x4 update in FP64                  */
#define QF_C64_REFINE_DF 4   /* bulk sweeps in QF_C64, then the tensor is
                                rebuilt in QF_DF64 for the final sweeps    */

/* Termination reasons. */
#define QF_STOP_CONVERGED   1   /* some start reached dist_tol               */
#define QF_STOP_PLATEAU     2   /* every start met a plateau test            */
#define QF_STOP_MAX_SWEEPS  3

/* Supported sizes. */
#define QF_MIN_QUBITS 2
#define QF_MAX_QUBITS 14

/*
 * Hyperparameters of Sec. III-A2.  qf_options_default() fills: dist_tol 1e-10,
 * max_sweeps 500, min_sweeps 0, reset_iter 40, diff_tol_a 0, diff_tol_r 0,
 * long_diff_count 0, long_diff_r 0.1, beta 0, precision QF_C128,
 * switch_tol 1e-6, max_c64_sweeps 1000, cost_history NULL.
 *   dist_tol      stop once a start's cost is <= dist_tol.
 *   max_sweeps    upper bound on two-sided sweeps (all phases together).
 *   min_sweeps    no stopping test before this many sweeps.
 *   reset_iter    rebuild every tensor from V and the gates after every
 *                 reset_iter sweeps (0 = never).
 *   diff_tol_a/r  short plateau: a start plateaus when
 *                 c_{i-1} - c_i <= diff_tol_a + diff_tol_r * c_i
 *                 (off when both are 0).
 *   long_diff_count/_r  long plateau: c_{i-L} - c_i < long_diff_r * c_{i-L},
 *                 L = long_diff_count (off when 0).
 *   beta          the update takes the SVD of (1-beta) E + beta u^dagger.
 *   precision     QF_C128, QF_C64, QF_C64_REFINE64, QF_DF64 or
 *                 QF_C64_REFINE_DF.
 *   switch_tol    QF_C64_REFINE64 / QF_C64_REFINE_DF: leave the c64 phase
 *                 once the best cost is <= switch_tol, or once ten c64
 *                 sweeps have lowered the cost by less than 1e-7 (the
 *                 complex64 noise floor) while the best cost is <= 1e-5 (a
 *                 stall at a larger cost is the method's own plateau and
 *                 stays in c64), or after max_c64_sweeps.  The plateau rules
 *                 apply in both phases.  Reported costs are always FP64
 *                 traces.
 *   cost_history  optional (NULL = off), host-or-device: the cost of every
 *                 start after every sweep (Alg. 1: the cost the stopping
 *                 rules of Sec. III-A2 test), row-major [start][sweep],
 *                 max_sweeps + 1 doubles per start (qf_instantiate_batched:
 *                 [instance][start][sweep]).  Entry 0 is the initial
 *                 circuit's cost, entry i the cost after sweep i: an FP64
 *                 trace of the tensor in the precision of that sweep (of the
 *                 rebuilt QF_C128/QF_DF64 tensor at the sweep that leaves the
 *                 complex64 phase).  Entries after a start's last sweep are
 *                 NaN.
 */
typedef struct {
    double dist_tol;
    int32_t max_sweeps;
    int32_t min_sweeps;
    int32_t reset_iter;
    int32_t long_diff_count;
    double diff_tol_a;
    double diff_tol_r;
    double long_diff_r;
    double beta;
    int32_t precision;
    int32_t max_c64_sweeps;
    double switch_tol;
    double* cost_history;
} qf_options;

/* Result summary of an instantiation. */
typedef struct {
    int32_t best_start;   /* start with the lowest final cost               */
    int32_t sweeps;       /* sweeps run (all phases)                        */
    int32_t c64_sweeps;   /* of which in complex64                          */
    int32_t reason;       /* QF_STOP_*                                      */
    double best_cost;     /* cost of best_start, from an FP64 trace          */
} qf_result;

/* Message for the calling thread's last error ("" if none). */
const char* qf_last_error(void);

/* Library version, major*10000 + minor*100 + patch. */
int qf_version(void);

/* Fill *opts with the defaults listed above.  Returns QF_EINVAL on NULL. */
int qf_options_default(qf_options* opts);

/*
 * qf_instantiate -- Qfactor of Alg. 1 for one start, in QF_C128.
 *   target         host-or-device, N x N unitary V.
 *   n_qubits       2 .. QF_MAX_QUBITS.
 *   n_gates        p >= 1.
 *   locations      host-or-device, p locations.
 *   initial_gates  host-or-device, p x 16.
 *   tol            dist_tol; max_sweeps >= 1.
 *   out_gates      host-or-device, p x 16 (may alias initial_gates).
 *   out_cost       host, final cost (FP64 trace of the tensor).
 *   out_sweeps     host, sweeps run; may be NULL.
 * Synchronises `stream`.
 */
int qf_instantiate(const qf_c128* target, int n_qubits, int n_gates,
                   const qf_loc* locations, const qf_c128* initial_gates,
                   double tol, int max_sweeps, qf_c128* out_gates,
                   double* out_cost, int* out_sweeps, void* stream);

/*
 * qf_instantiate_ex -- lock-step multistart Qfactor with all options.
 * All starts sweep together (Sec. IV-A): the run stops after the first sweep
 * in which any start reaches dist_tol, once every start has met a plateau
 * test (the mark is kept once set), or at max_sweeps.
 *   initial_gates  host-or-device, n_starts x p x 16.
 *   opts           host; NULL = defaults.
 *   out_gates      host-or-device, n_starts x p x 16.
 *   out_costs      host, n_starts final costs; may be NULL.
 *   out_result     host, summary; may be NULL.
 * Synchronises `stream`.
 */
int qf_instantiate_ex(const qf_c128* target, int n_qubits, int n_gates,
                      const qf_loc* locations, int n_starts,
                      const qf_c128* initial_gates, const qf_options* opts,
                      qf_c128* out_gates, double* out_costs,
                      qf_result* out_result, void* stream);

/*
 * qf_cost_and_env -- cost and every environment matrix of n_sets gate sets
 * (the adjoint walk: the tensor is built once, then each gate is moved from
 * the right of the tensor to its left with one pass, and its environment is
 * read on the way; O(4^n) memory for any p).
 *   gates      host-or-device, n_sets x p x 16.
 *   out_cost   host, n_sets costs; may be NULL.
 *   out_env    host-or-device, n_sets x p x 16: E_k of each set (FP64).
 *   out_trace  host, n_sets values Tr(V^dagger C); may be NULL.
 * Synchronises `stream`.
 */
int qf_cost_and_env(const qf_c128* target, int n_qubits, int n_gates,
                    const qf_loc* locations, int n_sets,
                    const qf_c128* gates, double* out_cost, qf_c128* out_env,
                    qf_c128* out_trace, void* stream);

/*
 * qf_cost_grad -- the differentiable cost: cost_s = 1 - |t_s|/N with
 * t_s = Tr(V^dagger C_s), and its gradient with respect to every gate entry
 * in the convention of PyTorch's complex autograd (d/dRe + i d/dIm):
 * grad_{s,k} = -(t_s / (N |t_s|)) E_{s,k}^dagger (E as in qf_cost_and_env,
 * Sec. III; a zero trace gives a zero gradient).  One forward trace plus one
 * adjoint walk gives all p gradients with O(4^n) memory.
 *   gates     host-or-device, n_sets x p x 16.
 *   out_cost  host, n_sets; may be NULL.
 *   out_grad  host-or-device, n_sets x p x 16.
 * Synchronises `stream`.
 */
int qf_cost_grad(const qf_c128* target, int n_qubits, int n_gates,
                 const qf_loc* locations, int n_sets, const qf_c128* gates,
                 double* out_cost, qf_c128* out_grad, void* stream);

/*
 * qf_instantiate_batched -- many small instantiations in one persistent
 * launch (captured as a CUDA graph).  Each (instance, start) problem runs the
 * whole Qfactor loop of Alg. 1 on one warp with its circuit tensor in shared
 * memory; the starts of an instance run side by side and stop at their next
 * sweep boundary once any of them has reached dist_tol, or once all of them
 * have met a plateau test (Sec. IV-A, without lock-step).  The number of
 * warps per CTA is chosen by a built-in autotuner (timed trial runs, cached
 * per largest qubit count, precision and device).
 *   n_qubits, n_gates  host, n_instances each; 2 <= n_qubits <= QF_BATCH_MAX_QUBITS.
 *   locations          host-or-device, concatenated over instances.
 *   targets            host-or-device, concatenated N_i x N_i targets.
 *   initial_gates      host-or-device, [instance][start][gate][16].
 *   opts               host; NULL = defaults (long_diff_count <= 127).
 *   out_gates          host-or-device, layout of initial_gates.
 *   out_costs          host, n_instances * n_starts final costs.
 *   out_sweeps         host, n_instances * n_starts; may be NULL.
 *   out_best           host, n_instances best start indices; may be NULL.
 *   stats              host; may be NULL.
 * Synchronises `stream`.
 */
#define QF_BATCH_MAX_QUBITS 6
typedef struct {
    int32_t warps_per_cta;     /* chosen by the autotuner                   */
    int32_t ctas;              /* persistent CTAs launched                  */
    double kernel_ms;          /* device time of the persistent launch      */
    int64_t total_sweeps;      /* over all problems                          */
    int64_t total_c64_sweeps;  /* of which in complex64                      */
} qf_batch_stats;
int qf_instantiate_batched(int n_instances, const int32_t* n_qubits,
                           const int32_t* n_gates, const qf_loc* locations,
                           const qf_c128* targets, int n_starts,
                           const qf_c128* initial_gates, const qf_options* opts,
                           qf_c128* out_gates, double* out_costs,
                           int32_t* out_sweeps, int32_t* out_best,
                           qf_batch_stats* stats, void* stream);

/* ------------------------------------------------------------------------
 * Gates on more than two qubits (the paper treats a multi-qubit unitary as
 * one variable with a 2^k x 2^k environment, Sec. III and Sec. VI).
 * Supported: k = 2, 3 and 4, mixed freely in one circuit.
 *
 * A gate on k qubits (q[0], ..., q[k-1]) acts on the local index
 * sum_i bit(q[i]) 2^(k-1-i) (k = 2: 2*bit(q[0]) + bit(q[1]), as qf_loc).
 * Gate arrays are concatenated per start in gate order: gate i has 4^k_i
 * entries (row-major 2^k x 2^k), a start's gates take E = sum_i 4^k_i
 * entries and start s's begin at s*E.
 * ---------------------------------------------------------------------- */
typedef struct {
    int32_t k;     /* 2, 3 or 4 */
    int32_t q[4];  /* qubits in local-index order; q[k..3] unused */
} qf_gate_loc;

/* qf_instantiate_ex for a circuit of 2-, 3- and 4-qubit gates.  locations:
 * host-or-device, n_gates entries; initial_gates and out_gates:
 * host-or-device, n_starts x E entries (see above).  The three-qubit
 * updates use the 8x8 polar on one warp, the four-qubit updates the 16x16
 * polar on one CTA of 256 threads: an FP32 one-sided Jacobi SVD, then FP64
 * refinement rounds (FP64 Jacobi sweeps when a singular value is below
 * 1e-3 of the largest), accurate to FP64 rounding within the polar
 * factor's conditioning; the look-ahead and the one-pass InitCircuitTensor apply to
 * two-qubit-only circuits, qf_instantiate_batched_k takes 2- and 3-qubit
 * gates.  Errors as qf_instantiate_ex, QF_EINVAL for k
 * outside {2, 3, 4}, k > n_qubits, repeated or out-of-range qubits. */
int qf_instantiate_k(const qf_c128* target, int n_qubits, int n_gates,
                     const qf_gate_loc* locations, int n_starts,
                     const qf_c128* initial_gates, const qf_options* opts,
                     qf_c128* out_gates, double* out_costs,
                     qf_result* out_result, void* stream);

/* qf_instantiate_batched for circuits of 2- and 3-qubit gates: the same
 * per-warp Qfactor (multistart rule, stopping rules, precisions, autotuner,
 * cost history), with the three-qubit updates as the band sum over 8x8
 * blocks, the warp 8x8 FP64 polar and the fused pass on 8x8 blocks in the
 * warp's shared memory.  locations: host-or-device, concatenated over
 * instances (n_gates[i] each); initial_gates and out_gates: host-or-device,
 * [instance][start][E_i entries] in the concatenated gate layout above.
 * Errors as qf_instantiate_batched, QF_EINVAL for k outside {2, 3}, k above
 * an instance's qubit count, repeated or out-of-range qubits. */
int qf_instantiate_batched_k(int n_instances, const int32_t* n_qubits,
                             const int32_t* n_gates, const qf_gate_loc* locations,
                             const qf_c128* targets, int n_starts,
                             const qf_c128* initial_gates, const qf_options* opts,
                             qf_c128* out_gates, double* out_costs,
                             int32_t* out_sweeps, int32_t* out_best,
                             qf_batch_stats* stats, void* stream);

/* qf_cost_and_env / qf_cost_grad for a circuit of 2-, 3- and 4-qubit gates
 * (the same adjoint walk; Sec. III: Tr(V^dagger C) = Tr(E_k u_k) for a gate
 * of any size, E_k its 2^k x 2^k environment).  gates, out_env and out_grad:
 * host-or-device, n_sets x E entries in the concatenated layout above;
 * out_cost, out_trace: host, n_sets each (may be NULL).  The gradient is
 * -(t_s / (N |t_s|)) E_{s,k}^dagger for every gate, in the convention of
 * PyTorch's complex autograd (d/dRe + i d/dIm).  Synchronises `stream`. */
int qf_cost_and_env_k(const qf_c128* target, int n_qubits, int n_gates,
                      const qf_gate_loc* locations, int n_sets, const qf_c128* gates,
                      double* out_cost, qf_c128* out_env, qf_c128* out_trace, void* stream);
int qf_cost_grad_k(const qf_c128* target, int n_qubits, int n_gates,
                   const qf_gate_loc* locations, int n_sets, const qf_c128* gates,
                   double* out_cost, qf_c128* out_grad, void* stream);

/* Steps for one gate of size k (parity tests; enqueue only):
 *   qf_apply_gate_k     T_s <- (L_s on q) T_s (R_s on q); L, R device
 *                       n_starts x 4^k (either may be NULL for identity).
 *                       Four-qubit complex64 calls with both operators at
 *                       n_qubits >= 7 run on the tensor cores (see
 *                       qf_set_tc_wait_limit); a wait that runs out leaves
 *                       NaN in the entries it did not finish.
 *   qf_partial_trace_k  P_s = partial trace of T_s over every qubit not in
 *                       q (CalcEnvMat, Alg. 1); P device n_starts x 4^k.
 *                       k = 3 and 4 allocate their scratch stream-ordered.
 *   qf_optimize_gates_k OptimizeGate (Eq. opt_u) on `count` dim x dim
 *                       matrices, dim 4, 8 or 16 (see qf_optimize_gates).
 *   qf_init_tensor_k    InitCircuitTensor with k-qubit gates (gates device,
 *                       n_starts x E).
 *   qf_circuit_unitary_k C = G_0 ... G_{p-1} (complex128, device N x N;
 *                       gates device, E entries).  Synchronises. */
int qf_apply_gate_k(void* T, int n_qubits, int n_starts,
                    const qf_gate_loc* location, const qf_c128* L,
                    const qf_c128* R, int precision, void* stream);
int qf_partial_trace_k(const void* T, int n_qubits, int n_starts,
                       const qf_gate_loc* location, qf_c128* P, int precision,
                       void* stream);
int qf_optimize_gates_k(const qf_c128* E, int dim, const qf_c128* u_old,
                        double beta, int count, qf_c128* u_out,
                        double* sigma_out, void* stream);
int qf_init_tensor_k(const qf_c128* target, int n_qubits, int n_gates,
                     const qf_gate_loc* locations, int n_starts,
                     const qf_c128* gates, void* T, int precision,
                     void* stream);
int qf_circuit_unitary_k(int n_qubits, int n_gates,
                         const qf_gate_loc* locations, const qf_c128* gates,
                         qf_c128* C_out, void* stream);

/* Four-qubit passes in complex64 with both operators at n_qubits >= 7 run
 * on the tensor cores (tcgen05, 3xTF32: FP32-level results).  Each of
 * their completion waits polls at most `polls` times (default 4194304,
 * well above any real wait); when one runs out, the pass writes NaN over
 * the tensor entries it has not finished and a plan returns QF_ETIMEOUT at
 * its next status check.  qf_set_tc_wait_limit sets the limit for later
 * launches (0 makes every wait run out at once, which tests that path) and
 * returns the previous limit; polls < 0 only returns it. */
int qf_set_tc_wait_limit(int polls);

/* ------------------------------------------------------------------------
 * Resident plan: device-resident tensors, target and gates for repeated
 * sweeps (the form the benchmark times).
 * ---------------------------------------------------------------------- */
typedef struct qf_plan qf_plan;

/* Allocate a plan for n_starts circuits of the given structure.  precision
 * is QF_C128 or QF_C64.  locations: host-or-device.  Allocates
 * n_starts*N*N tensor entries plus the target and gates on the current
 * device. */
int qf_plan_create(int n_qubits, int n_gates, const qf_loc* locations,
                   int n_starts, int precision, qf_plan** out_plan);
int qf_plan_destroy(qf_plan* plan);

/* Copy the target (host-or-device, N x N) and gates (host-or-device,
 * n_starts x p x 16) into the plan and build every tensor (InitCircuitTensor).
 * Enqueued on `stream`; the plan records `stream` for its later calls.  The
 * copies are checked for NaN/Inf on the device: a non-finite input sets the
 * plan's status word, which qf_plan_status reports as QF_ENONFINITE. */
int qf_plan_load(qf_plan* plan, const qf_c128* target, const qf_c128* gates,
                 void* stream);

/* Run n_sweeps two-sided sweeps on every start; the tensors are rebuilt after
 * every reset_iter-th sweep counted since qf_plan_load (reset_iter <= 0:
 * never).  With two or more starts the starts form two groups whose
 * environment kernels and passes run on two internal streams, so that one
 * group's gate update overlaps the other group's pass.  Without pass timing,
 * from the plan's second sweep on, a sweep is captured once as a CUDA graph
 * (per beta and precision) and replayed (the first sweep runs as live
 * launches, so one-sweep uses pay no capture).  Enqueue only. */
int qf_plan_sweep(qf_plan* plan, int n_sweeps, int reset_iter, double beta);

/* Rebuild every tensor from the target and the current gates, in
 * `precision` (QF_C128 or QF_C64; switching precision re-types the tensors). */
int qf_plan_rebuild(qf_plan* plan, int precision);

/* FP64 trace of every tensor -> host out_costs[s] = 1 - |Tr T_s|/N and, if
 * out_trace != NULL, Tr T_s.  Synchronises. */
int qf_plan_costs(qf_plan* plan, double* out_costs, qf_c128* out_trace);

/* Copy the current gates (n_starts x p x 16) to host-or-device `out`.
 * Synchronises. */
int qf_plan_get_gates(qf_plan* plan, qf_c128* out);

/* Kernel timing of the gate-application pass: when enabled, every pass
 * launch is bracketed by CUDA events on the stream it runs on (sweeps then
 * run as live launches instead of a replayed graph).  qf_plan_pass_stats
 * synchronises and returns, since the last call: the summed duration of the
 * timed passes (ms), their algorithmic bytes (one read and one write of every
 * tensor entry they cover; may be NULL), the pass-launch count and the count
 * of all kernel launches; then it resets them. */
int qf_plan_enable_pass_timing(qf_plan* plan, int enable);

/* Look-ahead sweeps (complex64 plans with n_qubits >= 8; elsewhere the flag
 * is kept but sweeps run one update per pass).  Each half-sweep (Alg. 1) is
 * split greedily into windows: two consecutive updates whose gates act on
 * four distinct qubits form a window, any other update a window of its own.
 * In a two-update window the second gate's environment is taken from the
 * tensor before the first update's pass, by carrying that pending update
 * through the partial trace (the same quantity as after the pass, so the
 * sweep follows the one-update order of Alg. 1 up to rounding), and one
 * pass applies both updates: half the tensor traffic for the pair.
 * qf_plan_lookahead_windows returns the two-update windows per sweep (0 when
 * look-ahead is off or unsupported for the plan). */
int qf_plan_set_lookahead(qf_plan* plan, int enable);
int qf_plan_lookahead_windows(qf_plan* plan, int* pairs_per_sweep);
int qf_plan_pass_stats(qf_plan* plan, double* pass_ms, int64_t* pass_launches,
                       int64_t* all_launches, double* pass_bytes);

/* Current device status word of the plan: 0 = clean, else the first error
 * recorded (QF_ENONFINITE: an update met a non-finite environment;
 * QF_ETIMEOUT: a tensor-core pass's completion wait ran out).  Synchronises. */
int qf_plan_status(qf_plan* plan);

/* A resident plan for a circuit of 2- and 3-qubit gates (as qf_plan_create;
 * qf_plan_load / qf_plan_get_gates then use the concatenated gate layout,
 * n_starts x E entries, E from qf_plan_gate_entries). */
int qf_plan_create_k(int n_qubits, int n_gates, const qf_gate_loc* locations,
                     int n_starts, int precision, qf_plan** out_plan);
int qf_plan_gate_entries(qf_plan* plan, int64_t* entries_per_start);

/* ------------------------------------------------------------------------
 * Specialised gate sets (Sec. III-A, "Specializing gate sets").  A circuit
 * may mix general unitaries with parameterised gates G(theta), whose
 * update is the closed-form theta' = argmax Re Tr(A G(theta)) (A = E, or
 * (1 - beta) E + beta u^dagger with damping) instead of the SVD:
 *   QF_GATE_RZ   Rz(theta) = diag(1, e^{i theta}) on q[0];
 *                theta' = -arg A1[1][1]
 *   QF_GATE_GPI  GPI(phi) = [[0, e^{-i phi}], [e^{i phi}, 0]] on q[0];
 *                phi' = -arg(A1[0][1] + conj A1[1][0])
 *   QF_GATE_MS   Moelmer-Soerensen MS(phi0, phi1) on (q[0], q[1]):
 *                (1/sqrt 2) [[1,0,0,-i e^{-i(phi0+phi1)}],
 *                            [0,1,-i e^{-i(phi0-phi1)},0],
 *                            [0,-i e^{i(phi0-phi1)},1,0],
 *                            [-i e^{i(phi0+phi1)},0,0,1]];
 *                phi0 + phi1 = -arg z_a, phi0 - phi1 = -arg z_b with
 *                z_a = -i (A[0][3] - conj A[3][0]), z_b = -i (A[1][2] - conj A[2][1])
 *   QF_GATE_U4, QF_GATE_U8  general unitaries on 2 or 3 qubits (SVD update).
 * An angle whose modulus is zero keeps its old value.  RZ and GPI run as
 * G (x) I in a 4x4 slot on (q[0], q[1]) (local index 2 bit(q[0]) +
 * bit(q[1])), q[1] being any other qubit, or, for q[1] < 0, q[0] + 1
 * (q[0] - 1 for the last qubit); A1[x][y] = sum_r A[2x+r][2y+r] is the
 * one-qubit environment.  Every gate takes a slot of E entries as in
 * qf_plan_create_k (16, or 64 for QF_GATE_U8), and two parameters per
 * (start, gate) (theta in the first for RZ and GPI; none used for general
 * gates), start stride 2 n_gates.
 * ---------------------------------------------------------------------- */
#define QF_GATE_U4 0
#define QF_GATE_U8 1
#define QF_GATE_RZ 2
#define QF_GATE_GPI 3
#define QF_GATE_MS 4

typedef struct {
    int32_t kind;  /* QF_GATE_* */
    int32_t q[3];  /* qubits (q[1] of RZ/GPI: the slot's partner qubit, < 0 automatic) */
} qf_gate_spec;

/* qf_instantiate_ex for a circuit of specialised and general gates: the
 * same stopping rules, multistart and precision phases.  initial_gates:
 * host-or-device n_starts x E entries, the general gates' matrices (the
 * parameterised slots ignored; NULL if every gate is parameterised);
 * initial_params / out_params: host-or-device n_starts x n_gates x 2
 * doubles; out_gates receives every slot matrix (n_starts x E).  Errors as
 * qf_instantiate_ex and qf_plan_create_spec. */
int qf_instantiate_spec(const qf_c128* target, int n_qubits, int n_gates,
                        const qf_gate_spec* gates, int n_starts,
                        const qf_c128* initial_gates, const double* initial_params,
                        const qf_options* opts, qf_c128* out_gates, double* out_params,
                        double* out_costs, qf_result* out_result, void* stream);

/* A resident plan for a circuit of specialised and general gates (as
 * qf_plan_create_k).  The look-ahead flag is ignored for these plans.
 * Errors: QF_EINVAL for an unknown kind, repeated or out-of-range qubits. */
int qf_plan_create_spec(int n_qubits, int n_gates, const qf_gate_spec* gates,
                        int n_starts, int precision, qf_plan** out_plan);

/* Load the target (N x N), the general gates' matrices (n_starts x E
 * entries, the slots of parameterised gates ignored; NULL if the circuit
 * has no general gate) and the parameters (n_starts x n_gates x 2 doubles),
 * all host-or-device; the parameterised gates' matrices are built from the
 * parameters on the device, then every tensor is built (InitCircuitTensor).
 * Non-finite inputs raise the plan status.  Enqueue only. */
int qf_plan_load_spec(qf_plan* plan, const qf_c128* target, const qf_c128* gates,
                      const double* params, void* stream);

/* The current parameters, n_starts x n_gates x 2 doubles (host or device).
 * Synchronises. */
int qf_plan_get_params(qf_plan* plan, double* out_params);

/* ------------------------------------------------------------------------
 * Single steps of the sweep (Alg. 1), on device arrays, enqueue only.
 * ---------------------------------------------------------------------- */

/* Step a1, InitCircuitTensor (Alg. 1): T_s <- V^dagger, then
 * T_s <- T_s (u_{s,k} on loc_k) for k = 0..p-1.
 *   target  device N x N (qf_c128);  locations host or device;
 *   gates   device n_starts x p x 16; T device n_starts x N x N of the
 *   given precision (QF_C128 | QF_C64). */
int qf_init_tensor(const qf_c128* target, int n_qubits, int n_gates,
                   const qf_loc* locations, int n_starts, const qf_c128* gates,
                   void* T, int precision, void* stream);

/* Steps a2+a5 fused (Alg. 1 ApplyRight/ApplyLeft on one location):
 * T_s <- (L_s on (a,b)) T_s (R_s on (a,b)) in one read and one write of T.
 * L, R: device n_starts x 16 (FP64; cast to the tensor's precision), either
 * may be NULL for the identity. */
int qf_apply_pair(void* T, int n_qubits, int n_starts, int a, int b,
                  const qf_c128* L, const qf_c128* R, int precision,
                  void* stream);

/* Steps a2+a5 for two updates on disjoint pairs in one pass (look-ahead):
 * T_s <- (L1_s on (a1,b1)) (L2_s on (a2,b2)) T_s (R1_s on (a1,b1))
 *        (R2_s on (a2,b2)).
 * a1, b1, a2, b2 must be four distinct qubits.  L1, R1, L2, R2: device
 * n_starts x 16 (FP64; cast to the tensor's precision).  complex64 tensors
 * with n_qubits >= 8 take the tiled one-pass kernel (one read and one write
 * of T); other cases run the two single-pair passes in order. */
int qf_apply_two_pairs(void* T, int n_qubits, int n_starts, int a1, int b1,
                       const qf_c128* L1, const qf_c128* R1, int a2, int b2,
                       const qf_c128* L2, const qf_c128* R2, int precision,
                       void* stream);

/* Look-ahead environment (Alg. 1 CalcEnvMat for the second gate of a
 * window): P_s = partial trace over every qubit except (a, b) of
 * (L1_s on (a1,b1)) T_s (R1_s on (a1,b1)), computed from T_s without
 * applying the pending update: with M = R1 L1,
 *   P[x][y] = sum_rest sum_{i,j} M[j][i] T[(rest,i,x),(rest,j,y)]
 * (i, j: local indices of (a1, b1); x, y: of (a, b)); 16 N entries of T are
 * read.  n_qubits >= 4; a1, b1, a, b four distinct qubits.  L1, R1: device
 * n_starts x 16; P: device n_starts x 16.  Accumulates in the tensor's
 * precision per CTA and in FP64 across CTAs. */
int qf_partial_trace_after(const void* T, int n_qubits, int n_starts, int a1,
                           int b1, const qf_c128* L1, const qf_c128* R1, int a,
                           int b, qf_c128* P, int precision, void* stream);

/* Step a3, CalcEnvMat (Alg. 1): P_s = partial trace of T_s over every qubit
 * except (a, b).  QF_C128 and QF_DF64 tensors are summed in FP64; QF_C64
 * tensors in FP32 within each CTA's slice of the band (error about 1e-6 of
 * the summed magnitudes) and in FP64 across CTAs.  P: device n_starts x 16. */
int qf_partial_trace(const void* T, int n_qubits, int n_starts, int a, int b,
                     qf_c128* P, int precision, void* stream);

/* Step a4, OptimizeGate (Sec. III-A1, Eq. opt_u): for each of `count`
 * matrices E_i, with A_i = (1-beta) E_i + beta u_old_i^dagger = X D Y^dagger,
 * u_out_i = Y X^dagger and sigma_out_i = sum(D).  All device arrays; u_old may
 * be NULL when beta == 0; sigma_out may be NULL. FP64. */
int qf_optimize_gates(const qf_c128* E, const qf_c128* u_old, double beta,
                      int count, qf_c128* u_out, double* sigma_out,
                      void* stream);

/* Precision conversion (no counterpart in the paper): dst[i] <- src[i] for
 * `count` tensor entries, src in src_precision and dst in dst_precision
 * (QF_C128, QF_C64 or QF_DF64), through FP64: exact from QF_C64 and
 * QF_DF64 sources; QF_C128 -> QF_DF64 keeps about 48 significant bits
 * (hi = float(x), lo = float(x - hi)); -> QF_C64 rounds to FP32.  Device
 * arrays; they must not overlap unless identical with equal precisions.
 * Enqueue only. */
int qf_convert_tensor(const void* src, int src_precision, void* dst,
                      int dst_precision, int64_t count, void* stream);

/* Step a7, periodic re-unitarisation (Sec. III-A2, reset_iter): three FP64
 * Newton-Schulz steps u <- u (3I - u^dagger u) / 2 on each of `count` device
 * gates (count x 16), in place.  The sweep engines run it on every gate
 * before each periodic rebuild of the circuit tensors. */
int qf_reunitarize_gates(qf_c128* gates, int count, void* stream);

/* Step a6: tr_out_s = Tr T_s (FP64 accumulation).  tr_out: device n_starts. */
int qf_trace(const void* T, int n_qubits, int n_starts, qf_c128* tr_out,
             int precision, void* stream);

/*
 * qf_partial_trace_noalloc -- qf_partial_trace without any device allocation.
 * The paper has no counterpart: this is a service to callers that cannot
 * allocate device memory inside the call (code that must not stall or
 * synchronise the device, embedders whose own caching allocator holds all
 * free device memory, code that must not fail on allocation once set up).
 * Same arguments, layout and result as qf_partial_trace.  The environment
 * kernel's scratch (n_starts * CTAs-per-start * 256 bytes of partial sums,
 * plus n_starts counters) lives in one static device array of
 * QF_NOALLOC_SCRATCH_BYTES per device, held until the process exits; a call
 * that needs more returns QF_EINVAL.  The first call on a device looks up the
 * array's device address (once per device, with that device current); make
 * that first call before any stream capture.  Every call shares the array:
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race on it and must be serialised by the caller.  Enqueue only.
 */
#define QF_NOALLOC_SCRATCH_BYTES (64 * 1024)
int qf_partial_trace_noalloc(const void* T, int n_qubits, int n_starts, int a,
                             int b, qf_c128* P, int precision, void* stream);

/* C = G_0 G_1 ... G_{p-1} (InitCircuitTensor with the identity target), FP64.
 *   locations host or device; gates device p x 16; C_out device N x N. */
int qf_circuit_unitary(int n_qubits, int n_gates, const qf_loc* locations,
                       const qf_c128* gates, qf_c128* C_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* QFACTOR_H */
