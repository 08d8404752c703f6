/*
 * lq.h -- C ABI of the GB300 (sm_103a) dense state-vector library for the
 * method of arXiv 2512.23183 ("LogosQ").
 *
 * State vectors are caller-owned device buffers of 2^n complex128 amplitudes
 * stored as interleaved (re, im) doubles (CUDA double2), the Complex64 dense
 * state of Sec. II-B.  Qubit q is bit n-1-q of the amplitude index
 * (MSB-first, Alg. 1 and Alg. 4).
 *
 * Conventions shared by every entry point:
 *   - return an lq_status, never throw, never exit; on failure
 *     lq_last_error() returns a message for the calling thread;
 *   - device memory (states, scratch, workspaces) is owned by the caller and
 *     never freed by the library; the library allocates no device memory;
 *   - host arrays (gate lists, parameters, Pauli terms) are read during the
 *     call only;
 *   - work is enqueued on `stream` (a cudaStream_t; NULL = the legacy default
 *     stream); calls are asynchronous unless they return host values, in which
 *     case they synchronise `stream` before returning;
 *   - sizes: 1 <= n <= 34 qubits;
 *   - constant device tables (dyadic phases for merged phase gates, QFT
 *     twiddles) are filled once per device by the first call that needs
 *     them, on a private stream that the call waits for, so a first call on
 *     any thread or stream sees complete tables; that first fill is refused
 *     with LQ_ERR_CUDA when `stream` is being captured into a CUDA graph:
 *     make one uncaptured call of the same kind on each device first.
 *
 * Validation stands in for the compile-time checks of Sec. III-B
 * (parameter bounds, parametrised versus fixed gates):
 *   LQ_ERR_INVALID_ARG for a qubit outside [0, n), a repeated qubit within a
 *   gate, a parameter index >= np, a parameter on a fixed gate, a Pauli mask
 *   with bits >= n, a NULL pointer where data is needed, or n out of range;
 *   LQ_ERR_NONFINITE for NaN/Inf in parameters, angles, matrices or
 *   coefficients (App. D: explicit error reporting instead of silent NaN).
 */
#ifndef LQ_API_H_
#define LQ_API_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* lq_stream; /* == cudaStream_t */

typedef enum {
  LQ_OK = 0,
  LQ_ERR_INVALID_ARG = 1,
  LQ_ERR_UNSUPPORTED = 2,
  LQ_ERR_NONFINITE = 3,
  LQ_ERR_OOM = 4,       /* workspace / scratch smaller than required */
  LQ_ERR_CUDA = 5,      /* a CUDA runtime call failed */
  LQ_ERR_TIMEOUT = 6    /* a bounded device-side wait gave up */
} lq_status;

/* Gate kinds.  Matrices are over the gate's listed qubits, the first listed
 * qubit being the most significant bit of the local index (the two-qubit
 * index (s1, s2) of Sec. II-C).  Controlled gates list their control(s)
 * first.  Rotations are R_P(theta) = exp(-i theta sigma_P / 2) (Sec. III-A). */
typedef enum {
  LQ_H = 0,   /* Hadamard [[1,1],[1,-1]]/sqrt2 (App. C)                     */
  LQ_X,       /* Pauli X                                                     */
  LQ_Y,       /* Pauli Y [[0,-i],[i,0]]                                      */
  LQ_Z,       /* Pauli Z                                                     */
  LQ_S,       /* diag(1, i)                                                  */
  LQ_SDG,     /* diag(1, -i)                                                 */
  LQ_T,       /* diag(1, e^{i pi/4})                                         */
  LQ_TDG,     /* diag(1, e^{-i pi/4})                                        */
  LQ_RX,      /* exp(-i theta X/2)                                           */
  LQ_RY,      /* exp(-i theta Y/2)                                           */
  LQ_RZ,      /* exp(-i theta Z/2)                                           */
  LQ_P,       /* diag(1, e^{i theta})                                        */
  LQ_U1,      /* 2x2 unitary in mat[0..7]                                    */
  LQ_CNOT,    /* Alg. 1: (control, target)                                   */
  LQ_CY,      /* controlled Y                                                */
  LQ_CZ,      /* diag(1,1,1,-1)                                              */
  LQ_CP,      /* diag(1,1,1,e^{i theta}), the controlled phase of Alg. 3     */
  LQ_SWAP,    /* Alg. 3 swaps                                                */
  LQ_CRX,     /* |0><0| (x) I + |1><1| (x) RX(theta)                         */
  LQ_CRY,     /* |0><0| (x) I + |1><1| (x) RY(theta) (App. D circuit)        */
  LQ_CRZ,     /* |0><0| (x) I + |1><1| (x) RZ(theta)                         */
  LQ_RXX,     /* exp(-i theta X(x)X / 2) (Sec. VII-A Trotter gates)          */
  LQ_RYY,     /* exp(-i theta Y(x)Y / 2)                                     */
  LQ_RZZ,     /* exp(-i theta Z(x)Z / 2)                                     */
  LQ_CCX,     /* Toffoli, Alg. 4: (control1, control2, target)               */
  LQ_U2,      /* 4x4 unitary in mat[0..31]                                   */
  LQ_GATE_KIND_COUNT
} lq_gate_kind;

/* One operation of a circuit (the Operation/Circuit of Sec. II-A flattened
 * into plain data).  The angle used is params[param] + angle when
 * param >= 0, else the fixed angle.  mat holds row-major (re, im) pairs for
 * LQ_U1 (8 doubles) and LQ_U2 (32 doubles). */
typedef struct {
  int32_t kind;
  int32_t qubits[3];
  int32_t param;
  int32_t reserved;
  double angle;
  double mat[32];
} lq_gate;

/* One term c * P of a Pauli sum H = sum_t c_t P_t (Sec. VI-A).  P acts on the
 * index as P|s> = i^{ny} (-1)^{popcount(s & zmask)} |s ^ xmask>, where bit b
 * of xmask (zmask) is set when the qubit n-1-b carries X or Y (Z or Y) and
 * ny counts the Y factors (popcount(xmask & zmask)). */
typedef struct {
  double coeff;
  uint64_t xmask;
  uint64_t zmask;
} lq_pauli_term;

/* Gradient methods of lq_param_shift_grad. */
typedef enum {
  LQ_PSR_PLAIN = 0,   /* 2P+1 separate circuit runs, as ParameterShift does  */
  LQ_PSR_BATCHED = 1  /* all shifted circuits in one persistent launch        */
} lq_psr_method;

/* QFT methods of lq_qft. */
typedef enum {
  LQ_QFT_FFT = 0,   /* Alg. 2: inverse FFT / sqrt(N) */
  LQ_QFT_GATES = 1  /* Alg. 3: H, CP(pi/2^(j-i)), SWAP on the dense state */
} lq_qft_method;

/* Message of the last failed call on this thread ("" if none). */
const char* lq_last_error(void);

/* Library version string. */
const char* lq_version(void);

/* Measured FP64 FMA throughput of the current device, in TFLOP/s (an FMA
 * counts 2 flops): `reps` timed launches (after one warm-up) of a kernel of
 * independent DFMA chains with no memory traffic, filling every SM, timed
 * with CUDA events on `stream`; the best launch is reported (and its
 * milliseconds in *ms_best when not NULL).  The roofline denominator of the
 * FP64-bound kernels (no paper counterpart: measurement only).  Allocates
 * nothing; synchronises `stream`.  LQ_ERR_INVALID_ARG for reps outside
 * [1, 1000] or a NULL tflops. */
lq_status lq_measure_fp64_fma(int reps, double* tflops, double* ms_best, lq_stream stream);

/* Measured FP64 rate, in TFLOP/s, of the access pattern every state-sized
 * tile pass runs, without its global-memory traffic: each CTA (as many as
 * fit per SM) holds a 2^12-amplitude complex128 tile in shared memory and
 * applies tangent-form rotations (two loads, four FMAs and two stores per
 * amplitude pair) on tile bits 0..11 in turn, 2400 sweeps with a barrier
 * after each.  The practical ceiling of the tile kernels, beside the DFMA
 * rate of lq_measure_fp64_fma (no paper counterpart: measurement only).
 * Timing, arguments and errors as lq_measure_fp64_fma. */
lq_status lq_measure_fp64_tile_sweep(int reps, double* tflops, double* ms_best, lq_stream stream);

/* Parse a Pauli string (character q acts on qubit q; one of I X Y Z, length
 * n) into a term.  Host only. */
lq_status lq_pauli_from_string(const char* s, int n, double coeff, lq_pauli_term* out);

/* |basis>: amplitude `basis` = 1, all others 0 (DenseState::zero_state,
 * Sec. II-B, for basis = 0).  amps: device, 2^n double2. */
lq_status lq_state_init(void* amps, int n, uint64_t basis, lq_stream stream);

/* Apply the circuit in list order (Circuit::execute, Sec. II-A) in place.
 * gates: host array of ng gates; params: host array of np doubles (may be
 * NULL when np == 0).  Each gate is a direct bitwise update of amplitude
 * pairs or quads (Sec. IV-A, Alg. 1, Alg. 4); gates are grouped into
 * shared-memory tile passes so each pass reads and writes the state once. */
lq_status lq_apply_circuit(void* amps, int n, const lq_gate* gates, int ng,
                           const double* params, int np, lq_stream stream);

/* QFT|x> = N^{-1/2} sum_k e^{2 pi i x k / N} |k> (Sec. IV-B) in place;
 * inverse = 1 applies the inverse QFT.  method LQ_QFT_FFT follows Alg. 2,
 * LQ_QFT_GATES follows Alg. 3.  Neither method needs scratch: pass NULL/0. */
lq_status lq_qft(void* amps, int n, int inverse, int method, void* scratch,
                 size_t scratch_bytes, lq_stream stream);

/* Bytes of device workspace lq_expval_pauli_sum needs. */
size_t lq_expval_workspace_size(int n, int nt);

/* E = sum_t c_t Re <psi|P_t|psi> (Sec. VI-A, Sec. VII-A-2) for the state in
 * `amps` (device, read only).  out: host double; the call synchronises
 * `stream`.  workspace: device, >= lq_expval_workspace_size(n, nt) bytes. */
lq_status lq_expval_pauli_sum(const void* amps, int n, const lq_pauli_term* terms, int nt,
                              double* out, void* workspace, size_t ws_bytes,
                              lq_stream stream);

/* Same, asynchronous: the result is written to the device double out_dev. */
lq_status lq_expval_pauli_sum_async(const void* amps, int n, const lq_pauli_term* terms,
                                    int nt, double* out_dev, void* workspace,
                                    size_t ws_bytes, lq_stream stream);

/* Allocation-free <H>.  The paper has no counterpart to this entry point.
 * It computes the same E as lq_expval_pauli_sum for callers that cannot
 * allocate device memory -- code embedded in a host application whose device
 * memory belongs to an allocator it cannot call, or a plugin that is handed
 * only a state pointer -- so it needs no workspace: its partial sums live in
 * one fixed array inside the library (4096 doubles = 32 KiB), which every GPU
 * that loads the library holds until the process exits.  Limits: at most 640
 * terms with at most 240 distinct X masks; larger sums return
 * LQ_ERR_INVALID_ARG with a message (use lq_expval_pauli_sum then).  The
 * first call on a device looks up the array's device address with that device
 * current; make that first call before any stream capture.  All calls share
 * the one array, so calls whose work overlaps on the GPU (several streams or
 * threads at once) race: serialise them.  No cudaMalloc, cudaFree or other
 * allocating call is made.  out: host double; the call synchronises
 * `stream`. */
lq_status lq_expval_pauli_sum_noalloc(const void* amps, int n, const lq_pauli_term* terms,
                                      int nt, double* out, lq_stream stream);

/* out = H psi for H = sum_t c_t P_t (device buffers, out != in). */
lq_status lq_apply_pauli_sum(void* out, const void* in, int n, const lq_pauli_term* terms,
                             int nt, lq_stream stream);

/* Bytes of device workspace lq_param_shift_grad needs for this problem. */
size_t lq_param_shift_workspace_size(int n, int np, int nt, int method);

/* Energy E(theta) and its parameter-shift gradient (Eq. parameter_shift,
 * s = pi/2; ParameterShift::compute_gradient of Sec. III-C):
 *   grad[i] = ( E(theta + s e_i) - E(theta - s e_i) ) / 2,
 * every evaluation starting from |0...0>.  Every parameter must drive exactly
 * one gate whose generator has two eigenvalues one apart (RX, RY, RZ, P, CP,
 * RXX, RYY, RZZ), else LQ_ERR_UNSUPPORTED (controlled rotations need the
 * four-term rule, see lq_param_shift_grad_general).  energy: host double;
 * grad: host array of np doubles; the call synchronises `stream`. */
lq_status lq_param_shift_grad(int n, const lq_gate* gates, int ng, const double* params,
                              int np, const lq_pauli_term* terms, int nt, int method,
                              double* energy, double* grad, void* workspace,
                              size_t ws_bytes, lq_stream stream);

/* Generalised shift rules: a parameter may drive several gates (the
 * derivative sums the per-occurrence shifts) and controlled rotations
 * CRX/CRY/CRZ use the four-term rule with shifts pi/2 and 3pi/2 and weights
 * (sqrt2 +- 1) / (4 sqrt2) (the generalised rules cited in Sec. III-A).
 * Always batched. */
size_t lq_param_shift_general_workspace_size(int n, const lq_gate* gates, int ng,
                                             int np, int nt);
lq_status lq_param_shift_grad_general(int n, const lq_gate* gates, int ng,
                                      const double* params, int np,
                                      const lq_pauli_term* terms, int nt, double* energy,
                                      double* grad, void* workspace, size_t ws_bytes,
                                      lq_stream stream);

/* Bytes of device workspace lq_adjoint_grad needs. */
size_t lq_adjoint_workspace_size(int n, int ng, int np, int nt);

/* Energy and exact gradient by reverse-mode (adjoint) differentiation: the
 * state psi_L = U_L...U_1|0>, lambda = H psi_L, then for k = L..1
 * grad[param(k)] += d/dtheta <psi|H|psi> through gate k, computed from
 * <lambda_k| dU_k |psi_{k-1}>, with psi_{k-1} = U_k^dag psi_k and
 * lambda_{k-1} = U_k^dag lambda_k.  Holds two states; any parametrised gate
 * kind is allowed and a parameter may drive several gates.  energy/grad:
 * host; the call synchronises `stream`. */
lq_status lq_adjoint_grad(int n, const lq_gate* gates, int ng, const double* params, int np,
                          const lq_pauli_term* terms, int nt, double* energy, double* grad,
                          void* workspace, size_t ws_bytes, lq_stream stream);

/* First-order Trotter-Suzuki evolution (Eq. trotter, Sec. VII-A):
 *   H(t) = sum_k c_k P_k + h(t) sum_f d_f F_f,  h(t) = A sin(omega t),
 * `steps` steps of dt; step j applies exp(-i c_k P_k dt) for the static
 * terms in order, then exp(-i h(t_j) d_f F_f dt) for the field terms in
 * order, t_j = j dt.  In place on `amps`. */
lq_status lq_trotter_evolve(void* amps, int n, const lq_pauli_term* terms, int nt,
                            const lq_pauli_term* field, int nf, double A, double omega,
                            double dt, int steps, lq_stream stream);

/* ---------------------------------------------------------------------------
 * Plans: what a call will launch, for measurement and tuning.  FP64 flops
 * count what the kernels execute (FMA = 2 flops, in the forms the library
 * uses: tangent-form rotations, deferred scalars); dram_bytes is the minimal
 * traffic of the launches (each tile pass reads and writes the state once:
 * 32 * 2^n bytes).
 */
typedef struct {
  int32_t npasses;      /* kernel launches of the state-vector passes */
  int32_t tile_bits;    /* tile width k of the passes (max over passes) */
  double dp_flops;      /* FP64 flops executed */
  double dram_bytes;    /* minimal DRAM bytes moved */
} lq_plan_info;

/* Plan of lq_apply_circuit for this circuit (host only, no GPU needed). */
lq_status lq_circuit_plan(int n, const lq_gate* gates, int ng, const double* params, int np,
                          lq_plan_info* out);

/* Plan of lq_qft (host only): the forward transform, or either direction. */
lq_status lq_qft_plan(int n, int method, lq_plan_info* out);
lq_status lq_qft_plan_dir(int n, int method, int inverse, lq_plan_info* out);

/* ---------------------------------------------------------------------------
 * Schedule autotuner (no counterpart in the paper, whose CPU library has no
 * tile schedule).  lq_autotune_circuit times the tile-pass schedules of
 * lq_apply_circuit for this circuit over tile width k (9..12, at most n),
 * contiguous low bits m (5, 6) and the per-CTA phase table (on, off), on the
 * caller's scratch state `scratch` (device, 2^n double2, overwritten; the
 * call synchronises `stream`), and records the fastest in a process-wide
 * cache keyed by (GPU name and SM count, n, circuit structure: gate kinds,
 * qubits, which gates take parameters, fixed angles).  lq_apply_circuit and
 * lq_circuit_plan then use the recorded schedule for every circuit of that
 * structure, whatever its parameter values.  The cache is saved to / loaded
 * from a text file (one entry per line); lq_tune_cache_load merges entries
 * and fails with LQ_ERR_INVALID_ARG (cache unchanged) on a malformed line.
 */
typedef struct {
  int32_t tile_bits;    /* chosen k */
  int32_t low_bits;     /* chosen m */
  int32_t phase_table;  /* chosen per-CTA phase-table option (0/1) */
  int32_t candidates;   /* schedules timed */
  double ms;            /* best time (ms, min of two timed runs) */
  double ms_default;    /* time of the default schedule (k = 10, m = 5, table on) */
} lq_tune_result;

lq_status lq_autotune_circuit(void* scratch, int n, const lq_gate* gates, int ng,
                              const double* params, int np, lq_tune_result* out,
                              lq_stream stream);
/* Autotune the gate form of lq_qft (its H / CP gate list, forward or
 * inverse) like lq_autotune_circuit; lq_qft(method = LQ_QFT_GATES) then uses
 * the recorded schedule. */
lq_status lq_autotune_qft(void* scratch, int n, int inverse, lq_tune_result* out,
                          lq_stream stream);
lq_status lq_tune_cache_save(const char* path);
lq_status lq_tune_cache_load(const char* path);
lq_status lq_tune_cache_clear(void);
int lq_tune_cache_size(void);

/* Plan of lq_expval_pauli_sum for this term list (host only): npasses counts
 * the reads of the state (tile passes of the tiled kernel, plus one per X-mask
 * group evaluated by the untiled kernel); dram_bytes = 16 * 2^n per read. */
lq_status lq_expval_plan(int n, const lq_pauli_term* terms, int nt, lq_plan_info* out);

/* Plan of lq_adjoint_grad (host only): npasses counts every kernel launch of
 * the call (initialisation, forward passes, <H>, H psi, reverse passes,
 * gradient reduction); dp_flops counts the forward and reverse passes. */
lq_status lq_adjoint_plan(int n, const lq_gate* gates, int ng, const double* params, int np,
                          int nt, lq_plan_info* out);

/* ---------------------------------------------------------------------------
 * Uneven batches: many independent problems (each its own n, circuit and
 * Hamiltonian) in one persistent launch.  Problems are described by
 * lq_problem; results go to host arrays.
 */
typedef struct {
  int32_t n;
  int32_t ng;
  int32_t np;
  int32_t nt;
  int32_t want_grad;            /* 0: energy only; 1: energy and gradient */
  int32_t reserved;
  const lq_gate* gates;         /* host */
  const double* params;         /* host */
  const lq_pauli_term* terms;   /* host */
  double* energy;               /* host out */
  double* grad;                 /* host out (np doubles) when want_grad */
} lq_problem;

/* Device workspace needed to run `count` problems in one batched launch. */
size_t lq_batch_workspace_size(const lq_problem* problems, int count);

/* Run every problem's 2P+1 (or 1, energy only) circuits in one persistent
 * launch and write the energies/gradients.  Same gate restrictions as
 * lq_param_shift_grad.  Synchronises `stream`. */
lq_status lq_batch_param_shift(const lq_problem* problems, int count, void* workspace,
                               size_t ws_bytes, lq_stream stream);

/* Tile width of the persistent batched launch (lq_batch_param_shift and the
 * batched lq_param_shift_grad) for states larger than 2^12 amplitudes, timed
 * over 9..12 on the caller's workspace (sized by lq_batch_workspace_size /
 * lq_param_shift_workspace_size, which cover every width) and recorded per
 * batch structure (every problem's n, gate structure, circuit and term
 * counts).  A batch whose states all fit shared memory has nothing to tune:
 * candidates = 1.  Gradients computed while tuning are discarded. */
lq_status lq_autotune_batch(const lq_problem* problems, int count, void* workspace,
                            size_t ws_bytes, lq_tune_result* out, lq_stream stream);
lq_status lq_autotune_param_shift(int n, const lq_gate* gates, int ng, const double* params,
                                  int np, const lq_pauli_term* terms, int nt, void* workspace,
                                  size_t ws_bytes, lq_tune_result* out, lq_stream stream);

/* ---------------------------------------------------------------------------
 * VQE outer loop (Sec. VI-B): Adam on E(theta), each gradient on the GPU.
 * The paper's settings are lr = 1e-2, at most 350 iterations, tolerance 1e-7
 * on the energy change; beta1 = 0.9, beta2 = 0.999, eps = 1e-8 are Adam's
 * usual constants.  method 0: adjoint gradient; 1: batched parameter shift.
 */
typedef struct {
  double lr, beta1, beta2, eps, tol;
  int32_t max_iters, method;
} lq_adam_options;

size_t lq_vqe_workspace_size(int n, int ng, int np, int nt, int method);

/* params: host, in/out (updated in place).  energies: host, max_iters
 * doubles; energies[i] is E at the parameters of iteration i+1 (before its
 * update).  *iters = gradient evaluations made (the loop stops at max_iters
 * or when |E_t - E_{t-1}| < tol, without updating after that evaluation). */
lq_status lq_vqe_adam(int n, const lq_gate* gates, int ng, double* params, int np,
                      const lq_pauli_term* terms, int nt, const lq_adam_options* opt,
                      double* energies, int* iters, void* workspace, size_t ws_bytes,
                      lq_stream stream);

/* ---------------------------------------------------------------------------
 * Serving: a continuous-batching request server (an addition: the paper
 * has no serving layer).  Requests carry one circuit, its parameters
 * and a Pauli sum, energy only or energy and gradient (adjoint).  The server
 * admits a request when its footprint (lq_server_footprint) fits in the free
 * part of the caller's device arena and a worker slot is free; work of
 * different requests overlaps on the device (one stream per slot), and
 * small energy-only requests waiting together run in one batched launch.
 * Gates, parameters and terms are copied at submit.  A result does not
 * depend on what else is in flight.
 */
typedef struct lq_server lq_server;

typedef struct {
  int32_t n, ng, np, nt;
  int32_t want_grad;            /* 0: energy only; 1: energy and gradient */
  int32_t reserved;
  const lq_gate* gates;         /* host, copied */
  const double* params;         /* host, copied */
  const lq_pauli_term* terms;   /* host, copied */
} lq_request;

typedef struct {
  int64_t id;
  int32_t status;               /* lq_status of the request */
  int32_t np;
  double energy;
  double t_submit, t_start, t_done;   /* seconds, one monotonic clock */
} lq_result;

/* Device bytes one request occupies in the arena while it runs. */
size_t lq_server_footprint(int n, int want_grad, int ng, int np, int nt);

/* Create a server over the caller's device arena (current device) with
 * `slots` concurrent workers.  The arena stays owned by the caller and must
 * outlive the server. */
lq_status lq_server_create(void* arena, size_t arena_bytes, int slots, lq_server** out);

/* Queue a request; *id identifies it.  LQ_ERR_OOM if it can never fit. */
lq_status lq_server_submit(lq_server* server, const lq_request* req, int64_t* id);

/* Wait up to timeout_s seconds for request `id`; fills `res` and, for a
 * gradient request, grad[0..np).  LQ_ERR_TIMEOUT if not done in time (the
 * request stays queued).  A finished request is forgotten after this call. */
lq_status lq_server_wait(lq_server* server, int64_t id, double timeout_s, lq_result* res,
                         double* grad);

/* Stop the workers (after the running requests finish) and free the server;
 * requests still queued are dropped. */
lq_status lq_server_destroy(lq_server* server);

#ifdef __cplusplus
}
#endif

#endif /* LQ_API_H_ */
