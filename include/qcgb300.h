/*
 * qcgb300.h -- C ABI of the GB300 (sm_103a) state-vector gate engine.
 *
 * The library applies quantum gates to a dense state |phi> in C^(2^n) held in
 * device memory, following QCLAB++ (arXiv 2303.00123), Sec. 2:
 *
 *   |psi> = (I_l (x) U (x) I_r) |phi>                              (Eq. (1))
 *
 * Qubit numbering is Definition 1 (big-endian): qubit 0 is the most
 * significant bit of a basis index j, so qubit q has stride 2^(n-q-1).
 * Amplitudes are stored interleaved (re, im): complex<float> (QC_C64, 8 bytes)
 * or complex<double> (QC_C128, 16 bytes), index j at byte offset j*E.
 * Every update is in place (the paper's kernels overwrite their input, Fig. 4).
 *
 * Matrices are always passed by the caller as host arrays of FP64 (re, im)
 * pairs, row-major, and are copied during the call (the caller may free or
 * reuse them on return).  For a gate on target qubits (t_0, ..., t_{k-1}) the
 * row/column index of U is the big-endian number formed by the target bits,
 * t_0 being the most significant -- the order that Eq. (1) fixes for a gate
 * on adjacent qubits, kept for any placement (Sec. 2.3 remarks that the
 * 2-qubit algorithm also covers non-adjacent qubits, Fig. 1(e)).
 *
 * Execution: every apply call only enqueues kernels on the state's stream
 * (qc_set_stream; default: the legacy default stream) and returns.  Calls that
 * return host data (qc_expect, qc_state_copy_to_host, qc_apply_circuit with
 * per-gate timing) synchronise that stream.  There is no CPU fallback: when no
 * CUDA device is usable every call returns QC_ERR_CUDA.
 *
 * Errors: every int-returning call returns QC_OK (0) or a negative QC_ERR_*
 * code and then leaves a message in qc_last_error() (thread-local).  A call
 * that fails argument validation has no effect.  Asynchronous kernel faults
 * surface as QC_ERR_CUDA on a later synchronising call.
 *
 * Thread safety: distinct states may be used from distinct threads; a single
 * state must not be used concurrently.
 */
#ifndef QCGB300_H
#define QCGB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define QC_OK 0
#define QC_ERR_ARG (-1)         /* invalid argument (qubit out of range, duplicate qubit, ...) */
#define QC_ERR_OOM (-2)         /* device allocation failed */
#define QC_ERR_CUDA (-3)        /* a CUDA runtime call failed / no device */
#define QC_ERR_TIMEOUT (-4)     /* a bounded device-side wait gave up */
#define QC_ERR_UNSUPPORTED (-5) /* valid request that this build does not implement */

/* ---- element types ------------------------------------------------------ */
typedef enum { QC_C64 = 0, QC_C128 = 1 } qc_dtype;

/*
 * Arithmetic used for QC_C128 states.  GB300 executes FP64 at about 1/64 of
 * its FP32 rate, so a dense complex128 gate sweep done in FP64 is bound by the
 * FP64 pipe, not by HBM.  QC_ARITH_F32X2 keeps the state in IEEE binary64 but
 * computes each gate in float-float arithmetic on the FP32/integer pipes
 * (operands split exactly into two floats, error-free products and sums),
 * with a per-gate relative error of about 2^-46.  QC_ARITH_AUTO picks F32X2
 * for complex128 and plain FP32 for complex64.
 */
typedef enum { QC_ARITH_AUTO = 0, QC_ARITH_NATIVE = 1, QC_ARITH_F32X2 = 2 } qc_arith;

/* ---- state ---------------------------------------------------------------
 * An opaque handle that owns (or borrows) 2^n amplitudes in device memory.
 * Limits: 1 <= n <= 36 (the amplitude count is indexed with 64-bit ints).   */
typedef struct qc_state qc_state;

/* Allocate a library-owned state on the current device, initialised to
 * |0...0>.  *out receives the handle.  QC_ERR_OOM if the device cannot hold
 * 2^n * E bytes. */
int qc_state_alloc(int n, int dtype, qc_state** out);

/* Borrow caller-owned device memory (for instance a torch tensor) of 2^n
 * amplitudes of `dtype`, 32-byte aligned (one 32-byte sector per access).  Its contents are used as the
 * state; qc_state_free does not free it. */
int qc_state_wrap(void* dev_ptr, int n, int dtype, qc_state** out);

/* Release the handle (and the memory, when library-owned).  NULL is a no-op. */
int qc_state_free(qc_state* s);

/* Set the state to the computational basis state |x>, 0 <= x < 2^n. */
int qc_state_set_basis(qc_state* s, uint64_t x);

/* Copy all 2^n amplitudes device -> host (synchronous; QC_ERR_TIMEOUT as
 * described at qc_device_status) or host -> device
 * (ordered on the state's stream; the host buffer must stay valid until the
 * stream reaches the copy when it is pinned, else the call is synchronous).
 * `host` holds 2^n interleaved (re, im) pairs of the state's element type.
 * Host -> device from page-locked host memory that CUDA has mapped
 * (cudaHostRegister, cudaHostAlloc; 16-byte aligned) is done by a kernel
 * reading the mapped memory, on the state's stream; from other memory by the
 * copy engine. */
int qc_state_copy_to_host(const qc_state* s, void* host);
int qc_state_copy_from_host(qc_state* s, const void* host);

/* Query: device pointer, qubit count, dtype. */
int qc_state_info(const qc_state* s, void** dev_ptr, int* n, int* dtype);

/* Bind a cudaStream_t (passed as void*) on which all later work on `s` is
 * enqueued.  NULL selects the legacy default stream. */
int qc_set_stream(qc_state* s, void* cuda_stream);

/* Select the arithmetic for complex128 gate sweeps (qc_arith). */
int qc_set_arith(qc_state* s, int arith);

/* Dense blocks on k = 3..5 qubits (fused gates, qc_apply_kq) run on the
 * tensor cores when enable != 0, else on the CUDA cores: complex64 with
 * split-TF32 products (hi*hi + hi*lo + lo*hi, FP32 accumulators); complex128
 * under QC_ARITH_F32X2 with exact fp16 digit slices (entries rounded to 48
 * bits against their group's largest exponent, six base-2^8 digits; the
 * matrix in seven; exact integer level sums; error about 2^-47 of each
 * 128-group's largest amplitude).  Every choice below computes the same
 * products in the same accumulators, so results are bit-identical; they differ
 * only in how a tile's work is scheduled:
 *   enable = 1 (the default): complex128 blocks on k = 4, 5 qubits in the
 *     warp-specialised pipeline (producer warps make the next tile's digits,
 *     an MMA warp and epilogue warps work on other tiles at the same time);
 *     complex128 k = 3 and all complex64 blocks in the one-role kernel (all
 *     warps load, split, wait for the MMAs and store; two CTAs per SM) --
 *     the faster of the two for each, as measured;
 *   enable = 2: the one-role kernel, with the tiles of complex128 blocks that
 *     hold exactly their groups (no control below the tile's run length)
 *     staged by the Tensor Memory Accelerator -- measured slower (the staging
 *     buffer's traffic competes with the MMAs' operand reads);
 *   enable = 3: the pipeline for every block of both types;
 *   enable = 4: the one-role kernel for every block. */
int qc_set_fused_tc(qc_state* s, int enable);

/* complex128 float-float dense and phase sweeps: enable = 0 scalar FP32
 * instructions; 1 packed FP32-pair instructions (add/mul/fma .f32x2, two FP32
 * operations per issue slot; the same operations in the same order as the
 * scalar form, so results are identical); 2 (the default) as 1, except that
 * dense 2-qubit gates sum their products in fixed-binade chains (per output
 * row, t <- fma(u, x, t) in one binade above every partial sum, so each
 * step's rounding error is recovered exactly; six instructions per product
 * instead of twelve) -- error about 2^-42 of (row sum of |u|) * (largest
 * input of the group), against about 2^-44 of the summed |products|. */
int qc_set_packed(qc_state* s, int enable);

/* Tensor-core waits.  A fused-block kernel on the tensor cores (qc_set_fused_tc)
 * waits for its MMAs on an mbarrier with a poll limit.  A wait that reaches it
 * counts on a per-device counter, stops the kernel from taking further tiles
 * (the state is then incomplete) and, before the kernel frees its tensor
 * memory, waits for the MMAs already committed (default limit).  The calls
 * that synchronise -- qc_synchronize, qc_state_copy_to_host, qc_expect,
 * qc_expect_noalloc and qc_apply_circuit with gate_ms -- return
 * QC_ERR_TIMEOUT when the counter of the state's device is non-zero, and reset
 * it: a wait that gave up in work on any state of that device is reported by
 * the next such call.
 *
 * qc_device_status: *tc_timeouts = the current device's counter (0 in normal
 * operation), not reset.  Ordered after work on the legacy default stream and
 * on blocking streams, not after non-blocking streams: synchronise those
 * first. */
int qc_device_status(int* tc_timeouts);

/* Wait for every call enqueued on the state's stream; QC_ERR_TIMEOUT as
 * described above. */
int qc_synchronize(const qc_state* s);

/* Poll limit of the state's tensor-core MMA waits: polls > 0 sets it, 0
 * restores the default (2^24 polls, seconds), polls < 0 makes every first
 * wait give up without polling -- for testing the time-out path: the kernels
 * stop after their first tile and the next synchronising call returns
 * QC_ERR_TIMEOUT. */
int qc_set_wait_limit(qc_state* s, long long polls);

/* ---- single gates --------------------------------------------------------
 * qc_apply_1q: Sec. 2.1, Alg. 1.  U[8] = 2x2 complex row-major
 * (u00, u01, u10, u11), each as (re, im).  For every pair of basis indices
 * (a_j, b_j) that differ only in the target bit (0 in a_j, 1 in b_j):
 *   psi[a_j] = u00 phi[a_j] + u01 phi[b_j];  psi[b_j] = u10 phi[a_j] + u11 phi[b_j].
 * Diagonal, anti-diagonal and permutation matrices are detected and applied
 * with the specialisations of Sec. 2.1 (Pauli X a swap, Z touching only b_j),
 * which only move the amplitudes they change. */
int qc_apply_1q(qc_state* s, const double U[8], int target);

/* qc_apply_c1q: Sec. 2.2, Alg. 2, and Sec. 2.4 (multi-controlled gates).
 * U acts on `target` only for basis indices whose bit of controls[i] equals
 * control_states[i] (0 or 1) for every i < ncontrols; all other amplitudes
 * are neither read nor written.  ncontrols may be 0.  Controls must be
 * distinct and differ from the target. */
int qc_apply_c1q(qc_state* s, const double U[8], const int* controls,
                 const int* control_states, int ncontrols, int target);

/* qc_apply_2q: Sec. 2.3, Alg. 3.  U4[32] = 4x4 complex row-major; the
 * row/column index is 2*bit(q0) + bit(q1) (Eq. (1) order; the paper's Alg. 3
 * labels the q0 offset as b_j, which contradicts Eq. (1) for non-symmetric
 * U4 -- this library follows Eq. (1)).  q0 != q1, any order, any distance.
 * SWAP is detected and only exchanges the two middle amplitudes. */
int qc_apply_2q(qc_state* s, const double U4[32], int q0, int q1);

/* qc_apply_kq: Sec. 2.4 (multi-qubit gates, generalised masks).  U is
 * 2^k x 2^k complex (2 * 4^k doubles), 1 <= k <= 5, targets `qubits[0..k)`
 * (qubits[0] = most significant index bit), optional controls as in
 * qc_apply_c1q.  Used for fused gate blocks. */
int qc_apply_kq(qc_state* s, const double* U, const int* qubits, int k,
                const int* controls, const int* control_states, int ncontrols);

/* ---- circuits ------------------------------------------------------------- */
#define QC_MAX_TARGETS 5
#define QC_MAX_CONTROLS 8

/* Named gates of the paper's circuits (Fig. 1 QFT: H, CP, SWAP; Fig. 5
 * Trotter circuit: Rz, Rx, CNOT) plus the usual Clifford+T set.
 * P(theta) = diag(1, e^{i theta}); RX/RY/RZ(theta) = exp(-i theta P / 2). */
typedef enum {
  QC_GATE_MATRIX = 0, /* explicit matrix (2^nq x 2^nq) in `matrix` */
  QC_GATE_H, QC_GATE_X, QC_GATE_Y, QC_GATE_Z, QC_GATE_S, QC_GATE_SDG,
  QC_GATE_T, QC_GATE_TDG, QC_GATE_P, QC_GATE_RX, QC_GATE_RY, QC_GATE_RZ,
  QC_GATE_SWAP
} qc_gate_kind;

typedef struct {
  int kind;                         /* qc_gate_kind */
  int nq;                           /* number of target qubits (1..5; SWAP: 2) */
  int nc;                           /* number of controls (0..QC_MAX_CONTROLS) */
  int qubits[QC_MAX_TARGETS];       /* targets, qubits[0] = MSB of U's index */
  int controls[QC_MAX_CONTROLS];
  int cstates[QC_MAX_CONTROLS];     /* 0 or 1 per control */
  double theta;                     /* angle of P, RX, RY, RZ */
  const double* matrix;             /* QC_GATE_MATRIX: 2 * 4^nq doubles, host memory */
} qc_gate;

typedef struct {
  int fuse_k;      /* 0 or 1: apply gate by gate; 2..5: greedy fusion into
                      k-qubit blocks applied as dense k-qubit gates, and runs
                      of commuting phase gates sharing a qubit applied as one
                      linear-phase sweep (qc_block kind 1) */
  int use_graph;   /* 1: capture the launches in a CUDA graph and replay it */
  float* gate_ms;  /* optional host array of at least ngates entries: entry i
                      receives the device time (ms) of launch i (a gate or a
                      fused block; *nlaunch entries are written); synchronises.
                      With use_graph the replay is timed as a whole and spread
                      evenly over the launches. */
  int* nlaunch;    /* optional out: number of kernel launches enqueued */
} qc_opts;

/* Apply `ngates` gates in order (Sec. 3: the circuit applies its gates one by
 * one to the state).  opts may be NULL (defaults: no fusion, no graph). */
int qc_apply_circuit(qc_state* s, const qc_gate* gates, int ngates, const qc_opts* opts);

/* One launch of a fusion plan.  kind 0: dense U on `qubits` (qubits[0] =
 * MSB of U's index), applied only where the controls hold.  kind 1: a run of
 * commuting phase gates that all involve qubit `anchor` (for instance the
 * controlled phases of one QFT stage, Fig. 1), applied in one sweep:
 * amplitudes whose anchor bit is 1 are multiplied by
 * exp(i (theta0 + sum_j bit(lin_qubits[j]) * lin_theta[j])).  A kind-1 block
 * with k = 1 first applies the 2x2 matrix U to qubits[0] == anchor in the same
 * sweep: a lone 1-qubit gate on the anchor right before the run (the Hadamard
 * of a QFT stage) joins it when the anchor's stride is at least 16
 * amplitudes (qubit index <= n - 5).  kind 2: a run of two or more SWAP
 * gates on disjoint qubit pairs (the final swaps of the QFT, Fig. 1) applied
 * as one sweep that permutes the index bits. */
#define QC_MAX_LIN 36
typedef struct {
  int k;
  int qubits[QC_MAX_TARGETS];
  int nc;
  int controls[QC_MAX_CONTROLS];
  int cstates[QC_MAX_CONTROLS];
  double U[2 * 32 * 32];            /* 2^k x 2^k complex, row-major (re, im) */
  int kind;                         /* 0: matrix block, 1: linear phase run,
                                       2: SWAPs on disjoint qubit pairs
                                       (lin_qubits[2j], lin_qubits[2j+1]),
                                       j < nlin / 2, as one bit permutation */
  int anchor;
  int nlin;
  int lin_qubits[QC_MAX_LIN];
  double lin_theta[QC_MAX_LIN];
  double theta0;
} qc_block;

/* Host-only: the launch plan qc_apply_circuit would execute for these gates
 * on an n-qubit state with fusion width fuse_k (0/1: none).  Writes at most
 * max_blocks blocks and the total count to *nblocks (QC_ERR_ARG if more than
 * max_blocks are needed).  Needs no GPU; used to inspect and test fusion. */
int qc_fuse_plan(int n, const qc_gate* gates, int ngates, int fuse_k,
                 qc_block* blocks, int max_blocks, int* nblocks);

/* ---- OpenQASM 2.0 input and output ----------------------------------------
 * The paper's library reads and writes circuits as openQASM (Sec. 3).
 * Register qubits are numbered in declaration order: element 0 of the first
 * qreg is qubit 0 (the most significant index bit, Definition 1).
 *
 * qc_qasm_parse: read an OpenQASM 2.0 program (text, NUL-terminated host
 * string) into a program object owned by the caller (free it with
 * qc_program_free).  Reads qreg/creg, gate definitions (expanded), parameter
 * expressions (numbers, pi, + - * / ^, sin cos tan exp ln sqrt), register
 * broadcasting and the gates U u3 u u2 u1 p CX cx id u0 x y z h s sdg t tdg sx
 * sxdg rx ry rz cy cz ch swap ccx cswap crx cry crz cu1 cp cu3 cu rzz rxx
 * (U(t,f,l) = [[cos t/2, -e^{il} sin t/2], [e^{if} sin t/2, e^{i(f+l)} cos t/2]]).
 * measure and barrier are skipped and counted; reset, if and opaque return
 * QC_ERR_UNSUPPORTED; syntax errors, unknown gates and registers, out-of-range
 * indices return QC_ERR_ARG with the line in qc_last_error(). */
typedef struct qc_program qc_program;
int qc_qasm_parse(const char* text, qc_program** out);
/* Number of qubits, of gates, and of skipped measure/barrier statements. */
int qc_program_info(const qc_program* p, int* nqubits, int* ngates, int* nignored);
/* The program's gate records (matrices owned by the program), ready for
 * qc_apply_circuit; valid until qc_program_free.  NULL for an empty program. */
const qc_gate* qc_program_gates(const qc_program* p);
int qc_program_free(qc_program* p);

/* qc_qasm_write: the gate list as an OpenQASM 2.0 program over one register
 * q[n].  Named gates map to their qelib1 names (controlled X/Y/Z/H, P, RX,
 * RY, RZ with one control, ccx, cswap); control states 0 are conjugated with
 * x; a 1-qubit matrix becomes u3 (its global phase, unobservable, dropped) and
 * a singly controlled one cu3 followed by u1 on the control (exact).  Other
 * gates (k >= 2 matrices, more controls) return QC_ERR_UNSUPPORTED.  Writes at
 * most cap bytes including the NUL to buf (buf may be NULL to query *len, the
 * length without the NUL). */
int qc_qasm_write(int n, const qc_gate* gates, int ngates, char* buf, size_t cap, size_t* len);

/* ---- batches of circuits -----------------------------------------------------
 * Many independent circuits of different sizes and depths run in one
 * persistent kernel launch (optionally captured in a CUDA graph and replayed).
 * A circuit whose state fits in a CTA's shared memory (complex64 n <= 13,
 * complex128 n <= 12) is simulated there from |0...0> and written to its state
 * once; larger ones are swept in global memory, by one CTA or by a team of up
 * to 16 CTAs (one per 8 MB of state, or the tuned size), which split every
 * gate block and meet at a bounded barrier between blocks; a barrier that
 * gives up makes qc_batch_launch return QC_ERR_TIMEOUT (results incomplete).
 * CTAs take work from two atomic queues: teams, largest work first, and
 * single-CTA circuits, smallest first; a share of the CTAs proportional to the
 * single-CTA work starts on the second queue, and a CTA whose queue is empty
 * moves to the other.  Fusion (greedy, k <= 4) is applied per circuit;
 * fuse_k < 0 lets the library time the candidates (k in {2, 3, 4}) x (4, 8 or
 * 16 MB of state per team member) on the batch once and keep the fastest. */
typedef struct {
  int n;                 /* qubits of the circuit (must equal its state's n) */
  int ngates;
  const qc_gate* gates;  /* host memory, read during qc_batch_create only */
} qc_circuit_desc;

typedef struct {
  int fuse_k;     /* -1: autotune; 0 or 1: gate by gate; 2..4: fusion width */
  int use_graph;  /* 1: capture the launch in a CUDA graph, replayed by qc_batch_launch */
  void* stream;   /* cudaStream_t or NULL */
  long long spin_limit;   /* team-barrier wait limit in polls (0: default 2^26, ~10 s) */
  int test_skip_circuit;  /* testing only: 1 + index of a circuit whose member ... */
  int test_skip_member;   /* ... never arrives at its team barriers (0 = off) */
} qc_batch_opts;

typedef struct qc_batch qc_batch;

/* Plan a batch: states[i] (all of one dtype/arith, on one device) receives
 * circuit i applied to |0...0> at every qc_batch_launch.  The plan owns its
 * device tables; the states stay owned by the caller and must outlive it. */
int qc_batch_create(qc_state* const* states, const qc_circuit_desc* circs, int ncirc,
                    const qc_batch_opts* opts, qc_batch** out);
/* Run the batch (asynchronous unless an output pointer is given).
 * completion_ms: optional host [ncirc], time from the launch start to the end
 * of each circuit (device clock); total_ms: optional, whole launch.  Either
 * output synchronises the stream. */
int qc_batch_launch(qc_batch* b, double* completion_ms, double* total_ms);
/* Chosen fusion width and total number of ops (gates or fused blocks). */
int qc_batch_info(const qc_batch* b, int* fuse_k, int* nops, int* nsmem_circuits);
int qc_batch_free(qc_batch* b);

/* ---- observables ---------------------------------------------------------
 * A Pauli sum H = sum_t coeffs[t] * P_t; term t consists of the (letter,
 * qubit) pairs with indices offsets[t] .. offsets[t+1]-1 of `letters`
 * ('X', 'Y', 'Z' or 'I') and `qubits`.  All arrays are host memory. */
typedef struct {
  int nterms;
  const double* coeffs;  /* nterms */
  const int* offsets;    /* nterms + 1 */
  const char* letters;
  const int* qubits;
} qc_pauli_sum;

/* *out = <psi| H |psi> (real part), copied to the host (synchronises the
 * state's stream); the state is not modified.  The terms are evaluated in
 * passes over tiles of the state (see qc_expect_passes).  complex128:
 * amplitudes split into float pairs (47 bits, truncated); each thread's sum of
 * a pair term's products over its share of a tile accumulates in a
 * fixed-exponent chain (hi*hi products added exactly to the high word, their
 * rounding remainders -- exact to 2^-24 of themselves -- and the hi*lo cross
 * terms in a second word); diagonal terms use |psi|^2 on the same fixed grid,
 * whose Walsh-Hadamard sums are exact in the high word and FP32 in the low
 * word; weights and the sum over a tile's terms in float-float, FP64 across
 * tiles.  Observed: about 1e-15 from the exact value for O(1) coefficients
 * (worst case, every rounding at its maximum and aligned: about
 * 2^-35 * sum |c_t|).  complex64: the same arithmetic on the FP32 amplitudes
 * as they are (their products are exact in two floats), so the result is the
 * expectation of the complex64 state to about 1e-13 * sum |c_t|.
 * QC_ERR_TIMEOUT as described at qc_device_status.
 * Deterministic (fixed grid, fixed reduction order). */
int qc_expect(const qc_state* s, const qc_pauli_sum* H, double* out);

/* Host only: the number of passes qc_expect makes over an n-qubit state of
 * the given dtype for H.  A pass reads the state once, a tile of 2^12
 * amplitudes at a time (n >= 12: 3 low index bits and 9 generator masks;
 * smaller states: one tile), and evaluates every term whose X/Y qubits fall
 * in the span of the tile's bits; the tiles' bits are chosen per pass so
 * that few passes cover all terms (a nearest-neighbour chain of n qubits:
 * ceil((n - 3) / 9)).  Validates H like qc_expect (QC_ERR_ARG on a malformed
 * sum); an empty sum needs 0 passes. */
int qc_expect_passes(int n, int dtype, const qc_pauli_sum* H, int* npasses);

/* <psi| H |psi> like qc_expect, for callers that cannot allocate device memory
 * -- for instance an application whose own memory manager (a framework's
 * caching allocator) has already reserved the whole device, or a
 * latency-critical loop in which a cudaMalloc, which may synchronise the
 * device, is not acceptable.  This entry point allocates nothing: its
 * partial sums live in a fixed array inside the library's device code
 * (4096 + 1024 doubles, about 40 KB, held on every device that loads the
 * library until the process exits).  The paper has no counterpart; this is an
 * interface choice of this library.
 * It evaluates the sum the simple way, one sweep per distinct X/Y pattern
 * with FP64 products (slower than qc_expect's tiled passes; the two agree to
 * about 1e-15 for complex128 states).
 * Limit: at most 1023 sweeps, one per distinct X/Y pattern of the terms per
 * 64 terms; larger sums return QC_ERR_ARG before any work is enqueued.
 * The first call on a device looks the array's device address up (with that
 * device current): the first call should come before any stream capture.  Every
 * call in the process uses the same array and leaves its own sums in it.
 * Calls whose work overlapped on the GPU would race on it; the library
 * prevents that within a process by serialising the calls -- each holds a
 * lock until its stream has finished -- so calls from several threads or on
 * several streams run one after another.  Host memory for grouping the terms
 * is the only memory the call takes.  Synchronises the state's stream
 * (QC_ERR_TIMEOUT as described at qc_device_status). */
int qc_expect_noalloc(const qc_state* s, const qc_pauli_sum* H, double* out);

/* ---- gradients ------------------------------------------------------------
 * Adjoint (reverse-sweep) gradients of E(theta) = <psi(theta)| H |psi(theta)>,
 * |psi(theta)> = U_L ... U_1 |0...0>, for every parametric gate
 * U_l = exp(-i theta_l P_l / 2) (RX, RY, RZ without controls; P_l = X, Y, Z):
 *   dE/dtheta_l = Im <lambda_l| P_l |phi_l>,
 *   phi_l = U_l ... U_1 |0>,  lambda_l = U_{l+1}^dag ... U_L^dag H |psi>
 * (Jones & Gacon 2020, arXiv:2009.02823).  The library keeps two states per
 * parameter set (phi and lambda), walks the circuit backwards once, and fuses
 * each parametric gate's reduction with undoing that gate on both states.
 * Reductions (energy, gradients) accumulate in FP64 on the device.
 *
 * gates/ngates: the circuit (gates with k <= 2 targets; any controls).
 * thetas: host [batch][nparams], nparams = number of parametric gates, in
 *   circuit order; NULL means "use each gate's own theta" (batch must be 1).
 * energies: host [batch] out; grads: host [batch][nparams] out.
 * dtype: QC_C64 (FP32 sweeps, FP64 reductions) or QC_C128 (arith as in
 *   qc_arith).  stream: cudaStream_t or NULL.  Device workspace: 2 * batch
 *   states plus partial sums, allocated on the first call and reused (it grows
 *   when a larger problem arrives).  Synchronises the stream. */
typedef struct {
  int dtype;
  int arith;
  void* stream;
} qc_grad_opts;

int qc_adjoint_grad(int n, const qc_gate* gates, int ngates, const double* thetas, int batch,
                    const qc_pauli_sum* H, double* energies, double* grads, const qc_grad_opts* opts);

/* Number of parametric gates (RX/RY/RZ without controls) in a gate list. */
int qc_count_params(const qc_gate* gates, int ngates, int* nparams);

/* ---- one state over several shards ------------------------------------------
 * A state of n qubits split over 2^g shards (one per rank or GPU): the g most
 * significant qubits (qubits 0 .. g-1, Definition 1) are global -- rank r
 * holds the 2^(n-g) amplitudes whose top g index bits equal r, global qubit p
 * being bit g-1-p of r -- and each shard is an (n-g)-qubit state whose qubit j
 * is qubit g + j of the register.  The paper simulates on one GPU; this
 * layout extends Eq. (1)'s gate application to a register larger than one
 * device's memory.
 *
 * qc_shard_plan (host only, no GPU needed): the steps that apply `gates` to
 * the sharded state, in order.  QC_SHARD_GATE: apply `gate` (qubits numbered
 * within a shard) on every rank r with (r & rank_mask) == rank_val -- its
 * controls on global qubits became that condition.  QC_SHARD_EXCHANGE: every
 * rank r trades the half of its shard whose bit `local_qubit` equals
 * 1 - bit(r, rank_bit) with the same half of rank r ^ (1 << rank_bit) (the
 * partner's half whose bit equals bit(r, rank_bit)), which swaps a global and
 * a local qubit; a target on a global qubit is brought local this way first.
 * Uncontrolled SWAP gates only relabel qubits and move no data.  The plan ends
 * with the identity layout.  Gate records of QC_SHARD_GATE steps point at the
 * caller's matrices.  steps == NULL: only *nsteps is written; otherwise
 * QC_ERR_ARG when more than max_steps steps are needed (*nsteps says how many). */
#define QC_SHARD_GATE 0
#define QC_SHARD_EXCHANGE 1
typedef struct {
  int kind;            /* QC_SHARD_GATE or QC_SHARD_EXCHANGE */
  qc_gate gate;        /* QC_SHARD_GATE: the gate in shard qubit numbering */
  uint32_t rank_mask;  /* QC_SHARD_GATE: ranks r with (r & rank_mask) == rank_val apply it */
  uint32_t rank_val;
  int rank_bit;        /* QC_SHARD_EXCHANGE: partner rank = r ^ (1 << rank_bit) */
  int local_qubit;     /* QC_SHARD_EXCHANGE: shard qubit whose halves are traded */
} qc_shard_step;
int qc_shard_plan(int n, int g, const qc_gate* gates, int ngates, qc_shard_step* steps, int max_steps,
                  int* nsteps);

/* One exchange between two shards held by this process: a's half with bit
 * `local_qubit` = 1 - bit_a trades places with b's half with that bit = bit_a
 * (bit_a = the rank bit of a; b is the partner).  Same n and dtype; b's memory
 * must be accessible from a's device (the same device, or peer access enabled
 * by the caller).  Enqueued on a's stream; in place, one pass over the halves. */
int qc_shard_exchange(qc_state* a, qc_state* b, int local_qubit, int bit_a);

/* Copy the half of s whose bit `local_qubit` equals `bit` into a contiguous
 * device buffer of 2^(n-1) amplitudes (16-byte aligned), and back -- the two
 * ends of an exchange between processes (the buffer travels by NCCL
 * send/recv or any other transport).  Enqueued on s's stream. */
int qc_shard_pack(const qc_state* s, int local_qubit, int bit, void* dev_buf);
int qc_shard_unpack(qc_state* s, int local_qubit, int bit, const void* dev_buf);

/* ---- diagnostics ---------------------------------------------------------- */
/* Message of the last failing call on this thread ("" if none). */
const char* qc_last_error(void);
/* Library version string. */
const char* qc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* QCGB300_H */
