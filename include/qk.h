/*
 * qk.h -- C ABI of libqk, a GB300 (sm_103a) dense state-vector engine for the
 * gate-application hot path of Quantum-Kit (Tankasala & Ilatikhameneh,
 * arXiv:1908.07187).
 *
 * The calls follow the paper's command set (Q-Kit section): (1) add qubits,
 * (2) perform a gate operation, (3) measure, (4) define a custom gate "as a
 * matrix or as a function"; plus classical bits, copying a measured qubit into a
 * classical bit and classically controlled gates (Q-Kit section; Appendix A
 * commands AddCbits, Copy and "SigmaX 0,-k"), and viewing the state (Q-Kit
 * section, Fig. 1b).
 *
 * State layout: one context holds one state of n qubits as 2^n complex
 * amplitudes in device memory, interleaved (re, im), complex64 (2 x float) or
 * complex128 (2 x double).  Logical qubit q is index bit q of the state as seen
 * by qk_get_state / qk_set_state / qk_device_state.  Internally a SWAP only
 * relabels qubits; the relabelling is undone before any state leaves the library.
 *
 * Register convention (Appendix A): in any target list the first-listed qubit is
 * the most significant bit of the register value.
 *
 * Ownership: every input array is copied (or consumed) before the call returns;
 * the context owns all device memory it allocates; outputs go into caller
 * buffers.  Device memory is taken stream-ordered from one memory pool per device
 * that the library keeps: blocks freed by a destroyed context or batch stay in it
 * for reuse while any context or batch exists on that device, and the pool is
 * trimmed to empty when the last one is destroyed.  Errors: every call returns a qk_status; nothing throws across the ABI.
 * A call that fails argument checks leaves the context unchanged and sets the
 * message returned by qk_last_error.  A QK_ECUDA status means a CUDA call failed;
 * the context should then be destroyed.
 *
 * Ordering: gate, measure and cbit calls are enqueued on the context's CUDA
 * stream and return without waiting, unless they have a host output
 * (qk_measure with a non-NULL outcome, qk_read_cbits, qk_get_state, qk_sync).
 * Measurement outcomes and classical conditions are evaluated on the device, so a
 * classically controlled gate needs no host round trip.
 *
 * Thread safety: a context must not be used from two host threads at once.
 */
#ifndef QK_H
#define QK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qk_ctx qk_ctx;

typedef enum {
    QK_OK = 0,
    QK_EINVAL = -1,          /* bad argument (qubit out of range, duplicate, size) */
    QK_ENOMEM = -2,          /* device or host allocation failed                   */
    QK_EBUDGET = -3,         /* request exceeds the context's HBM budget           */
    QK_ENOTBIJECTIVE = -4,   /* a function gate is not a permutation               */
    QK_ENOTUNITARY = -5,     /* a matrix gate fails the unitarity tolerance        */
    QK_ECUDA = -6,           /* a CUDA runtime call failed                         */
    QK_ETIMEOUT = -7,        /* a device-side bounded wait gave up                 */
    QK_ESTATE = -8           /* call not valid in the context's current state      */
} qk_status;

typedef enum { QK_C64 = 0, QK_C128 = 1 } qk_precision;

/* Execution modes.  PLAIN: one kernel pass over the state per gate (the
 * unfused baseline).  FUSED: gates are queued; at a flush point a planner groups
 * runs of gates into shared-memory tile passes, so several gates cost one HBM
 * read+write of the state. */
typedef enum { QK_EXEC_PLAIN = 0, QK_EXEC_FUSED = 1 } qk_exec_mode;

typedef struct {
    int exec_mode;            /* qk_exec_mode; default QK_EXEC_FUSED                 */
    int tile_qubits;          /* fused tile width: 0 or 13 (the kernel's fixed width;
                                 other values are rejected with QK_EINVAL)           */
    int max_pending;          /* queued ops that force a flush; 0 = default (4096)   */
    int profile;              /* 1: time every launch with CUDA events (qk_profile)  */
    size_t hbm_budget_bytes;  /* 0 = no limit beyond free device memory             */
    int no_tensor_cores;      /* 1: dense 3..5-qubit blocks on CUDA cores only        */
    int reserved[7];          /* must be zero                                         */
} qk_options;

/* Built-in gate ids for qk_apply_gate (negative; user gates get ids >= 0).
 * Matrices are the textbook ones, row/column index = register value. */
enum {
    QK_GATE_X = -1,      /* SigmaX (Appendix A)                            */
    QK_GATE_Y = -2,
    QK_GATE_Z = -3,
    QK_GATE_H = -4,      /* Hadamard (Appendix A)                          */
    QK_GATE_S = -5,
    QK_GATE_SDG = -6,
    QK_GATE_T = -7,
    QK_GATE_TDG = -8,
    QK_GATE_U3 = -9,     /* params (theta, phi, lambda), OpenQASM U        */
    QK_GATE_P = -10,     /* params (phi): diag(1, e^{i phi}); with one
                            control this is CPHASE of Appendix A           */
    QK_GATE_RZ = -11,    /* params (theta): diag(e^{-i theta/2}, e^{i theta/2}) */
    QK_GATE_SWAP = -12   /* 2 targets (Appendix A SWAP after the QFT)      */
};

#define QK_MAX_QUBITS 36
#define QK_MAX_CONTROLS 16
#define QK_MAX_COND 16
#define QK_MAX_MATRIX_QUBITS 6
#define QK_MAX_PERM_QUBITS 30
#define QK_MAX_RPHASE_CBITS 62
#define QK_MAX_MODEXP_CONTROLS 48

/* Create a context with no qubits.  cuda_stream: a cudaStream_t to enqueue on
 * (borrowed, must outlive the context), or NULL for a context-owned stream.
 * opt may be NULL for defaults.  Errors: QK_EINVAL, QK_ECUDA. */
qk_status qk_create(qk_ctx **out, qk_precision precision, void *cuda_stream, const qk_options *opt);

/* Free every device and host resource of the context (waits for its stream). */
qk_status qk_destroy(qk_ctx *ctx);

/* "AddQubits" (Q-Kit section, Appendix A): append n qubits in |0> as the new
 * highest index bits (the state becomes |0...0> (x) psi).  *first_qubit_out (may
 * be NULL) receives the first new qubit's id.  Errors: QK_EINVAL (n < 1 or total
 * above QK_MAX_QUBITS), QK_EBUDGET, QK_ENOMEM. */
qk_status qk_add_qubits(qk_ctx *ctx, int n, int *first_qubit_out);

/* "AddCbits" (Appendix A): append n classical bits, initialised to 0. */
qk_status qk_add_cbits(qk_ctx *ctx, int n, int *first_cbit_out);

/* Define a gate "as a matrix" (Q-Kit section, command 4): k qubits (1..6), u is the
 * 2^k x 2^k matrix, row-major, interleaved (re, im) doubles, copied.  The matrix
 * must satisfy max |U^dagger U - I| <= unitarity_tol (QK_ENOTUNITARY otherwise).
 * *gate_id receives an id >= 0 valid for the life of the context.  A 3-, 4- or
 * 5-qubit complex64 gate without controls or classical condition, on a state of
 * at least 5 qubits, runs on the tensor cores (3xTF32 batched complex GEMM; a
 * 3- or 4-qubit gate as the 5-qubit block U (x) I with the other lowest physical
 * qubits); when its targets are not among the lowest physical qubits, one
 * relabelling pass first moves them there (the qubit map records the move, no
 * extra memory beyond the context's gather buffer).  Other dense gates run on
 * CUDA cores in the working precision.  qk_sync reports QK_ETIMEOUT if a
 * tensor-core pass hit its bounded wait. */
qk_status qk_define_gate_matrix(qk_ctx *ctx, int k, const double *u, double unitarity_tol, int *gate_id);

/* Define a gate "as a function" (Q-Kit section, command 4; QuModExpUaj of
 * Appendix A): on a w-qubit register (1..30), x -> c*x mod N for x < N and x
 * unchanged for x >= N.  Requires 2 <= N <= 2^w, c < N and gcd(c, N) = 1
 * (QK_ENOTBIJECTIVE otherwise).  Index arithmetic is exact (64-bit). */
qk_status qk_define_gate_perm_mulmod(qk_ctx *ctx, int w, uint64_t c, uint64_t N, int *gate_id);

/* Allocation-free variant of the mul-mod permutation gate.  The paper has no
 * counterpart: it exists for callers that cannot allocate device memory --
 * latency-critical loops where an allocation's implicit device synchronisation
 * would stall every other stream, host applications whose own memory manager
 * owns all device memory, and embedded users that must stay inside a device
 * memory budget reserved up front.
 * Applies x -> c*x mod N (x < N; x >= N unchanged) to the w-qubit register
 * targets[0..w-1] (first-listed = MSB) of the caller's device state d_state
 * (2^n amplitudes, interleaved (re, im), complex64 or complex128, 16-byte
 * aligned, qubit q = index bit q) wherever every control qubit is |1>.  The work
 * is enqueued on cuda_stream (NULL = the legacy default stream) and the call
 * returns without waiting.  Requires gcd(c, N) = 1, c < N, 2 <= N <= 2^w.
 * No device memory is allocated: the gather goes through one fixed scratch
 * array of QK_NOALLOC_SCRATCH_BYTES (16 MiB) that every GPU loading the library
 * holds until the process exits, so states above that size (complex64 above 21
 * qubits, complex128 above 20) are rejected with QK_EBUDGET.  The first call on
 * each device looks up the array's device address with that device current;
 * make that first call before any stream capture.  All calls share the one
 * array: calls whose GPU work may overlap (different streams or threads without
 * ordering between them) race and corrupt each other's results.
 * Errors: QK_EINVAL (bad pointer, alignment, qubit lists, N or c),
 * QK_ENOTBIJECTIVE (gcd(c, N) != 1), QK_EBUDGET (state too large), QK_ECUDA. */
#define QK_NOALLOC_SCRATCH_BYTES (16u << 20)
qk_status qk_apply_perm_mulmod_noalloc(void *d_state, int n, qk_precision precision, const int *targets, int w,
                                       const int *controls, int nc, uint64_t c, uint64_t N, void *cuda_stream);

/* Define a gate as an arbitrary function f on a w-qubit register value (1..24):
 * f is 2^w entries, copied, and must be a bijection (QK_ENOTBIJECTIVE). */
qk_status qk_define_gate_perm_table(qk_ctx *ctx, int w, const uint64_t *f, int *gate_id);

/* "GateOp" (Q-Kit section, command 2; Appendix A): apply a built-in or defined
 * gate.  targets: nt qubits (1 for 1-qubit built-ins, 2 for SWAP, k or w for
 * defined gates; first-listed = register MSB).  controls: nc quantum controls
 * (the gate acts where all are |1>).  cond_cbits: ncc classical bits that must
 * all be 1 for the gate to act (checked on the device when the gate runs; the
 * classically controlled "SigmaX 0,-k" of Appendix A).  params: np doubles for
 * parametrised built-ins.  Targets, controls must be distinct and in range. */
qk_status qk_apply_gate(qk_ctx *ctx, int gate_id, const int *targets, int nt,
                        const int *controls, int nc, const int *cond_cbits, int ncc,
                        const double *params, int np);

/* "RPhase 0,-e..-1" (Appendix A, nx2n branch): multiply the |1> component of
 * target by exp(i theta), theta = -2 pi sum_{l=1..ncb} c[cbits[l-1]] / 2^(l+1),
 * where cbits lists the classical bits most recent first.  The angle is formed on
 * the device from the cbit values (no host round trip).  ncb <= 62. */
qk_status qk_apply_rphase_cbits(qk_ctx *ctx, int target, const int *cbits, int ncb);

/* One stage of Kitaev's one-control-qubit order finding (Shor section, Fig. 2b
 * and Fig. 6b; the nx2n command script of Appendix A), fused: H(control); the
 * permutation gate perm_gate_id (from qk_define_gate_perm_mulmod or _table) on
 * targets[0..nt-1] controlled by `control`; the phase correction of
 * qk_apply_rphase_cbits(control, phase_cbits, ncb); H(control); measure
 * `control` with `uniform` into dest_cbit; X(control) if the outcome is 1.
 * Precondition: `control` is |0> (every amplitude with the control bit set is
 * zero), which holds at the start and after every stage.  The result equals the
 * six separate calls; the stage costs two passes over the control = 0 half (the
 * reduction's last block takes the decision).  Stream-ordered, no host round trip.
 * Errors: QK_EINVAL (bad ids, lists or uniform), QK_ENOMEM, QK_ECUDA. */
qk_status qk_apply_kitaev_stage(qk_ctx *ctx, int control, int perm_gate_id, const int *targets, int nt,
                                const int *phase_cbits, int ncb, double uniform, int dest_cbit);

/* "Measure" (Q-Kit section, command 3) with "Copy" into classical bits:
 * measures qubits[0..nq-1] one after another in list order.  For each, P0 is the
 * probability of reading 0 (summed in FP64 on the device), the outcome is
 * m = (uniforms[i] >= P0), the other branch is zeroed and the kept branch scaled
 * by 1/sqrt(P_m).  uniforms: nq values in [0, 1), copied.  dest_cbits: nq cbits
 * to receive the outcomes, or NULL.  outcome: if non-NULL, the call waits and
 * stores the register value (first-listed qubit = MSB); if NULL it returns
 * without waiting. */
qk_status qk_measure(qk_ctx *ctx, const int *qubits, int nq, const double *uniforms,
                     const int *dest_cbits, uint64_t *outcome);

/* Copy n classical bits starting at cbit 0 to host (waits for the stream). */
qk_status qk_read_cbits(qk_ctx *ctx, uint8_t *out, int n);

/* Overwrite cbits[first..first+n-1] with values 0/1 (stream-ordered). */
qk_status qk_write_cbits(qk_ctx *ctx, int first, const uint8_t *in, int n);

/* Copy the whole state (2^n amplitudes, logical qubit order) into a host buffer
 * of exactly bytes = 2^n * sizeof(amplitude); waits for the stream. */
qk_status qk_get_state(qk_ctx *ctx, void *host_out, size_t bytes);

/* Overwrite the state from a host buffer of exactly 2^n amplitudes (logical
 * order); the buffer is copied before the call returns. */
qk_status qk_set_state(qk_ctx *ctx, const void *host_in, size_t bytes);

/* Reset the state to |0...0> (stream-ordered, no host copy). */
qk_status qk_reset(qk_ctx *ctx);

/* Run every queued gate, undo qubit relabelling, and return the device pointer
 * and size of the state (logical order).  The pointer stays valid until the next
 * call on the context that changes the qubit count or applies a permutation
 * gate.  Does not wait for the stream. */
qk_status qk_device_state(qk_ctx *ctx, void **dptr, size_t *bytes);

/* Run every queued gate (fused mode); stream-ordered, does not wait. */
qk_status qk_flush(qk_ctx *ctx);

/* Flush and wait until all work on the context's stream has finished.  Returns
 * QK_ETIMEOUT (and clears the condition) if a kernel's bounded device-side wait
 * gave up since the last qk_sync; the context stays usable, the state is not. */
qk_status qk_sync(qk_ctx *ctx);

/* Self-test of that failure path (the paper has no counterpart): enqueues one
 * kernel that waits, with the same bounded mbarrier wait the tensor-core pass
 * uses but a limit of about a millisecond, on a barrier nothing arrives at.  The
 * wait runs out, the kernel records the timeout in the context's error flag and
 * returns; the next qk_sync returns QK_ETIMEOUT.  Nothing faults and the state
 * is untouched.  Errors: QK_ECUDA (launch failed). */
qk_status qk_selftest_timeout(qk_ctx *ctx);

/* Number of qubits / cbits of the context. */
int qk_num_qubits(const qk_ctx *ctx);
int qk_num_cbits(const qk_ctx *ctx);

/* CUDA-graph capture of a sequence of calls (no counterpart in the paper; it
 * replaces a host loop of launches, e.g. a whole Kitaev order-finding run, by one
 * graph launch).  qk_capture_begin flushes queued gates, undoes qubit
 * relabelling, and starts capturing the context's stream.  Between begin and end
 * only stream-ordered calls are allowed (gates, stages, measurements without an
 * outcome, qk_reset, qk_flush); calls that allocate or wait return QK_ESTATE, so
 * define gates and apply one permutation (which allocates its gather buffer)
 * before capturing.  qk_capture_end flushes, restores the qubit map and the
 * state's buffer inside the capture (so that every replay starts and ends in the
 * same buffer with the same map), ends the capture and instantiates the graph.
 * Gate parameters and uniforms are fixed at capture time. */
typedef struct qk_graph qk_graph;
qk_status qk_capture_begin(qk_ctx *ctx);
qk_status qk_capture_end(qk_ctx *ctx, qk_graph **out);
/* Replay the graph on its context's stream (stream-ordered, does not wait). */
qk_status qk_graph_launch(qk_graph *g);
qk_status qk_graph_destroy(qk_graph *g);

/* Batched circuits (no counterpart in the paper; it serves many independent
 * circuits with few launches).  A batch holds up to thousands of circuits of
 * 1..24 qubits (complex64, up to 64 cbits each), each from |0...0> and cbits 0.
 * A circuit of 1..13 qubits runs entirely in one CTA's shared memory with the
 * same op semantics as a context: built-in 1-target gates with quantum controls
 * and classical conditions (qk_batch_apply_gate), the controlled mul-mod oracle
 * of Appendix A (qk_batch_apply_mulmod, register <= 16 qubits), and sequential
 * single-qubit measurement into cbits (qk_batch_measure).  A circuit of 14..24
 * qubits takes built-in 1-target gates with at most one quantum control and no
 * classical condition (QK_EINVAL otherwise); its state stays in device memory,
 * qk_batch_run plans it into fused tile passes (on the host's cores) and runs
 * pass k of every such circuit in one batched launch.  qk_batch_run uploads the
 * programs and launches (one launch per distinct small-circuit size, one per
 * pass index of the large circuits) on the batch's stream without waiting;
 * qk_batch_done polls; qk_batch_read waits and copies a circuit's cbits and
 * final state (always kept for large circuits, for small ones if stored).  Add
 * ops to the most recently added circuit.  qk_batch_clear waits for a previous
 * run and empties the batch.  Errors: QK_EINVAL (sizes, qubit lists, params),
 * QK_ENOTBIJECTIVE, QK_ESTATE (op before any circuit), QK_ENOMEM, QK_ECUDA;
 * message in qk_batch_last_error. */
typedef struct qk_batch qk_batch;
qk_status qk_batch_create(qk_batch **out, void *cuda_stream);
qk_status qk_batch_destroy(qk_batch *b);
qk_status qk_batch_clear(qk_batch *b);
qk_status qk_batch_add_circuit(qk_batch *b, int n, int ncbits, int *index);
qk_status qk_batch_apply_gate(qk_batch *b, int gate_id, const int *targets, int nt, const int *controls, int nc,
                              const int *cond_cbits, int ncc, const double *params, int np);
qk_status qk_batch_apply_mulmod(qk_batch *b, const int *targets, int w, const int *controls, int nc, uint64_t c,
                                uint64_t N);
/* One entry of a gate list for qk_batch_apply_gates: a built-in 1-target gate
 * with up to 4 quantum controls, up to 4 condition cbits and up to 3 parameters
 * (the meaning of each field as in qk_batch_apply_gate).  Plain C layout,
 * 80 bytes. */
typedef struct qk_gate_op {
    int gate_id;
    int target;
    int nc, ncc, np;
    int controls[4];
    int cond[4];
    double params[3];
} qk_gate_op;
/* Append `count` gates to the most recently added circuit, in order; the same
 * checks and errors as one qk_batch_apply_gate call per entry (on an error the
 * entries before the bad one stay appended and the message names its index).
 * The list is copied before the call returns. */
qk_status qk_batch_apply_gates(qk_batch *b, const qk_gate_op *ops, int count);
/* The same gate list on a context, in one call (GateOp of the Q-Kit section for
 * each entry, in order): exactly one qk_apply_gate per entry, with its checks and
 * errors; on an error the entries before it stay applied and qk_last_error names
 * the entry.  Lets a caller hand over a whole circuit with one call. */
qk_status qk_apply_gates(qk_ctx *ctx, const qk_gate_op *ops, int count);
/* Modular exponentiation of a register by a control register, as one gate: the
 * conventional order-finding circuit (Appendix A, 3nx1 branch; Fig. 6a) applies,
 * for c = 0 .. nCQ-1, the controlled x -> a^(2^c) x mod N on the work register
 * under control qubit nCQ-1-c.  Those gates act on the same register and commute,
 * so together they multiply the register value by the product of the multipliers
 * whose control qubits are 1.  This call applies that product in one pass.
 *   targets[0..nt)  the register, targets[0] its most significant bit;
 *                   N <= 2^nt <= 2^QK_MAX_PERM_QUBITS
 *   controls[j], mult[j] (j < nc <= QK_MAX_MODEXP_CONTROLS): control qubit j
 *                   selects multiplier j (mult[j] < N, gcd(mult[j], N) = 1);
 *                   controls distinct and not among the targets
 *   cond_cbits[0..ncc) classical condition, as for qk_apply_gate
 * For every basis state, the register value x < N becomes (prod over j with
 * control j = 1 of mult[j]) x mod N; x >= N is left alone.  The result equals
 * nc qk_apply_gate calls of qk_define_gate_perm_mulmod gates, one per (control,
 * multiplier), in any order, and is exact.  Errors: QK_EINVAL (bad lists, N,
 * multiplier >= N, condition), QK_ENOTBIJECTIVE (a multiplier not coprime to N),
 * QK_ESTATE (no qubits), QK_ENOMEM (the gather buffer); the state is unchanged
 * on an error.  Stream-ordered; one out-of-place gather, which allocates the
 * state-sized gather buffer on first use like the permutation gates. */
qk_status qk_apply_modexp(qk_ctx *ctx, const int *targets, int nt, const int *controls, const uint64_t *mult, int nc,
                          uint64_t N, const int *cond_cbits, int ncc);
qk_status qk_batch_measure(qk_batch *b, const int *qubits, int nq, const double *uniforms, const int *dest_cbits);
qk_status qk_batch_run(qk_batch *b, int store_states);
/* 1 when the last run has finished, 0 while it runs, -1 on error. */
int qk_batch_done(qk_batch *b);
qk_status qk_batch_read(qk_batch *b, int circuit, uint8_t *cbits, int ncb, void *state, size_t bytes);
/* All circuits' cbits, concatenated in circuit order (sum of their cbit counts). */
qk_status qk_batch_read_all_cbits(qk_batch *b, uint8_t *out, size_t n);
int qk_batch_num_circuits(const qk_batch *b);
/* Of the last qk_batch_run: host planning time (ms) of the large circuits, the
 * number of batched tile launches, and (waits for the run) the device time (ms)
 * from the end of the host planning to the end of the run's last launch. */
qk_status qk_batch_stats(qk_batch *b, double *plan_ms, int *tile_launches, double *device_ms);
const char *qk_batch_last_error(const qk_batch *b);

/* Counters since creation or the last reset_counters: kernel launches, passes
 * over the state (launches that stream the full state), and algorithmic bytes
 * (2^n * amplitude size * 2 per full pass, read + write). */
qk_status qk_get_counters(const qk_ctx *ctx, uint64_t *launches, uint64_t *state_passes,
                          uint64_t *algorithmic_bytes);
qk_status qk_reset_counters(qk_ctx *ctx);

/* With options.profile = 1: per launch class (0 = tile pass, 1 = 2x2 pass, 2 =
 * diagonal pass, 3 = k-qubit block, 4 = permutation, 5 = measurement, 6 = other)
 * the launches, summed CUDA-event milliseconds and algorithmic bytes since the
 * last reset.  Waits for the stream.  Errors: QK_ESTATE if profiling is off. */
#define QK_NUM_LAUNCH_CLASSES 7
qk_status qk_profile(qk_ctx *ctx, uint64_t launches[QK_NUM_LAUNCH_CLASSES],
                     double ms[QK_NUM_LAUNCH_CLASSES], double bytes[QK_NUM_LAUNCH_CLASSES]);

/* Message for the last failed call on this context ("" if none). */
const char *qk_last_error(const qk_ctx *ctx);

/* Human-readable name of a status code. */
const char *qk_status_str(qk_status s);

#ifdef __cplusplus
}
#endif
#endif /* QK_H */
