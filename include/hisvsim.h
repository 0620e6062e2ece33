/*
 * hisvsim.h - C ABI of the GB300 hierarchical state-vector simulator.
 *
 * The library applies a quantum circuit to a 2^n-amplitude state vector held
 * in GPU memory, one HBM pass per part of an acyclic partition of the circuit's
 * gate DAG (the Gather-Execute-Scatter model of Algorithm 1, Sec. III-C, with
 * the partitioning problem of Sec. IV-A and the Nat / DFS / dagP builders of
 * Sec. IV-B). The executor is offered as a library, as the paper does for its
 * own (Sec. III-D: "general interface for other simulators").
 *
 * Conventions shared by every entry point
 *   - Amplitude x of an n-qubit state is stored at index x = sum_q b_q 2^q
 *     (little-endian, Sec. II-B / Fig. 1), interleaved (re, im):
 *     SV_C64 = two floats (8 bytes), SV_C128 = two doubles (16 bytes),
 *     SV_C128DF = complex128 held as double-float pairs: each of the real and
 *     imaginary parts is the unevaluated sum hi + lo of two floats (Dekker's
 *     double-float format, about 48 significant bits), stored as (re.hi,
 *     re.lo, im.hi, im.lo), 16 bytes. Its arithmetic runs on the FP32 pipes
 *     (the FP64 rate of the GPU is a small fraction of its FP32 rate);
 *     sv_upload / sv_copy_state / sv_download / sv_export_c128 take and give
 *     double2 amplitudes, converted on the device; its parts always run on the
 *     plan's specialised kernels (SV_FLAG_SPECIALISE implied; no gate-by-gate
 *     or tensor-core path).
 *   - Handles (sv_state, sv_plan, sv_batch) are opaque, created and destroyed
 *     by the caller, and not thread-safe: one thread uses a handle at a time.
 *   - Device work is stream-ordered on the state's CUDA stream and the call
 *     returns once it is enqueued, unless the entry point says it synchronises.
 *     A device fault surfaces as SV_ERR_CUDA at the next synchronising call.
 *   - No entry point throws; every one returns an sv_status, and on a status
 *     other than SV_OK sv_last_error() describes it (thread-local string).
 *   - Argument errors are detected on the host before any device work.
 */
#ifndef HISVSIM_H
#define HISVSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SV_OK = 0,
    SV_ERR_ARG = 1,        /* bad argument: null pointer, size, qubit index, n out of range */
    SV_ERR_OOM = 2,        /* device or host allocation failed */
    SV_ERR_CUDA = 3,       /* a CUDA call failed (launch, copy, fault surfaced at a sync) */
    SV_ERR_PARTITION = 4,  /* a gate has more qubits than the part limit k (Sec. IV-A, L <= L_m) */
    SV_ERR_TIMEOUT = 5,    /* a bounded device wait gave up (batched / tensor-core kernels) */
    SV_ERR_BUSY = 6,       /* the handle has work that must complete first */
    SV_ERR_INTERNAL = 7
} sv_status;

typedef enum { SV_C64 = 0, SV_C128 = 1, SV_C128DF = 2 } sv_precision;

/* Part builders of Sec. IV-B; SV_PART_NONE runs gate by gate (one pass per gate).
 * SV_PART_EXACT: the minimum number of parts over all acyclic partitions with
 * L <= k (the optimum of the paper's ILP comparison, Sec. V-A), by breadth-first
 * search over the gate DAG's down-sets; for small circuits (at most 256
 * gates and a bounded search), SV_ERR_ARG beyond.
 * SV_PART_BEAM: beam search over the same down-sets for circuits of any size
 * (each kept prefix grows one candidate part from every available gate,
 * adding the qubit that lets the most gates in, up to k, looking one qubit
 * further at widths >= 32; the widest prefixes survive); deterministic; the
 * beam width is sv_plan_build's dfs_trials argument (<= 0: 16). */
typedef enum {
    SV_PART_NONE = 0, SV_PART_NAT = 1, SV_PART_DFS = 2, SV_PART_DAGP = 3, SV_PART_EXACT = 4, SV_PART_BEAM = 5
} sv_method;

/* Gate kinds. Matrices (Sec. II-A defines X, Y, Z, H; the rest are the
 * textbook conventions): RX(t) = [[c,-is],[-is,c]], RY(t) = [[c,-s],[s,c]]
 * with c = cos t/2, s = sin t/2; RZ(t) = diag(e^{-it/2}, e^{it/2});
 * P(t) = diag(1, e^{it}); S = P(pi/2); T = P(pi/4); CX(c,t) flips b_t when
 * b_c = 1; CZ = diag(1,1,1,-1); CP(t) = diag(1,1,1,e^{it}); SWAP exchanges
 * the two qubits. For two-qubit gates q[0] is the control. */
typedef enum {
    SV_GATE_H = 0, SV_GATE_X, SV_GATE_Y, SV_GATE_Z, SV_GATE_S, SV_GATE_T,
    SV_GATE_RX, SV_GATE_RY, SV_GATE_RZ, SV_GATE_P,
    SV_GATE_CX, SV_GATE_CZ, SV_GATE_CP, SV_GATE_SWAP,
    SV_GATE_COUNT
} sv_gate_kind;

/* One gate (24 bytes). arity must match the kind (1 or 2); q[arity..2] are ignored. */
typedef struct {
    uint16_t kind;
    uint16_t arity;
    uint32_t q[3];
    double theta;
} sv_gate;

typedef struct sv_state sv_state;
typedef struct sv_plan sv_plan;

/* Flags of sv_apply_parts. */
#define SV_FLAG_GATEWISE 0x1u   /* ignore the parts: one plain pass per gate (comparator) */
#define SV_FLAG_SYNC     0x2u   /* synchronise the stream before returning */
#define SV_FLAG_TC_DENSE 0x4u   /* complex64, n >= 13: parts of at most 6 qubits run as one fused
                                   64x64 unitary on the tensor cores (split BF16, FP32
                                   accumulation); other parts keep the gate-list kernel */
#define SV_FLAG_TC_PAIRS 0x10u  /* with SV_FLAG_TC_DENSE: two consecutive parts of at most 6
                                   qubits run in one pass where their qubits and qubits 0, 1
                                   fit a 13-qubit tile (the tile is read and written once,
                                   both unitaries applied on chip: multi-level partitioning,
                                   Sec. IV-B); the state must be 16-byte aligned */
/* Register bits per thread of the gate-list part kernels (amplitudes per
 * thread = 2^r, the register level of the tile): r in [3, 6] with
 * SV_FLAG_SPECIALISE (the tile must keep at least 2^5 threads, t - r >= 5);
 * 0 = the default (5 for complex64, 4 for complex128). The interpreter runs
 * the default only (SV_ERR_ARG otherwise). */
#define SV_FLAG_REGBITS(r) (((uint32_t)(r) & 0xFu) << 8)
#define SV_FLAG_SPECIALISE 0x8u /* gate-list parts run as kernels generated for this plan, with
                                   the tile layout, register phases and every gate (with its
                                   coefficients) compiled in (NVRTC, sm_103a); compiled at the
                                   first apply for the precision and tile (or by
                                   sv_plan_specialise) and kept in the plan. Same arithmetic as
                                   the interpreter kernel; SV_ERR_CUDA if NVRTC is missing */

/* ---------------------------------------------------------------- state ---
 * sv_create: make an n-qubit state (1 <= n <= 36) initialised to |0...0>.
 *   dev_buf       caller-owned device buffer of >= 2^n * amp bytes, or NULL to
 *                 let the library allocate (and free at sv_destroy). A caller
 *                 buffer must stay alive until sv_destroy.
 *   dev_buf_bytes size of dev_buf (ignored when dev_buf is NULL).
 *   stream        cudaStream_t the state's work is ordered on (NULL = legacy
 *                 default stream).
 *   out           receives the handle.
 * The amplitudes are the paper's state vector (Sec. II-B): 2^n entries. */
sv_status sv_create(int n_qubits, sv_precision prec, void *dev_buf, size_t dev_buf_bytes,
                    void *stream, sv_state **out);
/* sv_attach: a state handle over amplitudes already in dev_buf (required,
 * same layout and size rules as sv_create), left as they are: for callers
 * that own the amplitudes, e.g. one rank's slice of a distributed state
 * (Sec. III-D), whose local steps run through sv_apply_parts. */
sv_status sv_attach(int n_qubits, sv_precision prec, void *dev_buf, size_t dev_buf_bytes, void *stream,
                    sv_state **out);
sv_status sv_destroy(sv_state *s);
/* Set the state to the basis state |index> (index < 2^n). Stream-ordered. */
sv_status sv_set_basis(sv_state *s, uint64_t index);
/* Copy 2^n amplitudes from host memory (same layout/precision) into the state.
 * Stream-ordered; the host buffer must stay valid until the stream reaches the
 * copy (pinned memory makes it asynchronous). bytes must equal the state size. */
sv_status sv_upload(sv_state *s, const void *host_src, size_t bytes);
/* Copy the state to host memory; synchronises the stream. bytes = state size. */
sv_status sv_copy_state(sv_state *s, void *host_dst, size_t bytes);
/* Stream-ordered copy of the state to host memory (no synchronisation: the
 * data is in host_dst once the stream has passed the copy, e.g. after
 * sv_sync). host_dst must stay valid until then; pinned memory makes the
 * copy asynchronous, so a caller can overlap one state's transfers with
 * another state's passes. bytes = state size. */
sv_status sv_download(sv_state *s, void *host_dst, size_t bytes);
/* sv_export_c128: the state's amplitudes as 2^n double2 values into the
 * caller's device buffer dev_dst (bytes = 16 * 2^n), stream-ordered: a copy
 * for SV_C128, the conversion hi + lo (exact in FP64) for SV_C128DF;
 * SV_ERR_ARG for SV_C64. */
sv_status sv_export_c128(sv_state *s, void *dev_dst, size_t bytes);
/* Device address of the amplitudes and the number of bytes they occupy. */
sv_status sv_device_ptr(sv_state *s, void **ptr, size_t *bytes);
/* Synchronise the state's stream and report any pending device error; a
 * bounded device wait that gave up (tensor-core path) returns SV_ERR_TIMEOUT. */
sv_status sv_sync(sv_state *s);
/* CTA tile size used by the part kernels for this state: tile_qubits t in
 * [10, 13] for SV_C64 and [10, 12] for SV_C128 and SV_C128DF (2^t
 * amplitudes per CTA); 0 restores the default: 12 (complex64) / 11 (the
 * complex128 forms), grown to the plan's largest part plus the lowest free
 * qubits that make each contiguous run of the tile fill a 32-byte sector
 * (two for complex64, one for the complex128 forms), within the limits
 * above. The tile always contains the part's qubits and is padded with the
 * lowest remaining qubits (Sec. IV-B, multi-level: parts smaller than the
 * limit take extra qubits for spatial locality). */
sv_status sv_set_tile(sv_state *s, int tile_qubits);

/* ----------------------------------------------------------------- plan ---
 * sv_plan_build: build the gate DAG (Sec. IV-A) and partition it with method
 * m into acyclic parts of at most k qubits (Sec. IV-B); host only, synchronous.
 *   gates, n_gates  the circuit in execution order (copied; caller keeps ownership)
 *   n_qubits        qubits of the circuit (gate qubits must be < n_qubits)
 *   k               part qubit limit L_m (ignored for SV_PART_NONE)
 *   seed, dfs_trials  random DFS orders for SV_PART_DFS (dfs_trials <= 0: 16);
 *                   for SV_PART_BEAM dfs_trials is the beam width (<= 0: 16)
 * Parts are numbered in execution order: Kahn order of the part graph, ties to
 * the part holding the smallest gate index; gates of a part keep their order.
 * Returns SV_ERR_PARTITION if a gate has more than k qubits, SV_ERR_ARG for a
 * bad kind, arity, repeated or out-of-range qubit.
 * Threads: a plan may be applied to several states, from several host
 * threads at once (its compiled programs are built once, under a lock); a
 * state is used from one host thread at a time; sv_plan_destroy needs every
 * apply of the plan to have completed on the device. */
sv_status sv_plan_build(const sv_gate *gates, size_t n_gates, int n_qubits, sv_method m, int k,
                        uint64_t seed, int dfs_trials, sv_plan **out);
/* Copy the partition out: part_of_gate[n_gates] (may be NULL) and the number
 * of parts. n_gates must equal the plan's gate count. */
sv_status sv_plan_export(const sv_plan *p, uint32_t *part_of_gate, size_t n_gates, uint32_t *n_parts);
/* Statistics of the compiled device program for a precision, tile and apply
 * flags (SV_FLAG_TC_DENSE changes the program): passes = parts run on the
 * GPU, phases = register phases of the gate-list parts, ops = their kernel
 * ops, dense = parts run as fused unitaries on the tensor cores (any output
 * pointer may be NULL). Compiles on the host if needed; no device work. */
sv_status sv_plan_stats(sv_plan *p, sv_precision prec, int tile_qubits, uint32_t flags, uint32_t *passes,
                        uint32_t *phases, uint32_t *ops, uint32_t *dense);
/* sv_plan_build_ml: multi-level partitioning (Sec. IV-B, "Multi-level
 * partitioning"): the circuit is partitioned with builder m1 under the
 * first-level limit k1 (one HBM pass per first-level part, as for
 * sv_plan_build), then every first-level part, as a circuit of its own (its
 * gates in their original order), is partitioned again with builder m2 under
 * the second-level limit k2 <= k1. On the gate-list kernels each
 * second-level part becomes one register phase of its pass (the register
 * level is the tile's inner state vector), in place of the greedy phase
 * split, so k2 must not exceed the register bits (5 for complex64, 4 for
 * complex128; else sv_apply_parts reports SV_ERR_PARTITION). Same arguments
 * and errors as sv_plan_build, plus SV_ERR_ARG for m2 = SV_PART_NONE or k2
 * outside [1, k1] and SV_ERR_PARTITION for a gate wider than k2. Host only. */
sv_status sv_plan_build_ml(const sv_gate *gates, size_t n_gates, int n_qubits, sv_method m1, int k1, sv_method m2,
                           int k2, uint64_t seed, int dfs_trials, sv_plan **out);
/* sv_plan_export_inner: the second-level part of every gate (numbered over
 * the whole circuit: first-level parts in order, then each part's inner
 * schedule) and their count; SV_ERR_ARG for a one-level plan. */
sv_status sv_plan_export_inner(const sv_plan *p, uint32_t *inner_of_gate, size_t n_gates, uint32_t *n_inner);
/* sv_plan_specialise: generate and compile the plan's specialised part
 * kernels (SV_FLAG_SPECIALISE) for the precision, tile (0 = default) and
 * flags (SV_FLAG_TC_DENSE: only the parts that stay on the gate-list kernel)
 * now instead of at the first apply. load = 0 compiles on the host only and
 * discards the code (no device needed: a check of the generated source);
 * load = 1 loads it into the plan for the current device. *compile_seconds
 * (may be NULL) receives the wall time of the compilation. Errors: SV_ERR_ARG
 * (bad tile), SV_ERR_PARTITION (plan does not compile), SV_ERR_CUDA (NVRTC
 * missing, compile or load error; sv_last_error has the log). Host thread
 * safe like sv_apply_parts. */
sv_status sv_plan_specialise(sv_plan *p, sv_precision prec, int tile_qubits, uint32_t flags, int load,
                             double *compile_seconds);
/* sv_plan_source: the generated CUDA source of gate-list part i (execution
 * order among the gate-list parts) of the plan's program for prec, tile and
 * flags, copied NUL-terminated into buf (cap bytes); *len receives the
 * source length. Host only. */
sv_status sv_plan_source(sv_plan *p, sv_precision prec, int tile_qubits, uint32_t flags, uint32_t part, char *buf,
                         size_t cap, size_t *len);
/* sv_plan_flops: the floating-point operations one apply of the plan
 * executes for the precision, tile and flags (host only): *alu_flops on the
 * CUDA cores, counted per op of the compiled program as its arithmetic over
 * the amplitudes it touches (an FMA counts two; H 2, RX/RY 6, a fused 2x2
 * 14, a diagonal 6 on the amplitudes it scales; permutations and sign
 * changes 0; gate by gate: 14 per one-qubit and 30 per two-qubit gate, the
 * general matrices of Sec. III-A), and *tensor_flops on the tensor cores
 * (1536 per amplitude per dense part: three split-BF16 products of the
 * 128 x 128 real block form). Either pointer may be NULL. The basis of the
 * ALU roofline of the complex128 path. */
sv_status sv_plan_flops(sv_plan *p, sv_precision prec, int tile_qubits, uint32_t flags, double *alu_flops,
                        double *tensor_flops);
sv_status sv_plan_destroy(sv_plan *p);

/* ---------------------------------------------------------------- apply ---
 * Apply the plan's circuit to the state: for each part in order, one kernel
 * pass in which every CTA gathers a 2^t-amplitude tile (the part's qubits plus
 * padding), runs all of the part's gates on it in registers / shared memory,
 * and scatters it back (Algorithm 1). The plan's qubit count must equal the
 * state's. Stream-ordered (SV_FLAG_SYNC waits). The first call for a given
 * precision and tile uploads the part program to device memory (owned by the
 * plan). States with n < 10 run gate by gate. */
sv_status sv_apply_parts(sv_state *s, sv_plan *p, uint32_t flags);

/* -------------------------------------------------------------- measure ---
 * Probabilities p[x] = |a_x|^2 (Sec. II-A) into dev_out (device memory of
 * 2^n floats, or doubles when out_fp64 != 0; may be NULL to get the norm only)
 * and the norm sum_x |a_x|^2 accumulated in FP64 into *norm_out (host, may be
 * NULL). Synchronises the stream when norm_out is not NULL. */
sv_status sv_measure_probs(sv_state *s, void *dev_out, int out_fp64, double *norm_out);
/* Summary of the same distribution without writing it (no device memory
 * beyond the state's own scratch): *norm_out = sum_x |a_x|^2, *p0_out =
 * |a_0|^2, *pmax_out = max_x |a_x|^2 and *argmax_out = the smallest x that
 * reaches it, all computed in FP64 from the stored amplitudes (Sec. II-A:
 * measuring gives x with probability |a_x|^2). Any output may be NULL.
 * Synchronises the stream. */
sv_status sv_measure_summary(sv_state *s, double *norm_out, double *p0_out, uint64_t *argmax_out,
                             double *pmax_out);

/* ---------------------------------------------------------------- batch ---
 * Many small, independent circuits run in ONE persistent kernel launch that a
 * CUDA graph captures once and replays (the batched workload: thousands of
 * uneven circuits of 10..30 qubits). States are complex64, contiguous in one
 * device buffer in circuit order (circuit i starts after the 2^n_j amplitudes
 * of every j < i). Each plan's parts run on 2^9-amplitude tiles, one warp
 * per tile; parts of one circuit run in order (a device work list in wave
 * order with per-circuit tile counters and bounded waits), parts of different
 * circuits overlap. Parts are limited to 9 qubits (plans with k <= 9).
 *
 * sv_batch_create  n_qubits[n_circuits] in [10, 30]; states start in |0...0>;
 *                  stream NULL = a stream the library creates (graph capture
 *                  needs a non-legacy stream). Allocates the states.
 * sv_batch_set_plan  plan for circuit i (qubit count must match); the plan
 *                  must stay alive until the next sv_batch_run has returned.
 * sv_batch_config  warps per CTA (1..8) and tiles per work item (1..4096);
 *                  0 keeps the default (8, 16). Changing plans or the
 *                  configuration rebuilds the work list and the graph.
 * sv_batch_run     apply every circuit once to its current state; the first
 *                  run builds the work list, uploads it and captures the
 *                  graph (host work), later runs replay it. Stream-ordered;
 *                  SV_FLAG_SYNC waits and reports SV_ERR_TIMEOUT if a bounded
 *                  device wait gave up.
 * sv_batch_reset   every state back to |0...0> (stream-ordered).
 * sv_batch_probs   p[x] = |a_x|^2 of all states into dev_out (floats,
 *                  concatenated like the states; may be NULL) and each
 *                  state's norm (FP64 accumulation) into norms_host[n] (may
 *                  be NULL; synchronises when not NULL).
 * sv_batch_state   device address and byte size of circuit i's state.
 * sv_batch_copy_state  copy circuit i's state (bytes = its size) to host
 *                  memory; synchronises.
 * sv_batch_info    total amplitudes, work items and parts of the built
 *                  program's gate-list kernel.
 * sv_batch_set_dense  (Algorithm 1, Sec. III-C, with the execute step of a
 *                  part as one fused unitary) min_qubits > 0: every circuit of at least
 *                  max(min_qubits, 13) qubits whose plan has parts of at most
 *                  6 qubits runs on the batched tensor-core kernel, one
 *                  64x64 split-BF16 pass per part (the k_dense6 arithmetic);
 *                  its output is renormalised to unit norm after every pass
 *                  (the states start in |0...0>). tiles_per_item: tiles of
 *                  2^13 amplitudes per work item (0 = default 2).
 *                  group_tiles: the dense circuits, sorted by pass count, are
 *                  cut into groups holding about this many tiles of state
 *                  (64 KiB each), each group's passes in wave order, group
 *                  after group, so that a group's states can stay in L2
 *                  between passes (0 = default 1024, 64 MiB; a value above
 *                  the batch's total gives plain wave order).
 *                  min_qubits = 0 turns it off (the default). Rebuilds the
 *                  program.
 * sv_batch_dense_info  circuits, work items and passes on the dense kernel.
 * sv_batch_sync    synchronise and report device errors.
 * sv_batch_destroy free everything the batch allocated. */
typedef struct sv_batch sv_batch;
sv_status sv_batch_create(uint32_t n_circuits, const int *n_qubits, void *stream, sv_batch **out);
sv_status sv_batch_set_plan(sv_batch *b, uint32_t i, sv_plan *p);
sv_status sv_batch_config(sv_batch *b, int warps_per_cta, int tiles_per_item);
sv_status sv_batch_run(sv_batch *b, uint32_t flags);
/* sv_batch_prepare: build the batch's device program and capture its graph
 * (what the first sv_batch_run does) without launching it, so that a host
 * thread can prepare the next batch while another batch runs. It waits for
 * the batch's own stream (the program upload); the capture is thread-local. */
sv_status sv_batch_prepare(sv_batch *b);
sv_status sv_batch_reset(sv_batch *b);
sv_status sv_batch_probs(sv_batch *b, void *dev_out, double *norms_host);
sv_status sv_batch_state(sv_batch *b, uint32_t i, void **dev_ptr, size_t *bytes);
sv_status sv_batch_copy_state(sv_batch *b, uint32_t i, void *host_dst, size_t bytes);
sv_status sv_batch_info(sv_batch *b, uint64_t *total_amplitudes, uint32_t *n_items, uint32_t *n_parts);
sv_status sv_batch_sync(sv_batch *b);
sv_status sv_batch_set_dense(sv_batch *b, int min_qubits, int tiles_per_item, int group_tiles);
sv_status sv_batch_dense_info(sv_batch *b, uint32_t *n_circuits, uint32_t *n_items, uint32_t *n_passes);
/* Testing the failure path (no GPU fault involved): with on != 0 the last
 * work item waits for a tile count its circuit never reaches, so its bounded
 * wait gives up (about a second), the kernel records the error and ends, and
 * the run reports SV_ERR_TIMEOUT at the next synchronising call; the batch
 * stays usable. on = 0 restores the normal work list. Rebuilds the program. */
sv_status sv_batch_hold_last_item(sv_batch *b, int on);
sv_status sv_batch_destroy(sv_batch *b);

/* ------------------------------------------------- allocation-free probs ---
 * sv_probs_noalloc: the same probabilities and FP64-accumulated norm as
 * sv_measure_probs, for callers that must not allocate device memory: a host
 * framework that owns all device memory through its own pool under a fixed
 * budget, or a latency-critical loop where a device allocation could stall
 * the device. It allocates nothing (no cudaMalloc/cudaFree, no allocating
 * library call); its partial sums live in one static device array of
 * SV_NOALLOC_MAX_BLOCKS + 1 doubles (32 KiB) inside this library, which every
 * GPU that loads the library keeps until the process exits. The paper has no
 * counterpart; it is an interface addition of this library.
 *   dev_state  device pointer to 2^n amplitudes (layout of prec), caller-owned
 *   dev_probs  device output of 2^n floats (doubles if out_fp64), or NULL
 *   dev_norm   device output of one double (sum |a_x|^2), or NULL
 *   n_blocks   width of the FP64 reduction = partial sums used, 0 for the
 *              default (SV_NOALLOC_DEFAULT_BLOCKS); larger than
 *              SV_NOALLOC_MAX_BLOCKS is rejected with SV_ERR_ARG
 *   stream     cudaStream_t (NULL = legacy default stream); stream-ordered,
 *              no synchronisation.
 * Every call made outside a stream capture looks the array's device address
 * up (cudaGetSymbolAddress) with the caller's device current, so a device
 * reset or a new context never leaves a stale address; a call made during a
 * capture reuses the last address found on that device, so make the first
 * call on a device before any stream capture (otherwise SV_ERR_ARG). A device
 * ordinal of 64 or more is rejected with SV_ERR_ARG. Every call shares the
 * one array, which keeps
 * the last call's contents; each call writes every partial sum it reads, so
 * nothing needs clearing, but calls that overlap on the GPU (different
 * streams, or threads without ordering) race on it. */
#define SV_NOALLOC_MAX_BLOCKS 4096
#define SV_NOALLOC_DEFAULT_BLOCKS 1216
sv_status sv_probs_noalloc(const void *dev_state, int n_qubits, sv_precision prec, void *dev_probs,
                           int out_fp64, double *dev_norm, int n_blocks, void *stream);

/* sv_alu_probe: the measured FMA rate of the current device's CUDA cores in
 * FP64 (fp64 != 0) or FP32, in FLOP/s (an FMA counts two): the roofline of
 * the complex128 path, which is bound by FP64 arithmetic rather than by HBM
 * (Sec. III-A counts the flops of a gate). Best of a few timed launches of
 * independent FMA chains on every SM; synchronises the device's legacy
 * stream. Not part of the paper; a measurement helper of this library. */
sv_status sv_alu_probe(int fp64, double *flops_per_s);

/* Thread-local description of the last non-OK status (never NULL). */
const char *sv_last_error(void);
/* Library version string. */
const char *sv_version(void);

/* ----------------------------------------------------------- OpenQASM 2 ---
 * The paper's circuits are OpenQASM 2.0 files (Sec. V); this front-end turns
 * a program text into the gate list sv_plan_build takes.
 * sv_qasm_parse: text = the program (NUL-terminated). Registers are laid out
 *   one after another in declaration order (qubit index = register offset +
 *   index). Gates outside the library's set are decomposed exactly (u2, u3,
 *   sdg, tdg, cy, crz, crx, cry, ch, cu3, ccx, cswap, rzz; u1 = p); user gate
 *   definitions are expanded; barrier and a final measure are ignored.
 *   reset, if, opaque gates and gates after a measure are rejected with
 *   SV_ERR_ARG (the message names the line). On success *out_gates is a
 *   library-allocated array of *out_n_gates gates (free it with
 *   sv_free_gates) and *out_n_qubits the number of qubits. Host only. */
sv_status sv_qasm_parse(const char *text, sv_gate **out_gates, size_t *out_n_gates, int *out_n_qubits);
void sv_free_gates(sv_gate *gates);

#ifdef __cplusplus
}
#endif
#endif /* HISVSIM_H */
