/*
 * tz.h -- C ABI of the GB300 amplitude library for random quantum circuits.
 *
 * The library computes output amplitudes a(x) = <x| U_C |0^n> of the random
 * circuits of Sec. 1 (H layer; t cycles of CZ in 8 rotating patterns with
 * sqrt(X)/sqrt(Y)/T single-qubit gates; final H layer) by contracting the
 * circuit's tensor network (Sec. 1: each node a tensor, each hyperedge a
 * running index) along a contraction tree. A set of k indices is sliced:
 * the contraction splits into 2^k independent subtasks of equal cost
 * (Sec. 2) whose partial amplitudes add up to the amplitude (Sec. 1,
 * "preprocessing" and the agent's sum).
 *
 * Conventions for every function:
 *  - Return value: TZ_OK (0) on success, a negative TZ_E* code on failure.
 *    No function aborts the process. tz_last_error() returns a message for
 *    the last failure on the calling thread (valid until the next call).
 *  - Handles are opaque; the caller owns each handle it receives and frees
 *    it with the matching tz_*_destroy. Destroy functions accept NULL.
 *  - The library copies every input array it is given; it keeps no pointer
 *    to caller memory, except device memory bound as a workspace.
 *  - The library never allocates device memory. Device memory is supplied
 *    by the caller (tz_plan_bind_workspace, tz_server_opts.arena).
 *  - "Device pointer" means memory of the plan's CUDA device; "host
 *    pointer" means ordinary (pageable or pinned) host memory.
 *  - Bitstrings are uint8 arrays of n rows x n_qubits columns (row-major),
 *    each byte 0 or 1; column q is the bit of qubit q.
 *  - Amplitudes are returned as FP64 complex numbers: 2*n doubles,
 *    (re, im) interleaved.
 */
#ifndef TZ_H
#define TZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------- status */
#define TZ_OK            0
#define TZ_EINVAL       -1   /* invalid argument, shape or spec            */
#define TZ_ENOMEM       -2   /* host allocation failed or workspace too small */
#define TZ_EHBM_ADMIT   -3   /* server: query does not fit the HBM budget  */
#define TZ_ECUDA        -4   /* a CUDA runtime call failed                 */
#define TZ_ETIMEOUT     -5   /* a bounded wait ran out                     */
#define TZ_EUNSUPPORTED -6   /* valid request the build does not support  */
#define TZ_EBUSY        -7   /* server: no free slot (try again later)     */

const char *tz_last_error(void);

/* ------------------------------------------------------------ handles */
typedef struct tz_circuit tz_circuit;
typedef struct tz_network tz_network;
typedef struct tz_tree tz_tree;
typedef struct tz_plan tz_plan;
typedef struct tz_server tz_server;

/* --------------------------------------------------------- circuits
 * Sec. 1 (circuit prescription, items 1-4).
 */

/* Parse a plain-text circuit spec. First non-empty line: the qubit count.
 * Each further line: `cycle name q0 [q1]`, name in {h, cz, t, x_1_2, y_1_2}
 * (the GRCS gate names). Lines starting with '#' are skipped. Gates are
 * applied in line order. text need not be NUL-terminated; len is its length
 * in bytes. Malformed text, unknown gates, out-of-range or repeated qubits
 * give TZ_EINVAL. */
int tz_circuit_from_spec(const char *text, size_t len, tz_circuit **out);

#define TZ_LATTICE_GRID        0   /* rows x cols square lattice           */
#define TZ_LATTICE_BRISTLECONE 1   /* 72-site diamond, or 70 without (5,0),(5,11) */
typedef struct {
  int kind;      /* TZ_LATTICE_*                                         */
  int rows;      /* grid: rows (>= 1)                                    */
  int cols;      /* grid: cols (>= 1)                                    */
  int n_qubits;  /* bristlecone: 70 or 72                                */
} tz_lattice;

/* Generate a depth 1+t+1 circuit by the prescription of Sec. 1 with the
 * library's readings: CZ patterns H0,V0,H2,V2,H1,V1,H3,V3 (H_a: couplers
 * (r,c)-(r,c+1) with c = a + 2(r mod 2) mod 4; V_a: (r,c)-(r+1,c) with
 * r = a + 2(c mod 2) mod 4); sqrt(X)/sqrt(Y) after a CZ in the previous
 * cycle, chosen by the top bit of one SplitMix64 draw (seeded with `seed`;
 * cycle-major, qubit-minor order); T after H/sqrt(X)/sqrt(Y) in the previous
 * cycle. Qubits are the lattice sites in row-major order. */
int tz_circuit_generate(const tz_lattice *lat, int depth_t, uint64_t seed, tz_circuit **out);

int tz_circuit_n_qubits(const tz_circuit *c);
int tz_circuit_n_gates(const tz_circuit *c);
/* Write the spec text (NUL-terminated) into buf of capacity cap bytes;
 * *len receives the length without the NUL. If cap is too small, nothing is
 * written, *len receives the needed length and TZ_EINVAL is returned. */
int tz_circuit_to_spec(const tz_circuit *c, char *buf, size_t cap, size_t *len);
void tz_circuit_destroy(tz_circuit *c);

/* --------------------------------------------------------- networks
 * Sec. 1 (refactoring note): a node holds a tensor, a hyperedge is a running
 * index. Every index has dimension 2. A qubit's wire contributes one index
 * per segment: segment j is the stretch after the qubit's j-th non-diagonal
 * gate (H, sqrt(X), sqrt(Y)). Diagonal gates (T, CZ) create no index: T is
 * a rank-1 tensor and CZ a rank-2 tensor on the current segment indices.
 * The input |0> and the output <x_q| are rank-1 tensors. The builder then
 * merges rank-1 tensors into a neighbour and the last gate of each wire into
 * its output tensor (exact rewrites). Output tensors carry `batch_log2`
 * extra open indices (the bitstring batch): one call contracts 2^batch_log2
 * bitstrings at once.
 *
 * Open output qubits (the multi-amplitude trend of Sec. 2, Table 1: more
 * amplitudes per contraction, less time each): the listed qubits get no
 * output tensor; their last wire index stays open to the end of the
 * contraction, so one contraction yields the 2^n_open amplitudes of every
 * assignment of those qubits' output bits. Each bitstring then yields
 * 2^n_open amplitudes: amplitude o (0 <= o < 2^n_open) is that of the
 * bitstring with the output bit of open_qubits[j] (sorted ascending) set to
 * bit j of o; the bitstring's own bits on the open qubits are ignored.
 * TZ_EINVAL: more than 12 open qubits, a qubit out of range or listed twice,
 * or every qubit open (one must stay closed).
 */
typedef struct {
  int batch_log2;               /* 0..8: bitstrings contracted together per group */
  int n_open;                   /* 0..12 open output qubits                       */
  const int32_t *open_qubits;   /* n_open qubit numbers (any order; caller-owned,
                                   read during the call only)                     */
} tz_network_opts;

int tz_network_from_circuit(const tz_circuit *c, const tz_network_opts *opts, tz_network **out);
int tz_network_n_tensors(const tz_network *net);
int tz_network_n_indices(const tz_network *net);
/* Index info: *qubit = owning qubit and *segment = segment number for wire
 * indices; *qubit = -1 and *segment = bit number for batch indices;
 * *qubit = -2 and *segment = j for the index of open output qubit j (bit j of
 * the open value, the j-th smallest open qubit). */
int tz_network_index_info(const tz_network *net, int index, int *qubit, int *segment);
/* Indices of tensor t in storage order (bit p of a linear element offset is
 * the p-th index). cap = capacity of idx; *rank receives the rank. */
int tz_network_tensor_indices(const tz_network *net, int t, int32_t *idx, int cap, int *rank);
void tz_network_destroy(tz_network *net);

/* ------------------------------------------------------ contraction trees
 * The contraction algorithm of the paper is deferred to its earlier work;
 * the library builds its own trees, by two randomised heuristics:
 *   TZ_PATH_GREEDY      pairwise greedy over tensors that share an index,
 *                       cost size(out) - alpha (size(a) + size(b));
 *   TZ_PATH_ELIMINATION bucket elimination of indices in min-degree order
 *                       (merge every holder of the index, then sum it out);
 * TZ_PATH_AUTO alternates them. Each restart is scored by the estimated
 * GB300 time of the plan after slicing to log2_max_intermediate, and the
 * best tree is kept (the earliest restart among equal scores). Restarts run
 * on host threads: one per hardware thread (at most 64), or the number in
 * the environment variable TZ_PATH_THREADS; the tree returned does not depend
 * on the thread count.
 * Trees are lists of SSA pairs: leaves are ids 0..T-1, the i-th pair
 * creates id T+i. A complete tree has T-1 pairs.
 */
#define TZ_PATH_AUTO        0
#define TZ_PATH_GREEDY      1
#define TZ_PATH_ELIMINATION 2
typedef struct {
  int restarts;                 /* randomised trials (>= 1); the first trial of
                                   each algorithm is deterministic              */
  uint64_t seed;                /* seed of the randomisation                   */
  int log2_max_intermediate;    /* slicing target used to score trials (bits)  */
  int precision;                /* tz_precision used by the time model         */
  int algorithm;                /* TZ_PATH_*                                   */
  int reconfigure;              /* 0: off; 3..10: after the restarts, re-solve
                                   windows of up to this many subtrees exactly
                                   (dynamic programming over subsets) in the 8
                                   best trees, and keep the best result         */
} tz_path_opts;

int tz_path_greedy(const tz_network *net, const tz_path_opts *opts, tz_tree **out);
/* Build a tree from caller pairs (validated: complete, each id used once). */
int tz_tree_from_pairs(const tz_network *net, const int32_t *pairs, int n_pairs, tz_tree **out);
/* Copy the pairs out (2 int32 per pair). cap = capacity in pairs. */
int tz_tree_pairs(const tz_tree *tree, int32_t *pairs, int cap, int *n_pairs);
void tz_tree_destroy(tz_tree *tree);

/* ------------------------------------------------------------ slicing
 * Sec. 1 (preprocessing splits the contraction into subtasks). Greedily
 * picks indices whose fixing lowers the largest intermediate most (ties:
 * lower total cost) until it is <= 2^log2_max_intermediate elements or k_max
 * indices are chosen. sliced_edges receives the index ids (capacity k_max);
 * slice s fixes the i-th listed index to bit i of s. */
int tz_slice_select(const tz_network *net, const tz_tree *tree, int log2_max_intermediate,
                    int k_max, int32_t *sliced_edges, int *k_out);

/* ---------------------------------------------------------------- plans */
#define TZ_C64_SIMT     0   /* complex64, FP32 FMA on CUDA cores (4 real products) */
#define TZ_TF32X3       1   /* FP32 operands split hi+lo TF32, 3 tcgen05 products  */
#define TZ_BF16X3       2   /* FP32 operands split hi+lo BF16, 3 tcgen05 products  */
#define TZ_C128_SIMT    3   /* complex128, FP64 FMA on CUDA cores (reference-grade,
                               every tensor in FP64; slow on GB300's FP64 units)    */
#define TZ_FP16X3       4   /* FP32 operands scaled by a power of two per tensor,
                               split hi+lo FP16, 3 tcgen05 products; the scale is
                               undone exactly in the product's epilogue            */

typedef struct {
  int precision;         /* TZ_C64_SIMT, TZ_TF32X3, TZ_BF16X3, TZ_FP16X3 or TZ_C128_SIMT */
  int device;            /* CUDA device ordinal                                     */
  void *stream;          /* cudaStream_t the plan launches on (NULL = default)     */
  int small_log2;        /* steps with output and work below this use the direct SIMT kernel (0 = default) */
  int use_graph;         /* 1: replay the per-group launch sequence as a CUDA graph,
                            captured once per scratch part it runs on (the plan's
                            own, or a server slot's; up to 8 kept) and replayed on
                            any non-NULL stream                                    */
  int64_t max_bitstrings;/* bitstrings per call the workspace is sized for (0 = 4096) */
  int autotune;          /* 1: when the workspace is bound, time each tensor-core step's
                            launch choices (pairs of CTAs or single CTAs, K split or
                            not) on the plan's own buffers and keep the fastest; choices
                            are cached per device, precision, shape and output kind.
                            0: the built-in defaults                                  */
  int direct_queue;      /* 0: one launch of direct (small) steps per dependency level;
                            1: each run of direct steps between two products or
                            permutes is one persistent launch over a device work
                            queue, each step placed at the earliest point its inputs
                            exist (blocks wait, bounded, for the steps they read).
                            Same results; on GB300 with graph replay both forms
                            measure within 2 % of each other                         */
} tz_plan_opts;

typedef struct {
  int n_steps;                   /* contraction steps (tree pairs)                   */
  int n_const_steps;             /* steps computed once at bind time                 */
  int n_gemm_steps;              /* steps on the GEMM path (per group)               */
  int n_permutes;                /* operand permutes per group                       */
  int n_launches_per_group;      /* kernel launches per group                        */
  int k;                         /* sliced indices                                   */
  int batch_log2;                /* bitstrings per group = 2^batch_log2              */
  int max_log2;                  /* largest per-group intermediate (bits)            */
  double flops_per_group;        /* useful real flops per group, 8 per complex MAC   */
  double gemm_flops_per_group;   /* part of it on the GEMM path                      */
  double bytes_per_group;        /* algorithmic bytes: operands + results, complex64 */
  double permute_bytes_per_group;/* extra bytes moved by operand permutes            */
  size_t workspace_bytes;        /* device workspace the plan needs                  */
  size_t const_bytes;            /* part of it holding bind-time constants           */
  size_t scratch_bytes;          /* per-query scratch part (server admission unit)   */
  double const_flops;            /* useful flops of the bind-time (constant) steps,
                                    computed once per bind, not per group            */
  double bind_ms;                /* wall time of the last tz_plan_bind_workspace     */
  int n_tuned_steps;             /* tensor-core steps with an autotuned launch choice */
  int n_open;                    /* open output qubits: 2^n_open amplitudes per bitstring */
} tz_plan_stats;

/* Build a plan: classify steps, choose layouts, permutes and kernels, lay
 * out the device workspace. The network, tree and edge list are copied.
 * Errors: TZ_EINVAL for an incomplete tree, an edge that is not a wire index
 * or a repeated edge; TZ_EUNSUPPORTED for a tensor above 2^40 elements. */
int tz_plan_create(const tz_network *network, const tz_tree *contraction_tree,
                   const int32_t *sliced_edges, int k, const tz_plan_opts *opts, tz_plan **out);
int tz_plan_stats_get(const tz_plan *plan, tz_plan_stats *out);
/* Bind caller-owned device memory (>= workspace_bytes, 256-byte aligned) as
 * the plan's workspace; uploads the constant tensors and computes the
 * bind-time steps on the plan's stream (the memory must stay valid until
 * the plan is destroyed or rebound). TZ_ENOMEM if bytes is too small. */
int tz_plan_bind_workspace(tz_plan *plan, void *dev_ptr, size_t bytes);
/* Restrict contractions to slices [lo, hi) of [0, 2^k) (default: all).
 * Partial ranges give partial sums; ranges add up. */
int tz_plan_set_slice_range(tz_plan *plan, int64_t lo, int64_t hi);
/* The (qubit, segment) wire segment of each sliced index, in slice-bit order
 * (2 int32 per index; cap in pairs). */
int tz_plan_sliced_segments(const tz_plan *plan, int32_t *qubit_segment, int cap, int *k);

/* Text (JSON) description of the plan: tensors with their storage order,
 * steps with their GEMM shapes, the launch schedule. Same buffer protocol
 * as tz_circuit_to_spec. */
int tz_plan_describe(const tz_plan *plan, char *buf, size_t cap, size_t *len);

/* Amplitudes of n bitstrings (host pointers): copies the bitstrings in,
 * contracts every group of the slice range, sums partial amplitudes in
 * FP64, copies 2n doubles out (2n * 2^n_open with open output qubits: row r
 * holds the 2^n_open amplitudes of bitstring r, in open-value order), and
 * synchronises the plan's stream.
 * n = 0 does nothing and returns TZ_OK (the pointers are not read); n above
 * the plan's max_bitstrings, or negative, returns TZ_EINVAL. */
int tz_contract_amplitudes(tz_plan *plan, const uint8_t *bitstrings, int64_t n, double *out);
/* Same with device pointers; asynchronous on the plan's stream (no host
 * synchronisation). d_bitstrings: n x n_qubits uint8; d_out: 2n doubles
 * (2n * 2^n_open with open output qubits).
 * If a tensor-core product or a direct-step queue launch of the call times
 * out in one of its bounded waits, the amplitudes it could have affected
 * are written as NaN, and
 * tz_plan_status reports TZ_ETIMEOUT. (tz_contract_amplitudes returns
 * TZ_ETIMEOUT itself.) */
int tz_contract_amplitudes_device(tz_plan *plan, const uint8_t *d_bitstrings, int64_t n, double *d_out);
/* Synchronise the plan's stream and report how its last call (on the plan's
 * own workspace) ended: TZ_ETIMEOUT if a tensor-core product or a direct-step
 * queue launch ran out of time in a bounded wait (its amplitudes are then
 * NaN), else TZ_OK. Each call starts with a clear status. */
int tz_plan_status(tz_plan *plan);
void tz_plan_destroy(tz_plan *plan);

/* Per-kernel timing of a plan's launches (CUDA events around every launch on
 * the plan's stream; the captured-graph path is not used while enabled).
 * Kinds: 0 leaf builder, 1 direct small steps, 2 permute, 3 tiled SIMT
 * complex GEMM, 4 tensor-core complex GEMM, 5 FP64 accumulation, 6 skinny
 * streaming product (n <= 4, k <= 16), 7 long-k dot product. flops are useful
 * flops (8 per complex multiply-add); bytes are algorithmic bytes (each
 * operand read once, the result written once, complex64). */
#define TZ_PROFILE_KINDS 8
typedef struct {
  int64_t launches[TZ_PROFILE_KINDS];
  double ms[TZ_PROFILE_KINDS];
  double flops[TZ_PROFILE_KINDS];
  double bytes[TZ_PROFILE_KINDS];
} tz_plan_profile;
/* Turn profiling on (1) or off (0); either resets the counters. */
int tz_plan_profile_enable(tz_plan *plan, int on);
/* Synchronise the plan's stream and read the counters. */
int tz_plan_profile_get(tz_plan *plan, tz_plan_profile *out);
/* Per launch item of the group schedule, summed over profiled groups:
 * 6 doubles per item (kind, ms, flops, bytes, step or -1, launches), in
 * schedule order. cap = capacity in items; *n receives the item count. */
int tz_plan_profile_items(tz_plan *plan, double *out, int cap, int *n);

/* --------------------------------------------------------------- serving
 * A request loop for amplitude-batch queries over resident plans: plans
 * stay bound to their workspaces, queries are admitted while their device
 * footprint fits the budget and a slot is free, and admitted queries run
 * concurrently on separate streams. A query runs in chunks of its slice
 * range (each slice is an independent subtask, Sec. 1); between chunks a
 * query yields its slot to queries that wait for one and resumes later with
 * its partial sums kept, so long queries do not hold slots while short ones
 * queue.
 */
typedef struct {
  size_t hbm_budget;     /* bytes of device memory queries may hold at once         */
  int max_inflight;      /* concurrent queries (streams), 1..32                      */
  int device;            /* CUDA device ordinal                                      */
  void *arena;           /* caller-owned device memory of arena_bytes for query buffers */
  size_t arena_bytes;
  int wait_admit;        /* 1: submit queues a query that does not fit yet; 0: TZ_EHBM_ADMIT */
  double chunk_ms;       /* a query runs in chunks of its slice range of about this many
                            ms of estimated work (0 = 4 ms); between chunks it yields
                            its slot to waiting queries and keeps its partial sums   */
} tz_server_opts;

int tz_server_create(const tz_server_opts *opts, tz_server **out);
/* Queue a query (bitstrings copied). *ticket identifies it. */
int tz_server_submit(tz_server *srv, tz_plan *plan, const uint8_t *bitstrings, int64_t n, uint64_t *ticket);
/* Non-blocking: *done = 1 and out (2n doubles, 2n * 2^n_open with open
 * output qubits) filled once the query has
 * finished; *done = 0 otherwise. A finished ticket is released after a
 * successful poll. */
int tz_server_poll(tz_server *srv, uint64_t ticket, double *out, int *done);
/* Latency statistics (seconds) over finished queries since creation. */
int tz_server_latency(tz_server *srv, double *p50, double *p99, int64_t *n_done);
void tz_server_destroy(tz_server *srv);

/* ------------------------------------------------ per-step operations
 * The kernels of one contraction step, callable alone on device pointers
 * (asynchronous on `stream`). Used to test and tune the kernels.
 */

/* Bit permutation of a complex64 tensor of 2^rank elements: output bit p is
 * input bit perm[p] (out[j] = in[i] where bit perm[p] of i = bit p of j).
 * rank <= 40; perm must be a permutation of 0..rank-1. */
int tz_op_permute(const void *in, void *out, int rank, const int32_t *perm, void *stream);

/* Batched complex64 product C[z] = A[z] * B[z]^T, z < batch (the per-step
 * contraction of Sec. 1's network once operands are laid out):
 * A[z] is m x k row-major (k contiguous), B[z] is n x k row-major,
 * C[z] is m x n row-major; z-th matrices at element offsets z*sa, z*sb, z*sc.
 * precision: TZ_C64_SIMT, TZ_TF32X3, TZ_BF16X3, TZ_FP16X3, or TZ_C128_SIMT
 * (then A, B and C are complex128 arrays). The split-precision
 * modes need device scratch of tz_op_cgemm_scratch_bytes() bytes (256-byte
 * aligned): the hi/lo copies of B in the real view, the partial products
 * when a long K is split across CTAs (summed in a fixed order, so results do
 * not depend on scheduling), and for TZ_FP16X3 the partial maxima of |A| and
 * |B| that set each operand's power-of-two scale; they accumulate in FP32
 * over ranges of 128 real K values, added in FP32 with round to nearest.
 * TZ_EUNSUPPORTED for shapes they do not handle (m not a multiple of 128; k
 * odd for TF32, not a multiple of 4 for BF16 and FP16). */
int tz_op_cgemm(int precision, int64_t batch, int64_t m, int64_t n, int64_t k,
                const void *A, int64_t sa, const void *B, int64_t sb, void *C, int64_t sc,
                void *scratch, size_t scratch_bytes, void *stream);
int tz_op_cgemm_scratch_bytes(int precision, int64_t batch, int64_t m, int64_t n, int64_t k, size_t *bytes);
/* The split-precision products wait on on-chip barriers with a time limit
 * (2 s by default); when a wait runs out, the product stops, leaves C
 * invalid and sets an error word kept in the first 256 bytes of its scratch
 * (cleared on the stream when each tz_op_cgemm call starts). This call
 * synchronises `stream` and returns TZ_ETIMEOUT if the last product on
 * `scratch` set it, else TZ_OK (always TZ_OK for the CUDA-core modes). */
int tz_op_cgemm_status(int precision, const void *scratch, void *stream);

/* Allocation-free variant of tz_op_cgemm for the split-precision modes
 * (TZ_TF32X3, TZ_BF16X3, TZ_FP16X3). The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc (they hand all device memory
 * to another allocator, or must not pay for or fail in an allocation in a
 * latency-critical loop). The same arguments as tz_op_cgemm, without the
 * scratch buffer: the prepared copy of B goes to a 16 MiB array in device
 * global memory owned by the library, which every GPU that loads the library
 * holds until the process exits. Products needing more scratch than that
 * (tz_op_cgemm_scratch_bytes) return TZ_EINVAL. The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that
 * device current and keeps it; make that first call before any stream
 * capture, and do not reset the device (cudaDeviceReset) after it. All calls
 * share the array: calls that overlap on the GPU race on it and must be
 * serialised by the caller. The array keeps the last call's contents; each
 * call clears its error word (the array's first 256 bytes) on the stream and
 * writes every other byte it reads before reading it. Allocates no device
 * memory. */
int tz_op_cgemm_static(int precision, int64_t batch, int64_t m, int64_t n, int64_t k,
                       const void *A, int64_t sa, const void *B, int64_t sb, void *C, int64_t sc,
                       void *stream);
/* Status of the last tz_op_cgemm_static call on the current device, as
 * tz_op_cgemm_status: synchronises `stream`; TZ_ETIMEOUT if the product
 * timed out in a bounded wait. */
int tz_op_cgemm_static_status(void *stream);

/* Test hooks (current device; they change no result of a launch that
 * completes). tz_debug_set_wait_limit: the time limit of the bounded waits of
 * the tensor-core products and of the direct-step queue launches, in ns (0
 * restores the default 2 s); waits that let copies in flight land before a
 * stopped product exits always keep 2 s.
 * tz_debug_stall_tensor_core(1): every tensor-core product launched while it
 * is on first waits on a barrier that nothing arrives at, so the wait runs
 * out after the limit and the product reports TZ_ETIMEOUT; (0) turns it off.
 * tz_debug_stall_direct_queue(1): likewise, the first block of every
 * direct-step queue launch waits on a counter that nothing increments; the
 * launch stops and the plan's call reports TZ_ETIMEOUT.
 * Graph replays captured earlier pick these up (they are read on the device). */
int tz_debug_set_wait_limit(int64_t ns);
int tz_debug_stall_tensor_core(int on);
int tz_debug_stall_direct_queue(int on);
/* Test hook (process-wide): with on = 1, plans autotuned afterwards run every
 * tensor-core step with at most 32 complex K values on the tiled CUDA-core
 * complex64 kernel, whichever is faster; with on = 2, every complex64 step
 * with at most 32 complex K values that the stream kernel supports runs on
 * it (the autotuner otherwise takes either only where it measured faster);
 * 0 turns it off. Each call clears the autotuner's cache. */
int tz_debug_tune_force_simt(int on);
/* Preset one entry of the autotuner's cache on the current device: plans
 * autotuned afterwards whose step has this precision (a complex64 one),
 * shape (batch, m, n, k) and output kind (scatter = 0 row-major, 1 through
 * the scatter map) take this launch choice without timing it: pair (1 pairs
 * of CTAs, 0 single CTAs, -1 the process default), ksplit (1 never split K,
 * 0 the default split), simt (0 the step's own kernel; for k <= 32 only: 1
 * the tiled CUDA-core kernel, 2 the stream kernel). Lets a run reproduce the
 * choices of an earlier one, e.g. a profiler run, whose own timings would
 * differ. TZ_EINVAL for bad values. */
int tz_tune_preset(int precision, int64_t batch, int64_t m, int64_t n, int64_t k, int scatter, int pair, int ksplit,
                   int simt);
/* Test hook (host only, no device work): the tile the stream kernel would use
 * for a product of batch x m x n with k summed values (dimensions powers of
 * two), C row-major (scatter = 0) or written through the scatter map whose
 * output positions of the batch, row and column bits are pb, pm, pn
 * (log2 batch, log2 m, log2 n entries). *supported = 0 where the kernel does
 * not apply; else out (86 int32) = {bz, bm, bn, nl, kmax, dynamic shared
 * bytes; for each of 16 rank bits: source (0 batch, 1 row, 2 column, -1
 * none), bit, output position; the rank of each of the 32 lanes}. */
int tz_debug_stream_tile(int64_t batch, int64_t m, int64_t n, int64_t k, int scatter, const int8_t *pb,
                         const int8_t *pm, const int8_t *pn, int32_t *out, int *supported);

/* Process-wide default of how the split BF16 / FP16 products run where the
 * shape allows pairs (128-column tiles, m a multiple of 256): 1 on pairs of
 * CTAs on two SMs (cta_group::2, each CTA loading half of the B tile), 0 on
 * single CTAs, -1 back to the initial default (single CTAs, unless the
 * environment variable TZ_TC_PAIRS is 1). Plans autotuned at bind time keep
 * their own per-step choice. The two forms give the same results (the same
 * splits, products and accumulation ranges). */
int tz_tune_tc_pairs(int mode);
/* Process-wide default of how far ahead (in k-blocks of the product's K loop)
 * the tensor-core products prefetch their A tiles into L2, so that the tile
 * loads that follow hit L2; 0 turns it off, -1 restores the initial default
 * (the environment variable TZ_TC_PREFETCH, else 0). Results do not change. */
int tz_tune_tc_prefetch(int kblocks);

/* FP64 accumulation of partial amplitudes: acc[j] += scale * part[j] for
 * j < n, with part complex64 and acc, scale complex128 (re, im). */
int tz_op_accumulate(const void *part, double *acc, int64_t n, double scale_re, double scale_im, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* TZ_H */
