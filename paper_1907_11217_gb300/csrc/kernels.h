// Device-side descriptors and kernel launchers (host-callable).
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "tz.h"

namespace tz {
namespace dev {

constexpr int kMaxBits = 40;    // largest tensor rank handled (2^40 elements)
constexpr int kMaxDirect = 32;  // bits of C or K in a direct (SIMT) step
constexpr int kMaxBatch = 8;    // bitstring batch bits
constexpr int kMaxOpen = 12;    // open output qubits

// Which group (slice, bitstring chunk) the launches of one group work on.
// Read by the leaf builder and the accumulator; the accumulator advances it
// so that a captured group sequence can be replayed back to back.
struct GroupState {
  int64_t slice, chunk;  // current group
  int64_t lo, hi;        // slice range
  int64_t n_rows;        // bitstrings in the call
  int64_t groups_done;
  int tc_error;          // set by a tensor-core product or a direct-step queue
                         // launch whose bounded wait ran out; cleared when a
                         // call starts
  int pad0;
  int64_t pad[1];
};

// Device tables address tensors by region-relative byte offsets so that one
// plan can run in several scratch arenas at once: bit 62 set = offset into
// the per-query arena, clear = offset into the plan's resident constants.
constexpr int64_t kArenaTag = int64_t(1) << 62;
template <typename T = float2>
__host__ __device__ inline const T *region_ptr(int64_t off, const char *cbase, const char *abase) {
  return reinterpret_cast<const T *>(((off & kArenaTag) ? abase : cbase) + (off & (kArenaTag - 1)));
}

enum LeafKind { LJ_GATHER = 0, LJ_OUTPUT = 1 };
// One leaf tensor built per group.
struct LeafJob {
  int64_t dst;            // region-relative offset of the result
  int64_t src;            // gather: the full constant tensor
  int kind, rank;         // rank: bits of dst
  int n_fixed;            // gather: sliced bits of src
  int qubit;              // output: qubit
  int rc;                 // output: circuit indices in the table (0 or 1)
  int e_dst_pos;          // output: dst bit of the circuit index, -1 if none
  int e_slice_bit;        // output: slice bit fixing the circuit index, -1 if none
  int pad0;
  int8_t src_pos[24];     // gather: src bit of dst bit p
  int8_t fixed_src_pos[8];
  int8_t fixed_slice_bit[8];
  int8_t beta_dst_pos[8]; // output: dst bit of batch bit j, -1 if absent
  float2 M[4];            // output: table M[x * 2^rc + e] (complex64 plans)
  double2 Md[4];          // the same table for complex128 plans
};

// One small contraction step computed directly (no operand permute):
// C[c] = sum_k A[offA(c,k)] * B[offB(c,k)], offsets from bit positions.
struct DStep {
  int64_t A, B, C;      // region-relative offsets
  int64_t block_begin;  // first block of this step within its launch
  int nC, nK, split;    // output bits, contracted bits, log2 threads per output
  int nblk;             // blocks of this step
  int dep[2];           // queue launches: the steps of the same launch (indices
                        // from its first step) whose results A and B are, -1 none
  int dep_nblk[2];      // the blocks of those steps
  int8_t a_c[kMaxDirect], b_c[kMaxDirect];  // C bit -> A / B bit (-1 absent)
  int8_t a_k[kMaxDirect], b_k[kMaxDirect];  // K bit -> A / B bit
};

static_assert(offsetof(DStep, dep) % 16 == 0 && sizeof(DStep) % 16 == 0,
              "the queue kernel reads dep and dep_nblk with one 16-byte load");

// Where a GEMM writes its result: canonical element (z, m, n) of the
// row-major [batch][m][n] product goes to offset Sb(z) + Sm(m) + Sn(n),
// where bit j of m lands on bit pm[j] of the offset (likewise n, z). This
// writes the result directly in the storage order its consumer needs.
struct CScatter {
  int nm, nn, nb;
  int8_t pm[kMaxBits], pn[kMaxBits], pb[kMaxBits];
};

// Operand maps of a skinny product read in place (no permute): element
// (z, m, k) of X sits at offset sum of bit j of m << xm[j] (likewise k, z),
// and element (z, n, k) of Y at the offsets given by yn, yk, yb.
struct GatherMap {
  int nm, nn, nk, nb;
  int8_t xm[kMaxBits], xk[8], xb[kMaxBits];
  int8_t yn[8], yk[8], yb[kMaxBits];
};

struct PermuteArgs {
  int rank;
  int8_t perm[kMaxBits];  // out bit p = in bit perm[p]
};

struct AccumArgs {
  const void *root;           // complex64, or complex128 when dbl
  double2 *acc;               // [row][2^m open values]
  GroupState *gs;
  int g;                      // batch bits
  int m;                      // open output qubits
  int8_t beta_pos[kMaxBatch]; // root bit of batch bit j
  int8_t open_pos[kMaxOpen];  // root bit of open bit j
  double scale_re, scale_im;
  int advance;                // 1: advance gs to the next group
  int dbl;                    // root is complex128
};

// keep_error: a later part of the same call (the error word is kept)
cudaError_t launch_init_state(GroupState *gs, int64_t lo, int64_t hi, int64_t n_rows, cudaStream_t s,
                              int keep_error = 0);
// dbl: tensors are complex128 (else complex64)
cudaError_t launch_leaf_build(const LeafJob *jobs, int n_jobs, const GroupState *gs, const uint8_t *bits, int nq,
                              int g, const char *cbase, char *abase, int dbl, cudaStream_t s);
// bmap: the step (index from steps) of each of the launch's blocks.
cudaError_t launch_direct(const DStep *steps, int n_steps, const int *bmap, int64_t total_blocks, const char *cbase,
                          char *abase, int dbl, cudaStream_t s);
// The same steps in one persistent launch over a device work queue: blocks
// take the launch's blocks in order from a ticket counter, and a block whose
// step reads the result of an earlier step of the same launch (DStep::dep)
// first waits, bounded, until every block of that step has finished. So a
// run of dependent levels needs one launch instead of one per level.
// ctrl: direct_queue_ctrl_words(n_steps) zeroed words of device memory,
// owned by the caller; the launch leaves them zeroed again when it ends. A
// wait that runs out sets *err to 1 and stops the launch (the steps' results
// are then invalid).
// bmap: the step (index from the launch's first) of each of its blocks.
cudaError_t launch_direct_queue(const DStep *steps, int n_steps, const int *bmap, int64_t total_blocks,
                                const char *cbase, char *abase, unsigned *ctrl, int *err, int dbl, cudaStream_t s);
inline int64_t direct_queue_ctrl_words(int n_steps) { return 4 + (int64_t)n_steps; }
// Test hooks for the current device: the limit of the queue's bounded waits
// in ns (0 restores the default 2 s), and a switch that makes the first block
// of every queue launch wait on a counter that nothing increments.
cudaError_t direct_queue_set_wait_limit(unsigned long long ns);
cudaError_t direct_queue_set_stall(int on);
cudaError_t launch_permute(const float2 *in, float2 *out, const PermuteArgs &a, cudaStream_t s);
cudaError_t launch_permute_z(const double2 *in, double2 *out, const PermuteArgs &a, cudaStream_t s);
// complex128 products (FP64 FMA): tiled, skinny in place, long-k dot
cudaError_t launch_zgemm_simt(const double2 *A, const double2 *B, double2 *C, int64_t batch, int64_t M, int64_t N,
                              int64_t K, int64_t sA, int64_t sB, int64_t sC, const CScatter *sc, cudaStream_t s);
cudaError_t launch_zskinny_gather(const double2 *X, const double2 *Y, double2 *C, int64_t batch, int64_t M,
                                  int64_t N, int64_t K, const GatherMap &g, const CScatter *sc, cudaStream_t s);
// sc == nullptr: C row-major with batch stride sC.
cudaError_t launch_cgemm_simt(const float2 *A, const float2 *B, float2 *C, int64_t batch, int64_t M, int64_t N,
                              int64_t K, int64_t sA, int64_t sB, int64_t sC, const CScatter *sc, cudaStream_t s);
// Products with K <= 32 complex values on CUDA cores, organised around their
// writes: tiles of outputs that cover the lowest output positions, written in
// address order (launch_cgemm_stream returns cudaErrorNotSupported where
// cgemm_stream_supported is false: dimensions not powers of two, K above 32,
// or fewer than 256 outputs). Same FP32 arithmetic and summation order as
// launch_cgemm_simt's tiled kernel. sc == nullptr: C row-major (sC = M N).
bool cgemm_stream_supported(int64_t batch, int64_t M, int64_t N, int64_t K, const CScatter *sc);
cudaError_t launch_cgemm_stream(const float2 *A, const float2 *B, float2 *C, int64_t batch, int64_t M, int64_t N,
                                int64_t K, int64_t sA, int64_t sB, int64_t sC, const CScatter *sc, cudaStream_t s);
// Host-side tile of the stream kernel (no device work): 1 and out[] =
// {bz, bm, bn, nl, kmax, dynamic shared bytes, then per rank bit r < 16:
// source (0 batch, 1 row, 2 column, -1 none), bit, output position; then the
// 32 lanes' ranks}, or 0 where the kernel does not apply.
int cgemm_stream_describe(int64_t batch, int64_t M, int64_t N, int64_t K, const CScatter *sc, int32_t *out);
// Skinny product (n <= 4, k <= 16) reading X and Y through gather maps and
// writing C through sc (nullptr: row-major [batch][m][n]).
cudaError_t launch_cgemm_skinny_gather(const float2 *X, const float2 *Y, float2 *C, int64_t batch, int64_t M,
                                       int64_t N, int64_t K, const GatherMap &g, const CScatter *sc, cudaStream_t s);
// Split-precision tensor-core product; returns cudaErrorNotSupported when the
// shape is outside what the kernel handles (the planner checks first).
// *err (device memory) is set to 1 when one of the product's bounded waits
// runs out (its result is then invalid); the caller clears it.
// pair: 1 runs the product on pairs of CTAs (cta_group::2) where the shape
// allows it (tc_pair_supported), 0 on single CTAs, -1 the process default.
// ksplit: 1 never splits K across CTAs; 0 splits as cgemm_tc_split says.
cudaError_t launch_cgemm_tc(int precision, const float2 *A, const float2 *B, float2 *C, int64_t batch, int64_t M,
                            int64_t N, int64_t K, int64_t sA, int64_t sB, int64_t sC, const CScatter *sc,
                            void *scratch, size_t scratch_bytes, int *err, cudaStream_t s, int pair = -1,
                            int ksplit = 0);
// K ranges a row-major product of this shape is split into by default (1: none).
int cgemm_tc_split(int precision, int64_t batch, int64_t M, int64_t N, int64_t K);
bool cgemm_tc_supported(int precision, int64_t M, int64_t N, int64_t K);
// Split BF16 / FP16 products with 128-column tiles and whole 256-row tiles.
bool tc_pair_supported(int precision, int64_t M, int64_t N);
// Process default for pair = -1: 1 on, 0 off, -1 back to the initial default
// (off unless the environment variable TZ_TC_PAIRS is 1).
void tc_set_pairs(int mode);
// Process default of the L2 prefetch distance of A tiles, in k-blocks (0 off,
// -1 back to the initial default: the environment variable TZ_TC_PREFETCH, else 0).
void tc_set_prefetch(int kblocks);
// Test and debug hooks for the current device: the limit of the products'
// bounded waits in ns (0 restores the default 2 s), and a switch that makes
// every product first wait on a barrier that nothing arrives at.
cudaError_t tc_set_wait_limit(unsigned long long ns);
cudaError_t tc_set_stall(int on);
// Device scratch of one tensor-core product: the prepared hi/lo copies of B,
// for products that split K across CTAs the partial results, and in the FP16
// mode the partial maxima of |B|.
size_t cgemm_tc_scratch_bytes(int precision, int64_t batch, int64_t M, int64_t N, int64_t K);
// Kernel launches of one tensor-core product (FP16 mode: the maxima of |B|;
// B preparation, the product, and the sum of split-K partials when K is
// split; scatter outputs never split).
int cgemm_tc_launches(int precision, int64_t batch, int64_t M, int64_t N, int64_t K, bool scatter, int ksplit = 0);
cudaError_t launch_accumulate(const AccumArgs &a, cudaStream_t s);
// kernel launches of one launch_accumulate (2 when the root is too large for
// one block: the group state then advances in a launch of its own)
int accumulate_launches(int g, int m);
cudaError_t launch_accumulate_plain(const float2 *part, double2 *acc, int64_t n, double sre, double sim,
                                    cudaStream_t s);

}  // namespace dev
}  // namespace tz
