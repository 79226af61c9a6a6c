// Split-precision complex products on the tcgen05 tensor cores (sm_103a).
// Three modes share the pipeline: TF32x3 (operands split into TF32 hi + lo,
// kind::tf32), BF16x3 (operands split into BF16 hi + lo, kind::f16 with BF16
// inputs) and FP16x3 (operands scaled by powers of two into FP16's range, then
// split into FP16 hi + lo, kind::f16 with FP16 inputs: B by one exponent per
// tensor, A by one per row and k-block, chosen on chip). All accumulate in
// FP32 in TMEM.
//
// C[z] = A[z] B[z]^T in complex64, computed as one real product on the
// interleaved (re, im) view: A is read as an m x 2k FP32 matrix and C is
// written as an m x 2n FP32 matrix, with the 2n x 2k real matrix
//     row 2j   = ( Re b_jl, -Im b_jl )_l      (real part of column j)
//     row 2j+1 = ( Im b_jl,  Re b_jl )_l      (imaginary part)
// built from B by a small prep kernel. Each FP32 operand x is split exactly
// into hi = x rounded to the nearest TF32 value (10 explicit mantissa bits)
// and lo = x - hi (exact, |lo| <= 2^-11 |x|); three tensor-core products
// hi*hi + hi*lo + lo*hi accumulate in FP32 in tensor memory (TMEM); the
// dropped lo*lo term is below 2^-22 |a||b|.
//
// Pipeline per CTA (tiles of 128 rows of C by up to 64 complex columns):
//   warp 0     : TMA loads of the FP32 A tile (128 rows in boxes of 32 floats,
//                128B swizzle: one box TF32, two BF16) and of the prepared
//                hi/lo B tiles (128-byte rows), into a ring of stages;
//   warp 1     : TMEM allocation; one thread issues tcgen05.mma (A from
//                TMEM, B from shared memory) and commits stage, A-slot and
//                accumulator releases to mbarriers;
//   warps 2..5 : split each A tile: one row a thread, read from shared
//                memory, split in registers, written as hi and lo to a ring
//                of A slots in TMEM (tcgen05.st); so shared memory carries
//                only the raw A and the B operands;
//   warps 6..13: epilogue: every accumulation range of kFoldK real K values
//                ends in its own TMEM accumulator, which these warps add into
//                FP32 registers (per thread one row of the tile, half of its
//                columns: two warps per TMEM lane quarter) before the row
//                goes to global memory.
// Every wait is bounded in time; on timeout the kernel sets the caller's
// error word (TcArgs::err), drains its copies in flight, frees TMEM and
// returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "kernels.h"

namespace tz {
namespace dev {

namespace {

constexpr int BM = 128;           // C rows per tile = TMEM lanes
// K (real values) per stage: TF32 32, BF16 64, so that every TMA row is a
// whole 128-byte L2 line (64-byte rows measured slower): the FP32 A tile in
// one (TF32) or two (BF16) boxes of 128-byte rows, the split B in 128-byte
// rows.
template <int MODE>
__host__ __device__ constexpr int stage_k() { return MODE == 0 ? 32 : 64; }
// TMA, MMA, 4 split warps, 8 epilogue warps; registers are granted to warps
// in groups of four, so 14 warps leave 128 registers a thread
// warps: 0 TMA, 1 MMA issuer, 2..5 A split, 6..13 epilogue, 14 readiness
// waiter (hands the k-blocks over to the MMA warp through named barriers)
constexpr int kThreads = 480;
constexpr int kWaiterWarp = 14;
// named barriers of the MMA and waiter warps (64 threads): k-block g ready
// (kBarReady + g % kAhead), k-block g issued (kBarIssued + g % kAhead), and
// the status reduction at the end of each tile (kBarTile)
constexpr int kAhead = 2;
constexpr int kBarReady = 1, kBarIssued = kBarReady + kAhead, kBarTile = kBarIssued + kAhead;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait (default)
// Waits that let copies and products in flight finish before the CTA exits
// (after an abort) always use this limit, never the adjustable one.
constexpr unsigned long long kDrainNs = 2000000000ull;

// Per device: the limit of the ordinary bounded waits (tz_debug_set_wait_limit)
// and the test switch that makes every product's MMA issuer first wait on a
// barrier nothing arrives at (tz_debug_stall_tensor_core), so that the wait
// runs out and the product reports a timeout.
__device__ unsigned long long g_wait_ns = kWaitNs;
__device__ int g_stall;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase with the given parity; false on timeout (after limit_ns,
// which also raises the CTA's abort flag) or, with honour_abort, when another
// role has aborted (then the caller stops its work). Drains pass
// honour_abort = false and the fixed kDrainNs.
// The clock is read only every 256 unsuccessful polls (a wait that succeeds
// at once costs one try_wait): the time limit counts from the first of them.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          unsigned long long limit_ns, bool honour_abort = true) {
  unsigned long long t0 = 0;
  for (uint32_t i = 0;; i++) {
    if (mbar_try_wait(bar, parity)) return true;
    if (honour_abort && *abort_flag) return false;
    if ((i & 255) == 255) {
      const unsigned long long now = globaltimer();
      if (t0 == 0) {
        t0 = now;
      } else if (now - t0 > limit_ns) {
        *abort_flag = 1;
        return false;
      }
    }
  }
}

// Waits on barriers that the peer CTA of a pair also arrives on use the
// same (default-scope) wait: what a pair hands across is tensor memory and
// products, ordered by tcgen05 fences around the barrier.
template <bool CLUSTER>
__device__ __forceinline__ bool mbar_wait_t(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                            unsigned long long limit_ns, bool honour_abort = true) {
  return mbar_wait(bar, parity, abort_flag, limit_ns, honour_abort);
}

// Thread-block clusters of two CTAs (a pair shares one 256-row tile).
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_id_x() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t n_clusters_x() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
// shared::cluster address of the same shared-memory location in CTA `rank`
__device__ __forceinline__ uint32_t cluster_addr(const void *p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
// Arrival on a barrier of either CTA of the pair, with the default
// (CTA-scope) release: the tensor-memory writes and reads it publishes are
// ordered by tcgen05 fences, and a cluster-scope release would also wait for
// the thread's global stores to be acknowledged (a memory barrier per
// arrival, measured as the dominant stall of the epilogue warps).
__device__ __forceinline__ void mbar_arrive_remote(uint32_t caddr) {
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(caddr) : "memory");
}
__device__ __forceinline__ void st_remote_u32(uint32_t caddr, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(caddr), "r"(v) : "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// L2 policies for the TMA loads: B tiles are read by every row tile, so they
// are kept (evict last); A tiles are read by the few CTAs of one row tile at
// about the same time, then not again (normal priority by default, evict
// first as an option: TcArgs::l2_mode).
__device__ __forceinline__ uint64_t l2_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_evict_normal() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *tm, int x, int y, uint64_t *bar,
                                            uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%2, "
      "%3}], [%4], %5;" ::"r"(smem_u32(dst)),
      "l"((uint64_t)tm), "r"(x), "r"(y), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

// Hint that a tile will be loaded soon: bring it into L2 (no shared memory,
// no completion to wait for).
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap *tm, int x, int y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global [%0, {%1, %2}];" ::"l"((uint64_t)tm), "r"(x), "r"(y)
               : "memory");
}

// Instruction descriptor: FP32 accumulator, TF32 A and B, both K-major,
// N = n_cols, M = 128.
__host__ __device__ constexpr uint32_t idesc_tf32(int n_cols) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n_cols >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

// A from tensor memory (lane = row of A; one 32-bit column per TF32 value,
// or per pair of BF16 values with the lower k in the low half), B from
// shared memory.
__device__ __forceinline__ void umma_tf32_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t b, uint32_t idesc,
                                             uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::
          "r"(tmem_d),
      "r"(tmem_a), "l"(b), "r"(idesc), "r"(accum));
}
__device__ __forceinline__ void umma_f16_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t b, uint32_t idesc,
                                            uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::
          "r"(tmem_d),
      "r"(tmem_a), "l"(b), "r"(idesc), "r"(accum));
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// Pair products (cta_group::2, issued by the pair's first CTA): M = 256 rows,
// rows 0..127 of A and of the accumulator in the first CTA's tensor memory,
// rows 128..255 in the second's (same addresses); the first BNP/2 rows of B
// in the first CTA's shared memory, the rest in the second's (same offset).
__device__ __forceinline__ void umma_f16_ts_pair(uint32_t tmem_d, uint32_t tmem_a, uint64_t b, uint32_t idesc,
                                                 uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::2.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::
          "r"(tmem_d),
      "r"(tmem_a), "l"(b), "r"(idesc), "r"(accum));
}
// Commit of the pair's products to a barrier in either CTA of the pair.
__device__ __forceinline__ void umma_commit_pair(uint32_t caddr) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(caddr)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 columns of this warp's 32 TMEM lanes from registers (completion: tmem_st_wait).
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
// 8 columns (same layout as tmem_st16)
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
               "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 16 columns of this warp's 32 TMEM lanes; the wait is in the same asm
// statement, so the registers are only defined once the load has landed.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}

// Round to nearest TF32 on the bit pattern (a carry into the exponent is the
// correct rounding up); hi and x are within a factor of two, so x - hi is
// exact (Sterbenz).
__device__ __forceinline__ uint32_t split_hi(uint32_t x) { return (x + 0x1000u) & 0xFFFFE000u; }
__device__ __forceinline__ uint32_t split_lo(uint32_t x) {
  return __float_as_uint(__uint_as_float(x) - __uint_as_float(split_hi(x)));
}

// Two values at once (x0: lower k, in the low half of each result):
// hi = bf16(x) and lo = bf16(x - hi), both rounded to nearest even; the BF16
// hi values are widened back to FP32 by placing their bits in the top half.
__device__ __forceinline__ void split_bf16x2(float x0, float x1, uint32_t &hi, uint32_t &lo) {
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(x1), "f"(x0));
  const float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xFFFF0000u);
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(x1 - h1), "f"(x0 - h0));
}

// FP16 counterpart of split_bf16x2 (x0, x1 already scaled into FP16 range):
// hi = f16(x) and lo = f16(x - hi), both rounded to nearest even; x - hi is
// exact in FP32. (Computing hi by Veltkamp's splitting in FP32 arithmetic
// instead of converting it back from FP16 measured slower.)
__device__ __forceinline__ void split_f16x2(float x0, float x1, uint32_t &hi, uint32_t &lo) {
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(x1), "f"(x0));
  float h0, h1;
  asm("{\n .reg .b16 l, h;\n mov.b32 {l, h}, %2;\n cvt.f32.f16 %0, l;\n cvt.f32.f16 %1, h;\n}\n"
      : "=f"(h0), "=f"(h1)
      : "r"(hi));
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(x1 - h1), "f"(x0 - h0));
}
__device__ __forceinline__ void split_f16(float x, uint16_t &hi, uint16_t &lo) {
  const __half h = __float2half_rn(x);
  const __half l = __float2half_rn(x - __half2float(h));
  hi = __half_as_ushort(h);
  lo = __half_as_ushort(l);
}

// Per-tensor scaling of the FP16 mode (the paper's amplitudes sit near
// 2^(-n/2), far below FP16's normal range). The exponent s puts the largest
// magnitude of an operand in [2^14, 2^15): every scaled value stays below
// 65504 with its rounding, and FP16's subnormal spacing 2^-24 is 2^-38 of that
// maximum, so x = hi + lo keeps about 22 bits relative to the tensor's
// largest value. Scaling by 2^s is exact. maxbits is the FP32 bit pattern of
// the largest |x|; zero, subnormal and non-finite maxima are clamped so that
// 2^s and 2^-s stay normal FP32 numbers.
__device__ __forceinline__ int f16_scale_exp(uint32_t maxbits) {
  if (maxbits == 0 || maxbits >= 0x7f800000u) return 0;
  const int e = (int)(maxbits >> 23) - 127;  // max|x| in [2^e, 2^(e+1))
  return min(max(14 - e, -110), 110);
}
__device__ __forceinline__ float pow2i(int s) { return __int_as_float((s + 127) << 23); }  // s in [-126, 127]

// Round-to-nearest-even BF16 split: hi = bf16(x), lo = bf16(x - hi).
__device__ __forceinline__ void split_bf16(float x, uint16_t &hi, uint16_t &lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
  hi = __bfloat16_as_ushort(h);
  lo = __bfloat16_as_ushort(l);
}

// K-major operand in the 128-byte swizzled layout (rows of 128 bytes, 8-row
// atoms of 1024 bytes): 16-byte chunk c of row r sits at chunk c ^ (r & 7).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// FP32 accumulator, BF16 A and B, both K-major, N = n_cols, M = m (128, or
// 256 for a pair).
__host__ __device__ constexpr uint32_t idesc_bf16(int n_cols, int m = BM) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n_cols >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
// FP32 accumulator, FP16 A and B (format 0), both K-major, N = n_cols, M = m.
__host__ __device__ constexpr uint32_t idesc_f16(int n_cols, int m = BM) {
  return (1u << 4) | ((uint32_t)(n_cols >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

enum TcMode { MODE_TF32 = 0, MODE_BF16 = 1, MODE_F16 = 2 };

// FP16 mode: the largest |x| of B, as per-block partial maxima (FP32 bit
// patterns of |x|), at most kMaxPartials of them.
constexpr int kMaxPartials = 304;  // two blocks per SM of GB300

struct TcArgs {
  float2 *C;
  int64_t batch;
  int64_t M, N, K;     // complex sizes of one product
  int64_t sC;          // complex elements between batches of C
  int n_tiles_m, n_tiles_n, kblocks;
  int NT;              // rows of the prepared B per batch
  int scatter;         // 1: write C through sc; 2: likewise, the lowest bit of
                       // C being n bit 0 (stores of column pairs, staged per warp)
  int tma_store;       // 1: row-major C written by bulk tensor stores (tmC)
  int ksplit, kb_per;  // K split into ksplit ranges of kb_per k-blocks; with
  int64_t split_stride;  // ksplit > 1, range s writes row-major partials at C + s * split_stride
  const uint32_t *bmax;  // FP16 mode: pb partial maxima of |B|
  int pb;
  int *err;              // set to 1 when a bounded wait ran out (never cleared here)
  int prefetch;          // A tiles prefetched into L2 this many k-blocks ahead of their loads (0: off)
  int l2_mode;           // bit 0: A tiles loaded with the normal L2 priority (else evict first);
                         // bit 1: C written as streaming data (evict first)
  CScatter sc;
};

__device__ __forceinline__ int64_t scatter_bits(int64_t v, int n, const int8_t *pos) {
  int64_t o = 0;
  for (int j = 0; j < n; j++) o |= ((v >> j) & 1) << pos[j];
  return o;
}

// Accumulation range: the tensor cores sum at most kFoldK real K values (of
// each of the three products) in one TMEM accumulator. Their FP32
// accumulation rounds toward zero: on GB300 a product summed over K real
// values in one accumulator comes out smaller by about 6e-9 K (relative),
// whatever the total K. The epilogue warps add the ranges in FP32 registers
// (round to nearest), which bounds that bias at about 6e-9 kFoldK per product.
constexpr int kFoldK = 128;
// FP16 mode: the same ranges of 128 real K (two k-blocks); each range of a
// row of A carries its own scale exponent, chosen over the range's values.
template <int MODE>
__host__ __device__ constexpr int fold_k() { return kFoldK; }

// Per stage (shared memory): the FP32 A tile as loaded (128 rows in boxes of
// 128-byte rows: one TF32, two BF16) and the prepared B hi and lo tiles (BNP
// rows x 128 B).
// TMEM (all 512 columns): a ring of ASLOTS split A tiles (SLOT_COLS columns each:
// hi, then lo) in the top columns, below it a ring of NBUF accumulators of
// BNP columns (at least 32): the products of one range go to the next
// accumulator of the ring while the epilogue drains the previous ones.
// FP16 mode: a ring of XR x 128 scale exponents of A (one per row and
// k-block), written by the split warps and read by the epilogue, each ring
// entry with its own barrier.
template <int MODE, int BNP, int STAGES, int CG = 1>
struct TcSmem {
  static constexpr uint32_t A_BYTES = BM * stage_k<MODE>() * 4;         // FP32 tile as loaded (boxes of 128-byte rows)
  static constexpr uint32_t BROW = 128;                                  // bytes per split B row
  static constexpr uint32_t B_BYTES = (BNP / CG) * BROW;                 // a pair: this CTA's half of the rows
  static constexpr uint32_t SLOT_COLS = 64;                              // TMEM columns of a split A tile
  static constexpr uint32_t STAGE = A_BYTES + 2 * B_BYTES;
  static constexpr int EC = BNP >= 32 ? BNP / 2 : BNP;                // real columns per epilogue warp
  static constexpr uint32_t BARS = 512;                                // barriers and flags
  static constexpr uint32_t STAGING = 8 * 2048;                        // epilogue: 8 warps x (32 rows x 64 B)
  static constexpr uint32_t COLOFF = 8 * (EC / 2) * 8;                 // epilogue: 8 warps x column offsets
  static constexpr int XR = MODE == MODE_F16 ? 16 : 0;                 // FP16: ring of A exponents
  static constexpr uint32_t XEXP = XR * BM;                            // one int8 per row and entry
  static constexpr int XRI = XR > 0 ? XR : 1;                          // ring size for indexing
  static constexpr uint32_t TOTAL = STAGES * STAGE + STAGING + BARS + COLOFF + XEXP + 1024;  // + alignment
  static constexpr uint32_t ACC_COLS = BNP < 32 ? 32 : BNP;
  static constexpr uint32_t TMEM_COLS = 512;
  // the split warps cannot run more than STAGES k-blocks ahead (they read A
  // from a stage), so more slots than stages would stay unused
  static constexpr int ASLOTS = STAGES < 4 ? STAGES : 4;
  // one slot per stage: the products of a k-block release its stage and its
  // A slot together, on the stage's barrier (one commit instead of two)
  static constexpr bool SLOT_IS_STAGE = ASLOTS == STAGES;
  static constexpr uint32_t A_COL0 = TMEM_COLS - ASLOTS * SLOT_COLS;
  static constexpr int NBUF = A_COL0 / ACC_COLS;
  static_assert(BNP <= 128, "an epilogue thread holds half a row of the tile in registers");
  // barriers, then the TMEM address, the abort flag and two scale exponents
  static_assert((3 * STAGES + 2 * NBUF + ASLOTS + 2 + XR) * 8 + 16 <= BARS, "barriers and flags fit in BARS");
  // the split warps run at most ASLOTS k-blocks ahead of the products, which
  // run at most NBUF ranges ahead of the epilogue: a split warp never reaches
  // an exponent entry, or its barrier's next phase, that the epilogue has yet
  // to read
  static_assert(XR == 0 || XR >= ASLOTS + NBUF + 1, "exponent ring deep enough");
};

// Persistent: each CTA walks tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// (batch-major, then row tile, then column tile, so CTAs working at the same
// time share A tiles in L2). The stage ring and the accumulator ring run on
// across tiles.
// CG = 2: clusters of two CTAs on two SMs work as a pair on tiles of 256
// rows (cta_group::2 products issued by the first CTA): each CTA loads its
// own 128 rows of A and half of the B tile, so each SM takes in half the B
// bytes per product of the 1-CTA form. The split and epilogue warps of each
// CTA serve its own rows; the pair signals across the cluster (remote
// barrier arrivals, commits to both CTAs' barriers).
template <int MODE, int BNP, int STAGES, int CG>
__global__ void __launch_bounds__(kThreads, 1)
    tc_split3_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmBh,
                     const __grid_constant__ CUtensorMap tmBl, const __grid_constant__ CUtensorMap tmC, TcArgs a) {
  using L = TcSmem<MODE, BNP, STAGES, CG>;
  static_assert(CG == 1 || (MODE != MODE_TF32 && BNP == 128), "pairs: split BF16 / FP16, 128-column tiles");
  // who waits for a drained accumulator before a range's products: the split
  // warps when a range spans several k-blocks, else the MMA issuer
  constexpr bool kSplitWaitsDrain = fold_k<MODE>() / stage_k<MODE>() > 1;
  // who waits for each k-block's split A before its products: a waiter warp
  // that hands the k-blocks over (pairs and TF32: their products are bound
  // by the issuing thread, and a wait on it stalls the tensor pipe), or the
  // issuing thread itself (single-CTA BF16 / FP16: bound by the split warps,
  // where the extra hand-over only adds latency; measured 3-12 % slower with
  // the waiter, against 2-6 % faster for the others)
  constexpr bool kWaiter = CG == 2 || MODE == MODE_TF32;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * L::STAGE + L::STAGING);
  uint64_t *conv = full + STAGES;
  uint64_t *empty = conv + STAGES;
  uint64_t *tfull = empty + STAGES;     // [NBUF] accumulator ready for the epilogue
  uint64_t *tempty = tfull + L::NBUF;   // [NBUF] accumulator drained by the epilogue
  uint64_t *drain = tempty + L::NBUF;   // all products retired
  uint64_t *aempty_own = drain + 1;     // [ASLOTS] TMEM A slot read by its products
  uint64_t *aempty = L::SLOT_IS_STAGE ? empty : aempty_own;
  uint64_t *xfull = aempty_own + L::ASLOTS;  // [XR] FP16: exponent ring entry written
  uint64_t *stall = xfull + L::XR;       // test stall: nothing ever arrives here
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(stall + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  int *scale_exp = reinterpret_cast<int *>(tmem_slot + 2);  // FP16 mode: [1] = exponent of B
  int64_t *coloff_all = reinterpret_cast<int64_t *>(smem + STAGES * L::STAGE + L::STAGING + L::BARS);
  int8_t *aexp = reinterpret_cast<int8_t *>(smem + STAGES * L::STAGE + L::STAGING + L::BARS + L::COLOFF);
  uint8_t *staging = smem + STAGES * L::STAGE;  // 1024-aligned
  auto A_raw = [&](int s) { return smem + s * L::STAGE; };
  auto B_hi = [&](int s) { return smem + s * L::STAGE + L::A_BYTES; };
  auto B_lo = [&](int s) { return smem + s * L::STAGE + L::A_BYTES + L::B_BYTES; };

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t per_batch = (int64_t)a.n_tiles_m * a.n_tiles_n;
  const int64_t n_tiles = per_batch * a.batch * a.ksplit;
  // tile walkers: CTAs, or pairs of CTAs (clusters)
  const uint32_t rank = CG == 2 ? cluster_rank() : 0u;
  const int64_t walker = CG == 2 ? (int64_t)cluster_id_x() : (int64_t)blockIdx.x;
  const int64_t n_walkers = CG == 2 ? (int64_t)n_clusters_x() : (int64_t)gridDim.x;
  struct Tile {
    int64_t z;
    int mt, nt, rowA, rowB, ks, kb0, kb1;
    int64_t row0;  // first row of this CTA's part of the tile within its batch
  };
  auto decode = [&](int64_t t) {
    Tile d;
    d.ks = (int)(t % a.ksplit);
    t /= a.ksplit;
    d.kb0 = d.ks * a.kb_per;
    d.kb1 = min(a.kblocks, d.kb0 + a.kb_per);
    d.z = t / per_batch;
    const int64_t rem = t - d.z * per_batch;
    d.mt = (int)(rem / a.n_tiles_n);
    d.nt = (int)(rem % a.n_tiles_n);
    d.row0 = (int64_t)d.mt * (BM * CG) + (int64_t)rank * BM;
    d.rowA = (int)(d.z * a.M + d.row0);
    d.rowB = (int)(d.z * a.NT + (int64_t)d.nt * BNP + (int64_t)rank * (BNP / CG));
    return d;
  };

  if (threadIdx.x == 0) {
    // pairs: conv and tempty are counted per warp (one elected arrival of
    // each split or epilogue warp of both CTAs) on the first CTA's barriers
    for (int s = 0; s < STAGES; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], CG == 2 ? 8 : 128);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < L::NBUF; b++) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], CG == 2 ? 16 : 256);
    }
    mbar_init(drain, 1);
    if (!L::SLOT_IS_STAGE)
      for (int b = 0; b < L::ASLOTS; b++) mbar_init(&aempty_own[b], 1);
    for (int b = 0; b < L::XR; b++) mbar_init(&xfull[b], 128);
    mbar_init(stall, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    // a pair allocates collectively: one warp of each CTA, the same columns
    if constexpr (CG == 2) {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"((uint32_t)L::TMEM_COLS));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"((uint32_t)L::TMEM_COLS));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
  }
  if (MODE == MODE_F16 && warp == 2) {
    // B's exponent: reduce the partial maxima written by absmax_kernel
    // earlier on the stream
    uint32_t mb = 0;
    for (int j = lane; j < a.pb; j += 32) mb = max(mb, a.bmax[j]);
    mb = __reduce_max_sync(0xffffffffu, mb);
    if (lane == 0) scale_exp[1] = f16_scale_exp(mb);
  }
  tc_fence_before();
  __syncthreads();
  // a pair: the peer's barriers are initialised before anyone arrives on them
  if constexpr (CG == 2) cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const unsigned long long wait_ns = g_wait_ns;
  // named barriers of the MMA and waiter warps (64 threads, both whole warps)
  auto named_sync = [](int id) { asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory"); };
  auto named_arrive = [](int id) { asm volatile("bar.arrive %0, 64;" ::"r"(id) : "memory"); };
  // both warps meet; true when both pass ok_in true
  auto named_all = [](int id, bool ok_in) {
    uint32_t all;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.b32 q, %1, 0;\n bar.red.and.pred p, %2, 64, q;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(all)
        : "r"((uint32_t)ok_in), "r"(id)
        : "memory");
    return all != 0;
  };
  // a wait that gives up (timeout, or an abort) also stops the peer CTA
  auto wait = [&](uint64_t *bar, uint32_t parity) {
    const bool ok = mbar_wait_t<CG == 2>(bar, parity, abort_flag, wait_ns);
    if (CG == 2 && !ok) st_remote_u32(cluster_addr((const void *)abort_flag, rank ^ 1u), 1u);
    return ok;
  };

  if (warp == 0) {
    if (lane == 0) {
      const uint64_t keep = l2_evict_last(), stream = (a.l2_mode & 1) ? l2_evict_normal() : l2_evict_first();
      int64_t g = 0;  // k-blocks issued by this CTA
      bool ok = true;
      // L2 prefetch of A: a second cursor walks the same k-blocks a.prefetch
      // ahead of the loads, so that a load finds its A tile in L2
      int64_t pt = walker;
      int pkb = -1;
      Tile pd{};
      bool pf = a.prefetch > 0;
      auto prefetch_next = [&]() {
        if (!pf) return;
        if (pkb < 0 || ++pkb >= pd.kb1) {
          if (pkb >= 0) pt += n_walkers;
          if (pt >= n_tiles) {
            pf = false;
            return;
          }
          pd = decode(pt);
          pkb = pd.kb0;
        }
#pragma unroll
        for (int h = 0; h < stage_k<MODE>() / 32; h++) tma_prefetch_2d(&tmA, pkb * stage_k<MODE>() + 32 * h, pd.rowA);
      };
      for (int i = 0; i < a.prefetch; i++) prefetch_next();
      for (int64_t t = walker; t < n_tiles && ok; t += n_walkers) {
        const Tile d = decode(t);
        for (int kb = d.kb0; kb < d.kb1; kb++, g++) {
          prefetch_next();
          const int s = (int)(g % STAGES);
          const int64_t round = g / STAGES;
          if (round > 0 && !wait(&empty[s], (uint32_t)((round - 1) & 1))) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full[s], L::A_BYTES + 2 * L::B_BYTES);
          // A in boxes of 32 floats (128-byte rows), one after the other
#pragma unroll
          for (int h = 0; h < stage_k<MODE>() / 32; h++)
            tma_load_2d(A_raw(s) + h * BM * 128, &tmA, kb * stage_k<MODE>() + 32 * h, d.rowA, &full[s], stream);
          tma_load_2d(B_hi(s), &tmBh, kb * stage_k<MODE>(), d.rowB, &full[s], keep);
          tma_load_2d(B_lo(s), &tmBl, kb * stage_k<MODE>(), d.rowB, &full[s], keep);
        }
      }
      if (*abort_flag) {
        // drain: let the copies already issued land before the CTA exits
        for (int64_t q = g > STAGES ? g - STAGES : 0; q < g; q++)
          mbar_wait_t<CG == 2>(&full[q % STAGES], (uint32_t)((q / STAGES) & 1), abort_flag, kDrainNs, false);
      }
    }
  } else if (warp == 1) {
    if (CG == 2 && rank != 0) {
      // the pair's second CTA issues no products: it waits until the first
      // CTA's products (which use its tensor and shared memory) have retired
      if (lane == 0) mbar_wait_t<true>(drain, 0, abort_flag, kDrainNs, false);
    } else {
      constexpr uint32_t idesc = MODE == MODE_TF32   ? idesc_tf32(BNP)
                                 : MODE == MODE_BF16 ? idesc_bf16(BNP, BM * CG)
                                                     : idesc_f16(BNP, BM * CG);
      // commit to a barrier of this CTA and, for a pair, the same barrier of
      // the peer
      auto commit = [&](uint64_t *bar) {
        if constexpr (CG == 2) {
          umma_commit_pair(cluster_addr(bar, 0));
          umma_commit_pair(cluster_addr(bar, 1));
        } else {
          umma_commit(bar);
        }
      };
      // K per instruction: 8 TF32 or 16 BF16 values (32 bytes of a B row,
      // 8 TMEM columns of A)
      constexpr int kSteps = stage_k<MODE>() / (MODE == MODE_TF32 ? 8 : 16);
      constexpr int kFoldKb = fold_k<MODE>() / stage_k<MODE>();  // k-blocks per accumulation range
      // the products of k-block g (the kb - r0-th of its range) into d_acc,
      // then the release of its stage and A slot (one thread)
      auto issue = [&](int64_t g, int kr, uint32_t d_acc) {
        const int s = (int)(g % STAGES);
        const int slot = (int)(g % L::ASLOTS);
        const uint32_t ah = tmem + L::A_COL0 + (uint32_t)(slot * L::SLOT_COLS), al = ah + L::SLOT_COLS / 2;
        const uint32_t bh = smem_u32(B_hi(s)), bl = smem_u32(B_lo(s));
#pragma unroll
        for (int kk = 0; kk < kSteps; kk++) {
          // 8 TMEM columns and 32 bytes of each B row per instruction
          const uint64_t dbh = sw128_desc(bh + kk * 32), dbl = sw128_desc(bl + kk * 32);
          const uint32_t acc = (kr | kk) != 0;
          if (MODE == MODE_TF32) {
            umma_tf32_ts(d_acc, ah + kk * 8, dbh, idesc, acc);
            umma_tf32_ts(d_acc, ah + kk * 8, dbl, idesc, 1);
            umma_tf32_ts(d_acc, al + kk * 8, dbh, idesc, 1);
          } else if (CG == 2) {
            umma_f16_ts_pair(d_acc, ah + kk * 8, dbh, idesc, acc);
            umma_f16_ts_pair(d_acc, ah + kk * 8, dbl, idesc, 1);
            umma_f16_ts_pair(d_acc, al + kk * 8, dbh, idesc, 1);
          } else {
            umma_f16_ts(d_acc, ah + kk * 8, dbh, idesc, acc);
            umma_f16_ts(d_acc, ah + kk * 8, dbl, idesc, 1);
            umma_f16_ts(d_acc, al + kk * 8, dbh, idesc, 1);
          }
        }
        commit(&empty[s]);
        if (!L::SLOT_IS_STAGE) commit(&aempty[slot]);
      };
      int64_t g = 0, rg = 0;  // k-blocks and accumulation ranges issued
      if constexpr (kWaiter) {
        // No wait on the issuing thread: the waiter warp waits, up to kAhead
        // k-blocks ahead, and releases each k-block through a named barrier.
        // The whole warp runs the loop (named barriers count whole warps);
        // lane 0 issues. A wait of the waiter that gave up ends both warps at
        // the end of the tile (the products issued meanwhile read buffers that
        // may not be ready: their results are discarded with the call's error
        // status).
        for (int64_t t = walker; t < n_tiles; t += n_walkers) {
          const Tile d = decode(t);
          const int nkb = d.kb1 - d.kb0;
          for (int r0 = 0; r0 < nkb; r0 += kFoldKb, rg++) {
            const int buf = (int)(rg % L::NBUF);
            const uint32_t d_acc = tmem + (uint32_t)(buf * L::ACC_COLS);
            const int r1 = min(nkb, r0 + kFoldKb);
            for (int kb = r0; kb < r1; kb++, g++) {
              named_sync(kBarReady + (int)(g % kAhead));
              tc_fence_after();
              if (lane == 0) issue(g, kb - r0, d_acc);
              __syncwarp();
              named_arrive(kBarIssued + (int)(g % kAhead));
            }
            if (lane == 0) commit(&tfull[buf]);
            __syncwarp();
          }
          if (!named_all(kBarTile, true)) break;
        }
      } else if (lane == 0) {
        // the issuing thread waits itself
        bool ok = !g_stall || wait(stall, 0);  // test stall: nothing arrives there
        for (int64_t t = walker; t < n_tiles && ok; t += n_walkers) {
          const Tile d = decode(t);
          const int nkb = d.kb1 - d.kb0;
          for (int r0 = 0; r0 < nkb; r0 += kFoldKb, rg++) {
            const int buf = (int)(rg % L::NBUF);
            if (!kSplitWaitsDrain) {
              const int64_t use = rg / L::NBUF;
              if (use > 0 && !wait(&tempty[buf], (uint32_t)((use - 1) & 1))) {
                ok = false;
                break;
              }
              tc_fence_after();
            }
            const uint32_t d_acc = tmem + (uint32_t)(buf * L::ACC_COLS);
            const int r1 = min(nkb, r0 + kFoldKb);
            for (int kb = r0; kb < r1; kb++, g++) {
              if (!wait(&conv[(int)(g % STAGES)], (uint32_t)((g / STAGES) & 1))) {
                ok = false;
                break;
              }
              tc_fence_after();
              issue(g, kb - r0, d_acc);
            }
            if (!ok) break;
            commit(&tfull[buf]);
          }
        }
      }
      // every product issued by this thread has retired once this fires
      // (for a pair, in both CTAs)
      if (lane == 0) {
        commit(drain);
        mbar_wait_t<CG == 2>(drain, 0, abort_flag, kDrainNs, false);
      }
      __syncwarp();
    }
  } else if (warp == kWaiterWarp) {
    // readiness waiter of the issuing CTA: for each k-block it waits for the
    // split A (and, at a range's start, for the accumulator to be drained
    // where the split warps do not wait for that), then releases the k-block
    // to the MMA warp; it runs at most kAhead k-blocks ahead, so its waits
    // overlap the products of the k-blocks before. After a wait gives up it
    // waits no more and releases the rest of the tile at once; the status
    // reduction at the tile's end then stops both warps.
    if (kWaiter && (CG == 1 || rank == 0)) {
      constexpr int kFoldKb = fold_k<MODE>() / stage_k<MODE>();
      int64_t g = 0, rg = 0;
      bool ok = true;
      // test stall: a bounded wait on a barrier nothing arrives at
      if (lane == 0 && g_stall) ok = wait(stall, 0);
      for (int64_t t = walker; t < n_tiles; t += n_walkers) {
        const Tile d = decode(t);
        const int nkb = d.kb1 - d.kb0;
        for (int r0 = 0; r0 < nkb; r0 += kFoldKb, rg++) {
          const int r1 = min(nkb, r0 + kFoldKb);
          for (int kb = r0; kb < r1; kb++, g++) {
            if (lane == 0 && ok) {
              if (!kSplitWaitsDrain && kb == r0 && rg >= L::NBUF)
                ok = wait(&tempty[rg % L::NBUF], (uint32_t)(((rg / L::NBUF) - 1) & 1));
              if (ok) ok = wait(&conv[(int)(g % STAGES)], (uint32_t)((g / STAGES) & 1));
            }
            __syncwarp();
            // k-block g - kAhead issued: its ready barrier may be reused
            if (g >= kAhead) named_sync(kBarIssued + (int)(g % kAhead));
            named_arrive(kBarReady + (int)(g % kAhead));
          }
        }
        ok = __shfl_sync(0xffffffffu, (int)ok, 0) != 0;
        if (!named_all(kBarTile, ok)) break;
      }
      // take the last "issued" arrivals, so that every barrier generation
      // completes before the CTA exits
      for (int64_t q = g > kAhead ? g - kAhead : 0; q < g; q++) named_sync(kBarIssued + (int)(q % kAhead));
    }
  } else if (warp < 6) {
    // split warps: warp w takes TMEM lane quarter w % 4, one row of A a thread
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16) + L::A_COL0;
    constexpr int kFoldKb = fold_k<MODE>() / stage_k<MODE>();  // k-blocks per accumulation range
    int64_t g = 0, rg = 0;
    int range_se = 0;  // FP16: this row's scale exponent of the current range
    bool ok = true;
    for (int64_t tile = walker; tile < n_tiles && ok; tile += n_walkers) {
      const Tile d = decode(tile);
      const int nkb = d.kb1 - d.kb0;
      for (int kb = 0; kb < nkb; kb++, g++) {
        const int s = (int)(g % STAGES);
        const int slot = (int)(g % L::ASLOTS);
        const int64_t use = g / L::ASLOTS;
        // a range's first k-block is released to the products only once the
        // accumulator it goes to has been drained by the epilogue (a pair:
        // the first CTA's split warps wait, on the barrier both CTAs'
        // epilogues arrive at; the products wait for both CTAs' split warps)
        if (kSplitWaitsDrain && kb % kFoldKb == 0) {
          if ((CG == 1 || rank == 0) && rg >= L::NBUF &&
              !wait(&tempty[rg % L::NBUF], (uint32_t)(((rg / L::NBUF) - 1) & 1))) {
            ok = false;
            break;
          }
          rg++;
        }
        // the A slot is free once the products of k-block g - ASLOTS have
        // retired; with one slot per stage the stage's TMA load waited for
        // exactly that before it was issued, so its landing implies it
        if ((!L::SLOT_IS_STAGE && use > 0 && !wait(&aempty[slot], (uint32_t)((use - 1) & 1))) ||
            !wait(&full[s], (uint32_t)((g / STAGES) & 1))) {
          ok = false;
          break;
        }
        tc_fence_after();
        // boxes of 32 floats: 16-byte chunk c of a row at chunk c ^ (row & 7)
        const uint32_t ts = tq + (uint32_t)(slot * L::SLOT_COLS);
        if (MODE == MODE_TF32) {
          // one box; hi in columns 0..31 of the slot, lo in 32..63
          const uint4 *src = reinterpret_cast<const uint4 *>(A_raw(s) + row * 128);
#pragma unroll
          for (int h = 0; h < 2; h++) {
            uint32_t hi[16], lo[16];
#pragma unroll
            for (int c = 0; c < 4; c++) {
              const uint4 v = src[(4 * h + c) ^ (row & 7)];
              const uint32_t x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
              for (int j = 0; j < 4; j++) {
                hi[4 * c + j] = split_hi(x[j]);
                lo[4 * c + j] = __float_as_uint(__uint_as_float(x[j]) - __uint_as_float(hi[4 * c + j]));
              }
            }
            tmem_st16(ts + (uint32_t)(16 * h), hi);
            tmem_st16(ts + (uint32_t)(32 + 16 * h), lo);
          }
        } else if (MODE == MODE_BF16) {
          // two boxes (K 0..31, 32..63); BF16 pairs packed with the lower k
          // in the low half: hi in columns 0..31, lo in 32..63
#pragma unroll
          for (int h = 0; h < 2; h++) {
            const uint4 *src = reinterpret_cast<const uint4 *>(A_raw(s) + h * BM * 128 + row * 128);
            uint32_t hi[16], lo[16];
#pragma unroll
            for (int c = 0; c < 8; c++) {
              const uint4 v = src[c ^ (row & 7)];
              split_bf16x2(__uint_as_float(v.x), __uint_as_float(v.y), hi[2 * c], lo[2 * c]);
              split_bf16x2(__uint_as_float(v.z), __uint_as_float(v.w), hi[2 * c + 1], lo[2 * c + 1]);
            }
            tmem_st16(ts + (uint32_t)(16 * h), hi);
            tmem_st16(ts + (uint32_t)(32 + 16 * h), lo);
          }
        } else {
          // FP16: at a range's first k-block the row's values of the whole
          // range (this k-block and, if the range has one, the next: its
          // stage is waited for here) set the row's exponent for the range
          // (the largest magnitude scaled into [2^14, 2^15)); then as for
          // BF16, with FP16 pairs
          uint4 v[16];
#pragma unroll
          for (int c = 0; c < 16; c++)
            v[c] = reinterpret_cast<const uint4 *>(A_raw(s) + (c >> 3) * BM * 128 + row * 128)[(c & 7) ^ (row & 7)];
          if (kb % kFoldKb == 0) {
            // (FP32 max of magnitudes, one instruction a value; a NaN is
            // skipped here and still propagates through the products)
            float m = 0.f;
#pragma unroll
            for (int c = 0; c < 16; c++)
              m = fmaxf(fmaxf(m, fmaxf(fabsf(__uint_as_float(v[c].x)), fabsf(__uint_as_float(v[c].y)))),
                        fmaxf(fabsf(__uint_as_float(v[c].z)), fabsf(__uint_as_float(v[c].w))));
            for (int j = 1; j < kFoldKb && kb + j < nkb; j++) {
              const int64_t gj = g + j;
              if (!wait(&full[gj % STAGES], (uint32_t)((gj / STAGES) & 1))) {
                ok = false;
                break;
              }
              const uint8_t *aj = A_raw((int)(gj % STAGES));
#pragma unroll
              for (int c = 0; c < 16; c++) {
                const uint4 w = reinterpret_cast<const uint4 *>(aj + (c >> 3) * BM * 128 + row * 128)[(c & 7) ^ (row & 7)];
                m = fmaxf(fmaxf(m, fmaxf(fabsf(__uint_as_float(w.x)), fabsf(__uint_as_float(w.y)))),
                          fmaxf(fabsf(__uint_as_float(w.z)), fabsf(__uint_as_float(w.w))));
              }
            }
            if (!ok) break;
            range_se = f16_scale_exp(__float_as_uint(m));
            aexp[(int)((rg - 1) % L::XRI) * BM + row] = (int8_t)range_se;
          }
          const float sa = pow2i(range_se);
          // 8 columns at a time, so the raw values die as they are split
#pragma unroll
          for (int h = 0; h < 4; h++) {
            uint32_t hi[8], lo[8];
#pragma unroll
            for (int c = 0; c < 4; c++) {
              const uint4 w = v[4 * h + c];
              split_f16x2(__uint_as_float(w.x) * sa, __uint_as_float(w.y) * sa, hi[2 * c], lo[2 * c]);
              split_f16x2(__uint_as_float(w.z) * sa, __uint_as_float(w.w) * sa, hi[2 * c + 1], lo[2 * c + 1]);
            }
            tmem_st8(ts + (uint32_t)(8 * h), hi);
            tmem_st8(ts + (uint32_t)(32 + 8 * h), lo);
          }
        }
        tmem_st_wait();
        tc_fence_before();
        if constexpr (CG == 2) {
          // one arrival per warp on the first CTA's barrier: this CTA's
          // stage (its A rows and B half) has landed and its A is split
          __syncwarp();
          if (lane == 0) mbar_arrive_remote(cluster_addr(&conv[s], 0));
        } else {
          mbar_arrive(&conv[s]);
        }
        // FP16: the range's last k-block releases its exponent to the epilogue
        if (MODE == MODE_F16 && (kb % kFoldKb == kFoldKb - 1 || kb == nkb - 1)) mbar_arrive(&xfull[(rg - 1) % L::XRI]);
      }
    }
  } else {
    // epilogue: warps 6..13 read TMEM lane quarters 2, 3, 0, 1, 2, 3, 0, 1;
    // warps 6..9 take the first EC columns of the tile, warps 10..13 the
    // rest (none when the tile is narrower than 32 columns); each thread
    // sums its part of a row over the accumulation ranges in registers
    constexpr int kFoldKb = fold_k<MODE>() / stage_k<MODE>();
    constexpr int EC = L::EC;
    const int e = warp - 6;
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const int c0 = (e >> 2) * EC;  // first column (real) of this warp
    const bool active = c0 < BNP;
    int64_t *coloff = coloff_all + e * (EC / 2);  // this warp's copy
    // FP16 mode: the range of k-block g holds 2^(sa(row, g) + sb) times its
    // part of C; each range is added times 2^-sa(row, g) and the sum times
    // 2^-sb at the end (both exact: the exponents are clamped to +-110)
    const float ub = MODE == MODE_F16 ? pow2i(-scale_exp[1]) : 1.f;
    int64_t rg = 0;
    bool ok = true;
    for (int64_t tile = walker; tile < n_tiles && ok; tile += n_walkers) {
      const Tile d = decode(tile);
      const int64_t n0 = (int64_t)d.nt * (BNP / 2) + c0 / 2;  // first complex column of this warp
      if (a.scatter && active) {
        __syncwarp();  // the previous tile's offsets are no longer read
        for (int j = lane; j < EC / 2; j += 32) coloff[j] = scatter_bits(n0 + j, a.sc.nn, a.sc.pn);
        __syncwarp();
      }
      float acc[EC];
#pragma unroll
      for (int j = 0; j < EC; j++) acc[j] = 0.f;
      const int nkb = d.kb1 - d.kb0;
      for (int r0 = 0; r0 < nkb; r0 += kFoldKb, rg++) {
        const int buf = (int)(rg % L::NBUF);
        if (!wait(&tfull[buf], (uint32_t)((rg / L::NBUF) & 1))) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t taddr = tmem + (uint32_t)(buf * L::ACC_COLS + c0) + ((uint32_t)(q * 32) << 16);
        if (active) {
          float ua = 1.f;
          if (MODE == MODE_F16) {
            // the split warps released this entry before the products of the
            // range were issued, so the wait does not block in practice
            if (!wait(&xfull[rg % L::XRI], (uint32_t)((rg / L::XRI) & 1))) {
              ok = false;
              break;
            }
            ua = pow2i(-(int)aexp[(int)(rg % L::XRI) * BM + row]);
          }
#pragma unroll
          for (int c = 0; c < EC; c += 16) {
            uint32_t r[16];
            tmem_ld16(taddr + (uint32_t)c, r);
#pragma unroll
            for (int j = 0; j < 16; j++) {
              if (MODE == MODE_F16)
                acc[c + j] = fmaf(__uint_as_float(r[j]), ua, acc[c + j]);
              else
                acc[c + j] += __uint_as_float(r[j]);
            }
          }
        }
        tc_fence_before();
        if constexpr (CG == 2) {
          __syncwarp();
          if (lane == 0) mbar_arrive_remote(cluster_addr(&tempty[buf], 0));
        } else {
          mbar_arrive(&tempty[buf]);
        }
      }
      if (!ok) break;
      if (!active) continue;
      if (MODE == MODE_F16) {
#pragma unroll
        for (int j = 0; j < EC; j++) acc[j] *= ub;
      }
      if (a.scatter == 2) {
        // a warp's 32 rows x 8 complex go through its staging buffer (16-byte
        // chunk j of row r at chunk j ^ ((r >> 1) & 3), so both sides are
        // free of bank conflicts); then each store instruction writes 8 rows
        // x 4 column pairs (lane: row 8 u + lane / 4, pair lane % 4). A pair
        // is 16 contiguous bytes because n bit 0 is the lowest bit of C; when
        // n bits 1 and 2 follow it, a row's 4 pairs are 64 contiguous bytes.
        const int64_t om = scatter_bits(d.z, a.sc.nb, a.sc.pb) + scatter_bits(d.row0 + row, a.sc.nm, a.sc.pm);
        int64_t om_u[4];
#pragma unroll
        for (int u = 0; u < 4; u++) om_u[u] = __shfl_sync(0xffffffffu, om, 8 * u + (lane >> 2));
        uint8_t *buf = staging + e * 2048;
#pragma unroll
        for (int c = 0; c < EC; c += 16) {
          if (n0 + c / 2 < a.N) {  // N is a multiple of 8 here
            __syncwarp();  // the previous chunk's rows have been read
#pragma unroll
            for (int j = 0; j < 4; j++)
              *reinterpret_cast<float4 *>(buf + lane * 64 + ((j ^ ((lane >> 1) & 3)) << 4)) =
                  make_float4(acc[c + 4 * j], acc[c + 4 * j + 1], acc[c + 4 * j + 2], acc[c + 4 * j + 3]);
            __syncwarp();
            const int64_t col = coloff[c / 2 + 2 * (lane & 3)];
#pragma unroll
            for (int u = 0; u < 4; u++) {
              const int rr = 8 * u + (lane >> 2);
              const uint4 v =
                  *reinterpret_cast<const uint4 *>(buf + rr * 64 + (((lane & 3) ^ ((rr >> 1) & 3)) << 4));
              if (a.l2_mode & 2)
                __stcs(reinterpret_cast<uint4 *>(a.C + om_u[u] + col), v);
              else
                *reinterpret_cast<uint4 *>(a.C + om_u[u] + col) = v;
            }
          }
        }
      } else if (a.scatter) {
        const int64_t om = scatter_bits(d.z, a.sc.nb, a.sc.pb) + scatter_bits(d.row0 + row, a.sc.nm, a.sc.pm);
#pragma unroll
        for (int j = 0; j < EC / 2; j++)
          if (n0 + j < a.N) {
            if (a.l2_mode & 2)
              __stcs(a.C + om + coloff[j], make_float2(acc[2 * j], acc[2 * j + 1]));
            else
              a.C[om + coloff[j]] = make_float2(acc[2 * j], acc[2 * j + 1]);
          }
      } else if (a.tma_store) {
        // 16 columns (8 complex) at a time: this warp's 32 rows go to its
        // staging buffer in the 64-byte swizzled layout (16-byte chunk c of
        // row r at chunk c ^ ((r >> 1) & 3)), then one bulk tensor store.
        uint8_t *buf = staging + e * 2048;
        const int y = (int)(d.z * a.M + d.row0 + q * 32);
#pragma unroll
        for (int c = 0; c < EC; c += 16) {
          if (n0 + c / 2 < a.N) {
            // the previous store has read the buffer
            if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 4; j++) {
              const int pc = j ^ ((lane >> 1) & 3);
              *reinterpret_cast<float4 *>(buf + lane * 64 + pc * 16) =
                  make_float4(acc[c + 4 * j], acc[c + 4 * j + 1], acc[c + 4 * j + 2], acc[c + 4 * j + 3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
              if (a.l2_mode & 2)
                asm volatile(
                    "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group.L2::cache_hint [%0, {%1, %2}], [%3], %4;" ::"l"(
                        (uint64_t)&tmC),
                    "r"((int)(2 * n0 + c)), "r"(y), "r"(smem_u32(buf)), "l"(l2_evict_first())
                    : "memory");
              else
                asm volatile(
                    "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"((uint64_t)&tmC),
                    "r"((int)(2 * n0 + c)), "r"(y), "r"(smem_u32(buf))
                    : "memory");
              asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            }
          }
        }
      } else {
        float2 *crow = a.C + d.ks * a.split_stride + d.z * a.sC + (d.row0 + row) * a.N;
#pragma unroll
        for (int c = 0; c < EC; c += 16) {
          const int64_t nb = n0 + c / 2;
          if (nb + 8 <= a.N) {
            float4 *dst = reinterpret_cast<float4 *>(crow + nb);
#pragma unroll
            for (int j = 0; j < 4; j++) {
              const float4 v = make_float4(acc[c + 4 * j], acc[c + 4 * j + 1], acc[c + 4 * j + 2], acc[c + 4 * j + 3]);
              if (a.l2_mode & 2)
                __stcs(dst + j, v);
              else
                dst[j] = v;
            }
          } else {
#pragma unroll
            for (int j = 0; j < 8; j++)
              if (nb + j < a.N) crow[nb + j] = make_float2(acc[c + 2 * j], acc[c + 2 * j + 1]);
          }
        }
      }
    }
  }
  if (warp >= 6 && lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag && a.err) atomicExch(a.err, 1);
  // a pair: neither CTA leaves (or frees tensor memory) while the other may
  // still arrive on its barriers
  if constexpr (CG == 2) cluster_sync_all();
  if (warp == 1) {
    tc_fence_after();
    if constexpr (CG == 2)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)L::TMEM_COLS));
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)L::TMEM_COLS));
  }
}

// FP16 mode: per-block maxima of |x| over B (n2 float2 values), as FP32 bit
// patterns (ordered like the magnitudes); a fixed grid, so the consumers
// reduce a known number of partials. (A needs no such pass: its exponents
// are chosen per row and k-block on chip.)
__global__ void __launch_bounds__(512) absmax_kernel(const float2 *__restrict__ B, int64_t n2,
                                                     uint32_t *__restrict__ out) {
  uint32_t m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = B[i];
    m = max(m, max(__float_as_uint(v.x) & 0x7fffffffu, __float_as_uint(v.y) & 0x7fffffffu));
  }
  __shared__ uint32_t wm[16];
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t v = threadIdx.x < blockDim.x / 32 ? wm[threadIdx.x] : 0u;
    v = __reduce_max_sync(0xffffffffu, v);
    if (threadIdx.x == 0) out[blockIdx.x] = v;
  }
}

// B (batch x n x k complex) -> prepared real rows, hi and lo parts:
// row 2j = (Re b, -Im b) per k, row 2j+1 = (Im b, Re b); rows >= 2n are zero.
// FP16 mode: scaled by 2^sb first, sb from the pb partial maxima of B.
template <int MODE>
__global__ void prep_b_kernel(const float2 *__restrict__ B, void *__restrict__ Bh_, void *__restrict__ Bl_,
                              int64_t batch, int64_t N, int64_t K, int64_t sB, int NT, const uint32_t *bmax, int pb) {
  float sb = 1.f;
  if (MODE == MODE_F16) {
    __shared__ int s_exp;
    if (threadIdx.x < 32) {
      uint32_t m = 0;
      for (int j = threadIdx.x; j < pb; j += 32) m = max(m, bmax[j]);
      m = __reduce_max_sync(0xffffffffu, m);
      if (threadIdx.x == 0) s_exp = f16_scale_exp(m);
    }
    __syncthreads();
    sb = pow2i(s_exp);
  }
  const int64_t total = batch * NT * K;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i % K;
    const int64_t r = (i / K) % NT;
    const int64_t z = i / (K * NT);
    const int64_t j = r >> 1;
    float x0 = 0.f, x1 = 0.f;
    if (j < N) {
      const float2 b = B[z * sB + j * K + k];
      if (r & 1) {
        x0 = b.y;
        x1 = b.x;
      } else {
        x0 = b.x;
        x1 = -b.y;
      }
    }
    const int64_t o = (z * NT + r) * 2 * K + 2 * k;
    if (MODE == MODE_TF32) {
      uint32_t *Bh = static_cast<uint32_t *>(Bh_), *Bl = static_cast<uint32_t *>(Bl_);
      const uint32_t u0 = __float_as_uint(x0), u1 = __float_as_uint(x1);
      Bh[o] = split_hi(u0);
      Bh[o + 1] = split_hi(u1);
      Bl[o] = split_lo(u0);
      Bl[o + 1] = split_lo(u1);
    } else if (MODE == MODE_BF16) {
      uint16_t *Bh = static_cast<uint16_t *>(Bh_), *Bl = static_cast<uint16_t *>(Bl_);
      split_bf16(x0, Bh[o], Bl[o]);
      split_bf16(x1, Bh[o + 1], Bl[o + 1]);
    } else {
      uint16_t *Bh = static_cast<uint16_t *>(Bh_), *Bl = static_cast<uint16_t *>(Bl_);
      split_f16(x0 * sb, Bh[o], Bl[o]);
      split_f16(x1 * sb, Bh[o + 1], Bl[o + 1]);
    }
  }
}

// The same preparation, vectorised (B 16-byte aligned, K even): a thread
// takes one column j of B and two consecutive k, reads them with one 16-byte
// load and writes both prepared rows, 2j and 2j + 1, with 8-byte (BF16, FP16)
// or 16-byte (TF32) stores of hi and of lo.
template <int MODE>
__global__ void prep_b_vec_kernel(const float4 *__restrict__ B, void *__restrict__ Bh_, void *__restrict__ Bl_,
                                  int64_t batch, int64_t N, int64_t K, int64_t sB, int NT, const uint32_t *bmax,
                                  int pb) {
  float sb = 1.f;
  if (MODE == MODE_F16) {
    __shared__ int s_exp;
    if (threadIdx.x < 32) {
      uint32_t m = 0;
      for (int j = threadIdx.x; j < pb; j += 32) m = max(m, bmax[j]);
      m = __reduce_max_sync(0xffffffffu, m);
      if (threadIdx.x == 0) s_exp = f16_scale_exp(m);
    }
    __syncthreads();
    sb = pow2i(s_exp);
  }
  const int64_t K2 = K / 2, J = NT / 2;
  const int64_t total = batch * J * K2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t kp = i % K2;
    const int64_t j = (i / K2) % J;
    const int64_t z = i / (K2 * J);
    float4 b = make_float4(0.f, 0.f, 0.f, 0.f);  // (Re, Im) at k = 2 kp and 2 kp + 1
    if (j < N) b = B[(z * sB + j * K) / 2 + kp];
    const float r0[4] = {b.x, -b.y, b.z, -b.w};  // row 2j
    const float r1[4] = {b.y, b.x, b.w, b.z};    // row 2j + 1
    const int64_t o0 = (z * NT + 2 * j) * 2 * K + 4 * kp, o1 = o0 + 2 * K;
    if (MODE == MODE_TF32) {
      uint32_t *Bh = static_cast<uint32_t *>(Bh_), *Bl = static_cast<uint32_t *>(Bl_);
      uint32_t h0[4], l0[4], h1[4], l1[4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        h0[q] = split_hi(__float_as_uint(r0[q]));
        l0[q] = split_lo(__float_as_uint(r0[q]));
        h1[q] = split_hi(__float_as_uint(r1[q]));
        l1[q] = split_lo(__float_as_uint(r1[q]));
      }
      *reinterpret_cast<uint4 *>(Bh + o0) = make_uint4(h0[0], h0[1], h0[2], h0[3]);
      *reinterpret_cast<uint4 *>(Bl + o0) = make_uint4(l0[0], l0[1], l0[2], l0[3]);
      *reinterpret_cast<uint4 *>(Bh + o1) = make_uint4(h1[0], h1[1], h1[2], h1[3]);
      *reinterpret_cast<uint4 *>(Bl + o1) = make_uint4(l1[0], l1[1], l1[2], l1[3]);
    } else {
      uint16_t *Bh = static_cast<uint16_t *>(Bh_), *Bl = static_cast<uint16_t *>(Bl_);
      uint16_t h[8], l[8];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        if (MODE == MODE_BF16) {
          split_bf16(r0[q], h[q], l[q]);
          split_bf16(r1[q], h[4 + q], l[4 + q]);
        } else {
          split_f16(r0[q] * sb, h[q], l[q]);
          split_f16(r1[q] * sb, h[4 + q], l[4 + q]);
        }
      }
      auto pack = [](const uint16_t *v) {
        return make_uint2((uint32_t)v[0] | ((uint32_t)v[1] << 16), (uint32_t)v[2] | ((uint32_t)v[3] << 16));
      };
      *reinterpret_cast<uint2 *>(Bh + o0) = pack(h);
      *reinterpret_cast<uint2 *>(Bl + o0) = pack(l);
      *reinterpret_cast<uint2 *>(Bh + o1) = pack(h + 4);
      *reinterpret_cast<uint2 *>(Bl + o1) = pack(l + 4);
    }
  }
}

// Sum of the ksplit row-major partials of a split-K product, in a fixed order
// (so results do not depend on scheduling), written to row-major C whose
// batches are sC apart.
__global__ void split_reduce_kernel(const float2 *__restrict__ P, float2 *__restrict__ C, int ksplit,
                                    int64_t split_stride, int64_t MN, int64_t sC) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < split_stride;
       e += (int64_t)gridDim.x * blockDim.x) {
    float2 v = P[e];
    for (int s = 1; s < ksplit; s++) {
      const float2 w = P[s * split_stride + e];
      v.x += w.x;
      v.y += w.y;
    }
    C[(e / MN) * sC + e % MN] = v;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 2D tensor map: rows x cols (cols contiguous), box = box_cols x box_rows,
// zero fill outside; box rows of 128 bytes (128-byte swizzle) or 64 bytes
// (64-byte swizzle).
bool make_map(CUtensorMap *tm, const void *base, int64_t cols, int64_t rows, int box_cols, int box_rows,
              CUtensorMapDataType dt) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int esz = dt == CU_TENSOR_MAP_DATA_TYPE_FLOAT32 ? 4 : 2;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(cols * esz)};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(tm, dt, 2,
                  const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  box_cols * esz == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

constexpr int kMaxDevices = 64;

// Pairs of CTAs for the products that allow them: the process-wide default
// (tc_set_pairs; initially off unless the environment variable TZ_TC_PAIRS is
// 1: on the measured shapes pairs are no faster yet), which a launch's own
// choice (autotuned) overrides.
std::atomic<int> g_pairs{-1};
bool tc_pairs_default() {
  int v = g_pairs.load(std::memory_order_relaxed);
  if (v < 0) {
    const char *e = std::getenv("TZ_TC_PAIRS");
    v = (e && e[0] == '1') ? 1 : 0;
  }
  return v != 0;
}

int tile_cols(int64_t N) {  // real columns per tile (power of two, 16..128)
  int64_t c = 2 * N;
  if (c < 16) c = 16;
  if (c > 128) c = 128;
  int64_t p = 16;
  while (p < c) p <<= 1;
  return (int)p;
}

// Launches the persistent kernel on at most one CTA per tile (CG = 2: one
// pair per tile), as many as are resident at once (one CTA per SM).
template <int MODE, int BNP, int STAGES, int CG>
cudaError_t run_tc(const CUtensorMap &ta, const CUtensorMap &tbh, const CUtensorMap &tbl, const CUtensorMap &tc,
                   const TcArgs &args, int64_t n_tiles, cudaStream_t s) {
  using L = TcSmem<MODE, BNP, STAGES, CG>;
  static_assert(L::TOTAL <= 227 * 1024, "shared memory budget");
  // one CTA per SM: each allocates all of TMEM
  static_assert(L::TOTAL > 114 * 1024, "two CTAs would share an SM");
  auto kernel = tc_split3_kernel<MODE, BNP, STAGES, CG>;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = L::TOTAL;
  cfg.stream = s;
  if (CG == 2) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  // the shared-memory attribute is set, and the number of resident CTAs (or
  // pairs) read, once per device (server threads may launch concurrently)
  static std::mutex mu;
  static int resident[kMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  int walkers = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!resident[dev]) {
      e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::TOTAL);
      if (e != cudaSuccess) return e;
      int n = 0;
      if (CG == 2) {
        cfg.gridDim = dim3(2);
        if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) != cudaSuccess || n <= 0) n = 0;
      } else if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
        n = 148;
      }
      if (n <= 0) return cudaErrorLaunchOutOfResources;
      resident[dev] = n;
    }
    walkers = resident[dev];
  }
  cfg.gridDim = dim3((unsigned)(CG * std::min<int64_t>(n_tiles, walkers)));
  e = cudaLaunchKernelEx(&cfg, kernel, ta, tbh, tbl, tc, args);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int MODE>
cudaError_t dispatch(int bnp, int cg, const CUtensorMap &ta, const CUtensorMap &tbh, const CUtensorMap &tbl,
                     const CUtensorMap &tc, const TcArgs &args, int64_t n_tiles, cudaStream_t s) {
  // stages: at most what fits beside the epilogue staging (and at most 8);
  // for the 128-column tiles, the counts measured fastest
  constexpr bool T = MODE == MODE_TF32;
  if constexpr (!T) {
    if (cg == 2) return run_tc<MODE, 128, 4, 2>(ta, tbh, tbl, tc, args, n_tiles, s);
  }
  switch (bnp) {
    case 16: return run_tc<MODE, 16, T ? 8 : 5, 1>(ta, tbh, tbl, tc, args, n_tiles, s);
    case 32: return run_tc<MODE, 32, T ? 7 : 5, 1>(ta, tbh, tbl, tc, args, n_tiles, s);
    case 64: return run_tc<MODE, 64, T ? 5 : 4, 1>(ta, tbh, tbl, tc, args, n_tiles, s);
    default: return run_tc<MODE, 128, T ? 4 : 3, 1>(ta, tbh, tbl, tc, args, n_tiles, s);
  }
}

}  // namespace

static bool is_tc(int precision) {
  return precision == TZ_TF32X3 || precision == TZ_BF16X3 || precision == TZ_FP16X3;
}

bool cgemm_tc_supported(int precision, int64_t M, int64_t N, int64_t K) {
  if (!is_tc(precision)) return false;
  // M: whole 128-row tiles; K: rows of the operands a multiple of 16 bytes
  // for TMA (2 complex in FP32, 4 complex in BF16 or FP16)
  const int64_t kmin = precision == TZ_TF32X3 ? 2 : 4;
  if (M < BM || (M % BM) != 0 || K < kmin || (K % kmin) != 0 || N < 1) return false;
  return true;
}

// K ranges per product: products with fewer tiles than half the 152 SMs of
// GB300 and a long K split K so that the ranges fill the SMs, each range at
// least 32 k-blocks and the partials at most 64 MiB. A function of the shape
// alone, so scratch sized by a plan covers every launch (a launch writing C
// through a scatter map does not split).
static int split_k(int precision, int64_t batch, int64_t M, int64_t N, int64_t K) {
  const int bnp = tile_cols(N);
  const int64_t tiles = batch * (M / BM) * ((2 * N + bnp - 1) / bnp);
  const int sk = precision == TZ_TF32X3 ? stage_k<MODE_TF32>() : stage_k<MODE_BF16>();
  const int64_t kblocks = (2 * K + sk - 1) / sk;
  int64_t s = std::min<int64_t>({16, 152 / std::max<int64_t>(tiles, 1), kblocks / 32});
  while (s > 1 && s * batch * M * N * 8 > (int64_t(64) << 20)) s--;
  return s < 2 ? 1 : (int)s;
}

int cgemm_tc_launches(int precision, int64_t batch, int64_t M, int64_t N, int64_t K, bool scatter, int ksplit) {
  return 2 + (precision == TZ_FP16X3 ? 1 : 0) +
         (!scatter && ksplit != 1 && split_k(precision, batch, M, N, K) > 1 ? 1 : 0);
}

int cgemm_tc_split(int precision, int64_t batch, int64_t M, int64_t N, int64_t K) {
  return split_k(precision, batch, M, N, K);
}

// Scratch: prepared B hi | prepared B lo | split-K partials (when split) |
// FP16 mode: the partial maxima of |B| (kMaxPartials words).
size_t cgemm_tc_scratch_bytes(int precision, int64_t batch, int64_t M, int64_t N, int64_t K) {
  if (!is_tc(precision)) return 0;
  const int bnp = tile_cols(N);
  const int64_t nt = (2 * N + bnp - 1) / bnp;
  const int esz = precision == TZ_TF32X3 ? 4 : 2;
  const size_t half = ((size_t)(batch * nt * bnp * 2 * K * esz) + 255) & ~size_t(255);
  const int ks = split_k(precision, batch, M, N, K);
  const size_t part = ks > 1 ? (size_t)(ks * batch * M * N * 8) : 0;
  const size_t bmax = precision == TZ_FP16X3 ? kMaxPartials * sizeof(uint32_t) : 0;
  return 2 * half + ((part + 255) & ~size_t(255)) + bmax + 256;
}

bool tc_pair_supported(int precision, int64_t M, int64_t N) {
  return (precision == TZ_BF16X3 || precision == TZ_FP16X3) && tile_cols(N) == 128 && (M % (2 * BM)) == 0;
}

void tc_set_pairs(int mode) { g_pairs.store(mode < 0 ? -1 : (mode ? 1 : 0), std::memory_order_relaxed); }

// L2 prefetch distance of the A tiles in k-blocks: the process default
// (tc_set_prefetch; initially the environment variable TZ_TC_PREFETCH, else
// 0: measured no faster on the bench tree's products).
std::atomic<int> g_prefetch{-1};
int tc_prefetch_default() {
  int v = g_prefetch.load(std::memory_order_relaxed);
  if (v < 0) {
    const char *e = std::getenv("TZ_TC_PREFETCH");
    v = e ? std::max(0, std::min(64, std::atoi(e))) : 0;
  }
  return v;
}
// L2 priorities of the product (TcArgs::l2_mode): the environment variable
// TZ_TC_L2, else 3. A loaded with the normal priority and C written as
// streaming data: C's write-back lines are then evicted before the A tiles
// that the other column tiles of the same rows still have to read. On the
// Bristlecone-70 bench tree's products (scaled split FP16, pairs of CTAs)
// this took DRAM traffic from 1.34x to 1.02x the algorithmic bytes and the
// step 1.5 % faster; with A evict-first, pairs that drifted apart re-read A.
int tc_l2_mode_default() {
  static const int v = [] {
    const char *e = std::getenv("TZ_TC_L2");
    return e ? (std::atoi(e) & 3) : 3;
  }();
  return v;
}
void tc_set_prefetch(int kblocks) { g_prefetch.store(kblocks < 0 ? -1 : std::min(64, kblocks), std::memory_order_relaxed); }

cudaError_t launch_cgemm_tc(int precision, const float2 *A, const float2 *B, float2 *C, int64_t batch, int64_t M,
                            int64_t N, int64_t K, int64_t sA, int64_t sB, int64_t sC, const CScatter *sc,
                            void *scratch, size_t scratch_bytes, int *err, cudaStream_t s, int pair,
                            int ksplit) {
  if (!cgemm_tc_supported(precision, M, N, K)) return cudaErrorNotSupported;
  if (sA != M * K || sB != N * K) return cudaErrorNotSupported;  // contiguous batches only
  const int bnp = tile_cols(N);
  const int n_tiles_n = (int)((2 * N + bnp - 1) / bnp);
  const int NT = n_tiles_n * bnp;
  const int64_t rowsA = batch * M, rowsB = batch * (int64_t)NT;
  if (rowsA >= (int64_t(1) << 31) || rowsB >= (int64_t(1) << 31) || 2 * K >= (int64_t(1) << 31))
    return cudaErrorNotSupported;
  if (scratch_bytes < cgemm_tc_scratch_bytes(precision, batch, M, N, K) || !scratch) return cudaErrorInvalidValue;
  const bool tf32 = precision == TZ_TF32X3, f16 = precision == TZ_FP16X3;
  const size_t half = (size_t)(batch * NT * 2 * K) * (tf32 ? 4 : 2);
  char *Bh = static_cast<char *>(scratch);
  char *Bl = Bh + ((half + 255) & ~size_t(255));
  // after the prepared B: room for split-K partials (sized by the shape, as
  // in cgemm_tc_scratch_bytes), then the FP16 partial maxima
  const int ks_shape = split_k(precision, batch, M, N, K);
  const int ks = (sc || ksplit == 1) ? 1 : ks_shape;
  char *after_b = Bl + ((half + 255) & ~size_t(255));
  float2 *P = ks > 1 ? reinterpret_cast<float2 *>(after_b) : nullptr;
  const size_t part_all = ks_shape > 1 ? (size_t)(ks_shape * batch * M * N * 8) : 0;
  uint32_t *bmax = reinterpret_cast<uint32_t *>(after_b + ((part_all + 255) & ~size_t(255)));
  // pairs of CTAs (cta_group::2) take the split BF16 / FP16 products with
  // 128-column tiles and whole 256-row tiles: each CTA loads half of B
  const bool want_pair = pair < 0 ? tc_pairs_default() : pair != 0;
  const int cg = want_pair && tc_pair_supported(precision, M, N) ? 2 : 1;
  CUtensorMap ta, tbh, tbl;
  const int sk = tf32 ? stage_k<MODE_TF32>() : stage_k<MODE_BF16>();
  const CUtensorMapDataType bdt =
      tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : (f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
  if (!make_map(&ta, A, 2 * K, rowsA, 32, BM, CU_TENSOR_MAP_DATA_TYPE_FLOAT32) ||
      !make_map(&tbh, Bh, 2 * K, rowsB, sk, bnp / cg, bdt) || !make_map(&tbl, Bl, 2 * K, rowsB, sk, bnp / cg, bdt))
    return cudaErrorInvalidValue;
  int pb = 0;
  if (f16) {
    const int64_t nB2 = batch * N * K;
    pb = (int)std::min<int64_t>(kMaxPartials, std::max<int64_t>(1, nB2 / (512 * 8)));
    absmax_kernel<<<pb, 512, 0, s>>>(B, nB2, bmax);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if ((reinterpret_cast<uintptr_t>(B) & 15) == 0 && (K % 2) == 0) {
    // NT is even (whole tiles of at least 16 rows)
    const int64_t total = batch * (NT / 2) * (K / 2);
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 32);
    const float4 *B4 = reinterpret_cast<const float4 *>(B);
    if (tf32)
      prep_b_vec_kernel<MODE_TF32><<<blocks, 256, 0, s>>>(B4, Bh, Bl, batch, N, K, sB, NT, nullptr, 0);
    else if (f16)
      prep_b_vec_kernel<MODE_F16><<<blocks, 256, 0, s>>>(B4, Bh, Bl, batch, N, K, sB, NT, bmax, pb);
    else
      prep_b_vec_kernel<MODE_BF16><<<blocks, 256, 0, s>>>(B4, Bh, Bl, batch, N, K, sB, NT, nullptr, 0);
  } else {
    const int64_t total = batch * NT * K;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 32);
    if (tf32)
      prep_b_kernel<MODE_TF32><<<blocks, 256, 0, s>>>(B, Bh, Bl, batch, N, K, sB, NT, nullptr, 0);
    else if (f16)
      prep_b_kernel<MODE_F16><<<blocks, 256, 0, s>>>(B, Bh, Bl, batch, N, K, sB, NT, bmax, pb);
    else
      prep_b_kernel<MODE_BF16><<<blocks, 256, 0, s>>>(B, Bh, Bl, batch, N, K, sB, NT, nullptr, 0);
  }
  {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  TcArgs args{};
  args.err = err;
  args.prefetch = tc_prefetch_default();
  args.l2_mode = tc_l2_mode_default();
  args.bmax = bmax;
  args.pb = pb;
  args.C = C;
  args.batch = batch;
  args.M = M;
  args.N = N;
  args.K = K;
  args.sC = sC;
  args.n_tiles_m = (int)(M / (BM * cg));
  args.n_tiles_n = n_tiles_n;
  args.kblocks = (int)((2 * K + sk - 1) / sk);
  args.ksplit = ks;
  args.kb_per = (args.kblocks + ks - 1) / ks;
  args.split_stride = batch * M * N;
  args.NT = NT;
  args.scatter = sc ? 1 : 0;
  if (sc) {
    args.sc = *sc;
    // n bit 0 lowest in C (N a multiple of 8), C 16-byte aligned: stores of
    // 16-byte column pairs, instead of single columns at 32 different rows
    if (sc->nn >= 3 && sc->pn[0] == 0 && (reinterpret_cast<uintptr_t>(C) & 15) == 0) args.scatter = 2;
  }
  const int64_t n_tiles = batch * args.n_tiles_m * (int64_t)n_tiles_n * ks;
  // row-major C with 16-byte aligned rows: bulk tensor stores of 32-row x
  // 16-float boxes (64-byte swizzle), clipped at the tensor edge
  CUtensorMap tcm;
  std::memset(&tcm, 0, sizeof(tcm));
  if (ks > 1) {
    // partials row-major in scratch; the reduce kernel writes C
    args.C = P;
    args.sC = M * N;
    args.scatter = 0;
  } else if (!sc && sC == M * N && (N % 2) == 0 && (reinterpret_cast<uintptr_t>(C) & 15) == 0) {
    auto fn = encode_fn();
    cuuint64_t dims[2] = {(cuuint64_t)(2 * N), (cuuint64_t)(batch * M)};
    cuuint64_t strides[1] = {(cuuint64_t)(2 * N * 4)};
    cuuint32_t box[2] = {16, 32};
    cuuint32_t estr[2] = {1, 1};
    if (fn && fn(&tcm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, C, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                 CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
      args.tma_store = 1;
  }
  cudaError_t e = tf32  ? dispatch<MODE_TF32>(bnp, cg, ta, tbh, tbl, tcm, args, n_tiles, s)
                  : f16 ? dispatch<MODE_F16>(bnp, cg, ta, tbh, tbl, tcm, args, n_tiles, s)
                        : dispatch<MODE_BF16>(bnp, cg, ta, tbh, tbl, tcm, args, n_tiles, s);
  if (e != cudaSuccess || ks == 1) return e;
  const int64_t total = batch * M * N;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 8);
  split_reduce_kernel<<<blocks, 256, 0, s>>>(P, C, ks, total, M * N, sC);
  return cudaGetLastError();
}

cudaError_t tc_set_wait_limit(unsigned long long ns) {
  const unsigned long long v = ns ? ns : kWaitNs;
  return cudaMemcpyToSymbol(g_wait_ns, &v, sizeof(v));
}

cudaError_t tc_set_stall(int on) {
  const int v = on ? 1 : 0;
  return cudaMemcpyToSymbol(g_stall, &v, sizeof(v));
}

}  // namespace dev
}  // namespace tz
