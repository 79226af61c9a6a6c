// Per-group kernels: leaf builder, direct small-step contraction, FP64
// accumulation of partial amplitudes.
#include <algorithm>
#include <mutex>

#include "kernels.h"

namespace tz {
namespace dev {

// complex arithmetic on float2 (complex64) and double2 (complex128)
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
  c.x = fmaf(a.x, b.x, c.x);
  c.x = fmaf(-a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y);
  c.y = fmaf(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
  return c;
}
template <typename T>
__device__ __forceinline__ T czero();
template <>
__device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }
template <>
__device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
__device__ __forceinline__ float2 table_value(const LeafJob &j, int i, float2 *) { return j.M[i]; }
__device__ __forceinline__ double2 table_value(const LeafJob &j, int i, double2 *) { return j.Md[i]; }

__global__ void init_state_kernel(GroupState *gs, int64_t lo, int64_t hi, int64_t n_rows, int keep_error) {
  gs->slice = lo;
  gs->chunk = 0;
  gs->lo = lo;
  gs->hi = hi;
  gs->n_rows = n_rows;
  gs->groups_done = 0;
  if (!keep_error) gs->tc_error = 0;
}

cudaError_t launch_init_state(GroupState *gs, int64_t lo, int64_t hi, int64_t n_rows, cudaStream_t s,
                              int keep_error) {
  init_state_kernel<<<1, 1, 0, s>>>(gs, lo, hi, n_rows, keep_error);
  return cudaGetLastError();
}

// One block per leaf job. Gather: a constant tensor with its sliced bits
// fixed to the bits of the current slice id (Sec. 1 subtasks). Output: the
// tensor <x_q| (final gates folded in) for the current chunk of bitstrings.
template <typename T>
__global__ void leaf_kernel(const LeafJob *jobs, const GroupState *gs, const uint8_t *bits, int nq, int g,
                            const char *cbase, char *abase) {
  const LeafJob &j = jobs[blockIdx.x];
  T *dst = const_cast<T *>(region_ptr<T>(j.dst, cbase, abase));
  const T *src = j.kind == LJ_GATHER ? region_ptr<T>(j.src, cbase, abase) : nullptr;
  const int64_t slice = gs->slice, chunk = gs->chunk, n_rows = gs->n_rows;
  const int64_t n = int64_t(1) << j.rank;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    if (j.kind == LJ_GATHER) {
      int64_t so = 0;
      for (int p = 0; p < j.rank; p++) so |= ((e >> p) & 1) << j.src_pos[p];
      for (int f = 0; f < j.n_fixed; f++) so |= ((slice >> j.fixed_slice_bit[f]) & 1) << j.fixed_src_pos[f];
      dst[e] = src[so];
    } else {
      int64_t beta = 0;
      for (int b = 0; b < g; b++)
        if (j.beta_dst_pos[b] >= 0) beta |= ((e >> j.beta_dst_pos[b]) & 1) << b;
      const int64_t row = (chunk << g) | beta;
      const int x = row < n_rows ? (bits[row * nq + j.qubit] & 1) : 0;
      int ev = 0;
      if (j.rc) {
        if (j.e_dst_pos >= 0)
          ev = (int)((e >> j.e_dst_pos) & 1);
        else if (j.e_slice_bit >= 0)
          ev = (int)((slice >> j.e_slice_bit) & 1);
      }
      dst[e] = table_value(j, x * (1 << j.rc) + ev, (T *)nullptr);
    }
  }
}

cudaError_t launch_leaf_build(const LeafJob *jobs, int n_jobs, const GroupState *gs, const uint8_t *bits, int nq,
                              int g, const char *cbase, char *abase, int dbl, cudaStream_t s) {
  if (dbl)
    leaf_kernel<double2><<<n_jobs, 128, 0, s>>>(jobs, gs, bits, nq, g, cbase, abase);
  else
    leaf_kernel<float2><<<n_jobs, 128, 0, s>>>(jobs, gs, bits, nq, g, cbase, abase);
  return cudaGetLastError();
}

// Direct contraction of small steps. Each output element is summed by
// 2^split consecutive threads, each walking its share of the contracted bits
// in Gray-code order (one offset update per term), then reduced. blk is the
// block's number within its step.
template <typename T>
__device__ __forceinline__ void direct_block(const DStep &st, int64_t blk, const char *cbase, char *abase, T *red) {
  const T *__restrict__ Ap = region_ptr<T>(st.A, cbase, abase);
  const T *__restrict__ Bp = region_ptr<T>(st.B, cbase, abase);
  T *Cp = const_cast<T *>(region_ptr<T>(st.C, cbase, abase));
  const int split = st.split;
  const int64_t item = blk * 256 + threadIdx.x;
  const int64_t c = item >> split;
  const int part = (int)(item & ((1 << split) - 1));
  const bool active = c < (int64_t(1) << st.nC);
  T acc = czero<T>();
  if (active) {
    int64_t oa = 0, ob = 0;
    for (int q = 0; q < st.nC; q++) {
      if (!((c >> q) & 1)) continue;
      if (st.a_c[q] >= 0) oa += int64_t(1) << st.a_c[q];
      if (st.b_c[q] >= 0) ob += int64_t(1) << st.b_c[q];
    }
    const int nlow = st.nK - split;
    for (int q = 0; q < split; q++)
      if ((part >> q) & 1) {
        oa += int64_t(1) << st.a_k[nlow + q];
        ob += int64_t(1) << st.b_k[nlow + q];
      }
    acc = cmul(Ap[oa], Bp[ob]);
    const int64_t nt = int64_t(1) << nlow;
    for (int64_t t = 1; t < nt; t++) {
      const int q = __ffsll(t) - 1;
      const bool on = (((t ^ (t >> 1)) >> q) & 1) != 0;
      const int64_t da = int64_t(1) << st.a_k[q], db = int64_t(1) << st.b_k[q];
      oa += on ? da : -da;
      ob += on ? db : -db;
      acc = cfma(Ap[oa], Bp[ob], acc);
    }
  }
  if (split > 0) {
    red[threadIdx.x] = acc;
    __syncthreads();
    if (active && part == 0) {
      for (int q = 1; q < (1 << split); q++) {
        T v = red[threadIdx.x + q];
        acc.x += v.x;
        acc.y += v.y;
      }
    }
  }
  if (active && part == 0) Cp[c] = acc;
}

// A block's step descriptor, staged in shared memory by 12 threads at once
// (its fields are then read by every thread without further global loads).
__device__ __forceinline__ void stage_step(DStep *dst, const DStep *src) {
  static_assert(sizeof(DStep) % 16 == 0 && sizeof(DStep) / 16 <= 32, "DStep staged in 16-byte pieces");
  if (threadIdx.x < sizeof(DStep) / 16)
    reinterpret_cast<uint4 *>(dst)[threadIdx.x] = reinterpret_cast<const uint4 *>(src)[threadIdx.x];
}

// One launch per dependency level: block b of the launch belongs to step
// bmap[b].
template <typename T>
__global__ void __launch_bounds__(256) direct_kernel(const DStep *steps, const int *bmap, const char *cbase,
                                                     char *abase) {
  __shared__ __align__(16) DStep s_st;
  __shared__ T red[256];
  const int64_t blk = blockIdx.x;
  stage_step(&s_st, steps + bmap[blk]);
  __syncthreads();
  direct_block<T>(s_st, blk - s_st.block_begin, cbase, abase, red);
}

cudaError_t launch_direct(const DStep *steps, int n_steps, const int *bmap, int64_t total_blocks, const char *cbase,
                          char *abase, int dbl, cudaStream_t s) {
  if (n_steps <= 0) return cudaSuccess;
  if (total_blocks > 0x7fffffffLL || !bmap) return cudaErrorInvalidValue;
  if (dbl)
    direct_kernel<double2><<<(unsigned)total_blocks, 256, 0, s>>>(steps, bmap, cbase, abase);
  else
    direct_kernel<float2><<<(unsigned)total_blocks, 256, 0, s>>>(steps, bmap, cbase, abase);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- queue
// The persistent form. ctrl[0] hands out tickets (the launch's blocks in
// order), ctrl[1] counts blocks that have left, ctrl[2] is the stop flag,
// ctrl[3] is a counter nothing increments (the test stall waits on it), and
// ctrl[4 + j] counts the finished blocks of step j.
//
// Progress: a step's blocks come after the blocks of the steps it reads
// (DStep::dep < own index, tickets in block order). A block holding a
// ticket is resident, so the lowest unfinished ticket always has all of its
// inputs done and runs to the end; no wait can close a cycle, whatever the
// grid size. Every wait is still bounded. Block b's first ticket is b itself
// (no atomic); later tickets come from ctrl[0], which starts at the grid size.
//
// Visibility: a producer block's threads write their results, meet at a
// barrier, and one thread fences and counts the block done; a consumer's
// waiting thread reads the count with acquire semantics at GPU scope before
// its block's barrier, so the block's plain loads that follow see the
// results (the acquire also keeps the SM's L1 from serving older copies).
// Results of one launch never share a 128-byte line with anything else read
// in it: the tensors of a queue launch all live through the whole launch, so
// none reuses another's memory, and every tensor starts on 256 bytes.
constexpr unsigned long long kQueueWaitNs = 2000000000ull;  // 2 s (default)
__device__ unsigned long long g_dq_wait_ns = kQueueWaitNs;
__device__ int g_dq_stall;

__device__ __forceinline__ unsigned long long dq_globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Wait until *cnt >= target: 1 when it is, 0 when the launch was stopped or
// the wait ran out (then the error word and the stop flag are set).
__device__ __forceinline__ bool dq_wait(const unsigned *cnt, unsigned target, unsigned *stop, int *err,
                                        unsigned long long limit) {
  if (ld_acquire(cnt) >= target) return true;
  const unsigned long long t0 = dq_globaltimer();
  for (unsigned polls = 1;; polls++) {
    if (ld_acquire(cnt) >= target) return true;
    if ((polls & 15) == 0) {
      if (ld_acquire(stop)) return false;
      if (dq_globaltimer() - t0 > limit) {
        atomicExch(err, 1);
        atomicExch(stop, 1u);
        return false;
      }
      if (polls >= 256) __nanosleep(32);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) direct_queue_kernel(const DStep *steps, int n_steps, const int *bmap,
                                                           int64_t total, const char *cbase, char *abase,
                                                           unsigned *ctrl, int *err) {
  __shared__ int s_idx, s_go, s_last;
  __shared__ int64_t s_blk;
  __shared__ __align__(16) DStep s_st;
  __shared__ T red[256];
  unsigned *done = ctrl + 4;
  const unsigned long long limit = g_dq_wait_ns;
  // thread 0 takes the block's next ticket as soon as it has passed the
  // waits of the current one, so the atomic's latency hides behind the
  // block's work (a block holds at most one ticket it has not started, and
  // every ticket below it is finished or running: progress is unchanged)
  int64_t t_next = blockIdx.x;
  for (;;) {
    if (threadIdx.x == 0) {
      const int64_t t = t_next;
      int go = t < total;
      int idx = 0;
      if (go) {
        idx = bmap[t];
        if (g_dq_stall && t == 0) go = dq_wait(&ctrl[3], 1u, &ctrl[2], err, limit);
        const int4 dp = *reinterpret_cast<const int4 *>(steps[idx].dep);  // dep[2], dep_nblk[2]
        if (go && dp.x >= 0) go = dq_wait(&done[dp.x], (unsigned)dp.z, &ctrl[2], err, limit);
        if (go && dp.y >= 0) go = dq_wait(&done[dp.y], (unsigned)dp.w, &ctrl[2], err, limit);
        if (go) t_next = (int64_t)gridDim.x + atomicAdd(&ctrl[0], 1u);
      }
      s_idx = idx;
      s_blk = t;
      s_go = go;
    }
    __syncthreads();
    if (!s_go) break;
    stage_step(&s_st, steps + s_idx);
    __syncthreads();
    direct_block<T>(s_st, s_blk - s_st.block_begin, cbase, abase, red);
    __syncthreads();  // every result of this block is written
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(&done[s_idx], 1u);
    }
  }
  // the last block to leave zeroes the counters for the next launch
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&ctrl[1], 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    for (int j = threadIdx.x; j < n_steps; j += blockDim.x) done[j] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
      ctrl[0] = 0;
      ctrl[2] = 0;
      ctrl[3] = 0;
      __threadfence();
      ctrl[1] = 0;
    }
  }
}

namespace {
// resident blocks of the queue kernel per device (blocks per SM x SMs)
std::mutex g_dq_mu;
int g_dq_resident[2][64];
}  // namespace

template <typename T>
static int dq_resident(int dbl) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  std::lock_guard<std::mutex> lk(g_dq_mu);
  int &r = g_dq_resident[dbl][dev];
  if (r == 0) {
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, direct_queue_kernel<T>, 256, 0) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return 0;
    r = std::max(1, per_sm) * std::max(1, sms);
  }
  return r;
}

cudaError_t launch_direct_queue(const DStep *steps, int n_steps, const int *bmap, int64_t total_blocks,
                                const char *cbase, char *abase, unsigned *ctrl, int *err, int dbl, cudaStream_t s) {
  if (n_steps <= 0) return cudaSuccess;
  if (total_blocks > 0x7fffffffLL || !ctrl || !err || !bmap) return cudaErrorInvalidValue;
  const int resident = dbl ? dq_resident<double2>(1) : dq_resident<float2>(0);
  if (resident <= 0) return cudaErrorInvalidDevice;
  const unsigned grid = (unsigned)std::min<int64_t>(total_blocks, resident);
  if (dbl)
    direct_queue_kernel<double2><<<grid, 256, 0, s>>>(steps, n_steps, bmap, total_blocks, cbase, abase, ctrl, err);
  else
    direct_queue_kernel<float2><<<grid, 256, 0, s>>>(steps, n_steps, bmap, total_blocks, cbase, abase, ctrl, err);
  return cudaGetLastError();
}

cudaError_t direct_queue_set_wait_limit(unsigned long long ns) {
  const unsigned long long v = ns ? ns : kQueueWaitNs;
  return cudaMemcpyToSymbol(g_dq_wait_ns, &v, sizeof(v));
}

cudaError_t direct_queue_set_stall(int on) {
  const int v = on ? 1 : 0;
  return cudaMemcpyToSymbol(g_dq_stall, &v, sizeof(v));
}

// acc[row][o] += scale * root[beta, o] in FP64 for the current chunk (o the
// value of the open output qubits; m = 0 without them); then advance the
// group state (next slice, wrapping to the next chunk).
template <typename T>
__global__ void accum_kernel(AccumArgs a) {
  const T *root = static_cast<const T *>(a.root);
  GroupState *gs = a.gs;
  const int64_t chunk = gs->chunk, n_rows = gs->n_rows;
  const int total = 1 << (a.g + a.m);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int beta = e >> a.m, o = e & ((1 << a.m) - 1);
    int64_t off = 0;
    for (int j = 0; j < a.g; j++) off |= int64_t((beta >> j) & 1) << a.beta_pos[j];
    for (int j = 0; j < a.m; j++) off |= int64_t((o >> j) & 1) << a.open_pos[j];
    const int64_t row = (chunk << a.g) | beta;
    if (row < n_rows) {
      const T v = root[off];
      const double vr = v.x, vi = v.y;
      const int64_t at = (row << a.m) | o;
      double2 r = a.acc[at];
      r.x += a.scale_re * vr - a.scale_im * vi;
      r.y += a.scale_re * vi + a.scale_im * vr;
      // a product of this call timed out: its rows are poisoned, so a
      // caller that only reads the amplitudes still sees the failure
      if (gs->tc_error) r = make_double2(__longlong_as_double(0x7ff8000000000000ll),
                                         __longlong_as_double(0x7ff8000000000000ll));
      a.acc[at] = r;
    }
  }
  if (gridDim.x > 1) return;  // the state advances in a launch of its own
  __syncthreads();
  if (threadIdx.x == 0 && a.advance) {
    int64_t sl = gs->slice + 1;
    if (sl >= gs->hi) {
      sl = gs->lo;
      gs->chunk = chunk + 1;
    }
    gs->slice = sl;
    gs->groups_done++;
  }
}

__global__ void advance_kernel(GroupState *gs) {
  int64_t sl = gs->slice + 1;
  if (sl >= gs->hi) {
    sl = gs->lo;
    gs->chunk = gs->chunk + 1;
  }
  gs->slice = sl;
  gs->groups_done++;
}

// one block up to 4096 root values; beyond, one value per thread over
// several blocks, and a separate launch advances the state once they are done
constexpr int kAccumOneBlock = 12;

int accumulate_launches(int g, int m) { return g + m <= kAccumOneBlock ? 1 : 2; }

cudaError_t launch_accumulate(const AccumArgs &a, cudaStream_t s) {
  if (a.g < 0 || a.m < 0 || a.g > kMaxBatch || a.m > kMaxOpen) return cudaErrorInvalidValue;
  const int bits = a.g + a.m;
  const unsigned blocks = bits <= kAccumOneBlock ? 1u : (unsigned)(((1 << bits) + 255) / 256);
  if (a.dbl)
    accum_kernel<double2><<<blocks, 256, 0, s>>>(a);
  else
    accum_kernel<float2><<<blocks, 256, 0, s>>>(a);
  if (blocks > 1 && a.advance) advance_kernel<<<1, 1, 0, s>>>(a.gs);
  return cudaGetLastError();
}

__global__ void accum_plain_kernel(const float2 *part, double2 *acc, int64_t n, double sre, double sim) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const double vr = part[j].x, vi = part[j].y;
    double2 r = acc[j];
    r.x += sre * vr - sim * vi;
    r.y += sre * vi + sim * vr;
    acc[j] = r;
  }
}

cudaError_t launch_accumulate_plain(const float2 *part, double2 *acc, int64_t n, double sre, double sim,
                                    cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 65536) blocks = 65536;
  accum_plain_kernel<<<(unsigned)blocks, 256, 0, s>>>(part, acc, n, sre, sim);
  return cudaGetLastError();
}

}  // namespace dev
}  // namespace tz
