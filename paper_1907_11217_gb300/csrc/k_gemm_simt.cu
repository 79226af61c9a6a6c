// Batched complex64 product on CUDA cores (FP32 FMA, four real products per
// complex multiply-add): C[z] = A[z] B[z]^T with A[z] m x k, B[z] n x k and
// C[z] m x n, all row-major. This is the plain complex64 precision mode and
// the baseline of the split-precision tensor-core modes.
#include <algorithm>
#include <utility>
#include <vector>

#include "kernels.h"

namespace tz {
namespace dev {

namespace {

// multiply-add and zero on complex64 / complex128
__device__ __forceinline__ void cmac(float2 &acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cmac(double2 &acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
template <typename T>
__device__ __forceinline__ T zero_c() {
  T z;
  z.x = 0;
  z.y = 0;
  return z;
}

__device__ __forceinline__ int64_t scatter_bits(int64_t v, int n, const int8_t *pos) {
  int64_t o = 0;
  for (int j = 0; j < n; j++) o |= ((v >> j) & 1) << pos[j];
  return o;
}

template <typename T, int BM, int BN, int TM, int TN, int BK>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    cgemm_simt_kernel(const T *__restrict__ A, const T *__restrict__ B, T *__restrict__ C,
                      int64_t batch, int64_t M, int64_t N, int64_t K, int64_t sA, int64_t sB, int64_t sC,
                      const __grid_constant__ CScatter sc, int scatter) {
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int TX = BN / TN;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int64_t mt = (M + BM - 1) / BM, nt = (N + BN - 1) / BN;
  const int64_t tiles = mt * nt * batch;
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t z = tile / (mt * nt);
    const int64_t rem = tile - z * mt * nt;
    const int64_t m0 = (rem / nt) * BM, n0 = (rem % nt) * BN;
    const T *Az = A + z * sA;
    const T *Bz = B + z * sB;
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; i++)
#pragma unroll
      for (int j = 0; j < TN; j++) acc[i][j] = zero_c<T>();
    for (int64_t k0 = 0; k0 < K; k0 += BK) {
      for (int l = threadIdx.x; l < BM * BK; l += NT) {
        const int i = l / BK, kk = l % BK;
        const int64_t m = m0 + i, k = k0 + kk;
        As[kk][i] = (m < M && k < K) ? Az[m * K + k] : zero_c<T>();
      }
      for (int l = threadIdx.x; l < BN * BK; l += NT) {
        const int i = l / BK, kk = l % BK;
        const int64_t n = n0 + i, k = k0 + kk;
        Bs[kk][i] = (n < N && k < K) ? Bz[n * K + k] : zero_c<T>();
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; kk++) {
        T a[TM], b[TN];
#pragma unroll
        for (int i = 0; i < TM; i++) a[i] = As[kk][ty + i * (BM / TM)];
#pragma unroll
        for (int j = 0; j < TN; j++) b[j] = Bs[kk][tx + j * TX];
#pragma unroll
        for (int i = 0; i < TM; i++)
#pragma unroll
          for (int j = 0; j < TN; j++) cmac(acc[i][j], a[i], b[j]);
      }
      __syncthreads();
    }
    if (!scatter) {
      T *Cz = C + z * sC;
#pragma unroll
      for (int i = 0; i < TM; i++) {
        const int64_t m = m0 + ty + i * (BM / TM);
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < TN; j++) {
          const int64_t n = n0 + tx + j * TX;
          if (n < N) Cz[m * N + n] = acc[i][j];
        }
      }
    } else {
      const int64_t ob = scatter_bits(z, sc.nb, sc.pb);
      int64_t on[TN];
#pragma unroll
      for (int j = 0; j < TN; j++) on[j] = scatter_bits(n0 + tx + j * TX, sc.nn, sc.pn);
#pragma unroll
      for (int i = 0; i < TM; i++) {
        const int64_t m = m0 + ty + i * (BM / TM);
        if (m >= M) continue;
        const int64_t om = ob + scatter_bits(m, sc.nm, sc.pm);
#pragma unroll
        for (int j = 0; j < TN; j++) {
          const int64_t n = n0 + tx + j * TX;
          if (n < N) C[om + on[j]] = acc[i][j];
        }
      }
    }
  }
}

// Skinny products (n <= NMAX complex columns, k <= KMAX): memory-bound, so
// each thread streams RPT rows of A (k contiguous complex values, 16-byte
// loads, all issued before any use) against B held in shared memory and
// writes its n results per row.
template <int NMAX, int KMAX, int RPT>
__global__ void __launch_bounds__(256)
    cgemm_skinny_kernel(const float2 *__restrict__ A, const float2 *__restrict__ B, float2 *__restrict__ C,
                        int64_t batch, int64_t M, int N, int K, int64_t sA, int64_t sB, int64_t sC,
                        const __grid_constant__ CScatter sc, int scatter) {
  __shared__ float2 Bs[NMAX * KMAX];
  constexpr int ROWS = 256 * RPT;
  const int64_t blocks_per_batch = (M + ROWS - 1) / ROWS;
  for (int64_t blk = blockIdx.x; blk < blocks_per_batch * batch; blk += gridDim.x) {
    const int64_t z = blk / blocks_per_batch;
    const int64_t m0 = (blk - z * blocks_per_batch) * ROWS + threadIdx.x;
    __syncthreads();
    for (int i = threadIdx.x; i < N * K; i += 256) Bs[i] = B[z * sB + i];
    __syncthreads();
    float2 a[RPT][KMAX];
#pragma unroll
    for (int r = 0; r < RPT; r++) {
      const int64_t m = m0 + r * 256;
      const float2 *arow = A + z * sA + m * K;
      if ((K & 1) == 0) {
        // K even: every row starts on a 16-byte boundary
#pragma unroll
        for (int k = 0; k < KMAX; k += 2)
          if (m < M && k < K) {
            const float4 v = __ldcs(reinterpret_cast<const float4 *>(arow + k));
            a[r][k] = make_float2(v.x, v.y);
            a[r][k + 1] = make_float2(v.z, v.w);
          }
      } else {
#pragma unroll
        for (int k = 0; k < KMAX; k++)
          if (m < M && k < K) a[r][k] = arow[k];
      }
    }
#pragma unroll
    for (int r = 0; r < RPT; r++) {
      const int64_t m = m0 + r * 256;
      if (m >= M) continue;
      const int64_t om = scatter ? scatter_bits(z, sc.nb, sc.pb) + scatter_bits(m, sc.nm, sc.pm) : z * sC + m * N;
#pragma unroll
      for (int n = 0; n < NMAX; n++) {
        if (n >= N) break;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < KMAX; k++)
          if (k < K) {
            const float2 b = Bs[n * K + k];
            acc.x = fmaf(a[r][k].x, b.x, acc.x);
            acc.x = fmaf(-a[r][k].y, b.y, acc.x);
            acc.y = fmaf(a[r][k].x, b.y, acc.y);
            acc.y = fmaf(a[r][k].y, b.x, acc.y);
          }
        C[om + (scatter ? scatter_bits(n, sc.nn, sc.pn) : n)] = acc;
      }
    }
  }
}

template <int NMAX, int KMAX, int RPT>
cudaError_t run_skinny(const float2 *A, const float2 *B, float2 *C, int64_t batch, int64_t M, int64_t N, int64_t K,
                       int64_t sA, int64_t sB, int64_t sC, const CScatter *sc, cudaStream_t s) {
  const int64_t blocks = ((M + 256 * RPT - 1) / (256 * RPT)) * batch;
  CScatter none{};
  cgemm_skinny_kernel<NMAX, KMAX, RPT><<<(unsigned)std::min<int64_t>(blocks, 152 * 16), 256, 0, s>>>(
      A, B, C, batch, M, (int)N, (int)K, sA, sB, sC, sc ? *sc : none, sc ? 1 : 0);
  return cudaGetLastError();
}

// complex128 version of the long-k dot product (element loads)
__global__ void __launch_bounds__(256)
    zdot_kernel(const double2 *__restrict__ A, const double2 *__restrict__ B, double2 *__restrict__ C, int64_t batch,
                int64_t M, int64_t N, int64_t K, int64_t sA, int64_t sB, int64_t sC, const __grid_constant__ CScatter sc,
                int scatter) {
  __shared__ double2 red[8];
  const int64_t n_out = batch * M * N;
  for (int64_t o = blockIdx.x; o < n_out; o += gridDim.x) {
    const int64_t z = o / (M * N);
    const int64_t m = (o / N) % M;
    const int64_t n = o % N;
    const double2 *a = A + z * sA + m * K;
    const double2 *b = B + z * sB + n * K;
    double2 acc = zero_c<double2>();
    for (int64_t k = threadIdx.x; k < K; k += blockDim.x) cmac(acc, a[k], b[k]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double2 t = red[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
        t.x += red[w].x;
        t.y += red[w].y;
      }
      const int64_t off = scatter ? scatter_bits(z, sc.nb, sc.pb) + scatter_bits(m, sc.nm, sc.pm) +
                                        scatter_bits(n, sc.nn, sc.pn)
                                  : z * sC + m * N + n;
      C[off] = t;
    }
  }
}

// Few outputs per batch, moderate summed index (m*n small, 64 <= k < 2048,
// many batches): one warp per output element streams its A row and B row
// (k-contiguous) with 16-byte loads and sums in FP32 (a shuffle reduction);
// HBM-bound. The tiled kernels waste their tiles on such shapes (a batch of
// 8192 1 x 1 products with k = 1024 ran 100x slower there).
__global__ void __launch_bounds__(256)
    cgemm_dot_warp_kernel(const float2 *__restrict__ A, const float2 *__restrict__ B, float2 *__restrict__ C,
                          int64_t batch, int64_t M, int64_t N, int64_t K, int64_t sA, int64_t sB, int64_t sC,
                          const __grid_constant__ CScatter sc, int scatter) {
  const int lane = threadIdx.x & 31;
  const int64_t n_out = batch * M * N;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t o = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); o < n_out; o += warps) {
    const int64_t z = o / (M * N);
    const int64_t m = (o / N) % M;
    const int64_t n = o % N;
    const float4 *a = reinterpret_cast<const float4 *>(A + z * sA + m * K);
    const float4 *b = reinterpret_cast<const float4 *>(B + z * sB + n * K);
    float2 acc = make_float2(0.f, 0.f);
    for (int64_t k = lane; k < K / 2; k += 32) {
      const float4 va = a[k], vb = b[k];
      acc.x = fmaf(va.x, vb.x, acc.x);
      acc.x = fmaf(-va.y, vb.y, acc.x);
      acc.y = fmaf(va.x, vb.y, acc.y);
      acc.y = fmaf(va.y, vb.x, acc.y);
      acc.x = fmaf(va.z, vb.z, acc.x);
      acc.x = fmaf(-va.w, vb.w, acc.x);
      acc.y = fmaf(va.z, vb.w, acc.y);
      acc.y = fmaf(va.w, vb.z, acc.y);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
    }
    if (lane == 0) {
      const int64_t off = scatter ? scatter_bits(z, sc.nb, sc.pb) + scatter_bits(m, sc.nm, sc.pm) +
                                        scatter_bits(n, sc.nn, sc.pn)
                                  : z * sC + m * N + n;
      C[off] = acc;
    }
  }
}

// Few outputs, long summed index (m*n small, k large): one block per output
// element streams its A row and B row (both k-contiguous) with 16-byte loads;
// each thread sums its strided share in FP32, then a tree reduction.
__global__ void __launch_bounds__(256)
    cgemm_dot_kernel(const float2 *__restrict__ A, const float2 *__restrict__ B, float2 *__restrict__ C,
                     int64_t batch, int64_t M, int64_t N, int64_t K, int64_t sA, int64_t sB, int64_t sC,
                     const __grid_constant__ CScatter sc, int scatter) {
  __shared__ float2 red[8];
  const int64_t n_out = batch * M * N;
  for (int64_t o = blockIdx.x; o < n_out; o += gridDim.x) {
    const int64_t z = o / (M * N);
    const int64_t m = (o / N) % M;
    const int64_t n = o % N;
    const float4 *a = reinterpret_cast<const float4 *>(A + z * sA + m * K);
    const float4 *b = reinterpret_cast<const float4 *>(B + z * sB + n * K);
    float2 acc = make_float2(0.f, 0.f);
    for (int64_t k = threadIdx.x; k < K / 2; k += blockDim.x) {
      const float4 va = a[k], vb = b[k];
      acc.x = fmaf(va.x, vb.x, acc.x);
      acc.x = fmaf(-va.y, vb.y, acc.x);
      acc.y = fmaf(va.x, vb.y, acc.y);
      acc.y = fmaf(va.y, vb.x, acc.y);
      acc.x = fmaf(va.z, vb.z, acc.x);
      acc.x = fmaf(-va.w, vb.w, acc.x);
      acc.y = fmaf(va.z, vb.w, acc.y);
      acc.y = fmaf(va.w, vb.z, acc.y);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      float2 t = red[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
        t.x += red[w].x;
        t.y += red[w].y;
      }
      const int64_t off = scatter ? scatter_bits(z, sc.nb, sc.pb) + scatter_bits(m, sc.nm, sc.pm) +
                                        scatter_bits(n, sc.nn, sc.pn)
                                  : z * sC + m * N + n;
      C[off] = t;
    }
  }
}

template <int BM, int BN, int TM, int TN, int BK, typename T>
cudaError_t run(const T *A, const T *B, T *C, int64_t batch, int64_t M, int64_t N, int64_t K, int64_t sA, int64_t sB,
                int64_t sC, const CScatter *sc, cudaStream_t s) {
  const int64_t tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN) * batch;
  const int blocks = (int)std::min<int64_t>(tiles, 152 * 64);
  CScatter none{};
  cgemm_simt_kernel<T, BM, BN, TM, TN, BK><<<blocks, (BM / TM) * (BN / TN), 0, s>>>(A, B, C, batch, M, N, K, sA, sB,
                                                                               sC, sc ? *sc : none, sc ? 1 : 0);
  return cudaGetLastError();
}

// Skinny products read in place: X and Y in any bit layout (gather maps),
// C through a scatter map. One thread per row of X; rows are numbered so that
// the lowest row bits are the lowest bits of X where possible, which keeps
// the loads of a warp in few sectors.
template <typename T, int NMAX, int KMAX, int RPT>
__global__ void __launch_bounds__(256)
    skinny_gather_kernel(const T *__restrict__ X, const T *__restrict__ Y, T *__restrict__ C,
                         int64_t batch, int64_t M, int N, int K, const __grid_constant__ GatherMap g,
                         const __grid_constant__ CScatter sc, int scatter) {
  __shared__ T Ys[NMAX * KMAX];
  __shared__ int64_t xk_off[KMAX];
  __shared__ int64_t cn_off[NMAX];
  __shared__ int64_t hi_off[2];  // block-uniform part of the X and C offsets
  constexpr int ROWS = 256 * RPT;
  static_assert(ROWS == 1024 || ROWS == 512, "rows per block");
  constexpr int LOW = ROWS == 1024 ? 10 : 9;  // row bits owned by the thread
  // offsets of this thread's rows within a block: the row index bits below
  // LOW come from threadIdx and r only, so they are computed once
  int64_t xlo[RPT], clo[RPT];
#pragma unroll
  for (int r = 0; r < RPT; r++) {
    const int64_t m = threadIdx.x + r * 256;
    xlo[r] = scatter_bits(m, g.nm < LOW ? g.nm : LOW, g.xm);
    clo[r] = scatter ? scatter_bits(m, sc.nm < LOW ? sc.nm : LOW, sc.pm) : m * N;
  }
  const int64_t blocks_per_batch = (M + ROWS - 1) / ROWS;
  for (int64_t blk = blockIdx.x; blk < blocks_per_batch * batch; blk += gridDim.x) {
    const int64_t z = blk / blocks_per_batch;
    const int64_t mb = (blk - z * blocks_per_batch) * ROWS;
    __syncthreads();
    if (threadIdx.x < N * K) {
      const int n = threadIdx.x / K, k = threadIdx.x % K;
      Ys[threadIdx.x] = Y[scatter_bits(z, g.nb, g.yb) + scatter_bits(n, g.nn, g.yn) + scatter_bits(k, g.nk, g.yk)];
    }
    if (threadIdx.x < K) xk_off[threadIdx.x] = scatter_bits(threadIdx.x, g.nk, g.xk);
    if (threadIdx.x >= 64 && threadIdx.x < 64 + N)
      cn_off[threadIdx.x - 64] = scatter ? scatter_bits(threadIdx.x - 64, sc.nn, sc.pn) : threadIdx.x - 64;
    if (threadIdx.x == 128) {
      int64_t xh = scatter_bits(z, g.nb, g.xb), ch = scatter ? scatter_bits(z, sc.nb, sc.pb) : z * M * N;
      for (int j = LOW; j < g.nm; j++) xh |= ((mb >> j) & 1) << g.xm[j];
      if (scatter)
        for (int j = LOW; j < sc.nm; j++) ch |= ((mb >> j) & 1) << sc.pm[j];
      else
        ch += mb * N;
      hi_off[0] = xh;
      hi_off[1] = ch;
    }
    __syncthreads();
    const int64_t xh = hi_off[0], ch = hi_off[1];
    T a[RPT][KMAX];
#pragma unroll
    for (int r = 0; r < RPT; r++) {
      if (mb + threadIdx.x + r * 256 >= M) continue;
      const T *xr = X + xh + xlo[r];
#pragma unroll
      for (int k = 0; k < KMAX; k++)
        if (k < K) a[r][k] = __ldcs(xr + xk_off[k]);
    }
#pragma unroll
    for (int r = 0; r < RPT; r++) {
      if (mb + threadIdx.x + r * 256 >= M) continue;
      const int64_t om = ch + clo[r];
#pragma unroll
      for (int n = 0; n < NMAX; n++) {
        if (n >= N) break;
        T acc = zero_c<T>();
#pragma unroll
        for (int k = 0; k < KMAX; k++)
          if (k < K) cmac(acc, a[r][k], Ys[n * K + k]);
        __stcs(C + om + cn_off[n], acc);
      }
    }
  }
}

template <typename T, int NMAX, int KMAX, int RPT>
cudaError_t run_skinny_gather(const T *X, const T *Y, T *C, int64_t batch, int64_t M, int64_t N, int64_t K,
                              const GatherMap &g, const CScatter *sc, cudaStream_t s) {
  const int64_t blocks = ((M + 256 * RPT - 1) / (256 * RPT)) * batch;
  CScatter none{};
  skinny_gather_kernel<T, NMAX, KMAX, RPT><<<(unsigned)std::min<int64_t>(blocks, 152 * 16), 256, 0, s>>>(
      X, Y, C, batch, M, (int)N, (int)K, g, sc ? *sc : none, sc ? 1 : 0);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- stream
// Products with few summed values (K <= 32) write far more than they read,
// and through a scatter map their outputs land wherever the consumer wants
// them. This kernel is built around the writes: a tile is the set of
// outputs whose local bits (the low bz bits of the batch index, bm of the row
// index, bn of the column index) vary, chosen so that they cover the lowest
// output positions. Its outputs are numbered ("ranks") in the order of
// their output positions, so a warp's 32 consecutive ranks write consecutive
// addresses; the tile's rows of A and B are staged in shared memory
// (K padded to KMAX with zeros) and every output is a short dot product in
// FP32 FMA, summed in k order like the tiled kernel.
constexpr int kStreamMaxLocal = 16;
struct StreamTile {
  int bz, bm, bn, nl;               // local bits of batch, row, column; total
  int8_t rsrc[kStreamMaxLocal];     // rank bit r: 0 batch, 1 row, 2 column
  int8_t rbit[kStreamMaxLocal];     // its bit within that index
  int8_t rpos[kStreamMaxLocal];     // its output position
  int8_t lane_rank[32];             // rank (within its warp's 32) that lane l computes
};
// Shared-memory layout of the staged rows: a row of KMAX values takes
// KMAX / 2 + 1 chunks of 16 bytes (an odd count, so 8 consecutive rows start
// in 8 different banks), and each block of rows with the same batch bits is
// shifted by one more chunk (rows that differ only in batch bits would
// otherwise share banks). shift = log2 of the rows per batch value.
__host__ __device__ inline int stream_row_chunk(int row, int ch, int shift) { return row * (ch + 1) + (row >> shift); }

template <int KMAX>
__global__ void __launch_bounds__(256)
    cgemm_stream_kernel(const float2 *__restrict__ A, const float2 *__restrict__ B, float2 *__restrict__ C,
                        int64_t batch, int64_t M, int64_t N, int K, const __grid_constant__ CScatter sc,
                        const __grid_constant__ StreamTile st) {
  // rows in shared memory: KMAX / 2 chunks of 16 bytes each, and every block
  // of rows with the same batch bits shifted by one more chunk, so that the
  // rows a warp reads at once (different batch bits) sit in different banks
  extern __shared__ float4 stream_smem[];
  constexpr int CH = KMAX / 2;
  const int rowsA = 1 << (st.bz + st.bm), rowsB = 1 << (st.bz + st.bn);
  float4 *As4 = stream_smem;
  float4 *Bs4 = As4 + (size_t)rowsA * (CH + 1) + (1 << st.bz);
  auto rowA = [&](int row) { return As4 + stream_row_chunk(row, CH, st.bm); };
  auto rowB = [&](int row) { return Bs4 + stream_row_chunk(row, CH, st.bn); };
  // the rank bits from 8 up, decoded once per launch: entry j holds the local
  // batch, row and column bits and the output offset of rank j * 256
  __shared__ int s_hz[1 << (kStreamMaxLocal - 8)], s_hm[1 << (kStreamMaxLocal - 8)],
      s_hn[1 << (kStreamMaxLocal - 8)];
  __shared__ int64_t s_ho[1 << (kStreamMaxLocal - 8)];
  __shared__ int8_t s_pos[kMaxBits];      // output position of bit t of (batch, row, column)
  __shared__ unsigned s_base[2][2];       // a tile's output base, OR-reduced by warps 0 and 1
  const int gz = sc.nb, gm = sc.nm, gn = sc.nn, total = gz + gm + gn;
  const int nhi = st.nl > 8 ? 1 << (st.nl - 8) : 1;
  for (int j = threadIdx.x; j < nhi; j += 256) {
    int hz = 0, hm = 0, hn = 0;
    int64_t ho = 0;
    for (int r = 8; r < st.nl; r++)
      if ((j >> (r - 8)) & 1) {
        const int v = 1 << st.rbit[r];
        if (st.rsrc[r] == 0) hz |= v;
        else if (st.rsrc[r] == 1) hm |= v;
        else hn |= v;
        ho |= int64_t(1) << st.rpos[r];
      }
    s_hz[j] = hz;
    s_hm[j] = hm;
    s_hn[j] = hn;
    s_ho[j] = ho;
  }
  for (int t = threadIdx.x; t < total; t += 256)
    s_pos[t] = t < gz ? sc.pb[t] : t < gz + gm ? sc.pm[t - gz] : sc.pn[t - gz - gm];
  // the rank bits below 8 come from the thread
  // the thread's rank within its block of 256: the warp's 32 ranks are a
  // fixed permutation of its lanes (chosen on the host so that the lanes a
  // shared-memory phase serves read rows in different banks); the warp
  // still writes one contiguous run
  const int trank = (int)(threadIdx.x & ~31u) | st.lane_rank[threadIdx.x & 31];
  int tz0 = 0, tm0 = 0, tn0 = 0;
  int64_t to0 = 0;
  for (int r = 0; r < st.nl && r < 8; r++)
    if ((trank >> r) & 1) {
      const int v = 1 << st.rbit[r];
      if (st.rsrc[r] == 0) tz0 |= v;
      else if (st.rsrc[r] == 1) tm0 |= v;
      else tn0 |= v;
      to0 |= int64_t(1) << st.rpos[r];
    }
  __syncthreads();
  const int sn = gn - st.bn, sm = gm - st.bm;  // log2 of the column and row tiles
  const int64_t tiles = (batch * M * N) >> st.nl;
  const int R = 1 << st.nl;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t nt = tile & ((int64_t(1) << sn) - 1);
    const int64_t mt = (tile >> sn) & ((int64_t(1) << sm) - 1);
    const int64_t zt = tile >> (sn + sm);
    const int64_t z0 = zt << st.bz, m0 = mt << st.bm, n0 = nt << st.bn;
    if (threadIdx.x < 64) {
      // bit t of (z0, m0, n0) contributes 1 << s_pos[t] to the tile's base
      const int t = threadIdx.x;
      int64_t c = 0;
      if (t < total) {
        const int64_t v = t < gz ? (z0 >> t) : t < gz + gm ? (m0 >> (t - gz)) : (n0 >> (t - gz - gm));
        c = (v & 1) ? int64_t(1) << s_pos[t] : 0;
      }
      const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)c);
      const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(c >> 32));
      if ((t & 31) == 0) {
        s_base[t >> 5][0] = lo;
        s_base[t >> 5][1] = hi;
      }
    }
    __syncthreads();  // the previous tile's rows are no longer read; base ready
    const int64_t base = (int64_t)((uint64_t)(s_base[0][0] | s_base[1][0]) |
                                   ((uint64_t)(s_base[0][1] | s_base[1][1]) << 32));
    // rows (z0 + lz, m0 .. m0 + 2^bm) of A are one contiguous run of 2^bm K
    // values; two complex values (16 bytes) per load where K is even
    for (int i = threadIdx.x; i < rowsA * CH; i += 256) {
      const int row = i / CH, c = i - row * CH;
      const int lz = row >> st.bm, lm = row & ((1 << st.bm) - 1);
      const float2 *src = A + ((z0 + lz) * M + m0 + lm) * K;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if ((K & 1) == 0) {
        if (2 * c < K) v = *reinterpret_cast<const float4 *>(src + 2 * c);
      } else {
        if (2 * c < K) v.x = src[2 * c].x, v.y = src[2 * c].y;
        if (2 * c + 1 < K) v.z = src[2 * c + 1].x, v.w = src[2 * c + 1].y;
      }
      rowA(row)[c] = v;
    }
    for (int i = threadIdx.x; i < rowsB * CH; i += 256) {
      const int row = i / CH, c = i - row * CH;
      const int lz = row >> st.bn, ln = row & ((1 << st.bn) - 1);
      const float2 *src = B + ((z0 + lz) * N + n0 + ln) * K;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if ((K & 1) == 0) {
        if (2 * c < K) v = *reinterpret_cast<const float4 *>(src + 2 * c);
      } else {
        if (2 * c < K) v.x = src[2 * c].x, v.y = src[2 * c].y;
        if (2 * c + 1 < K) v.z = src[2 * c + 1].x, v.w = src[2 * c + 1].y;
      }
      rowB(row)[c] = v;
    }
    __syncthreads();
    if (trank >= R) continue;
    // (keeping a thread's rows in registers across its outputs measured
    // slower: the registers cost more occupancy than the reads they save)
    for (int rr = 0; rr < R; rr += 256) {
      const int j = rr >> 8;
      const int lz = tz0 | s_hz[j];
      const float4 *a = rowA((lz << st.bm) + (tm0 | s_hm[j]));
      const float4 *b = rowB((lz << st.bn) + (tn0 | s_hn[j]));
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < CH; k++) {
        const float4 x = a[k], y = b[k];
        cmac(acc, make_float2(x.x, x.y), make_float2(y.x, y.y));
        cmac(acc, make_float2(x.z, x.w), make_float2(y.z, y.w));
      }
      __stcs(C + base + (to0 | s_ho[j]), acc);
    }
  }
}

// Tile of the stream kernel for this product, or false when it does not
// apply (dimensions not powers of two, K above 32, or no tile within the
// shared-memory budget). The output position of every index bit comes from
// the scatter map (row-major: column bits lowest, then row, then batch).
bool stream_tile(int64_t batch, int64_t M, int64_t N, int64_t K, const CScatter &sc, StreamTile *t, int *kmax) {
  auto lg = [](int64_t v) { int b = 0; while ((int64_t(1) << b) < v) b++; return (int64_t(1) << b) == v ? b : -1; };
  const int gz = lg(batch), gm = lg(M), gn = lg(N);
  if (gz < 0 || gm < 0 || gn < 0 || K < 1 || K > 32) return false;
  if (sc.nb != gz || sc.nm != gm || sc.nn != gn) return false;
  const int total = gz + gm + gn;
  if (total > kMaxBits) return false;
  *kmax = K <= 4 ? 4 : K <= 8 ? 8 : K <= 16 ? 16 : 32;
  const int64_t budget = 40 * 1024 / 8;  // float2 values of dynamic shared memory (48 KB with the static part)
  // owner of each output position
  std::vector<std::pair<int, int>> owner(total, {-1, -1});
  const int8_t *pos[3] = {sc.pb, sc.pm, sc.pn};
  const int g[3] = {gz, gm, gn};
  for (int x = 0; x < 3; x++)
    for (int j = 0; j < g[x]; j++) {
      if (pos[x][j] < 0 || pos[x][j] >= total || owner[pos[x][j]].first >= 0) return false;
      owner[pos[x][j]] = {x, j};
    }
  auto fits = [&](const int *b) {
    return ((int64_t(1) << (b[0] + b[1])) + (int64_t(1) << (b[0] + b[2]))) * (*kmax + 2) + (int64_t(4) << b[0]) <=
               budget &&
           b[0] + b[1] + b[2] <= kStreamMaxLocal;
  };
  int b[3] = {0, 0, 0};
  for (int L = std::min(total, 6); L >= 0; L--) {
    int c[3] = {0, 0, 0};
    for (int p = 0; p < L; p++) c[owner[p].first] = std::max(c[owner[p].first], owner[p].second + 1);
    if (fits(c)) {
      std::copy(c, c + 3, b);
      break;
    }
  }
  // more rows and columns while they fit: each A row is then read by more
  // columns and each B row by more rows (up to 4096 outputs a tile)
  for (;;) {
    if (b[0] + b[1] + b[2] >= 12) break;
    int c[3] = {b[0], b[1], b[2]};
    const int pick = (b[2] < g[2] && (b[2] <= b[1] || b[1] >= g[1])) ? 2 : 1;
    if (c[pick] >= g[pick]) break;
    c[pick]++;
    if (!fits(c)) break;
    std::copy(c, c + 3, b);
  }
  t->bz = b[0];
  t->bm = b[1];
  t->bn = b[2];
  t->nl = b[0] + b[1] + b[2];
  // ranks: the local bits in the order of their output positions
  int r = 0;
  for (int p = 0; p < total; p++) {
    const int x = owner[p].first, j = owner[p].second;
    if (j < b[x]) {
      t->rsrc[r] = (int8_t)x;
      t->rbit[r] = (int8_t)j;
      t->rpos[r] = (int8_t)p;
      r++;
    }
  }
  if (r != t->nl) return false;
  // lanes of a warp: a shared-memory phase of 128-bit loads serves 8
  // consecutive lanes, and its cost is the largest number of different rows
  // that fall in one 16-byte bank group. Ranks are dealt to lanes to keep
  // that low for both operands (pairwise swaps while the cost drops); the
  // pattern is the same in every warp and for every chunk of the rows.
  for (int l = 0; l < 32; l++) t->lane_rank[l] = (int8_t)l;
  if (t->nl >= 5) {
    const int ch = *kmax / 2;
    int slot[2][32], row[2][32];
    for (int q = 0; q < 32; q++) {
      int lz = 0, lm = 0, ln = 0;
      for (int j = 0; j < 5; j++)
        if ((q >> j) & 1) {
          const int v = 1 << t->rbit[j];
          if (t->rsrc[j] == 0) lz |= v;
          else if (t->rsrc[j] == 1) lm |= v;
          else ln |= v;
        }
      row[0][q] = (lz << t->bm) | lm;
      row[1][q] = (lz << t->bn) | ln;
      slot[0][q] = stream_row_chunk(row[0][q], ch, t->bm) & 7;
      slot[1][q] = stream_row_chunk(row[1][q], ch, t->bn) & 7;
    }
    auto phase_cost = [&](int ph) {
      int c = 0;
      for (int o = 0; o < 2; o++) {
        int worst = 0;
        for (int sl = 0; sl < 8; sl++) {
          int rows_here[8], nr = 0;
          for (int l = 8 * ph; l < 8 * ph + 8; l++) {
            const int q = t->lane_rank[l];
            if (slot[o][q] != sl) continue;
            bool seen = false;
            for (int i = 0; i < nr; i++) seen |= rows_here[i] == row[o][q];
            if (!seen) rows_here[nr++] = row[o][q];
          }
          worst = std::max(worst, nr);
        }
        c += worst;
      }
      return c;
    };
    for (int pass = 0; pass < 8; pass++) {
      bool better = false;
      for (int a = 0; a < 32; a++)
        for (int b = a + 1; b < 32; b++) {
          if ((a >> 3) == (b >> 3)) continue;
          const int before = phase_cost(a >> 3) + phase_cost(b >> 3);
          std::swap(t->lane_rank[a], t->lane_rank[b]);
          if (phase_cost(a >> 3) + phase_cost(b >> 3) < before) {
            better = true;
          } else {
            std::swap(t->lane_rank[a], t->lane_rank[b]);
          }
        }
      if (!better) break;
    }
  }
  return true;
}

CScatter row_major_map(int64_t batch, int64_t M, int64_t N) {
  auto lg = [](int64_t v) { int b = 0; while ((int64_t(1) << b) < v) b++; return b; };
  CScatter sc{};
  sc.nn = lg(N);
  sc.nm = lg(M);
  sc.nb = lg(batch);
  for (int j = 0; j < sc.nn; j++) sc.pn[j] = (int8_t)j;
  for (int j = 0; j < sc.nm; j++) sc.pm[j] = (int8_t)(sc.nn + j);
  for (int j = 0; j < sc.nb; j++) sc.pb[j] = (int8_t)(sc.nn + sc.nm + j);
  return sc;
}

}  // namespace

bool cgemm_stream_supported(int64_t batch, int64_t M, int64_t N, int64_t K, const CScatter *sc) {
  StreamTile t{};
  int kmax = 0;
  if (batch * M * N < 256) return false;
  return stream_tile(batch, M, N, K, sc ? *sc : row_major_map(batch, M, N), &t, &kmax);
}

int cgemm_stream_describe(int64_t batch, int64_t M, int64_t N, int64_t K, const CScatter *sc, int32_t *out) {
  StreamTile t{};
  int kmax = 0;
  if (batch * M * N < 256 || !stream_tile(batch, M, N, K, sc ? *sc : row_major_map(batch, M, N), &t, &kmax)) return 0;
  out[0] = t.bz;
  out[1] = t.bm;
  out[2] = t.bn;
  out[3] = t.nl;
  out[4] = kmax;
  out[5] = (int32_t)(((((int64_t)1 << (t.bz + t.bm)) + ((int64_t)1 << (t.bz + t.bn))) * (kmax / 2 + 1) +
                      ((int64_t)2 << t.bz)) * 16);
  for (int r = 0; r < kStreamMaxLocal; r++) {
    out[6 + 3 * r] = r < t.nl ? t.rsrc[r] : -1;
    out[7 + 3 * r] = r < t.nl ? t.rbit[r] : -1;
    out[8 + 3 * r] = r < t.nl ? t.rpos[r] : -1;
  }
  for (int l = 0; l < 32; l++) out[6 + 3 * kStreamMaxLocal + l] = t.lane_rank[l];
  return 1;
}

cudaError_t launch_cgemm_stream(const float2 *A, const float2 *B, float2 *C, int64_t batch, int64_t M, int64_t N,
                                int64_t K, int64_t sA, int64_t sB, int64_t sC, const CScatter *sc, cudaStream_t s) {
  if (sA != M * K || sB != N * K || (!sc && sC != M * N)) return cudaErrorNotSupported;
  const CScatter map = sc ? *sc : row_major_map(batch, M, N);
  StreamTile t{};
  int kmax = 0;
  if (batch * M * N < 256 || !stream_tile(batch, M, N, K, map, &t, &kmax)) return cudaErrorNotSupported;
  const size_t smem = ((((size_t)1 << (t.bz + t.bm)) + ((size_t)1 << (t.bz + t.bn))) * (kmax / 2 + 1) +
                       ((size_t)2 << t.bz)) * sizeof(float4);
  const int64_t tiles = batch * M * N >> t.nl;
  const unsigned grid = (unsigned)std::min<int64_t>(tiles, 152 * 8);
  switch (kmax) {
    case 4: cgemm_stream_kernel<4><<<grid, 256, smem, s>>>(A, B, C, batch, M, N, (int)K, map, t); break;
    case 8: cgemm_stream_kernel<8><<<grid, 256, smem, s>>>(A, B, C, batch, M, N, (int)K, map, t); break;
    case 16: cgemm_stream_kernel<16><<<grid, 256, smem, s>>>(A, B, C, batch, M, N, (int)K, map, t); break;
    default: cgemm_stream_kernel<32><<<grid, 256, smem, s>>>(A, B, C, batch, M, N, (int)K, map, t); break;
  }
  return cudaGetLastError();
}

namespace {
}  // namespace

cudaError_t launch_cgemm_skinny_gather(const float2 *X, const float2 *Y, float2 *C, int64_t batch, int64_t M,
                                       int64_t N, int64_t K, const GatherMap &g, const CScatter *sc, cudaStream_t s) {
  if (batch <= 0 || M <= 0 || N <= 0 || K <= 0 || N > 4 || K > 16) return cudaErrorInvalidValue;
  if (K <= 4) return run_skinny_gather<float2, 4, 4, 4>(X, Y, C, batch, M, N, K, g, sc, s);
  return run_skinny_gather<float2, 4, 16, 2>(X, Y, C, batch, M, N, K, g, sc, s);
}

cudaError_t launch_zskinny_gather(const double2 *X, const double2 *Y, double2 *C, int64_t batch, int64_t M,
                                  int64_t N, int64_t K, const GatherMap &g, const CScatter *sc, cudaStream_t s) {
  if (batch <= 0 || M <= 0 || N <= 0 || K <= 0 || N > 4 || K > 16) return cudaErrorInvalidValue;
  if (K <= 4) return run_skinny_gather<double2, 4, 4, 2>(X, Y, C, batch, M, N, K, g, sc, s);
  return run_skinny_gather<double2, 4, 16, 2>(X, Y, C, batch, M, N, K, g, sc, s);
}

cudaError_t launch_zgemm_simt(const double2 *A, const double2 *B, double2 *C, int64_t batch, int64_t M, int64_t N,
                              int64_t K, int64_t sA, int64_t sB, int64_t sC, const CScatter *sc, cudaStream_t s) {
  if (batch <= 0 || M <= 0 || N <= 0 || K <= 0) return cudaErrorInvalidValue;
  if (M * N <= 64 && K >= 2048) {
    CScatter none{};
    zdot_kernel<<<(unsigned)std::min<int64_t>(batch * M * N, 152 * 8), 256, 0, s>>>(A, B, C, batch, M, N, K, sA, sB,
                                                                                 sC, sc ? *sc : none, sc ? 1 : 0);
    return cudaGetLastError();
  }
  if (N >= 48) return run<64, 64, 4, 4, 8>(A, B, C, batch, M, N, K, sA, sB, sC, sc, s);
  if (N >= 12) return run<128, 16, 4, 2, 8>(A, B, C, batch, M, N, K, sA, sB, sC, sc, s);
  if (N >= 3) return run<256, 4, 4, 1, 8>(A, B, C, batch, M, N, K, sA, sB, sC, sc, s);
  return run<256, 2, 2, 1, 8>(A, B, C, batch, M, N, K, sA, sB, sC, sc, s);
}

cudaError_t launch_cgemm_simt(const float2 *A, const float2 *B, float2 *C, int64_t batch, int64_t M, int64_t N,
                              int64_t K, int64_t sA, int64_t sB, int64_t sC, const CScatter *sc, cudaStream_t s) {
  if (batch <= 0 || M <= 0 || N <= 0 || K <= 0) return cudaErrorInvalidValue;
  const bool aligned = (K % 2) == 0 && (sA % 2) == 0 && (sB % 2) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0 &&
                       (reinterpret_cast<uintptr_t>(B) & 15) == 0;
  if (M * N <= 64 && K >= 2048 && aligned) {
    CScatter none{};
    const int64_t outs = batch * M * N;
    cgemm_dot_kernel<<<(unsigned)std::min<int64_t>(outs, 152 * 8), 256, 0, s>>>(A, B, C, batch, M, N, K, sA, sB, sC,
                                                                             sc ? *sc : none, sc ? 1 : 0);
    return cudaGetLastError();
  }
  if (M * N <= 64 && K >= 64 && aligned) {
    CScatter none{};
    const int64_t outs = batch * M * N;
    const int64_t blocks = std::min<int64_t>((outs + 7) / 8, 152 * 16);
    cgemm_dot_warp_kernel<<<(unsigned)blocks, 256, 0, s>>>(A, B, C, batch, M, N, K, sA, sB, sC, sc ? *sc : none,
                                                           sc ? 1 : 0);
    return cudaGetLastError();
  }
  if (N <= 4 && K <= 16 && M >= 256) {
    if (K <= 4) return run_skinny<4, 4, 4>(A, B, C, batch, M, N, K, sA, sB, sC, sc, s);
    return run_skinny<4, 16, 2>(A, B, C, batch, M, N, K, sA, sB, sC, sc, s);
  }
  if (N >= 48) return run<64, 64, 4, 4, 8>(A, B, C, batch, M, N, K, sA, sB, sC, sc, s);
  if (N >= 12) return run<128, 16, 4, 2, 8>(A, B, C, batch, M, N, K, sA, sB, sC, sc, s);
  if (N >= 3) return run<256, 4, 4, 1, 8>(A, B, C, batch, M, N, K, sA, sB, sC, sc, s);
  return run<256, 2, 2, 1, 8>(A, B, C, batch, M, N, K, sA, sB, sC, sc, s);
}

}  // namespace dev
}  // namespace tz
