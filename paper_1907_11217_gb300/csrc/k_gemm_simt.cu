// Batched complex64 product on CUDA cores (FP32 FMA, four real products per
// complex multiply-add): C[z] = A[z] B[z]^T with A[z] m x k, B[z] n x k and
// C[z] m x n, all row-major. This is the plain complex64 precision mode and
// the baseline of the split-precision tensor-core modes.
#include <algorithm>

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
