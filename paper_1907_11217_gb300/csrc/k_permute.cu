// Bit permutation of a complex64 tensor (every index has dimension 2, so a
// tensor transpose is a permutation of the bits of the element offset).
// HBM-bound. A tile spans the 5 lowest input bits, the input bits that land
// on the 5 lowest output bits, and further low input bits up to 10 bits
// (1024 elements, 8 KB of shared memory), so loads and stores both move
// runs of >= 32 consecutive elements (256 bytes per warp access). The
// tile-local offsets are the same for every tile and are computed once per
// thread. Each thread moves pairs of consecutive elements (16-byte global
// accesses: input bit 0 and output bit 0 are both inside the tile's runs);
// shared memory is XOR-swizzled on index bits 1..4 (by bits 5..8), which
// keeps pair partners adjacent and spreads both access orders over banks.
#include <algorithm>

#include "kernels.h"

namespace tz {
namespace dev {

namespace {

constexpr int kW = 5;       // bits of a contiguous run on either side
constexpr int kTile = 10;   // bits of a tile (1024 elements, 8 KB)
constexpr int kThreads = 256;
constexpr int kPer = (1 << kTile) / kThreads;  // elements per thread per tile

struct TileMap {
  int r, u;                 // tensor rank, tile bits
  int8_t uin[kTile];        // input bit of tile bit j (load order)
  int8_t vout[kTile];       // output bit of tile bit j (store order)
  int8_t vsrc[kTile];       // store-order tile bit j -> load-order tile bit
  int8_t rin[kMaxBits];     // input bit of tile-index bit j
  int8_t rout[kMaxBits];    // output bit of tile-index bit j
};

__device__ __forceinline__ int swz(int e) { return e ^ (((e >> 5) & 15) << 1); }

template <typename T>
__global__ void permute_small_kernel(const T *__restrict__ in, T *__restrict__ out, PermuteArgs a) {
  const int64_t n = int64_t(1) << a.rank;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = 0;
    for (int p = 0; p < a.rank; p++) i |= ((o >> p) & 1) << a.perm[p];
    out[o] = in[i];
  }
}

// u == kTile (rank >= 10): every thread moves kPer elements (kPer/2 pairs)
// per tile.
__global__ void __launch_bounds__(kThreads) permute_tiled_kernel(const float2 *__restrict__ in,
                                                                 float2 *__restrict__ out,
                                                                 const __grid_constant__ TileMap m, int64_t n_tiles) {
  __shared__ __align__(16) float2 tile[1 << kTile];
  constexpr int kPairs = kPer / 2;
  // tile-local offsets of each pair, identical for every tile
  int64_t ld_off[kPairs], st_off[kPairs];
  int ld_s[kPairs], st_s0[kPairs], st_s1[kPairs];
#pragma unroll
  for (int i = 0; i < kPairs; i++) {
    const int e = 2 * (threadIdx.x + i * kThreads);  // load order, even
    int64_t o = 0;
    for (int j = 0; j < kTile; j++) o |= int64_t((e >> j) & 1) << m.uin[j];
    ld_off[i] = o;
    ld_s[i] = swz(e);
    const int f = e;  // store order, even
    int64_t oo = 0;
    int src0 = 0, src1 = 0;
    for (int j = 0; j < kTile; j++) {
      const int b0 = (f >> j) & 1, b1 = ((f + 1) >> j) & 1;
      oo |= int64_t(b0) << m.vout[j];
      src0 |= b0 << m.vsrc[j];
      src1 |= b1 << m.vsrc[j];
    }
    st_off[i] = oo;
    st_s0[i] = swz(src0);
    st_s1[i] = swz(src1);
  }
  __shared__ int64_t base[2];
  const int nr = m.r - kTile;
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    // the tile's base offsets are block-uniform: one thread computes them
    if (threadIdx.x == 0) {
      int64_t bin = 0, bout = 0;
      for (int j = 0; j < nr; j++) {
        const int64_t b = (t >> j) & 1;
        bin |= b << m.rin[j];
        bout |= b << m.rout[j];
      }
      base[0] = bin;
      base[1] = bout;
    }
    __syncthreads();
    const int64_t bin = base[0], bout = base[1];
    float4 v[kPairs];
#pragma unroll
    for (int i = 0; i < kPairs; i++) v[i] = __ldcs(reinterpret_cast<const float4 *>(in + bin + ld_off[i]));
#pragma unroll
    for (int i = 0; i < kPairs; i++) *reinterpret_cast<float4 *>(&tile[ld_s[i]]) = v[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kPairs; i++) {
      const float2 a = tile[st_s0[i]], b = tile[st_s1[i]];
      __stcs(reinterpret_cast<float4 *>(out + bout + st_off[i]), make_float4(a.x, a.y, b.x, b.y));
    }
    __syncthreads();
  }
}

// complex128: 16-byte elements, moved one by one (already 16-byte accesses)
__global__ void __launch_bounds__(kThreads) permute_tiled_z_kernel(const double2 *__restrict__ in,
                                                                   double2 *__restrict__ out,
                                                                   const __grid_constant__ TileMap m,
                                                                   int64_t n_tiles) {
  __shared__ double2 tile[1 << kTile];
  __shared__ int64_t base[2];
  int64_t ld_off[kPer], st_off[kPer];
  int ld_s[kPer], st_s[kPer];
#pragma unroll
  for (int i = 0; i < kPer; i++) {
    const int e = threadIdx.x + i * kThreads;
    int64_t o = 0, oo = 0;
    int src = 0;
    for (int j = 0; j < kTile; j++) {
      o |= int64_t((e >> j) & 1) << m.uin[j];
      oo |= int64_t((e >> j) & 1) << m.vout[j];
      src |= ((e >> j) & 1) << m.vsrc[j];
    }
    ld_off[i] = o;
    ld_s[i] = swz(e);
    st_off[i] = oo;
    st_s[i] = swz(src);
  }
  const int nr = m.r - kTile;
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    if (threadIdx.x == 0) {
      int64_t bin = 0, bout = 0;
      for (int j = 0; j < nr; j++) {
        const int64_t b = (t >> j) & 1;
        bin |= b << m.rin[j];
        bout |= b << m.rout[j];
      }
      base[0] = bin;
      base[1] = bout;
    }
    __syncthreads();
    const int64_t bin = base[0], bout = base[1];
    double2 v[kPer];
#pragma unroll
    for (int i = 0; i < kPer; i++) v[i] = in[bin + ld_off[i]];
#pragma unroll
    for (int i = 0; i < kPer; i++) tile[ld_s[i]] = v[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kPer; i++) out[bout + st_off[i]] = tile[st_s[i]];
    __syncthreads();
  }
}

bool tile_map(const PermuteArgs &a, TileMap *mp);

}  // namespace

cudaError_t launch_permute_z(const double2 *in, double2 *out, const PermuteArgs &a, cudaStream_t s) {
  const int r = a.rank;
  if (r < 0 || r > kMaxBits) return cudaErrorInvalidValue;
  const int64_t n = int64_t(1) << r;
  if (r < kTile) {
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    permute_small_kernel<double2><<<blocks, 256, 0, s>>>(in, out, a);
    return cudaGetLastError();
  }
  TileMap m{};
  tile_map(a, &m);
  const int64_t n_tiles = n >> kTile;
  permute_tiled_z_kernel<<<(int)std::min<int64_t>(n_tiles, 152 * 8), kThreads, 0, s>>>(in, out, m, n_tiles);
  return cudaGetLastError();
}

cudaError_t launch_permute(const float2 *in, float2 *out, const PermuteArgs &a, cudaStream_t s) {
  const int r = a.rank;
  if (r < 0 || r > kMaxBits) return cudaErrorInvalidValue;
  const int64_t n = int64_t(1) << r;
  if (r < kTile) {
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    permute_small_kernel<float2><<<blocks, 256, 0, s>>>(in, out, a);
    return cudaGetLastError();
  }
  TileMap m{};
  tile_map(a, &m);
  const int64_t n_tiles = n >> kTile;
  const int blocks = (int)std::min<int64_t>(n_tiles, 152 * 8);
  permute_tiled_kernel<<<blocks, kThreads, 0, s>>>(in, out, m, n_tiles);
  return cudaGetLastError();
}

namespace {
bool tile_map(const PermuteArgs &a, TileMap *mp) {
  TileMap &m = *mp;
  const int r = a.rank;
  int inv[kMaxBits];
  for (int p = 0; p < r; p++) inv[a.perm[p]] = p;
  m.r = r;
  // load order: input bits 0..kW-1, then input bits feeding output bits
  // 0..kW-1, then the next lowest input bits until the tile has kTile bits
  bool in_tile[kMaxBits] = {};
  int u = 0;
  for (int b = 0; b < kW; b++) {
    m.uin[u++] = (int8_t)b;
    in_tile[b] = true;
  }
  for (int p = 0; p < kW; p++)
    if (!in_tile[(int)a.perm[p]]) {
      m.uin[u++] = a.perm[p];
      in_tile[(int)a.perm[p]] = true;
    }
  for (int b = 0; b < r && u < kTile; b++)
    if (!in_tile[b]) {
      m.uin[u++] = (int8_t)b;
      in_tile[b] = true;
    }
  m.u = u;
  // store order: tile members by increasing output bit
  int k = 0;
  for (int p = 0; p < r; p++)
    if (in_tile[(int)a.perm[p]]) {
      m.vout[k] = (int8_t)p;
      for (int j = 0; j < u; j++)
        if (m.uin[j] == a.perm[p]) m.vsrc[k] = (int8_t)j;
      k++;
    }
  int j = 0;
  for (int b = 0; b < r; b++)
    if (!in_tile[b]) {
      m.rin[j] = (int8_t)b;
      m.rout[j] = (int8_t)inv[b];
      j++;
    }
  return true;
}
}  // namespace

}  // namespace dev
}  // namespace tz
