// Bit permutation of a complex64 tensor (every index has dimension 2, so a
// tensor transpose is a permutation of the bits of the element offset).
// Tiled through shared memory: a tile spans the 5 lowest input bits and the
// input bits that land on the 5 lowest output bits (topped up to 10 bits),
// so both the loads and the stores move runs of >= 32 consecutive elements.
#include <algorithm>

#include "kernels.h"

namespace tz {
namespace dev {

namespace {

constexpr int kW = 5;       // bits of a contiguous run on either side
constexpr int kTile = 10;   // bits of a tile (1024 elements, 8 KB)

struct TileMap {
  int r, u;                 // tensor rank, tile bits
  int8_t uin[kTile];        // input bit of tile bit j (load order)
  int8_t vout[kTile];       // output bit of tile bit j (store order)
  int8_t vsrc[kTile];       // store-order tile bit j -> load-order tile bit
  int8_t rin[kMaxBits];     // input bit of tile-index bit j
  int8_t rout[kMaxBits];    // output bit of tile-index bit j
};

__global__ void permute_small_kernel(const float2 *__restrict__ in, float2 *__restrict__ out, PermuteArgs a) {
  const int64_t n = int64_t(1) << a.rank;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = 0;
    for (int p = 0; p < a.rank; p++) i |= ((o >> p) & 1) << a.perm[p];
    out[o] = in[i];
  }
}

__global__ void __launch_bounds__(256) permute_tiled_kernel(const float2 *__restrict__ in, float2 *__restrict__ out,
                                                            TileMap m, int64_t n_tiles) {
  __shared__ float2 tile[1 << kTile];
  const int nt = 1 << m.u;
  const int nr = m.r - m.u;
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    int64_t bin = 0, bout = 0;
    for (int j = 0; j < nr; j++) {
      const int64_t b = (t >> j) & 1;
      bin |= b << m.rin[j];
      bout |= b << m.rout[j];
    }
    for (int e = threadIdx.x; e < nt; e += blockDim.x) {
      int64_t off = bin;
      for (int j = 0; j < m.u; j++) off |= int64_t((e >> j) & 1) << m.uin[j];
      tile[e] = in[off];
    }
    __syncthreads();
    for (int f = threadIdx.x; f < nt; f += blockDim.x) {
      int64_t off = bout;
      int e = 0;
      for (int j = 0; j < m.u; j++) {
        const int b = (f >> j) & 1;
        off |= int64_t(b) << m.vout[j];
        e |= b << m.vsrc[j];
      }
      out[off] = tile[e];
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_permute(const float2 *in, float2 *out, const PermuteArgs &a, cudaStream_t s) {
  const int r = a.rank;
  if (r < 0 || r > kMaxBits) return cudaErrorInvalidValue;
  const int64_t n = int64_t(1) << r;
  if (r <= kTile) {
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    permute_small_kernel<<<blocks, 256, 0, s>>>(in, out, a);
    return cudaGetLastError();
  }
  int inv[kMaxBits];
  for (int p = 0; p < r; p++) inv[a.perm[p]] = p;
  TileMap m{};
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
    if (!in_tile[a.perm[p]]) {
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
  const int64_t n_tiles = n >> u;
  const int blocks = (int)std::min<int64_t>(n_tiles, 152 * 16);
  permute_tiled_kernel<<<blocks, 256, 0, s>>>(in, out, m, n_tiles);
  return cudaGetLastError();
}

}  // namespace dev
}  // namespace tz
