// Helpers shared by the large-block kernels (trace_big.cu, trace_big64.cu):
// the bounded grid barrier of the persistent cooperative launches and the
// tile orders.
#pragma once

#include <cstdint>

#include "tc_ptx.cuh"

namespace ctq {
namespace bigc {

__device__ __forceinline__ int rup(int x, int m) { return (x + m - 1) / m * m; }

// Grid barrier with a bounded wait (sense reversal on a generation word).
__device__ __forceinline__ bool grid_sync(unsigned* count, volatile unsigned* gen, uint64_t timeout_ns) {
  __syncthreads();
  __shared__ int ok_s;
  if (threadIdx.x == 0) {
    ok_s = 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(count, 1u) == gridDim.x - 1) {
      *count = 0;
      __threadfence();
      atomicAdd(const_cast<unsigned*>(gen), 1u);
    } else {
      const uint64_t t0 = ptx::globaltimer();
      while (*gen == g) {
        if (ptx::globaltimer() - t0 > timeout_ns) {
          ok_s = 0;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok_s != 0;
}

// Tile (row mt, column nt) of linear tile index t in a product of n_mt x n_nt
// tiles: order 0 column-major (consecutive CTAs share a B tile), 1 row-major
// (they share an A tile), 2 groups of 8 column tiles, row-major inside a group.
__device__ __forceinline__ void tile_coords(int t, int n_mt, int n_nt, int order, int& mt, int& nt) {
  if (order == 1) {
    mt = t / n_nt;
    nt = t - mt * n_nt;
  } else if (order == 2) {
    constexpr int G = 8;
    const int g = t / (G * n_mt);
    const int width = min(G, n_nt - g * G);
    const int local = t - g * G * n_mt;
    mt = local / width;
    nt = g * G + (local - mt * width);
  } else {
    nt = t / n_mt;
    mt = t - nt * n_mt;
  }
}

}  // namespace bigc
}  // namespace ctq
