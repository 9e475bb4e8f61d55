// sectors.cuh -- total-S^z sector weights of a state (sm_103a).
#pragma once
#include "kernels.cuh"

namespace spinrp {

// ---------------------------------------------------------------------------
// Total-S^z sector weights n_k = sum over x with k bits set of |psi_x|^2,
// k = 0..M (k = number of up spins; every Hamiltonian of the paper conserves
// them).  The physical layout permutes bits, so the count of set bits of a
// physical index equals that of its logical index.  A block walks chunks of
// 2^13 amplitudes: thread t takes x = chunk + t + 256 j, j = 0..31, so
// popcount(x) = popcount(chunk) + popcount(t) + popcount(j) over disjoint
// bit fields; each thread sums its 32 weights by popcount(j) (six FP64
// registers), the block adds them into 14 sub-bins popcount(t) + i by warp
// trees and a fixed-order sum over warps, then into the bins of the chunk.
// Everything is summed in a fixed order: the result is reproducible.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256)
sector_kernel(const typename CT<R>::T *__restrict__ psi, int M, double *__restrict__ part, int nblk) {
  __shared__ double s_w[8][14];
  __shared__ double s_bins[kMaxM + 1];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int k = t; k <= M; k += 256) s_bins[k] = 0.0;
  const uint64_t N = 1ull << M;
  const uint64_t nchunks = (N + 8191) >> 13;
  const int pt = __popc(t);
  for (uint64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const uint64_t x0 = c << 13;
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const uint64_t x = x0 + (uint64_t)t + 256ull * j;
      if (x < N) {
        const typename CT<R>::T v = psi[x];
        acc[(j & 1) + ((j >> 1) & 1) + ((j >> 2) & 1) + ((j >> 3) & 1) + ((j >> 4) & 1)] +=
            (double)v.x * v.x + (double)v.y * v.y;
      }
    }
    // sub-bin s = popcount(t) + i
    for (int sb = 0; sb < 14; ++sb) {
      const int i = sb - pt;
      double v = 0.0;
#pragma unroll
      for (int q = 0; q < 6; ++q)
        if (q == i) v = acc[q];
      for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) s_w[warp][sb] = v;
    }
    __syncthreads();
    if (t < 14) {
      double v = 0.0;
      for (int w = 0; w < 8; ++w) v += s_w[w][t];
      const int k = (int)__popcll(x0) + t;
      if (k <= M) s_bins[k] += v;
    }
    __syncthreads();
  }
  for (int k = t; k <= M; k += 256) part[(size_t)k * nblk + blockIdx.x] = s_bins[k];
}

// n_k = sum of the nblk block rows of column k in a fixed order (block k).
__global__ void __launch_bounds__(256)
sector_finalize_kernel(const double *__restrict__ part, int nblk, double *__restrict__ out) {
  const double *__restrict__ col = part + (size_t)blockIdx.x * nblk;
  double v = 0.0;
  for (int r = threadIdx.x; r < nblk; r += blockDim.x) v += col[r];
  __shared__ double s[256];
  s[threadIdx.x] = v;
  __syncthreads();
  for (int h = 128; h; h >>= 1) {
    if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = s[0];
}

}  // namespace spinrp
