// Mutual check (a reading beyond the paper, CASHASH_FLAG_MUTUAL): a plan with
// the flag matches its P pairs (A, B) and, as pairs P..2P-1, their reversals
// (B, A).  Reversed, the epipolar constraint x_B^T F x_A = 0 reads
// x_A^T F^T x_B = 0, so the band of the reverse pair uses F transposed.
// After both directions are matched, a forward match q -> j is kept only when
// the reverse result of j is q.
#include "internal.h"

namespace chx {

// F2[i] = F[i], F2[P + i] = F[i]^T (row-major 3 x 3).
__global__ void k_mutual_F(const double* __restrict__ F, uint32_t P, double* __restrict__ F2) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < 9ull * P;
       e += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = e / 9;
    const uint32_t r = (uint32_t)(e % 9) / 3, c = (uint32_t)(e % 9) % 3;
    const double v = F[e];
    F2[e] = v;
    F2[9ull * (P + i) + 3 * c + r] = v;
  }
}

// One CTA per forward pair (grid-stride): queries whose match j does not
// match back are set to NO_MATCH and the pair's count is lowered.  Reverse
// results are only read, forward results only written by their own thread.
__global__ void __launch_bounds__(256) k_mutual(const PairInfo* __restrict__ pairs, uint32_t P,
                                                uint32_t* __restrict__ res, unsigned long long* __restrict__ pair_cnt) {
  __shared__ uint32_t s_drop[8];
  for (uint32_t i = blockIdx.x; i < P; i += gridDim.x) {
    const PairInfo f = pairs[i], r = pairs[P + i];
    uint32_t drop = 0;
    for (uint32_t q = threadIdx.x; q < f.nA; q += blockDim.x) {
      const uint32_t j = res[f.qbase + q];
      if (j < PENDING && j < r.nA && res[r.qbase + j] != q) {
        res[f.qbase + q] = NO_MATCH;
        ++drop;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) drop += __shfl_xor_sync(0xFFFFFFFFu, drop, o);
    if ((threadIdx.x & 31) == 0) s_drop[threadIdx.x >> 5] = drop;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t t = 0;
      for (uint32_t w = 0; w < blockDim.x / 32; ++w) t += s_drop[w];
      if (t) atomicAdd(pair_cnt + i, (unsigned long long)(-(long long)t));
    }
    __syncthreads();
  }
}

cudaError_t launch_mutual_F(const double* F, uint32_t P, double* F2, cudaStream_t s) {
  if (P == 0) return cudaSuccess;
  const uint64_t n = 9ull * P;
  const unsigned grid = (unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_mutual_F<<<grid, 256, 0, s>>>(F, P, F2);
  return cudaGetLastError();
}

cudaError_t launch_mutual(const PairInfo* pairs, uint32_t P, uint32_t* res, unsigned long long* pair_cnt,
                          cudaStream_t s) {
  if (P == 0) return cudaSuccess;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = P < (uint32_t)nsm * 8 ? P : (unsigned)nsm * 8;
  k_mutual<<<grid, 256, 0, s>>>(pairs, P, res, pair_cnt);
  return cudaGetLastError();
}

}  // namespace chx
