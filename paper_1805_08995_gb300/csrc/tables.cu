// Lookup tables of Step 1 (Sec. 3.1): for each candidate image, each table t
// and each m-bit short code v, the list of points whose code in table t is v.
//
// Layout (private to the library): each image's features are cut into chunks
// of JC features; chunk k (numbered over the whole set) occupies
// chunk_bytes(T) bytes at tables + k * chunk_bytes(T):
//   uint16 off[T][OFF_STRIDE]  bucket v of table t holds local indices
//                              idx[t][off[t][v] .. off[t][v+1])
//   uint16 idx[T][JC]          local feature indices (0..JC-1), ascending
//                              within a bucket (stable counting sort)
// A chunk is staged whole into shared memory by the matcher.
#include "internal.h"

namespace chx {

// One warp per (chunk, table).
__global__ void __launch_bounds__(256) k_build_tables(const uint8_t* __restrict__ buckets,
                                                      const uint64_t* __restrict__ chunk_feat0,
                                                      const uint32_t* __restrict__ chunk_len, uint32_t n_chunks,
                                                      uint32_t T, uint8_t* __restrict__ tables) {
  __shared__ uint32_t cur_all[8][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint64_t task = (uint64_t)blockIdx.x * 8 + w;
  if (task >= (uint64_t)n_chunks * T) return;  // whole warp leaves together
  const uint32_t c = (uint32_t)(task / T), t = (uint32_t)(task % T);
  const uint64_t f0 = chunk_feat0[c];
  const uint32_t len = chunk_len[c];
  uint16_t* base = reinterpret_cast<uint16_t*>(tables + (uint64_t)c * chunk_bytes(T));
  uint16_t* off = base + (size_t)t * OFF_STRIDE;
  uint16_t* idx = base + (size_t)T * OFF_STRIDE + (size_t)t * JC;
  uint32_t* cur = cur_all[w];
#pragma unroll
  for (int k = 0; k < 8; ++k) cur[lane * 8 + k] = 0;
  __syncwarp();
  for (uint32_t j = lane; j < len; j += 32) atomicAdd(&cur[buckets[(f0 + j) * 8 + t]], 1u);
  __syncwarp();
  // exclusive scan of the 256 counts: lane owns 8 consecutive buckets
  uint32_t v[8], run = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    v[k] = run;
    run += cur[lane * 8 + k];
  }
  uint32_t incl = run;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, incl, d);
    if (lane >= d) incl += o;
  }
  const uint32_t excl = incl - run;
  __syncwarp();
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    off[lane * 8 + k] = (uint16_t)(excl + v[k]);
    cur[lane * 8 + k] = excl + v[k];
  }
  if (lane == 31) off[256] = (uint16_t)incl;
  __syncwarp();
  // stable scatter in feature order
  const uint32_t lt = (1u << lane) - 1u;
  for (uint32_t j0 = 0; j0 < len; j0 += 32) {
    const uint32_t j = j0 + lane;
    const bool valid = j < len;
    const uint32_t b = valid ? (uint32_t)buckets[(f0 + j) * 8 + t] : 256u + lane;
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, b);
    const uint32_t rank = __popc(peers & lt);
    uint32_t pos = 0;
    if (valid) pos = cur[b] + rank;
    __syncwarp();
    if (valid) {
      idx[pos] = (uint16_t)j;
      if (rank == 0) cur[b] += __popc(peers);
    }
    __syncwarp();
  }
}

// Bucket-sorted tables with inline codes: one warp per (image, table), a
// stable counting sort over the whole image.
__global__ void __launch_bounds__(256) k_build_join(const uint8_t* __restrict__ buckets,
                                                    const uint32_t* __restrict__ codes,
                                                    const uint64_t* __restrict__ img_f0,
                                                    const uint32_t* __restrict__ img_n,
                                                    const uint64_t* __restrict__ img_join, uint32_t n_images,
                                                    uint32_t T, uint8_t* __restrict__ join) {
  __shared__ uint32_t cur_all[8][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint64_t task = (uint64_t)blockIdx.x * 8 + w;
  if (task >= (uint64_t)n_images * T) return;  // whole warp leaves together
  const uint32_t im = (uint32_t)(task / T), t = (uint32_t)(task % T);
  const uint64_t f0 = img_f0[im];
  const uint32_t n = img_n[im];
  uint8_t* blk = join + img_join[im] + (uint64_t)t * join_block(n);
  uint32_t* off = reinterpret_cast<uint32_t*>(blk);
  uint32_t* idx = reinterpret_cast<uint32_t*>(blk + 1040);
  uint4* rec = reinterpret_cast<uint4*>(blk + 1040 + 4 * ((n + 3) / 4 * 4));
  uint32_t* cur = cur_all[w];
#pragma unroll
  for (int k = 0; k < 8; ++k) cur[lane * 8 + k] = 0;
  __syncwarp();
  for (uint32_t j = lane; j < n; j += 32) atomicAdd(&cur[buckets[(f0 + j) * 8 + t]], 1u);
  __syncwarp();
  uint32_t v[8], run = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    v[k] = run;
    run += cur[lane * 8 + k];
  }
  uint32_t incl = run;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, incl, d);
    if (lane >= d) incl += o;
  }
  const uint32_t excl = incl - run;
  __syncwarp();
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    off[lane * 8 + k] = excl + v[k];
    cur[lane * 8 + k] = excl + v[k];
  }
  if (lane == 31) off[256] = incl;
  __syncwarp();
  const uint32_t lt = (1u << lane) - 1u;
  const uint4* cd = reinterpret_cast<const uint4*>(codes) + f0;
  for (uint32_t j0 = 0; j0 < n; j0 += 32) {
    const uint32_t j = j0 + lane;
    const bool valid = j < n;
    const uint32_t b = valid ? (uint32_t)buckets[(f0 + j) * 8 + t] : 256u + lane;
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, b);
    const uint32_t rank = __popc(peers & lt);
    uint32_t pos = 0;
    if (valid) pos = cur[b] + rank;
    __syncwarp();
    if (valid) {
      idx[pos] = j;
      rec[pos] = __ldg(cd + j);
      if (rank == 0) cur[b] += __popc(peers);
    }
    __syncwarp();
  }
}

cudaError_t launch_build_join(const uint8_t* buckets, const uint32_t* codes, const uint64_t* img_f0,
                              const uint32_t* img_n, const uint64_t* img_join, uint32_t n_images, uint32_t n_tables,
                              uint8_t* join, cudaStream_t s) {
  const uint64_t tasks = (uint64_t)n_images * n_tables;
  if (tasks == 0) return cudaSuccess;
  k_build_join<<<(unsigned)((tasks + 7) / 8), 256, 0, s>>>(buckets, codes, img_f0, img_n, img_join, n_images,
                                                          n_tables, join);
  return cudaGetLastError();
}

cudaError_t launch_build_tables(const uint8_t* buckets, const uint64_t* chunk_feat0, const uint32_t* chunk_len,
                                uint32_t n_chunks, uint32_t n_tables, uint8_t* tables, cudaStream_t s) {
  const uint64_t tasks = (uint64_t)n_chunks * n_tables;
  if (tasks == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((tasks + 7) / 8);
  k_build_tables<<<grid, 256, 0, s>>>(buckets, chunk_feat0, chunk_len, n_chunks, n_tables, tables);
  return cudaGetLastError();
}

}  // namespace chx
