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

// Stable counting sort of one (image or chunk, table) in shared memory, one
// CTA of 8 warps, for at most BJ_MAX_N features.  Warp w takes the w-th eighth
// of the features; its bucket cursors start after the earlier warps' entries
// of the same bucket, so the order within a bucket is the feature order.  The
// sorted local indices are then written out in order (and, for the join
// tables, the codes gathered behind them), so every global write is
// coalesced.
//   CHUNK = false: the join tables of image blockIdx.x / T (the join_block
//                  layout: uint32 offsets, uint32 indices, inline codes);
//   CHUNK = true:  lookup-table chunk blockIdx.x / T of the layout above.
constexpr uint32_t BJ_MAX_N = 65535;  // local indices held as uint16 in shared memory

template <bool CHUNK>
__global__ void __launch_bounds__(256) k_sort_tables(const uint8_t* __restrict__ buckets,
                                                     const uint32_t* __restrict__ codes,
                                                     const uint64_t* __restrict__ feat0,
                                                     const uint32_t* __restrict__ count,
                                                     const uint64_t* __restrict__ img_join, uint32_t T,
                                                     uint8_t* __restrict__ out) {
  extern __shared__ __align__(16) uint32_t bsm[];
  uint32_t* hist = bsm;  // [8 warps][256 buckets]
  __shared__ uint32_t s_wsum[8];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint32_t u = blockIdx.x / T, t = blockIdx.x % T;
  const uint64_t f0 = feat0[u];
  const uint32_t n = count[u];
  uint16_t* sidx = reinterpret_cast<uint16_t*>(bsm + 8 * 256);       // [n] sorted local indices
  uint8_t* sb = reinterpret_cast<uint8_t*>(sidx + (n + 7) / 8 * 8);  // [n] bucket of each feature
  for (int k = tid; k < 8 * 256; k += 256) hist[k] = 0;
  for (uint32_t j = tid; j < n; j += 256) sb[j] = buckets[(f0 + j) * 8 + t];
  __syncthreads();
  const uint32_t seg = (n + 7) / 8, j_lo = min(n, w * seg), j_hi = min(n, j_lo + seg);
  uint32_t* hw = hist + w * 256;
  for (uint32_t j = j_lo + lane; j < j_hi; j += 32) atomicAdd(&hw[sb[j]], 1u);
  __syncthreads();
  // thread b: bucket b's total, its exclusive offset over buckets, and the
  // warps' starting cursors in bucket b
  const uint32_t b = (uint32_t)tid;
  uint32_t tot = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) tot += hist[k * 256 + b];
  uint32_t incl = tot;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, incl, d);
    if (lane >= d) incl += o;
  }
  if (lane == 31) s_wsum[w] = incl;
  __syncthreads();
  uint32_t base = 0;
  for (int k = 0; k < w; ++k) base += s_wsum[k];
  const uint32_t excl = base + incl - tot;
  uint8_t* blk;
  if constexpr (CHUNK) {
    blk = out + (uint64_t)u * chunk_bytes(T);
    uint16_t* off = reinterpret_cast<uint16_t*>(blk) + (size_t)t * OFF_STRIDE;
    off[b] = (uint16_t)excl;
    if (b == 255) off[256] = (uint16_t)(excl + tot);
  } else {
    blk = out + img_join[u] + (uint64_t)t * join_block(n);
    uint32_t* off = reinterpret_cast<uint32_t*>(blk);
    off[b] = excl;
    if (b == 255) off[256] = excl + tot;
  }
  uint32_t run = excl;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint32_t c = hist[k * 256 + b];
    hist[k * 256 + b] = run;
    run += c;
  }
  __syncthreads();
  // stable scatter of each warp's range, 32 features at a time in feature order
  const uint32_t lt = (1u << lane) - 1u;
  for (uint32_t j0 = j_lo; j0 < j_hi; j0 += 32) {
    const uint32_t j = j0 + lane;
    const bool valid = j < j_hi;
    const uint32_t bk = valid ? (uint32_t)sb[j] : 256u + lane;
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, bk);
    const uint32_t rank = __popc(peers & lt);
    uint32_t pos = 0;
    if (valid) pos = hw[bk] + rank;
    __syncwarp();
    if (valid) {
      sidx[pos] = (uint16_t)j;
      if (rank == 0) hw[bk] += __popc(peers);
    }
    __syncwarp();
  }
  __syncthreads();
  if constexpr (CHUNK) {
    uint16_t* idx = reinterpret_cast<uint16_t*>(blk) + (size_t)T * OFF_STRIDE + (size_t)t * JC;
    for (uint32_t p = tid; p < n; p += 256) idx[p] = sidx[p];
  } else {
    uint32_t* idx = reinterpret_cast<uint32_t*>(blk + 1040);
    uint4* rec = reinterpret_cast<uint4*>(blk + 1040 + 4 * ((n + 3) / 4 * 4));
    const uint4* cd = reinterpret_cast<const uint4*>(codes) + f0;
    for (uint32_t p = tid; p < n; p += 256) {
      const uint32_t j = sidx[p];
      idx[p] = j;
      rec[p] = __ldg(cd + j);
    }
  }
}

static size_t sort_smem(uint32_t n_max) { return 8 * 256 * 4 + (size_t)(n_max + 7) / 8 * 8 * 3; }

// Join tables of a set with an image of more than BJ_MAX_N features: one warp
// per (image, table), a stable counting sort over the whole image with global
// scatters.
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
                              uint32_t n_max, uint8_t* join, cudaStream_t s) {
  const uint64_t tasks = (uint64_t)n_images * n_tables;
  if (tasks == 0) return cudaSuccess;
  if (tasks > 0x7FFFFFFFull) return cudaErrorInvalidValue;  // one CTA (or warp) per image and table
  if (n_max <= BJ_MAX_N) {
    static int attr_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (attr_dev != dev) {
      e = cudaFuncSetAttribute(k_sort_tables<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sort_smem(BJ_MAX_N));
      if (e != cudaSuccess) return e;
      attr_dev = dev;
    }
    k_sort_tables<false><<<(unsigned)tasks, 256, sort_smem(n_max), s>>>(buckets, codes, img_f0, img_n, img_join,
                                                                        n_tables, join);
    return cudaGetLastError();
  }
  k_build_join<<<(unsigned)((tasks + 7) / 8), 256, 0, s>>>(buckets, codes, img_f0, img_n, img_join, n_images,
                                                          n_tables, join);
  return cudaGetLastError();
}

cudaError_t launch_build_tables(const uint8_t* buckets, const uint64_t* chunk_feat0, const uint32_t* chunk_len,
                                uint32_t n_chunks, uint32_t n_tables, uint8_t* tables, cudaStream_t s) {
  const uint64_t tasks = (uint64_t)n_chunks * n_tables;
  if (tasks == 0) return cudaSuccess;
  if (tasks > 0x7FFFFFFFull) return cudaErrorInvalidValue;  // one CTA per chunk and table
  static_assert(JC <= (int)BJ_MAX_N, "chunk tables sort in shared memory");
  k_sort_tables<true><<<(unsigned)tasks, 256, sort_smem(JC), s>>>(buckets, nullptr, chunk_feat0, chunk_len, nullptr,
                                                                  n_tables, tables);
  return cudaGetLastError();
}

}  // namespace chx
