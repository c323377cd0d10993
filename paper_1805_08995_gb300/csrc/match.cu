// Matching of image pairs: Steps 1-4 of Sec. 3.1, the tau threshold of Sec. 5
// and the epipolar band of Sec. 6.2 (Eq. 1-2), fused in one kernel.
//
// Work item = (pair, tile of TPB queries of the query image); thread = query.
// The candidate image is streamed through shared memory in chunks of JC
// features: its 128-bit codes (16 B each) and the chunk's lookup tables.
// For each table the thread walks the bucket of its query and, per
// candidate, forms the key (Hamming << 24 | candidate index); the KC smallest
// distinct keys are kept in registers by a branch-free insertion network that
// also drops a key equal to one already kept (the same candidate met through
// another table), so the candidate set is a set as Step 1 requires and ties
// are broken by the smaller index.  Then each warp computes the exact
// squared distances of its 32 queries' k candidates with 8 lanes per
// 128-byte row (d = |a|^2 + |b|^2 - 2 a.b, dp4a on uint8, exact in int32),
// and each thread applies Lowe's ratio test den^2 d1 < num^2 d2.
#include "internal.h"

namespace chx {

template <int KC>
__device__ __forceinline__ void topk_insert(uint32_t (&top)[KC], uint32_t k) {
#pragma unroll
  for (int s = 0; s < KC; ++s) {
    const uint32_t t = top[s];
    const bool dup = (t == k);
    top[s] = min(t, k);
    k = dup ? KEY_INF : max(t, k);
  }
}

__host__ __device__ inline size_t match_smem_bytes(uint32_t T, bool epi, int KC, int TPB) {
  size_t scan = (size_t)JC * 16 + (size_t)T * (OFF_STRIDE + JC) * 2 + (epi ? (size_t)JC * 8 : 0);
  size_t fin = (size_t)2 * KC * TPB * 4;
  return scan > fin ? scan : fin;
}

template <int KC, int TPB, bool EPI>
__global__ void __launch_bounds__(TPB, 1) k_match(MatchArgs a, int persistent) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ uint32_t s_item;
  const KParams kp = a.kp;
  const uint32_t T = kp.n_tables;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint4* codes_s = reinterpret_cast<uint4*>(smem);
  uint16_t* tab_s = reinterpret_cast<uint16_t*>(smem + (size_t)JC * 16);
  float2* kp_s = reinterpret_cast<float2*>(smem + (size_t)JC * 16 + (size_t)T * (OFF_STRIDE + JC) * 2);
  constexpr bool epi = EPI;
  const double dd = kp.epi_px * kp.epi_px;

  for (uint32_t round = 0;; ++round) {
    uint32_t it;
    if (persistent) {
      __syncthreads();
      if (tid == 0) s_item = atomicAdd(a.item_ctr, 1u);
      __syncthreads();
      it = s_item;
    } else {
      if (round > 0) break;
      it = blockIdx.x;
    }
    if (it >= a.n_items) break;
    const uint2 item = a.items[it];
    const PairInfo P = a.pairs[item.x];
    const uint32_t q = item.y + tid;
    const bool valid = q < P.nA;
    uint4 qc = make_uint4(0u, 0u, 0u, 0u);
    uint2 qb = make_uint2(0u, 0u);
    double la = 0.0, lb = 0.0, lc = 0.0, rhs = 0.0;
    if (valid) {
      qc = __ldg(reinterpret_cast<const uint4*>(a.codes) + P.a0 + q);
      qb = __ldg(reinterpret_cast<const uint2*>(a.buckets) + P.a0 + q);
      if (epi) {
        // Sec. 6.2: epipolar line l_q = F p_q of the query in the candidate image
        const double* F = a.F + 9 * (size_t)item.x;
        const float2 pq = __ldg(reinterpret_cast<const float2*>(a.kpts) + P.a0 + q);
        const double x = (double)pq.x, y = (double)pq.y;
        la = __dadd_rn(__dadd_rn(__dmul_rn(F[0], x), __dmul_rn(F[1], y)), F[2]);
        lb = __dadd_rn(__dadd_rn(__dmul_rn(F[3], x), __dmul_rn(F[4], y)), F[5]);
        lc = __dadd_rn(__dadd_rn(__dmul_rn(F[6], x), __dmul_rn(F[7], y)), F[8]);
        rhs = __dmul_rn(dd, __dadd_rn(__dmul_rn(la, la), __dmul_rn(lb, lb)));
      }
    }
    uint32_t top[KC];
#pragma unroll
    for (int s = 0; s < KC; ++s) top[s] = KEY_INF;

    const uint32_t nch = (P.nB + JC - 1) / JC;
    for (uint32_t c = 0; c < nch; ++c) {
      const uint32_t len = min((uint32_t)JC, P.nB - c * JC);
      __syncthreads();
      {  // stage the chunk's codes, lookup tables (and key-points)
        const uint4* gc = reinterpret_cast<const uint4*>(a.codes) + P.b0 + (uint64_t)c * JC;
        for (uint32_t i = tid; i < len; i += TPB) codes_s[i] = __ldg(gc + i);
        const uint4* gt = reinterpret_cast<const uint4*>(a.tables + (uint64_t)(P.bchunk0 + c) * chunk_bytes(T));
        uint4* st = reinterpret_cast<uint4*>(tab_s);
        const uint32_t noff = T * (OFF_STRIDE / 8);
        for (uint32_t i = tid; i < noff; i += TPB) st[i] = __ldg(gt + i);
        const uint32_t n16 = (len + 7) / 8;
        for (uint32_t i = tid; i < T * n16; i += TPB) {
          const uint32_t t = i / n16, r = i - t * n16;
          const uint32_t o = noff + t * (JC / 8) + r;
          st[o] = __ldg(gt + o);
        }
        if (epi) {
          const float2* gk = reinterpret_cast<const float2*>(a.kpts) + P.b0 + (uint64_t)c * JC;
          for (uint32_t i = tid; i < len; i += TPB) kp_s[i] = __ldg(gk + i);
        }
      }
      __syncthreads();
      if (valid) {
        const uint32_t cb = c * JC;
        const uint16_t* il0 = tab_s + T * OFF_STRIDE;
        for (uint32_t t = 0; t < T; ++t) {
          // Step 1: the query's bucket in table t
          const uint32_t v = (t < 4 ? (qb.x >> (8 * t)) : (qb.y >> (8 * (t - 4)))) & 0xFFu;
          const uint32_t s0 = tab_s[t * OFF_STRIDE + v], s1 = tab_s[t * OFF_STRIDE + v + 1];
          const uint16_t* il = il0 + t * JC;
          for (uint32_t pos = s0; pos < s1; ++pos) {
            const uint32_t jl = il[pos];
            const uint4 cc = codes_s[jl];
            // Step 2: Hamming distance of the n-bit remapping codes
            const uint32_t h = __popc(cc.x ^ qc.x) + __popc(cc.y ^ qc.y) + __popc(cc.z ^ qc.z) + __popc(cc.w ^ qc.w);
            uint32_t key = (h << 24) | (cb + jl);
            if (h > kp.tau) key = KEY_INF;  // Sec. 5
            if (epi && key != KEY_INF) {    // Sec. 6.2 Eq. 1-2, squared
              const float2 pc = kp_s[jl];
              const double num = __dadd_rn(__dadd_rn(__dmul_rn(la, (double)pc.x), __dmul_rn(lb, (double)pc.y)), lc);
              if (!(__dmul_rn(num, num) <= rhs)) key = KEY_INF;
            }
            // Step 3: keep the KC smallest distinct keys
            if (key < top[KC - 1]) topk_insert<KC>(top, key);
          }
        }
      }
    }

    // Step 4: exact squared distances of the k ranked candidates
    __syncthreads();
    uint32_t* key_s = reinterpret_cast<uint32_t*>(smem);
    uint32_t* dist_s = key_s + KC * TPB;
#pragma unroll
    for (int s = 0; s < KC; ++s) key_s[s * TPB + tid] = valid ? top[s] : KEY_INF;
    __syncwarp();
    const uint32_t K = kp.top_k;
    const uint32_t wbase = warp * 32;
    const int grp = lane >> 3, sub = lane & 7;
    for (uint32_t t0 = 0; t0 < 32 * K; t0 += 4) {
      const uint32_t task = t0 + grp;
      const uint32_t qq = task & 31, s = task >> 5;
      const uint32_t key = (s < K) ? key_s[s * TPB + wbase + qq] : KEY_INF;
      uint32_t dot = 0;
      uint64_t fa = 0, fb = 0;
      if (key != KEY_INF) {
        fa = P.a0 + item.y + wbase + qq;
        fb = P.b0 + (key & 0xFFFFFFu);
        const uint4 av = __ldg(reinterpret_cast<const uint4*>(a.desc + fa * DIM) + sub);
        const uint4 bv = __ldg(reinterpret_cast<const uint4*>(a.desc + fb * DIM) + sub);
        dot = __dp4a(av.x, bv.x, dot);
        dot = __dp4a(av.y, bv.y, dot);
        dot = __dp4a(av.z, bv.z, dot);
        dot = __dp4a(av.w, bv.w, dot);
      }
      dot += __shfl_xor_sync(0xFFFFFFFFu, dot, 1);
      dot += __shfl_xor_sync(0xFFFFFFFFu, dot, 2);
      dot += __shfl_xor_sync(0xFFFFFFFFu, dot, 4);
      if (sub == 0 && key != KEY_INF) dist_s[s * TPB + wbase + qq] = __ldg(a.sqnorm + fa) + __ldg(a.sqnorm + fb) - 2u * dot;
    }
    __syncwarp();
    bool matched = false;
    uint32_t j1 = NO_MATCH;
    if (valid) {
      uint32_t nv = 0, d1 = 0xFFFFFFFFu, d2 = 0xFFFFFFFFu;
      for (uint32_t s = 0; s < K; ++s) {
        const uint32_t key = key_s[s * TPB + tid];
        if (key == KEY_INF) continue;
        ++nv;
        const uint32_t d = dist_s[s * TPB + tid], j = key & 0xFFFFFFu;
        if (d < d1 || (d == d1 && j < j1)) {
          d2 = d1;
          d1 = d;
          j1 = j;
        } else if (d < d2) {
          d2 = d;
        }
      }
      // Lowe's ratio test on distances, strict: sqrt(d1) < (num/den) sqrt(d2)
      matched = nv >= 2 && (uint64_t)kp.ratio_den * kp.ratio_den * d1 < (uint64_t)kp.ratio_num * kp.ratio_num * d2;
      a.res[P.qbase + q] = matched ? j1 : NO_MATCH;
    }
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, matched);
    if (lane == 0 && bal) atomicAdd(a.pair_cnt + item.x, (unsigned long long)__popc(bal));
  }
}

template <int KC, int TPB, bool EPI>
static cudaError_t launch_epi(const MatchArgs& a, int persistent, uint32_t grid, cudaStream_t s) {
  static int attr_dev = -1;  // the shared-memory opt-in is set once per device
  const size_t smem = match_smem_bytes(a.kp.n_tables, EPI, KC, TPB);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (attr_dev != dev) {
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_match<KC, TPB, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 1024);
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  k_match<KC, TPB, EPI><<<grid, TPB, smem, s>>>(a, persistent);
  return cudaGetLastError();
}

template <int KC, int TPB>
static cudaError_t launch_one(const MatchArgs& a, int persistent, uint32_t grid, cudaStream_t s) {
  if (a.kp.epi_px >= 0.0) return launch_epi<KC, TPB, true>(a, persistent, grid, s);
  return launch_epi<KC, TPB, false>(a, persistent, grid, s);
}

int match_tile_size(uint32_t top_k, int persistent) {
  if (!persistent) return 256;
  if (top_k <= 10) return 1024;
  if (top_k <= 16) return 512;
  return 256;
}

cudaError_t launch_match(const MatchArgs& a, int persistent, uint32_t grid, cudaStream_t s) {
  if (grid == 0 || a.n_items == 0) return cudaSuccess;
  const uint32_t k = a.kp.top_k;
  if (!persistent) {
    if (k <= 4) return launch_one<4, 256>(a, 0, grid, s);
    if (k <= 8) return launch_one<8, 256>(a, 0, grid, s);
    if (k <= 10) return launch_one<10, 256>(a, 0, grid, s);
    if (k <= 16) return launch_one<16, 256>(a, 0, grid, s);
    return launch_one<32, 256>(a, 0, grid, s);
  }
  if (k <= 4) return launch_one<4, 1024>(a, 1, grid, s);
  if (k <= 8) return launch_one<8, 1024>(a, 1, grid, s);
  if (k <= 10) return launch_one<10, 1024>(a, 1, grid, s);
  if (k <= 16) return launch_one<16, 512>(a, 1, grid, s);
  return launch_one<32, 256>(a, 1, grid, s);
}

// ---------------------------------------------------------------------------
// Output compaction: exclusive scan of per-pair counts, then a stable
// per-pair compaction of the per-query results (ascending query index).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_scan_counts(const unsigned long long* __restrict__ cnt, uint32_t P,
                                                      uint64_t* __restrict__ off, uint64_t cap,
                                                      uint32_t* __restrict__ status,
                                                      unsigned long long* __restrict__ total) {
  __shared__ unsigned long long ws[32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint32_t per = (P + 1023) / 1024;
  const uint32_t b = min(P, tid * per), e = min(P, b + per);
  unsigned long long s = 0;
  for (uint32_t i = b; i < e; ++i) s += cnt[i];
  unsigned long long incl = s;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long o = __shfl_up_sync(0xFFFFFFFFu, incl, d);
    if (lane >= d) incl += o;
  }
  if (lane == 31) ws[w] = incl;
  __syncthreads();
  if (w == 0) {
    unsigned long long x = ws[lane], y = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long o = __shfl_up_sync(0xFFFFFFFFu, y, d);
      if (lane >= d) y += o;
    }
    ws[lane] = y - x;  // exclusive prefix of warp totals
    if (lane == 31) {
      off[P] = y;
      *total = y;
      if (y > cap) atomicOr(status, DST_OVERFLOW);
    }
  }
  __syncthreads();
  unsigned long long run = ws[w] + incl - s;
  for (uint32_t i = b; i < e; ++i) {
    off[i] = run;
    run += cnt[i];
  }
}

__global__ void __launch_bounds__(256) k_compact(const PairInfo* __restrict__ pairs, const uint32_t* __restrict__ res,
                                                 const uint64_t* __restrict__ off, uint32_t* __restrict__ matches,
                                                 uint64_t cap) {
  __shared__ uint32_t wsum[8];
  const uint32_t p = blockIdx.x;
  const PairInfo pi = pairs[p];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint64_t base = off[p];
  uint64_t run = 0;
  for (uint32_t q0 = 0; q0 < pi.nA; q0 += 256) {
    const uint32_t q = q0 + tid;
    const uint32_t r = q < pi.nA ? res[pi.qbase + q] : NO_MATCH;
    const bool f = r != NO_MATCH;
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, f);
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    uint32_t woff = 0, tot = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t x = wsum[k];
      if (k < w) woff += x;
      tot += x;
    }
    if (f) {
      const uint64_t pos = base + run + woff + __popc(bal & ((1u << lane) - 1u));
      if (pos < cap) {
        matches[2 * pos] = q;
        matches[2 * pos + 1] = r;
      }
    }
    run += tot;
    __syncthreads();
  }
}

cudaError_t launch_scan_counts(const unsigned long long* pair_cnt, uint32_t P, uint64_t* match_off, uint64_t cap,
                               uint32_t* status, unsigned long long* total, cudaStream_t s) {
  k_scan_counts<<<1, 1024, 0, s>>>(pair_cnt, P, match_off, cap, status, total);
  return cudaGetLastError();
}

cudaError_t launch_compact(const PairInfo* pairs, uint32_t P, const uint32_t* res, const uint64_t* match_off,
                           uint32_t* matches, uint64_t cap, cudaStream_t s) {
  if (P == 0) return cudaSuccess;
  k_compact<<<P, 256, 0, s>>>(pairs, res, match_off, matches, cap);
  return cudaGetLastError();
}

}  // namespace chx
