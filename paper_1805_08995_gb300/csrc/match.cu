// Matching of image pairs: Steps 1-4 of Sec. 3.1, the tau threshold of Sec. 6
// and the epipolar band of Sec. 7.2 (Eq. 1-2), fused in one kernel.
//
// Work item = (pair, tile of TPB queries of the query image); thread = query.
// The candidate image is streamed through shared memory in chunks of JC
// features: its 128-bit codes (16 B each) and the chunk's lookup tables.
// For each table the thread walks the bucket of its query and, per
// candidate, forms the key (Hamming << 24 | candidate index).  The k
// smallest distinct keys are the ranked candidates of Step 3: distinct
// because a point met through several tables is one candidate (Step 1 is a
// set), and ordered by (Hamming, index).
//
// Two forms of the selection:
//  * direct (one pair per launch): every key below the current k-th key goes
//    through a branch-free insertion network in registers that also drops a
//    key equal to one already kept;
//  * speculative (batched): the hot loop only appends keys below a threshold
//    to the thread's survivor queue in global memory (L2-resident).  The
//    threshold is per pair: without the band a plan's first launch starts
//    from the calibrated guess of k_join_calibrate (sampled queries), and
//    every launch raises it to the largest k-th Hamming distance any tile of
//    the pair has produced (kept across launches); a
//    typical query then keeps about a tenth of its candidates, and the
//    insertion network runs once per query over the survivors.  Exactness never depends on the guess: a
//    query whose survivors hold fewer than k distinct keys while some
//    candidate was turned away is marked PENDING and re-matched exactly by
//    k_match_fallback.  A full queue is folded into the registers at once and
//    the threshold tightened to the exact k-th key.
// Then each warp computes the exact squared distances of its 32 queries' k
// candidates with 8 lanes per 128-byte row (d = |a|^2 + |b|^2 - 2 a.b, dp4a
// on uint8, exact in int32), and each thread applies Lowe's ratio test
// den^2 d1 < num^2 d2 (Step 4, Sec. 5.2).
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

template <int KC>
__device__ __forceinline__ uint32_t topk_kth(const uint32_t (&top)[KC], uint32_t K) {
  uint32_t v = KEY_INF;
#pragma unroll
  for (int s = 0; s < KC; ++s)
    if ((uint32_t)s + 1 == K) v = top[s];
  return v;
}

__host__ __device__ inline size_t match_smem_bytes(uint32_t T, bool epi, int KC, int TPB) {
  size_t scan = (size_t)JC * 16 + (size_t)T * (OFF_STRIDE + JC) * 2 + (epi ? (size_t)JC * 8 : 0);
  size_t fin = (size_t)2 * KC * TPB * 4;
  return scan > fin ? scan : fin;
}

__device__ __forceinline__ uint32_t hamming128(uint4 a, uint4 b) {
  return __popc(a.x ^ b.x) + __popc(a.y ^ b.y) + __popc(a.z ^ b.z) + __popc(a.w ^ b.w);
}

template <int KC, int TPB, bool EPI, bool SPEC>
__global__ void __launch_bounds__(TPB, (TPB <= 512 ? 2 : 1)) k_match(MatchArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ uint32_t s_item, s_tau, s_tau_next;
  __shared__ PairInfo s_P;
  const KParams kp = a.kp;
  const uint32_t T = kp.n_tables;
  const uint32_t K = kp.top_k;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint4* codes_s = reinterpret_cast<uint4*>(smem);
  uint16_t* tab_s = reinterpret_cast<uint16_t*>(smem + (size_t)JC * 16);
  float2* kp_s = reinterpret_cast<float2*>(smem + (size_t)JC * 16 + (size_t)T * (OFF_STRIDE + JC) * 2);
  const double dd = kp.epi_px * kp.epi_px;
  // Sec. 6: candidates farther than tau are not candidates at all
  const uint32_t thr_user = kp.tau < kp.code_bits ? ((kp.tau + 1u) << 24) : KEY_INF;
  const bool filtered = EPI || thr_user != KEY_INF;
  uint32_t* qreg = nullptr;
  if (SPEC) qreg = a.queue + ((size_t)blockIdx.x * TPB + tid) * QCAP;

  for (;;) {
    __syncthreads();
    if (tid == 0) {
      const uint32_t it0 = atomicAdd(a.item_ctr, 1u);
      s_item = it0;
      if (it0 < a.n_items) {
        const uint2 item0 = a.items[it0];
        s_P = a.pairs[item0.x];
        if (SPEC) s_tau = *reinterpret_cast<volatile uint32_t*>(a.tau_pair + item0.x);
      }
      if (SPEC) s_tau_next = 0;
    }
    __syncthreads();
    const uint32_t it = s_item;
    if (it >= a.n_items) break;
    const uint2 item = a.items[it];
    const PairInfo P = s_P;
    const uint32_t q = item.y + tid;
    const bool valid = q < P.nA;
    uint4 qc = make_uint4(0u, 0u, 0u, 0u);
    uint2 qb = make_uint2(0u, 0u);
    EpiQ eq{};
    if (valid) {
      qc = __ldg(reinterpret_cast<const uint4*>(a.codes) + P.a0 + q);
      qb = __ldg(reinterpret_cast<const uint2*>(a.buckets) + P.a0 + q);
      if (EPI) eq = epi_query(a.F + 9 * (size_t)item.x, __ldg(reinterpret_cast<const float2*>(a.kpts) + P.a0 + q), dd);
    }
    uint32_t top[KC];
#pragma unroll
    for (int s = 0; s < KC; ++s) top[s] = KEY_INF;
    uint32_t thr = thr_user;
    uint32_t cnt = 0, nflushed = 0, nlook = 0;
    if (SPEC) {
      const uint32_t ts = s_tau;  // 0: no guess yet; else threshold + 1
      if (ts != 0 && ts <= kp.code_bits) thr = min(thr, ts << 24);
    }

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
        if (EPI) {
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
          if (SPEC) nlook += s1 - s0;
          for (uint32_t pos = s0; pos < s1; ++pos) {
            const uint32_t jl = il[pos];
            // Step 2: Hamming distance of the n-bit remapping codes
            const uint32_t h = hamming128(codes_s[jl], qc);
            uint32_t key = (h << 24) | (cb + jl);
            if (key >= thr_user) key = KEY_INF;                                 // Sec. 6
            if (EPI && key != KEY_INF && !epi_keep_fast(eq, kp_s[jl])) key = KEY_INF;  // Sec. 7.2
            if (SPEC) {
              if (filtered && key == KEY_INF) --nlook;
              const bool keep = key < thr;
              st_global_if(qreg + cnt, key, keep);  // cnt < QCAP here
              cnt += keep ? 1u : 0u;
              if (cnt == QCAP) {  // fold a full queue into the registers, tighten the threshold
                for (uint32_t e = 0; e < QCAP; ++e) {
                  const uint32_t k2 = qreg[e];
                  if (k2 < top[KC - 1]) topk_insert<KC>(top, k2);
                }
                nflushed += QCAP;
                cnt = 0;
                thr = min(thr, top[KC - 1]);
              }
            } else {
              // Step 3: keep the KC smallest distinct keys
              if (key < top[KC - 1]) topk_insert<KC>(top, key);
            }
          }
        }
      }
    }

    bool pending = false;
    if (SPEC && valid) {
      for (uint32_t e = 0; e < cnt; ++e) {
        const uint32_t k2 = qreg[e];
        if (k2 < top[KC - 1]) topk_insert<KC>(top, k2);
      }
      const uint32_t kth = topk_kth<KC>(top, K);
      // fewer than k distinct survivors although a candidate was turned away
      pending = kth == KEY_INF && nlook > nflushed + cnt;
      if (kth != KEY_INF) atomicMax(&s_tau_next, (kth >> 24) + 1u);
    }

    // Step 4 (Sec. 5.2): exact squared distances of the k ranked candidates
    __syncthreads();
    uint32_t* key_s = reinterpret_cast<uint32_t*>(smem);
    uint32_t* dist_s = key_s + KC * TPB;
#pragma unroll
    for (int s = 0; s < KC; ++s) key_s[s * TPB + tid] = (valid && !pending) ? top[s] : KEY_INF;
    __syncwarp();
    const uint32_t wbase = warp * 32;
    const int grp = lane >> 3, sub = lane & 7;
    // 8 lanes per 128-byte row; each group of 8 lanes takes one query and
    // issues the loads of DB rows at once (independent, so their latencies overlap)
    constexpr int DB = 5;
    for (uint32_t qq0 = 0; qq0 < 32; qq0 += 4) {
      const uint32_t qq = qq0 + grp;
      const uint32_t qi = wbase + qq;
      const bool has = key_s[qi] != KEY_INF;  // slot 0 filled <=> the query has candidates
      const uint64_t fa = P.a0 + item.y + qi;
      uint4 av = make_uint4(0u, 0u, 0u, 0u);
      if (has) av = __ldg(reinterpret_cast<const uint4*>(a.desc + fa * DIM) + sub);
      for (uint32_t s0 = 0; s0 < K; s0 += DB) {
        uint32_t key[DB];
        uint4 bv[DB];
#pragma unroll
        for (int d = 0; d < DB; ++d) {
          key[d] = (has && s0 + d < K) ? key_s[(s0 + d) * TPB + qi] : KEY_INF;
          bv[d] = make_uint4(0u, 0u, 0u, 0u);
          if (key[d] != KEY_INF)
            bv[d] = __ldg(reinterpret_cast<const uint4*>(a.desc + (P.b0 + (key[d] & 0xFFFFFFu)) * DIM) + sub);
        }
#pragma unroll
        for (int d = 0; d < DB; ++d) {
          uint32_t dot = 0;
          dot = __dp4a(av.x, bv[d].x, dot);
          dot = __dp4a(av.y, bv[d].y, dot);
          dot = __dp4a(av.z, bv[d].z, dot);
          dot = __dp4a(av.w, bv[d].w, dot);
          dot += __shfl_xor_sync(0xFFFFFFFFu, dot, 1);
          dot += __shfl_xor_sync(0xFFFFFFFFu, dot, 2);
          dot += __shfl_xor_sync(0xFFFFFFFFu, dot, 4);
          if (sub == 0 && key[d] != KEY_INF) {
            const uint64_t fb = P.b0 + (key[d] & 0xFFFFFFu);
            dist_s[(s0 + d) * TPB + qi] = __ldg(a.sqnorm + fa) + __ldg(a.sqnorm + fb) - 2u * dot;
          }
        }
      }
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
      matched = ratio_ok(kp, nv, d1, d2);
      a.res[P.qbase + q] = pending ? PENDING : (matched ? j1 : NO_MATCH);
    }
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, matched);
    if (lane == 0 && bal) atomicAdd(a.pair_cnt + item.x, (unsigned long long)__popc(bal));
    if (SPEC) {
      __syncthreads();
      if (tid == 0 && s_tau_next && !a.tau_fixed) atomicMax(a.tau_pair + item.x, s_tau_next);
    }
  }
}

// ---------------------------------------------------------------------------
// Exact fallback for PENDING queries, one warp per query.  Warps stream the
// per-query result array (128 entries per step, coalesced); for each PENDING
// entry the warp finds its pair with a 32-way search over the pairs' first
// result index, then walks the query's buckets in the chunked lookup tables
// with the lanes side by side.  Each lane keeps the k smallest distinct keys
// it met; the warp merges them by k rounds of minimum extraction (equal keys
// of several lanes leave together, so a point met through several tables
// counts once), k lanes compute the exact distances and lane 0 applies the
// ratio test.
// ---------------------------------------------------------------------------
// One query g of the per-query result array, by one warp (exact): the pair
// holding g, the query's buckets walked with the lanes side by side, the
// merge of the lanes' k smallest distinct keys, distances and the ratio test.
template <int KC, bool EPI>
__device__ __forceinline__ void fallback_query(const MatchArgs& a, uint64_t g, int lane, uint32_t thr_user,
                                               double dd) {
  const KParams& kp = a.kp;
  const uint32_t T = kp.n_tables, K = kp.top_k;
  // pair: the last with qbase <= g.  32-way search; invariant: pairs[lo].qbase <= g
  // and the answer lies in [lo, hi].  Lane l probes lo + 1 + l * span / 32.
  uint32_t lo = 0, hi = a.n_pairs - 1;
  while (lo < hi) {
    const uint32_t lo0 = lo, span = hi - lo;
    const uint32_t piv = lo0 + 1u + (uint32_t)(((uint64_t)lane * span) / 32u);  // in [lo + 1, hi]
    const uint32_t m = __ballot_sync(0xFFFFFFFFu, a.pairs[piv].qbase <= g);  // a prefix of the lanes
    if (m == 0u) {
      hi = lo0;
    } else {
      const int l = 31 - __clz(m);  // lane l + 1 probes a later pair, past g
      lo = lo0 + 1u + (uint32_t)(((uint64_t)l * span) / 32u);
      if (l < 31) hi = lo0 + (uint32_t)(((uint64_t)(l + 1) * span) / 32u);
    }
  }
  const PairInfo P = a.pairs[lo];
  const uint32_t q = (uint32_t)(g - P.qbase);
  const uint4 qc = __ldg(reinterpret_cast<const uint4*>(a.codes) + P.a0 + q);
  const uint2 qb = __ldg(reinterpret_cast<const uint2*>(a.buckets) + P.a0 + q);
  EpiQ eq{};
  if (EPI) eq = epi_query(a.F + 9 * (size_t)lo, __ldg(reinterpret_cast<const float2*>(a.kpts) + P.a0 + q), dd);
  uint32_t top[KC];
#pragma unroll
  for (int s = 0; s < KC; ++s) top[s] = KEY_INF;
  const uint32_t nch = (P.nB + JC - 1) / JC;
  for (uint32_t c = 0; c < nch; ++c) {
    const uint16_t* blk =
        reinterpret_cast<const uint16_t*>(a.tables + (uint64_t)(P.bchunk0 + c) * chunk_bytes(T));
    const uint4* gc = reinterpret_cast<const uint4*>(a.codes) + P.b0 + (uint64_t)c * JC;
    for (uint32_t t = 0; t < T; ++t) {
      const uint32_t v = (t < 4 ? (qb.x >> (8 * t)) : (qb.y >> (8 * (t - 4)))) & 0xFFu;
      const uint32_t s0 = blk[t * OFF_STRIDE + v], s1 = blk[t * OFF_STRIDE + v + 1];
      const uint16_t* il = blk + T * OFF_STRIDE + t * JC;
      for (uint32_t pos = s0 + lane; pos < s1; pos += 32) {
        const uint32_t jl = il[pos];
        const uint32_t key = (hamming128(__ldg(gc + jl), qc) << 24) | (c * JC + jl);
        if (key >= thr_user) continue;
        if (EPI && !epi_keep_fast(eq, __ldg(reinterpret_cast<const float2*>(a.kpts) + P.b0 + (uint64_t)c * JC + jl)))
          continue;
        if (key < top[KC - 1]) topk_insert<KC>(top, key);
      }
    }
  }
  // merge: round r leaves the r-th smallest distinct key in lane r
  uint32_t mine = KEY_INF;
  for (uint32_t r = 0; r < K; ++r) {
    uint32_t m = top[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
    if (m == KEY_INF) break;  // warp-uniform
    if ((uint32_t)lane == r) mine = m;
    if (top[0] == m) {
#pragma unroll
      for (int s = 0; s + 1 < KC; ++s) top[s] = top[s + 1];
      top[KC - 1] = KEY_INF;
    }
  }
  // exact distances of the k ranked candidates (Step 4), ratio test
  const uint64_t fa = P.a0 + q;
  uint64_t dj = ~0ull;  // (d << 32) | j
  if (mine != KEY_INF) {
    const uint32_t j = mine & 0xFFFFFFu;
    const uint64_t fb = P.b0 + j;
    const uint4* arow = reinterpret_cast<const uint4*>(a.desc + fa * DIM);
    const uint4* brow = reinterpret_cast<const uint4*>(a.desc + fb * DIM);
    uint32_t dot = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const uint4 av = __ldg(arow + w), bv = __ldg(brow + w);
      dot = __dp4a(av.x, bv.x, dot);
      dot = __dp4a(av.y, bv.y, dot);
      dot = __dp4a(av.z, bv.z, dot);
      dot = __dp4a(av.w, bv.w, dot);
    }
    const uint32_t d = __ldg(a.sqnorm + fa) + __ldg(a.sqnorm + fb) - 2u * dot;
    dj = ((uint64_t)d << 32) | j;
  }
  const uint32_t nv = __popc(__ballot_sync(0xFFFFFFFFu, mine != KEY_INF));
  uint64_t best = dj;  // smallest (d, j)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xFFFFFFFFu, best, o));
  uint64_t second = dj == best ? ~0ull : dj;  // keys are distinct, so exactly one lane holds best
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) second = min(second, __shfl_xor_sync(0xFFFFFFFFu, second, o));
  if (lane == 0) {
    const uint32_t d1 = (uint32_t)(best >> 32), j1 = (uint32_t)best, d2 = (uint32_t)(second >> 32);
    const bool matched = ratio_ok(kp, nv, d1, d2);
    a.res[g] = matched ? j1 : NO_MATCH;
    if (matched) atomicAdd(a.pair_cnt + lo, 1ull);
  }
}

template <int KC, bool EPI>
__global__ void __launch_bounds__(128) k_match_fallback(MatchArgs a) {
  const KParams kp = a.kp;
  const uint32_t thr_user = kp.tau < kp.code_bits ? ((kp.tau + 1u) << 24) : KEY_INF;
  const double dd = kp.epi_px * kp.epi_px;
  const int lane = threadIdx.x & 31;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarp = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  if (a.all_queries) {  // every query, one warp each (the exact warp-per-query configuration)
    for (uint64_t g = warp; g < a.n_res; g += nwarp) {
      fallback_query<KC, EPI>(a, g, lane, thr_user, dd);
      __syncwarp();
    }
    return;
  }
  for (uint64_t g0 = warp * 128; g0 < a.n_res; g0 += nwarp * 128) {
    uint32_t pend[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint64_t g = g0 + 32 * i + lane;
      pend[i] = __ballot_sync(0xFFFFFFFFu, g < a.n_res && a.res[g] == PENDING);
    }
#pragma unroll 1
    for (int i = 0; i < 4; ++i) {
      while (pend[i]) {
        const int b = __ffs(pend[i]) - 1;
        pend[i] &= pend[i] - 1u;
        fallback_query<KC, EPI>(a, g0 + 32 * i + b, lane, thr_user, dd);
        __syncwarp();
      }
    }
  }
}

// ---------------------------------------------------------------------------
// launch plumbing
// ---------------------------------------------------------------------------
namespace {

template <int KC, int TPB, bool EPI, bool SPEC>
cudaError_t run_match(const MatchArgs* a, uint32_t grid, cudaStream_t s, uint32_t* occ) {
  static int attr_dev = -1;  // the shared-memory opt-in is set once per device
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (attr_dev != dev) {
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_match<KC, TPB, EPI, SPEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 1024);
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  const uint32_t T = a ? a->kp.n_tables : (occ ? *occ : 6u);
  const size_t smem = match_smem_bytes(T, EPI, KC, TPB);
  if (occ) {
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_match<KC, TPB, EPI, SPEC>, TPB, smem);
    *occ = (uint32_t)(nb > 0 ? nb : 1);
    return e;
  }
  k_match<KC, TPB, EPI, SPEC><<<grid, TPB, smem, s>>>(*a);
  return cudaGetLastError();
}

template <int KC, int TPB>
cudaError_t run_kc(const MatchArgs* a, int spec, bool epi, uint32_t grid, cudaStream_t s, uint32_t* occ) {
  if (spec) return epi ? run_match<KC, TPB, true, true>(a, grid, s, occ) : run_match<KC, TPB, false, true>(a, grid, s, occ);
  return epi ? run_match<KC, TPB, true, false>(a, grid, s, occ) : run_match<KC, TPB, false, false>(a, grid, s, occ);
}

// Queries per CTA of the speculative form: 512 (k <= 16 only) or 256.
uint32_t spec_tpb(uint32_t k, uint32_t tile) {
  if (k > 16) return 256;
  return tile == 256 ? 256u : 512u;
}

cudaError_t dispatch(uint32_t k, const MatchArgs* a, int spec, bool epi, uint32_t grid, cudaStream_t s, uint32_t* occ,
                     uint32_t tile) {
  if (!spec) {
    if (k <= 4) return run_kc<4, 256>(a, 0, epi, grid, s, occ);
    if (k <= 8) return run_kc<8, 256>(a, 0, epi, grid, s, occ);
    if (k <= 10) return run_kc<10, 256>(a, 0, epi, grid, s, occ);
    if (k <= 16) return run_kc<16, 256>(a, 0, epi, grid, s, occ);
    return run_kc<32, 256>(a, 0, epi, grid, s, occ);
  }
  if (spec_tpb(k, tile) == 256) {
    if (k <= 4) return run_kc<4, 256>(a, 1, epi, grid, s, occ);
    if (k <= 8) return run_kc<8, 256>(a, 1, epi, grid, s, occ);
    if (k <= 10) return run_kc<10, 256>(a, 1, epi, grid, s, occ);
    if (k <= 16) return run_kc<16, 256>(a, 1, epi, grid, s, occ);
    return run_kc<32, 256>(a, 1, epi, grid, s, occ);
  }
  if (k <= 4) return run_kc<4, 512>(a, 1, epi, grid, s, occ);
  if (k <= 8) return run_kc<8, 512>(a, 1, epi, grid, s, occ);
  if (k <= 10) return run_kc<10, 512>(a, 1, epi, grid, s, occ);
  return run_kc<16, 512>(a, 1, epi, grid, s, occ);
}

}  // namespace

int match_tile_size(uint32_t top_k, int spec, uint32_t tile) {
  if (!spec) return 256;
  return (int)spec_tpb(top_k, tile);
}

uint32_t match_grid(uint32_t top_k, int spec, bool epi, uint32_t n_tables, uint32_t n_items, uint32_t tile) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  uint32_t occ = n_tables;
  if (dispatch(top_k, nullptr, spec, epi, 0, 0, &occ, tile) != cudaSuccess) {
    cudaGetLastError();
    occ = 1;
  }
  const uint64_t g = (uint64_t)nsm * occ;
  return (uint32_t)(n_items < g ? n_items : g);
}

cudaError_t launch_match(const MatchArgs& a, int spec, uint32_t grid, cudaStream_t s, uint32_t tile) {
  if (grid == 0 || a.n_items == 0) return cudaSuccess;
  return dispatch(a.kp.top_k, &a, spec, a.kp.epi_px >= 0.0, grid, s, nullptr, tile);
}

cudaError_t launch_match_fallback(const MatchArgs& a, cudaStream_t s) {
  if (a.n_res == 0 || a.n_pairs == 0) return cudaSuccess;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t want = a.all_queries ? (a.n_res + 3) / 4 : (a.n_res + 127) / 128;  // 4 warps per CTA
  const unsigned grid = (unsigned)(want < (uint64_t)nsm * 16 ? want : (uint64_t)nsm * 16);
  const bool epi = a.kp.epi_px >= 0.0;
  const uint32_t k = a.kp.top_k;
#define CHX_FB(KC)                                                              \
  do {                                                                          \
    if (epi) k_match_fallback<KC, true><<<grid, 128, 0, s>>>(a);               \
    else k_match_fallback<KC, false><<<grid, 128, 0, s>>>(a);                  \
  } while (0)
  if (k <= 4) CHX_FB(4);
  else if (k <= 8) CHX_FB(8);
  else if (k <= 10) CHX_FB(10);
  else if (k <= 16) CHX_FB(16);
  else CHX_FB(32);
#undef CHX_FB
  return cudaGetLastError();
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

template <int NT>
__global__ void __launch_bounds__(NT) k_compact(const PairInfo* __restrict__ pairs, const uint32_t* __restrict__ res,
                                                const uint64_t* __restrict__ off, uint32_t* __restrict__ matches,
                                                uint64_t cap) {
  constexpr int NW = NT / 32;
  __shared__ uint32_t wsum[NW];
  const uint32_t p = blockIdx.x;
  const PairInfo pi = pairs[p];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint64_t base = off[p];
  uint64_t run = 0;
  for (uint32_t q0 = 0; q0 < pi.nA; q0 += NT) {
    const uint32_t q = q0 + tid;
    const uint32_t r = q < pi.nA ? res[pi.qbase + q] : NO_MATCH;
    const bool f = r < PENDING;
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, f);
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    uint32_t woff = 0, tot = 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
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
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // one CTA per pair; a list of fewer pairs than SMs takes CTAs of 1024 threads (fewer steps each)
  if (P < (uint32_t)nsm) k_compact<1024><<<P, 1024, 0, s>>>(pairs, res, match_off, matches, cap);
  else k_compact<256><<<P, 256, 0, s>>>(pairs, res, match_off, matches, cap);
  return cudaGetLastError();
}

}  // namespace chx
