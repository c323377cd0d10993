// Device helpers shared by the two bucket-join kernels (mma.sync form in
// join.cu, tcgen05 form in join_tc.cu): the top-k insertion network, the view
// of one image's bucket-sorted table, the per-pair Hamming threshold and the
// finalisation of a pair's survivor lists.
#pragma once

#include <cuda_fp16.h>

#include "internal.h"

namespace chx {

constexpr int JT = 256;  // threads of a join CTA (one query per thread in the finalisation)

template <int KC>
__device__ __forceinline__ void jt_insert(uint32_t (&top)[KC], uint32_t k) {
#pragma unroll
  for (int s = 0; s < KC; ++s) {
    const uint32_t t = top[s];
    const bool dup = (t == k);
    top[s] = min(t, k);
    k = dup ? KEY_INF : max(t, k);
  }
}

template <int KC>
__device__ __forceinline__ uint32_t jt_kth(const uint32_t (&top)[KC], uint32_t K) {
  uint32_t v = KEY_INF;
#pragma unroll
  for (int s = 0; s < KC; ++s)
    if ((uint32_t)s + 1 == K) v = top[s];
  return v;
}

__device__ __forceinline__ uint32_t jt_hamming(uint4 a, uint4 b) {
  return __popc(a.x ^ b.x) + __popc(a.y ^ b.y) + __popc(a.z ^ b.z) + __popc(a.w ^ b.w);
}

struct JView {  // one image's bucket-sorted table t
  const uint32_t* off;
  const uint32_t* idx;
  const uint4* rec;
};

__device__ __forceinline__ JView jview(const uint8_t* join, uint64_t base, uint32_t n, uint32_t t) {
  const uint8_t* b = join + base + (uint64_t)t * join_block(n);
  JView v;
  v.off = reinterpret_cast<const uint32_t*>(b);
  v.idx = reinterpret_cast<const uint32_t*>(b + 1040);
  v.rec = reinterpret_cast<const uint4*>(b + 1040 + 4 * ((n + 3) / 4 * 4));
  return v;
}

// Hamming threshold for a pair: the 99.5th percentile of the k-th distances
// seen so far (histogram kept across launches), else the calibration / host
// hint; 0 = none.  Computed by warp 0.
__device__ __forceinline__ uint32_t pair_threshold(const MatchArgs& a, uint32_t p, int lane) {
  const uint32_t* h = a.jhist + (size_t)p * HBINS;
  uint32_t v[5], tot = 0;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const uint32_t b = lane * 5 + k;  // lanes own 5 consecutive bins
    v[k] = b < HBINS ? *reinterpret_cast<const volatile uint32_t*>(h + b) : 0u;
    tot += v[k];
  }
  uint32_t incl = tot;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, incl, d);
    if (lane >= d) incl += o;
  }
  const uint32_t all = __shfl_sync(0xFFFFFFFFu, incl, 31);
  uint32_t guess = *reinterpret_cast<const volatile uint32_t*>(a.tau_pair + p);
  if (!a.tau_fixed && all >= 64) {
    const uint32_t want = all - all / 200;  // 99.5 %
    uint32_t run = incl - tot, bin = 0xFFFFFFFFu;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      run += v[k];
      if (bin == 0xFFFFFFFFu && run >= want) bin = lane * 5 + k;
    }
    uint32_t best = bin;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xFFFFFFFFu, best, o));
    if (best != 0xFFFFFFFFu) guess = best + 1u;
  }
  return guess;
}

// Finalisation of one pair (one thread per query, JT threads): the k
// smallest distinct survivors of each query's list (Step 3), exact squared
// distances of those k with 4 lanes per 128-byte row (Step 4, Sec. 5.2) and
// Lowe's ratio test.  A query whose list overflowed, or that holds fewer than
// k survivors while the guess may have turned a candidate away (cut), is left
// PENDING for the exact fallback.  key_s / dist_s: KC * JT words each.
template <int KC, bool EPI>
__device__ __forceinline__ void join_finalise(const MatchArgs& a, const PairInfo& P, uint32_t it, bool cut,
                                              const uint32_t* cnt_s, const uint32_t* seg, uint32_t* key_s,
                                              uint32_t* dist_s, uint32_t* s_hist) {
  const KParams& kp = a.kp;
  const uint32_t T = kp.n_tables, K = kp.top_k;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (uint32_t q0 = 0; q0 < P.nA; q0 += JT) {
    const uint32_t q = q0 + tid;
    const bool valid = q < P.nA;
    uint32_t top[KC];
#pragma unroll
    for (int s = 0; s < KC; ++s) top[s] = KEY_INF;
    bool pending = false;
    if (valid) {
      const uint32_t n = cnt_s[q];
      pending = n > JSEG;  // survivors were dropped
      const uint4* ql = reinterpret_cast<const uint4*>(seg + (size_t)q * JSEG);
      const uint32_t m = min(n, JSEG);
      // the next 16 survivors are loaded while the current 16 are inserted; a key at or above
      // the list's last entry when its group starts cannot enter it
      const uint4 INF4 = make_uint4(KEY_INF, KEY_INF, KEY_INF, KEY_INF);
      uint4 x[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) x[i] = 4 * i < m ? ql[i] : INF4;
      for (uint32_t e0 = 0; e0 < m; e0 += 16) {
        uint4 y[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) y[i] = e0 + 16 + 4 * i < m ? ql[(e0 + 16) / 4 + i] : INF4;
        const uint32_t lim = top[KC - 1];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const uint32_t kk[4] = {x[i].x, x[i].y, x[i].z, x[i].w};
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (e0 + 4 * i + u < m && kk[u] < lim) jt_insert<KC>(top, kk[u]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) x[i] = y[i];
      }
      const uint32_t kth = jt_kth<KC>(top, K);
      if (!pending && kth == KEY_INF && cut) {
        // fewer than k: exact only if no candidate was turned away by the guess
        const uint2 qbk = __ldg(reinterpret_cast<const uint2*>(a.buckets) + P.a0 + q);
        uint32_t nlook = 0;
        for (uint32_t t = 0; t < T; ++t) {
          const JView B = jview(a.join, P.bjoin, P.nB, t);
          const uint32_t v = (t < 4 ? (qbk.x >> (8 * t)) : (qbk.y >> (8 * (t - 4)))) & 0xFFu;
          nlook += __ldg(B.off + v + 1) - __ldg(B.off + v);
        }
        pending = nlook > n;
      }
      if (!EPI && !pending && kth != KEY_INF && !a.tau_fixed) atomicAdd(s_hist + (kth >> 24), 1u);
    }
#pragma unroll
    for (int s = 0; s < KC; ++s) key_s[s * JT + tid] = (valid && !pending) ? top[s] : KEY_INF;
    __syncwarp();
    // 4 lanes per 128-byte row (32 bytes each), 8 queries per step, the k rows in flight
    const uint32_t wbase = warp * 32;
    const int grp = lane >> 2, sub = lane & 3;
    constexpr int DB = KC <= 10 ? (KC + 1) / 2 : 8;  // rows in flight per batch (measured: 5 of 10 is fastest)
    for (uint32_t qq0 = 0; qq0 < 32; qq0 += 8) {
      const uint32_t qi = wbase + qq0 + grp;
      const bool has = key_s[qi] != KEY_INF;
      const uint64_t fa = P.a0 + q0 + qi;
      const uint4* arow = reinterpret_cast<const uint4*>(a.desc + fa * DIM) + 2 * sub;
      uint4 av0 = make_uint4(0u, 0u, 0u, 0u), av1 = av0;
      if (has) {
        av0 = __ldg(arow);
        av1 = __ldg(arow + 1);
      }
      for (uint32_t s0 = 0; s0 < K; s0 += DB) {
        uint32_t key[DB];
        uint4 bv0[DB], bv1[DB];
#pragma unroll
        for (int d = 0; d < DB; ++d) {
          key[d] = (has && s0 + d < K) ? key_s[(s0 + d) * JT + qi] : KEY_INF;
          bv0[d] = bv1[d] = make_uint4(0u, 0u, 0u, 0u);
          if (key[d] != KEY_INF) {
            const uint4* brow = reinterpret_cast<const uint4*>(a.desc + (P.b0 + (key[d] & 0xFFFFFFu)) * DIM) + 2 * sub;
            bv0[d] = __ldg(brow);
            bv1[d] = __ldg(brow + 1);
          }
        }
#pragma unroll
        for (int d = 0; d < DB; ++d) {
          uint32_t dot = 0;
          dot = __dp4a(av0.x, bv0[d].x, dot);
          dot = __dp4a(av0.y, bv0[d].y, dot);
          dot = __dp4a(av0.z, bv0[d].z, dot);
          dot = __dp4a(av0.w, bv0[d].w, dot);
          dot = __dp4a(av1.x, bv1[d].x, dot);
          dot = __dp4a(av1.y, bv1[d].y, dot);
          dot = __dp4a(av1.z, bv1[d].z, dot);
          dot = __dp4a(av1.w, bv1[d].w, dot);
          dot += __shfl_xor_sync(0xFFFFFFFFu, dot, 1);
          dot += __shfl_xor_sync(0xFFFFFFFFu, dot, 2);
          if (sub == 0 && key[d] != KEY_INF) {
            const uint64_t fb = P.b0 + (key[d] & 0xFFFFFFu);
            dist_s[(s0 + d) * JT + qi] = __ldg(a.sqnorm + fa) + __ldg(a.sqnorm + fb) - 2u * dot;
          }
        }
      }
    }
    __syncwarp();
    bool matched = false;
    if (valid) {
      uint32_t nv = 0, d1 = 0xFFFFFFFFu, d2 = 0xFFFFFFFFu, j1 = NO_MATCH;
      for (uint32_t s = 0; s < K; ++s) {
        const uint32_t key = key_s[s * JT + tid];
        if (key == KEY_INF) continue;
        ++nv;
        const uint32_t d = dist_s[s * JT + tid], j = key & 0xFFFFFFu;
        if (d < d1 || (d == d1 && j < j1)) {
          d2 = d1;
          d1 = d;
          j1 = j;
        } else if (d < d2) {
          d2 = d;
        }
      }
      matched = ratio_ok(kp, nv, d1, d2);
      a.res[P.qbase + q] = pending ? PENDING : (matched ? j1 : NO_MATCH);
    }
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, matched);
    if (lane == 0 && bal) atomicAdd(a.pair_cnt + it, (unsigned long long)__popc(bal));
    __syncwarp();
  }
}

}  // namespace chx
