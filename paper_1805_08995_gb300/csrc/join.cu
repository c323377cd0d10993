// Batched matching as a bucket join on the tensor cores: Steps 1-4 of
// Sec. 3.1 (+ the Sec. 6 threshold tau) organised around the lookup tables.
//
// Step 1 pairs a query with exactly the candidates that share its bucket in
// some table, so for table t and short code v the work is the dense block
// (queries of A in bucket v) x (candidates of B in bucket v).  With the
// bucket-sorted tables (codes stored inline) a warp takes one (t, v) block
// and computes its Hamming distances (Step 2) as one +-1 contraction: with a
// code bit mapped to +1 / -1, the dot product of two 128-bit codes is
// 128 - 2 H.  The +-1 values are exact in FP8 (e4m3) and every partial sum is
// an integer of magnitude <= 128, so mma.m16n8k32 (FP8 in, f16 accumulators)
// gives H exactly.  The query side enters negated and the accumulators start
// at 1152, so each result is 1024 + 2 H: in [1024, 2048) an f16 has unit
// spacing, so its low ten bits are 2 H and the key needs no conversion.
// Because the Hamming distance does not depend on the order of the bits, each
// lane expands one 32-bit code word of its row / column into eight FP8
// registers (register i, byte b <- bit 8b + i); rows and columns use the same
// map.
//
// Keys H <= theta (theta: the pair's threshold guess, learned per pair from the
// k-th distances of earlier launches, capped by the Sec. 6 tau) are appended to
// the query's survivor list: a counter per query in shared memory, a list of
// JSEG entries per query in global memory.  After the scan the CTA finalises
// the pair's queries, one thread per query: the k smallest distinct survivors
// (Step 3; a point met through several tables appears once), exact squared
// distances with 8 lanes per 128-byte row (Step 4, Sec. 5.2) and Lowe's ratio test.  A
// query whose list overflowed, or that holds fewer than k distinct survivors
// while the guess turned some candidate away, is left PENDING for the exact
// fallback kernel, so results never depend on the guess.
//
// With the Sec. 7.2 band (EPI) a candidate outside the band is no candidate at
// all, so there is no Hamming guess: each entry is tested against the query's
// epipolar line (FP32 roundings of the FP64 line, computed once per query and
// pair; undecided entries in FP64) and only entries inside the band survive.
#include <cuda_fp16.h>

#include "join_common.cuh"

namespace chx {

constexpr int CAL_SAMPLES = 128;   // calibration: sampled queries per pair
constexpr uint32_t CAL_MARGIN = 1; // calibration: Hamming margin over the second largest sample

// Dynamic shared memory: survivor counters of the pair's queries, then the
// finalisation's keys and distances.
__host__ __device__ inline size_t join_smem_bytes(int KC, uint32_t na_max) {
  return (size_t)4 * ((na_max + 3) / 4 * 4) + (size_t)2 * KC * JT * 4;
}

// One 32-bit code word as eight FP8 registers of +-1 (byte b of register i is
// bit 8b + i of w; e4m3 0x38 = +1, 0xB8 = -1): bit 1 -> +1 (NEG = false) or
// -1 (NEG = true); on = false gives zeros for padding rows and columns.
template <bool NEG>
__device__ __forceinline__ void pm1_expand(uint32_t w, bool on, uint32_t (&r)[8]) {
  const uint32_t m = on ? 0x80808080u : 0u, c = on ? (NEG ? 0xB8B8B8B8u : 0x38383838u) : 0u;
#pragma unroll
  for (int i = 0; i < 8; ++i) r[i] = NEG ? (((w << (7 - i)) & m) ^ c) : (((w << (7 - i)) & m) | c);
}

// D += A (16x32, FP8) * B (32x8, FP8), f16 accumulators: d0 holds row g,
// d1 row g + 8 (columns 2 (lane % 4) and +1), g = lane / 4.
__device__ __forceinline__ void mma_pm1(uint32_t& d0, uint32_t& d1, uint32_t a0, uint32_t a1, uint32_t a2,
                                        uint32_t a3, uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k32.row.col.f16.e4m3.e4m3.f16 {%0,%1}, {%2,%3,%4,%5}, {%6,%7}, {%0,%1};"
      : "+r"(d0), "+r"(d1)
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t le_mask(uint32_t d, __half2 t) {
  __half2 h;
  memcpy(&h, &d, 4);
  return __hle2_mask(h, t);
}

constexpr uint32_t ACC0 = 0x64806480u;  // f16 (1152, 1152): results are 1024 + 2 H

// Key H << 24 | j from the low / high f16 result (bits 0x6400 + 2 H), as an integer multiply-add:
// d * 2^23 keeps (mod 2^32) only bits 1-8 of the low f16, i.e. 2 H << 23 = H << 24, and j < 2^24
// adds without carry.
__device__ __forceinline__ uint32_t key_lo(uint32_t d, uint32_t j) { return d * 0x800000u + j; }
__device__ __forceinline__ uint32_t key_hi(uint32_t d, uint32_t j) { return (d >> 16) * 0x800000u + j; }

// *(base + pos) = v and ++pos when (bits & mask) != 0: one predicate for a predicated store and a
// predicated add (survivors are sparse and scattered over the lanes, so nearly every warp has some
// in every slot position and a branch per slot would diverge).  The stores are read only after the
// CTA barrier that ends the scan.
__device__ __forceinline__ void append_if(uint32_t* base, uint32_t& pos, uint32_t bits, uint32_t mask, uint32_t v) {
  asm volatile(
      "{\n .reg .pred q;\n .reg .b32 t;\n and.b32 t, %2, %3;\n setp.ne.b32 q, t, 0;\n"
      " @q st.global.u32 [%1], %4;\n @q add.u32 %0, %0, 1;\n}"
      : "+r"(pos)
      : "l"(__cvta_generic_to_global(base + pos)), "r"(bits), "r"(mask), "r"(v));
}

// Bucket offsets of join task `task` (table task / nbk, bucket task % nbk) in
// both images; zeros past the last task.
__device__ __forceinline__ void load_offsets(const uint8_t* join, const PairInfo& P, uint64_t ablk, uint64_t bblk,
                                             uint32_t nbk, uint32_t ntask, uint32_t task, uint32_t (&o)[4]) {
  o[0] = o[1] = o[2] = o[3] = 0u;
  if (task < ntask) {
    const uint32_t t = task / nbk, v = task - t * nbk;
    const uint32_t* ao = reinterpret_cast<const uint32_t*>(join + P.ajoin + t * ablk) + v;
    const uint32_t* bo = reinterpret_cast<const uint32_t*>(join + P.bjoin + t * bblk) + v;
    o[0] = __ldg(ao);
    o[1] = __ldg(ao + 1);
    o[2] = __ldg(bo);
    o[3] = __ldg(bo + 1);
  }
}

// NTC: candidate tiles (of 8 columns) held in registers at a time.
template <int KC, bool TAU, int NTC, bool EPI>
__global__ void __launch_bounds__(JT, 2) k_join(MatchArgs a) {
  extern __shared__ __align__(16) uint8_t jsm[];
  __shared__ uint32_t s_item, s_tau, s_task, s_kx, s_ky;
  __shared__ uint32_t s_hist[HBINS];
  __shared__ PairInfo s_P;
  const KParams kp = a.kp;
  const uint32_t T = kp.n_tables, K = kp.top_k, nbk = 1u << kp.bits_per_table;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t g = (uint32_t)lane >> 2, l4 = (uint32_t)lane & 3u;
  uint32_t* cnt_s = reinterpret_cast<uint32_t*>(jsm);
  uint32_t* key_s = cnt_s + (a.na_max + 3) / 4 * 4;
  uint32_t* dist_s = key_s + KC * JT;
  uint32_t* seg = a.jqueue + (size_t)blockIdx.x * a.na_max * JSEG;
  const uint32_t h_user = TAU ? kp.tau : 128u;  // Sec. 6: keys with H > tau are no candidates
  // per query: FP32 a, b, c and the thresholds w_lo, w_hi on |a x' + b y' + c| (band_thresholds)
  float4* lines = EPI ? a.jline + (size_t)blockIdx.x * jline_stride(a.na_max) : nullptr;
  float* lhi = EPI ? reinterpret_cast<float*>(lines + a.na_max) : nullptr;
  const double dd = kp.epi_px * kp.epi_px;
  const float2* kpts = reinterpret_cast<const float2*>(a.kpts);

  for (;;) {
    __syncthreads();
    if (tid == 0) {
      const uint32_t it0 = atomicAdd(a.item_ctr, 1u);
      uint32_t p0 = 0xFFFFFFFFu;
      if (it0 < a.n_items) {
        p0 = a.items[it0].x;
        s_P = a.pairs[p0];
      }
      s_item = p0;
      s_task = 0;
      s_kx = s_ky = 0u;
    }
    for (uint32_t b = tid; b < HBINS; b += JT) s_hist[b] = 0;
    __syncthreads();
    const uint32_t it = s_item;  // pair index
    if (it == 0xFFFFFFFFu) break;
    if (warp == 0) {
      const uint32_t gs = pair_threshold(a, it, lane);
      if (lane == 0) s_tau = gs;
    }
    const PairInfo P = s_P;
    const double* Fp = EPI ? a.F + 9 * (size_t)it : nullptr;
    if constexpr (EPI) {  // max |x'|, |y'| over the candidate image (non-negative floats order as integers)
      float mx = 0.f, my = 0.f;
      for (uint32_t j = tid; j < P.nB; j += JT) {
        const float2 pc = __ldg(kpts + P.b0 + j);
        mx = fmaxf(mx, fabsf(pc.x));
        my = fmaxf(my, fabsf(pc.y));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
        my = fmaxf(my, __shfl_xor_sync(0xFFFFFFFFu, my, o));
      }
      if (lane == 0) {
        atomicMax(&s_kx, __float_as_uint(mx));
        atomicMax(&s_ky, __float_as_uint(my));
      }
      __syncthreads();
    }
    for (uint32_t q = tid; q < P.nA; q += JT) {
      cnt_s[q] = 0;
      if constexpr (EPI) {
        const EpiQ e = epi_query(Fp, __ldg(kpts + P.a0 + q), dd);
        float wlo, whi;
        band_thresholds(e, __uint_as_float(s_kx), __uint_as_float(s_ky), wlo, whi);
        lines[q] = make_float4(e.a, e.b, e.c, wlo);
        lhi[q] = whi;
      }
    }
    __syncthreads();
    // survivors: H <= h_thr
    uint32_t h_thr = h_user;
    if (!EPI) {
      const uint32_t ts = s_tau;  // 0: no guess; else threshold + 1
      if (ts != 0 && ts - 1u < h_thr) h_thr = ts - 1u;
    }
    const bool cut = h_thr < h_user;  // the guess may turn candidates away
    const __half2 t2 = __float2half2_rn(1024.f + 2.f * (float)min(h_thr, 128u));
    // the pair's two images: table t of image X starts at join + Xjoin + t * Xblk
    const uint64_t ablk = join_block(P.nA), bblk = join_block(P.nB);
    const uint64_t arec = 1040u + 4u * ((P.nA + 3) / 4 * 4), brec = 1040u + 4u * ((P.nB + 3) / 4 * 4);

    // ---- scan: (table, bucket) blocks on the tensor cores, one warp per block ----
    // The bucket offsets of the next block are loaded while the current one runs.
    const uint32_t ntask = T * nbk;
    uint32_t task = 0;
    if (lane == 0) task = atomicAdd(&s_task, 1u);
    task = __shfl_sync(0xFFFFFFFFu, task, 0);
    uint32_t ob[4];  // off_A[v], off_A[v + 1], off_B[v], off_B[v + 1] of `task`
    load_offsets(a.join, P, ablk, bblk, nbk, ntask, task, ob);
    while (task < ntask) {
      uint32_t nxt = 0;
      if (lane == 0) nxt = atomicAdd(&s_task, 1u);
      nxt = __shfl_sync(0xFFFFFFFFu, nxt, 0);
      uint32_t onx[4];
      load_offsets(a.join, P, ablk, bblk, nbk, ntask, nxt, onx);
      const uint32_t t = task / nbk;
      const uint8_t* Ab = a.join + P.ajoin + t * ablk;
      const uint8_t* Bb = a.join + P.bjoin + t * bblk;
      const uint32_t qs = ob[0], nq = ob[1] - ob[0];
      const uint32_t cs = ob[2], nc = ob[3] - ob[2];
      task = nxt;
#pragma unroll
      for (int k = 0; k < 4; ++k) ob[k] = onx[k];
      if (nq == 0 || nc == 0) continue;
      const uint32_t* Aidx = reinterpret_cast<const uint32_t*>(Ab + 1040) + qs;
      const uint32_t* Bidx = reinterpret_cast<const uint32_t*>(Bb + 1040) + cs;
      const uint32_t* Aw = reinterpret_cast<const uint32_t*>(Ab + arec) + 4 * qs + l4;
      const uint32_t* Bw = reinterpret_cast<const uint32_t*>(Bb + brec) + 4 * cs + l4;
      for (uint32_t c0 = 0; c0 < nc; c0 += 8 * NTC) {
        const uint32_t ntiles = min((uint32_t)NTC, (nc - c0 + 7) / 8);
        uint32_t bf[NTC][8], jc[NTC][2], jok = 0;  // jok bit 2n + c: column 2 (lane % 4) + c of tile n exists
#pragma unroll
        for (int n = 0; n < NTC; ++n) {
          const uint32_t col = c0 + n * 8 + g;
          const bool on = (uint32_t)n < ntiles && col < nc;
          pm1_expand<false>(on ? __ldg(Bw + (size_t)col * 4) : 0u, on, bf[n]);
          const uint32_t cc = c0 + n * 8 + 2 * l4;
          const bool o0 = (uint32_t)n < ntiles && cc < nc, o1 = (uint32_t)n < ntiles && cc + 1 < nc;
          jc[n][0] = o0 ? __ldg(Bidx + cc) : 0u;
          jc[n][1] = o1 ? __ldg(Bidx + cc + 1) : 0u;
          jok |= ((o0 ? 1u : 0u) | (o1 ? 2u : 0u)) << (2 * n);
        }
        // rows g and g + 8 of the first row tile; each iteration loads the next tile's
        uint32_t wa = g < nq ? __ldg(Aw + (size_t)g * 4) : 0u;
        uint32_t wb = g + 8 < nq ? __ldg(Aw + (size_t)(g + 8) * 4) : 0u;
        uint32_t qa = g < nq ? __ldg(Aidx + g) : 0u;
        uint32_t qb = g + 8 < nq ? __ldg(Aidx + g + 8) : 0u;
        for (uint32_t r0 = 0; r0 < nq; r0 += 16) {
          const bool va = r0 + g < nq, vb = r0 + g + 8 < nq;
          uint32_t af[8], ag[8];
          pm1_expand<true>(wa, va, af);
          pm1_expand<true>(wb, vb, ag);
          const uint32_t qa_c = qa, qb_c = qb;
          {
            const uint32_t ra = r0 + 16 + g, rb = r0 + 24 + g;
            wa = ra < nq ? __ldg(Aw + (size_t)ra * 4) : 0u;
            wb = rb < nq ? __ldg(Aw + (size_t)rb * 4) : 0u;
            qa = ra < nq ? __ldg(Aidx + ra) : 0u;
            qb = rb < nq ? __ldg(Aidx + rb) : 0u;
          }
          uint32_t d[NTC][2];
          uint32_t acc_a = 0, acc_b = 0;  // survivors: bit 2n (low f16 of tile n) and bit 17 + 2n (high)
#pragma unroll
          for (int n = 0; n < NTC; ++n) {
            d[n][0] = d[n][1] = ACC0;
            if ((uint32_t)n < ntiles) {  // warp-uniform
#pragma unroll
              for (int s = 0; s < 4; ++s)
                mma_pm1(d[n][0], d[n][1], af[2 * s], ag[2 * s], af[2 * s + 1], ag[2 * s + 1], bf[n][2 * s],
                        bf[n][2 * s + 1]);
              const uint32_t sel = (1u << (2 * n)) | (1u << (17 + 2 * n));
              acc_a |= le_mask(d[n][0], t2) & sel;
              acc_b |= le_mask(d[n][1], t2) & sel;
            }
          }
          // bit 2n + c: entry (row, column 2 (lane % 4) + c of tile n) survives
          uint32_t ka = (acc_a | (acc_a >> 16)) & 0xFFu, kb = (acc_b | (acc_b >> 16)) & 0xFFu;
          ka &= va ? jok : 0u;
          kb &= vb ? jok : 0u;
          if constexpr (EPI) {  // Sec. 7.2: only candidates inside the band
            const float4 La = va ? lines[qa_c] : make_float4(0.f, 0.f, 0.f, -1.f);
            const float4 Lb = vb ? lines[qb_c] : make_float4(0.f, 0.f, 0.f, -1.f);
            const float ha = va ? lhi[qa_c] : 0.f, hb = vb ? lhi[qb_c] : 0.f;
            uint32_t ba = 0, bb = 0, ua = 0, ub = 0;  // inside / undecided in FP32
#pragma unroll
            for (int n = 0; n < NTC; ++n)
#pragma unroll
              for (int c = 0; c < 2; ++c) {
                const int bit = 2 * n + c;
                {  // every slot, without a branch (a column past the run reads feature 0 of B; masked below)
                  const float2 pc = __ldg(kpts + P.b0 + jc[n][c]);
                  const float na = fabsf(fmaf(La.x, pc.x, fmaf(La.y, pc.y, La.z)));
                  const float nb = fabsf(fmaf(Lb.x, pc.x, fmaf(Lb.y, pc.y, Lb.z)));
                  if (na <= La.w) ba |= 1u << bit;
                  if (!(na <= La.w) && !(na >= ha)) ua |= 1u << bit;
                  if (nb <= Lb.w) bb |= 1u << bit;
                  if (!(nb <= Lb.w) && !(nb >= hb)) ub |= 1u << bit;
                }
              }
            ua &= ka;
            ub &= kb;
            if (ua | ub) {  // near the band's edge: the FP64 expression decides
#pragma unroll
              for (int n = 0; n < NTC; ++n)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                  const int bit = 2 * n + c;
                  if (((ua | ub) >> bit) & 1u) {
                    const float2 pc = __ldg(kpts + P.b0 + jc[n][c]);
                    if (((ua >> bit) & 1u) && epi_keep_fp64_F(Fp, __ldg(kpts + P.a0 + qa_c), dd, pc)) ba |= 1u << bit;
                    if (((ub >> bit) & 1u) && epi_keep_fp64_F(Fp, __ldg(kpts + P.a0 + qb_c), dd, pc)) bb |= 1u << bit;
                  }
                }
            }
            ka &= ba;
            kb &= bb;
          }
          // with tau or the band survivors are sparse, and a warp whose lanes have none skips the
          // appends (without them nearly every warp has some, and the vote would only cost)
          if (!(TAU || EPI) || __any_sync(0xFFFFFFFFu, (ka | kb) != 0u)) {
            // one counter update per row, then the row's survivors at consecutive slots
            uint32_t pa = ka ? atomicAdd(cnt_s + qa_c, (uint32_t)__popc(ka)) : 0u;
            uint32_t pb = kb ? atomicAdd(cnt_s + qb_c, (uint32_t)__popc(kb)) : 0u;
            // a row that would overflow its list stores nothing (its query is left PENDING)
            const uint32_t sta = pa + __popc(ka) <= JSEG ? ka : 0u, stb = pb + __popc(kb) <= JSEG ? kb : 0u;
            uint32_t* sa = seg + (size_t)qa_c * JSEG;
            uint32_t* sb = seg + (size_t)qb_c * JSEG;
#pragma unroll
            for (int n = 0; n < NTC; ++n)
#pragma unroll
              for (int c = 0; c < 2; ++c) {
                const int bit = 2 * n + c;
                append_if(sa, pa, sta, 1u << bit, c ? key_hi(d[n][0], jc[n][1]) : key_lo(d[n][0], jc[n][0]));
                append_if(sb, pb, stb, 1u << bit, c ? key_hi(d[n][1], jc[n][1]) : key_lo(d[n][1], jc[n][0]));
              }
          }
        }
      }
    }
    __syncthreads();

    // ---- finalise: top-k of the survivors, distances, ratio test ----
    join_finalise<KC, EPI>(a, P, it, cut, cnt_s, seg, key_s, dist_s, s_hist);
    __syncthreads();
    if (!a.tau_fixed)
      for (uint32_t b = tid; b < HBINS; b += JT)
        if (s_hist[b]) atomicAdd(a.jhist + (size_t)it * HBINS + b, s_hist[b]);
  }
}

// Threshold guess for pairs that have none yet, from CAL_SAMPLES sampled
// queries (one CTA per pair, one thread per query): the exact k-th Hamming
// distance of each, then the second largest of them plus CAL_MARGIN.  Only a
// performance hint; results never depend on it.
template <int KC, bool TAU>
__global__ void __launch_bounds__(CAL_SAMPLES) k_join_calibrate(MatchArgs a) {
  __shared__ uint32_t s_top[CAL_SAMPLES / 32][2];
  const KParams kp = a.kp;
  const uint32_t T = kp.n_tables, K = kp.top_k;
  const uint32_t thr_user = TAU ? ((kp.tau + 1u) << 24) : KEY_INF;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t p = blockIdx.x; p < a.n_pairs; p += gridDim.x) {
    if (*reinterpret_cast<volatile uint32_t*>(a.tau_pair + p) != 0) continue;  // uniform over the CTA
    const PairInfo P = a.pairs[p];
    if (P.nA == 0 || P.nB == 0) continue;
    const uint32_t q = (uint32_t)(((uint64_t)threadIdx.x * P.nA) / CAL_SAMPLES);
    const uint4 qc = __ldg(reinterpret_cast<const uint4*>(a.codes) + P.a0 + q);
    const uint2 qb = __ldg(reinterpret_cast<const uint2*>(a.buckets) + P.a0 + q);
    uint32_t top[KC];
#pragma unroll
    for (int s = 0; s < KC; ++s) top[s] = KEY_INF;
    for (uint32_t t = 0; t < T; ++t) {
      const JView B = jview(a.join, P.bjoin, P.nB, t);
      const uint32_t v = (t < 4 ? (qb.x >> (8 * t)) : (qb.y >> (8 * (t - 4)))) & 0xFFu;
      const uint32_t cs = __ldg(B.off + v), ce = __ldg(B.off + v + 1);
      for (uint32_t c = cs; c < ce; ++c) {
        const uint32_t key = (jt_hamming(__ldg(B.rec + c), qc) << 24) | __ldg(B.idx + c);
        if (TAU && key >= thr_user) continue;
        if (key < top[KC - 1]) jt_insert<KC>(top, key);
      }
    }
    const uint32_t kth = jt_kth<KC>(top, K);
    const uint32_t hk = kth == KEY_INF ? 0xFFFFFFFFu : (kth >> 24);  // fewer than k candidates: largest
    // the two largest values of the warp, then of the CTA
    uint32_t m1 = hk;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m1 = max(m1, __shfl_xor_sync(0xFFFFFFFFu, m1, o));
    const uint32_t eq = __ballot_sync(0xFFFFFFFFu, hk == m1);
    uint32_t m2 = (hk == m1 && (eq & ((1u << lane) - 1u)) == 0) ? 0u : hk;  // drop one copy of the maximum
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m2 = max(m2, __shfl_xor_sync(0xFFFFFFFFu, m2, o));
    if (lane == 0) {
      s_top[warp][0] = m1;
      s_top[warp][1] = m2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t b1 = 0, b2 = 0;
      for (int w = 0; w < CAL_SAMPLES / 32; ++w)
        for (int k = 0; k < 2; ++k) {
          const uint32_t x = s_top[w][k];
          if (x > b1) {
            b2 = b1;
            b1 = x;
          } else if (x > b2) {
            b2 = x;
          }
        }
      // two or more samples with fewer than k candidates: leave the pair without a guess
      if (b2 != 0xFFFFFFFFu) atomicMax(a.tau_pair + p, b2 + CAL_MARGIN + 1u);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
namespace {

template <int KC, bool TAU, int NTC, bool EPI>
cudaError_t run_join(const MatchArgs* a, uint32_t grid, cudaStream_t s, uint32_t* occ, uint32_t na_max,
                     bool calibrate) {
  static int attr_dev = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (attr_dev != dev) {
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_join<KC, TAU, NTC, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 2048);
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  const size_t smem = join_smem_bytes(KC, na_max);
  if (occ) {
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_join<KC, TAU, NTC, EPI>, JT, smem);
    *occ = (uint32_t)(nb > 0 ? nb : 0);
    return e;
  }
  if (calibrate) {
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t want = a->n_pairs;
    k_join_calibrate<KC, TAU><<<want < (uint32_t)nsm * 8 ? want : (uint32_t)nsm * 8, CAL_SAMPLES, 0, s>>>(*a);
    return cudaGetLastError();
  }
  k_join<KC, TAU, NTC, EPI><<<grid, JT, smem, s>>>(*a);
  return cudaGetLastError();
}

// The band form is built with 4 candidate tiles only.
template <int KC, bool TAU>
cudaError_t run_join_nt(const MatchArgs* a, uint32_t ntc, bool epi, uint32_t grid, cudaStream_t s, uint32_t* occ,
                        uint32_t na_max, bool cal) {
  if (epi) return run_join<KC, TAU, 4, true>(a, grid, s, occ, na_max, cal);
  return ntc <= 2 ? run_join<KC, TAU, 2, false>(a, grid, s, occ, na_max, cal)
                  : run_join<KC, TAU, 4, false>(a, grid, s, occ, na_max, cal);
}

template <int KC>
cudaError_t run_join_kc(const MatchArgs* a, bool tau, uint32_t ntc, bool epi, uint32_t grid, cudaStream_t s,
                        uint32_t* occ, uint32_t na_max, bool cal) {
  return tau ? run_join_nt<KC, true>(a, ntc, epi, grid, s, occ, na_max, cal)
             : run_join_nt<KC, false>(a, ntc, epi, grid, s, occ, na_max, cal);
}

cudaError_t join_dispatch(uint32_t k, const MatchArgs* a, bool tau, uint32_t ntc, bool epi, uint32_t grid,
                          cudaStream_t s, uint32_t* occ, uint32_t na_max, bool cal) {
  if (k <= 4) return run_join_kc<4>(a, tau, ntc, epi, grid, s, occ, na_max, cal);
  if (k <= 8) return run_join_kc<8>(a, tau, ntc, epi, grid, s, occ, na_max, cal);
  if (k <= 10) return run_join_kc<10>(a, tau, ntc, epi, grid, s, occ, na_max, cal);
  if (k <= 16) return run_join_kc<16>(a, tau, ntc, epi, grid, s, occ, na_max, cal);
  return run_join_kc<32>(a, tau, ntc, epi, grid, s, occ, na_max, cal);
}

int kc_of(uint32_t k) { return k <= 4 ? 4 : k <= 8 ? 8 : k <= 10 ? 10 : k <= 16 ? 16 : 32; }

}  // namespace

uint32_t join_grid(const KParams& kp, uint32_t na_max, uint32_t n_items, uint32_t ntc, uint32_t ctas_per_sm) {
  int dev = 0, nsm = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (join_smem_bytes(kc_of(kp.top_k), na_max) + 4096 > (size_t)optin) return 0;
  uint32_t occ = 0;
  if (join_dispatch(kp.top_k, nullptr, kp.tau < kp.code_bits, ntc, kp.epi_px >= 0.0, 0, 0, &occ, na_max, false) !=
      cudaSuccess) {
    cudaGetLastError();
    occ = 0;
  }
  if (ctas_per_sm && ctas_per_sm < occ) occ = ctas_per_sm;
  const uint64_t gr = (uint64_t)nsm * occ;
  return (uint32_t)(n_items < gr ? n_items : gr);
}

cudaError_t launch_join_calibrate(const MatchArgs& a, cudaStream_t s) {
  if (a.n_pairs == 0 || a.kp.epi_px >= 0.0) return cudaSuccess;  // the band form uses no threshold guess
  return join_dispatch(a.kp.top_k, &a, a.kp.tau < a.kp.code_bits, 4, false, 0, s, nullptr, a.na_max, true);
}

cudaError_t launch_join(const MatchArgs& a, uint32_t grid, uint32_t ntc, cudaStream_t s) {
  if (a.n_items == 0 || grid == 0) return cudaSuccess;
  return join_dispatch(a.kp.top_k, &a, a.kp.tau < a.kp.code_bits, ntc, a.kp.epi_px >= 0.0, grid, s, nullptr,
                       a.na_max, false);
}

}  // namespace chx
