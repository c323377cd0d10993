// Batched matching as a bucket join on the 5th-generation tensor cores
// (tcgen05.mma with tensor-memory accumulators, sm_103a): the same results as
// k_join (Steps 1-4 of Sec. 3.1, the Sec. 6 threshold tau, the Sec. 7.2
// band), with the Hamming contraction of Step 2 moved from warp-level mma.sync
// to tcgen05.
//
// For table t the query image's features are taken in the order of its
// bucket-sorted table, so each bucket is a run of consecutive rows; a tile is
// 128 such rows (TMEM lanes).  The candidates a row needs (its bucket in the
// candidate image's table t) are a run of consecutive positions of that
// table, and the runs of a tile's rows are consecutive too: their union is
// the tile's columns, processed in chunks of at most 256.  Codes are expanded
// to +-1 FP8 (e4m3) rows of 128 bytes in shared memory (canonical K-major
// layout, no swizzle) and four tcgen05.mma.kind::f8f6f4 (M = 128, N <= 256,
// K = 32 each) give D = 128 - 2 H in FP32 tensor memory, exactly (integers of
// magnitude at most 128; both sides use the same bit-to-element map, so the
// dot product does not depend on it).
//
// Epilogue: each warp owns 32 TMEM lanes (rows) and half of the column chunks
// of their union; a thread keeps the entries of its own row's run with
// H <= theta (the pair's threshold guess, capped by tau; with the band, tau
// alone and the band test) and appends keys H << 24 | j to its query's
// survivor list: one counter update per row and chunk, keys at consecutive
// slots.  The lists, the per-pair thresholds, the finalisation and the PENDING
// rule are those of k_join, so the two kernels give identical results.
//
// One MMA group per CTA (accumulator of 256 TMEM columns); the dynamic shared
// memory is at least 80 KB, so at most two CTAs share an SM and the 512
// columns of tensor memory.  Every mbarrier wait is bounded: on timeout the
// CTA records DST_INDEX, waits once more for its MMAs and stops, and still
// releases its tensor memory.
#include "join_common.cuh"
#include "tc_common.cuh"

namespace chx {

constexpr int TJ_M = 128;                     // rows (queries) per tile = TMEM lanes
constexpr uint32_t TJ_NMAX = 256;             // columns (candidates) per MMA chunk
constexpr uint32_t TJ_TMEM_COLS = 256;
constexpr uint32_t TJ_A_BYTES = TJ_M * 128;   // +-1 FP8 rows of 128 bytes
constexpr uint32_t TJ_B_BYTES = TJ_NMAX * 128;
constexpr size_t TJ_MIN_SMEM = 80 * 1024;     // keeps two CTAs per SM at most (TMEM: 2 x 256 columns)
constexpr uint32_t TJ_SCRATCH_WORDS = 16;     // epilogue: one 16-column chunk per thread

// Dynamic shared memory: [operands A | B, reused by the finalisation's keys
// and distances][column indices][row query, run begin, run end][bucket
// offsets of A and B][survivor counters].
__host__ __device__ inline size_t tj_op_bytes(int KC) {
  const size_t ops = TJ_A_BYTES + TJ_B_BYTES, fin = (size_t)2 * KC * JT * 4;
  return ops > fin ? ops : fin;
}
__host__ __device__ inline size_t tj_smem_bytes(int KC, uint32_t na_max) {
  const size_t b = tj_op_bytes(KC) + 4 * (TJ_NMAX + 3 * TJ_M + 2 * 260) + (size_t)4 * ((na_max + 3) / 4 * 4);
  return b < TJ_MIN_SMEM ? TJ_MIN_SMEM : b;
}

// Byte offset of the 16-byte chunk c (0..7) of row r in a K-major operand of
// 128-byte rows: core matrix (r / 8, c) at ((r / 8) * 8 + c) * 128.
__device__ __forceinline__ uint32_t tj_off(uint32_t r, uint32_t c) { return ((r >> 3) * 8 + c) * 128 + (r & 7) * 16; }

// Code word w of a row (bits 32 cw .. 32 cw + 31) as 32 FP8 values: chunk
// 2 cw + i / 4, word i % 4, byte b <- bit 8 b + i of w (e4m3 0x38 = +1 for
// a 0 bit, 0xB8 = -1 for a 1 bit); on = false writes zeros (padding rows).
__device__ __forceinline__ void tj_expand(uint8_t* base, uint32_t r, uint32_t cw, uint32_t w, bool on) {
  uint32_t o[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) o[i] = on ? (((w << (7 - i)) & 0x80808080u) | 0x38383838u) : 0u;
  *reinterpret_cast<uint4*>(base + tj_off(r, 2 * cw)) = make_uint4(o[0], o[1], o[2], o[3]);
  *reinterpret_cast<uint4*>(base + tj_off(r, 2 * cw + 1)) = make_uint4(o[4], o[5], o[6], o[7]);
}

// Epilogue scratch of one thread (16 words in the B operand region, free once
// the MMAs completed): 16-byte slots rotated by the thread index so that a
// warp's 16-byte stores do not collide in the banks.
__device__ __forceinline__ uint32_t* tj_scratch(uint8_t* bbase, int tid) {
  return reinterpret_cast<uint32_t*>(bbase + (size_t)tid * (TJ_SCRATCH_WORDS * 4));
}
__device__ __forceinline__ uint32_t tj_slot(int tid, uint32_t c) { return ((c ^ ((uint32_t)tid >> 1)) & 3u); }

// One tile of a table: rows [r0, r0 + nrows) of the query image's table order
// (buckets v0..v1), columns [c0, c0 + w) of the candidate run [cb0, cb1) of
// those buckets in the candidate image's table (N = w rounded up to 16);
// first: the first column chunk of its rows (the rows are staged then).
struct TjTile {
  uint32_t r0, nrows, v0, v1, cb0, cb1, c0, w, N, first;
};

// From t.r0 (and a bucket t.v0 at or before it): the rows' buckets and run;
// tiles whose rows have no candidate are skipped; t.r0 >= n marks the end.
__device__ __forceinline__ void tj_first_tile(TjTile& t, const uint32_t* aoff, const uint32_t* boff, uint32_t n) {
  for (; t.r0 < n; t.r0 += TJ_M) {
    t.nrows = min((uint32_t)TJ_M, n - t.r0);
    while (aoff[t.v0 + 1] <= t.r0) ++t.v0;
    t.v1 = t.v0;
    while (aoff[t.v1 + 1] <= t.r0 + t.nrows - 1) ++t.v1;
    t.cb0 = boff[t.v0];
    t.cb1 = boff[t.v1 + 1];
    if (t.cb1 > t.cb0) break;
    t.v0 = t.v1;
  }
  t.c0 = t.cb0;
  t.w = min(TJ_NMAX, t.cb1 - t.c0);
  t.N = (t.w + 15u) & ~15u;
  t.first = 1;
}

__device__ __forceinline__ void tj_next_tile(TjTile& t, const uint32_t* aoff, const uint32_t* boff, uint32_t n) {
  if (t.c0 + TJ_NMAX < t.cb1) {  // the next column chunk of the same rows
    t.c0 += TJ_NMAX;
    t.w = min(TJ_NMAX, t.cb1 - t.c0);
    t.N = (t.w + 15u) & ~15u;
    t.first = 0;
    return;
  }
  t.r0 += TJ_M;
  t.v0 = t.v1;
  tj_first_tile(t, aoff, boff, n);
}

// This thread's global loads of a tile: the code words of rows tid / 4 and
// (tid + JT) / 4 (word tid % 4) with their query indices, and of columns
// (tid + u JT) / 4 with their candidate indices; zeros outside the tile.
__device__ __forceinline__ void tj_load(const TjTile& t, int tid, const uint32_t* Aw, const uint32_t* Aidx,
                                        const uint32_t* Bw, const uint32_t* Bidx, uint32_t (&pa)[2],
                                        uint32_t (&pq)[2], uint32_t (&pb)[4], uint32_t (&pi)[4]) {
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const uint32_t i = (uint32_t)tid + u * JT, r = i >> 2, cw = i & 3u;
    const bool on = t.first && r < t.nrows;
    pa[u] = on ? __ldg(Aw + 4ull * (t.r0 + r) + cw) : 0u;
    pq[u] = (on && cw == 0) ? __ldg(Aidx + t.r0 + r) : 0u;
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const uint32_t i = (uint32_t)tid + u * JT, c = i >> 2, cw = i & 3u;
    const bool on = c < t.w;
    pb[u] = on ? __ldg(Bw + 4ull * (t.c0 + c) + cw) : 0u;
    pi[u] = (on && cw == 0) ? __ldg(Bidx + t.c0 + c) : 0u;
  }
}

template <int KC, bool TAU, bool EPI>
__global__ void __launch_bounds__(JT, 2) k_join_tc(MatchArgs a) {
  extern __shared__ __align__(1024) uint8_t tsm[];
  __shared__ __align__(8) uint64_t s_mbar;
  __shared__ uint32_t s_tmem, s_item, s_tau;
  __shared__ uint32_t s_hist[HBINS];
  __shared__ PairInfo s_P;
  const KParams kp = a.kp;
  const uint32_t T = kp.n_tables, nbk = 1u << kp.bits_per_table;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint8_t* As = tsm;
  uint8_t* Bs = tsm + TJ_A_BYTES;
  const size_t opb = tj_op_bytes(KC);
  uint32_t* s_bidx = reinterpret_cast<uint32_t*>(tsm + opb);  // [TJ_NMAX] candidate index of each column
  uint32_t* s_rq = s_bidx + TJ_NMAX;                          // [TJ_M] query of each row
  uint32_t* s_rbs = s_rq + TJ_M;                              // [TJ_M] run of the row's bucket in B: begin
  uint32_t* s_rbe = s_rbs + TJ_M;                             //                                      end
  uint32_t* s_aoff = s_rbe + TJ_M;                            // [260] bucket offsets of A, table t
  uint32_t* s_boff = s_aoff + 260;                            // [260] bucket offsets of B, table t
  uint32_t* cnt_s = s_boff + 260;                             // [na_max] survivor counters
  uint32_t* key_s = reinterpret_cast<uint32_t*>(tsm);         // finalisation (aliases the operands)
  uint32_t* dist_s = key_s + KC * JT;
  uint32_t* seg = a.jqueue + (size_t)blockIdx.x * a.na_max * JSEG;
  const uint32_t h_user = TAU ? kp.tau : 128u;
  float4* lines = EPI ? a.jline + (size_t)blockIdx.x * a.na_max : nullptr;
  const double dd = kp.epi_px * kp.epi_px;
  const float2* kpts = reinterpret_cast<const float2*>(a.kpts);

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(TJ_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  const uint32_t mbar = smem_u32(&s_mbar);
  const uint32_t qd = (uint32_t)warp & 3u, half = (uint32_t)warp >> 2;  // TMEM lanes 32 qd .. 32 qd + 31
  const uint32_t r_ep = 32u * qd + (uint32_t)lane;                       // this thread's row in the epilogue
  uint32_t* scr = tj_scratch(Bs, tid);
  uint32_t phase = 0;
  bool failed = false;

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
    for (uint32_t q = tid; q < P.nA; q += JT) {
      cnt_s[q] = 0;
      if constexpr (EPI) {
        const EpiQ e = epi_query(Fp, __ldg(kpts + P.a0 + q), dd);
        lines[q] = make_float4(e.a, e.b, e.c, e.r);
      }
    }
    __syncthreads();
    uint32_t h_thr = h_user;
    if (!EPI) {
      const uint32_t ts = s_tau;  // 0: no guess; else threshold + 1
      if (ts != 0 && ts - 1u < h_thr) h_thr = ts - 1u;
    }
    const bool cut = h_thr < h_user;  // the guess may turn candidates away
    const float tf = 128.0f - 2.0f * (float)min(h_thr, 128u);  // keep D = 128 - 2 H >= tf
    const uint64_t ablk = join_block(P.nA), bblk = join_block(P.nB);
    const uint64_t arec = 1040u + 4u * ((P.nA + 3) / 4 * 4), brec = 1040u + 4u * ((P.nB + 3) / 4 * 4);

    for (uint32_t t = 0; t < T && P.nA && P.nB && !failed; ++t) {
      const uint8_t* Ab = a.join + P.ajoin + t * ablk;
      const uint8_t* Bb = a.join + P.bjoin + t * bblk;
      const uint32_t* Aidx = reinterpret_cast<const uint32_t*>(Ab + 1040);
      const uint32_t* Bidx = reinterpret_cast<const uint32_t*>(Bb + 1040);
      const uint32_t* Aw = reinterpret_cast<const uint32_t*>(Ab + arec);  // 4 code words per position
      const uint32_t* Bw = reinterpret_cast<const uint32_t*>(Bb + brec);
      for (uint32_t v = tid; v <= nbk; v += JT) {
        s_aoff[v] = __ldg(reinterpret_cast<const uint32_t*>(Ab) + v);
        s_boff[v] = __ldg(reinterpret_cast<const uint32_t*>(Bb) + v);
      }
      __syncthreads();
      // Tiles of this table in order: rows [r0, r0 + 128) (buckets v0..v1), columns [c0, c0 + w)
      // of the rows' run [cb0, cb1) in B.  Every thread steps the same (uniform) iterator.
      TjTile cur, nxt;
      cur.r0 = 0;
      cur.v0 = 0;
      tj_first_tile(cur, s_aoff, s_boff, P.nA);
      // registers of the next tile's loads (issued while the current tile's MMA and epilogue run)
      uint32_t pa[2], pq[2], pb[4], pi[4];
      bool have = false;  // pa..pi hold cur's data
      while (cur.r0 < P.nA && !failed) {
        if (!have) tj_load(cur, tid, Aw, Aidx, Bw, Bidx, pa, pq, pb, pi);
        // ---- stage: the tile's rows (first column chunk only) and its columns as +-1 FP8 ----
        if (cur.first) {
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const uint32_t i = (uint32_t)tid + u * JT, r = i >> 2, cw = i & 3u;
            const bool on = r < cur.nrows;
            tj_expand(As, r, cw, pa[u], on);
            if (cw == 0) {
              uint32_t rb = 0, re = 0;
              if (on) {  // the row's bucket: a short walk from the tile's first bucket
                uint32_t v = cur.v0;
                while (s_aoff[v + 1] <= cur.r0 + r) ++v;
                rb = s_boff[v];
                re = s_boff[v + 1];
              }
              s_rq[r] = pq[u];
              s_rbs[r] = rb;
              s_rbe[r] = re;
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const uint32_t i = (uint32_t)tid + u * JT, c = i >> 2, cw = i & 3u;
          if (c < cur.N) {
            tj_expand(Bs, c, cw, pb[u], c < cur.w);
            if (cw == 0) s_bidx[c] = pi[u];
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // ---- D = A x B^T over K = 128 (four K = 32 steps of 32 bytes = two core matrices) ----
        if (tid == 0) {
          const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
          const uint32_t idesc = tc_idesc_e4m3(TJ_M, cur.N);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            tc_mma_f8(tmem, tc_desc(a0 + kk * 256, 128, 1024), tc_desc(b0 + kk * 256, 128, 1024), idesc,
                      kk ? 1u : 0u);
          tc_commit(mbar);
        }
        // the next tile of this table, and its loads while the MMAs run
        nxt = cur;
        tj_next_tile(nxt, s_aoff, s_boff, P.nA);
        have = nxt.r0 < P.nA;
        if (have) tj_load(nxt, tid, Aw, Aidx, Bw, Bidx, pa, pq, pb, pi);
        bool ok = true;
        if (tid == 0) ok = mbar_wait(mbar, phase);  // one thread polls, the others wait at the barrier
        if (__syncthreads_or(!ok)) {  // never expected: record it, let the MMAs drain, stop
          if (tid == 0) atomicOr(a.status, DST_INDEX);
          mbar_wait(mbar, phase);
          failed = true;
          break;
        }
        if (tid != 0) mbar_wait(mbar, phase);  // completed: returns at once
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t c0 = cur.c0, w = cur.w;
        // ---- epilogue: this thread's row, the warp's share of the column chunks ----
        {
          const uint32_t q = s_rq[r_ep];
          const uint32_t rbs = s_rbs[r_ep], rbe = s_rbe[r_ep];
          const uint32_t cs = rbs > c0 ? min(rbs - c0, w) : 0u;  // the row's run within this chunk
          const uint32_t ce = rbe > c0 ? min(rbe - c0, w) : 0u;
          const bool any = ce > cs;
          const uint32_t u0 = __reduce_min_sync(0xFFFFFFFFu, any ? cs : 0xFFFFFFFFu);
          const uint32_t u1 = __reduce_max_sync(0xFFFFFFFFu, any ? ce : 0u);
          float4 L = make_float4(0.f, 0.f, 0.f, 0.f);
          float2 pqa = make_float2(0.f, 0.f);
          if constexpr (EPI) {
            if (any) {
              L = lines[q];
              pqa = __ldg(kpts + P.a0 + q);
            }
          }
          const uint32_t taddr = tmem + ((32u * qd) << 16);
          uint32_t* lst = seg + (size_t)q * JSEG;
          if (u1 > u0) {  // warp-uniform
            for (uint32_t k = (u0 >> 4) + half; k <= ((u1 - 1) >> 4); k += 2) {
              uint32_t v[16];
              tmem_ld16_nowait(taddr + 16u * k, v);
              tmem_wait_ld();
              const int lo = (int)cs - (int)(16u * k), hi = (int)ce - (int)(16u * k);
              uint32_t m = 0;
              if (any && hi > 0 && lo < 16) {
                const int l2 = lo > 0 ? lo : 0, h2 = hi < 16 ? hi : 16;
                const uint32_t rm = (uint32_t)((1ull << h2) - (1ull << l2));
#pragma unroll
                for (int i = 0; i < 16; ++i) m |= (__uint_as_float(v[i]) >= tf) ? (1u << i) : 0u;
                m &= rm;
              }
              if (m) {
#pragma unroll
                for (uint32_t c = 0; c < 4; ++c)
                  *reinterpret_cast<uint4*>(scr + 4 * tj_slot(tid, c)) =
                      make_uint4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
                if constexpr (EPI) {  // Sec. 7.2: only candidates inside the band
                  uint32_t keep = 0, mm = m;
                  while (mm) {
                    const uint32_t i = __ffs(mm) - 1u;
                    mm &= mm - 1u;
                    const float2 pc = __ldg(kpts + P.b0 + s_bidx[16u * k + i]);
                    int d = epi_test32(L.x, L.y, L.z, L.w, pc);
                    if (d == 2) d = epi_keep_fp64_F(Fp, pqa, dd, pc) ? 1 : 0;
                    keep |= (uint32_t)d << i;
                  }
                  m = keep;
                }
              }
              if (m) {
                uint32_t pos = atomicAdd(cnt_s + q, (uint32_t)__popc(m));
                while (m) {
                  const uint32_t i = __ffs(m) - 1u;
                  m &= m - 1u;
                  if (pos < JSEG) {
                    const float f = __uint_as_float(scr[4 * tj_slot(tid, i >> 2) + (i & 3u)]);
                    const uint32_t H = (uint32_t)(128 - __float2int_rn(f)) >> 1;
                    lst[pos] = (H << 24) | s_bidx[16u * k + i];
                  }
                  ++pos;
                }
              }
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();  // the columns, the scratch and TMEM are reused by the next tile
        cur = nxt;
      }
      __syncthreads();
    }
    if (failed) break;
    __syncthreads();

    // ---- finalise: top-k of the survivors, distances, ratio test (as k_join) ----
    join_finalise<KC, EPI>(a, P, it, cut, cnt_s, seg, key_s, dist_s, s_hist);
    __syncthreads();
    if (!a.tau_fixed)
      for (uint32_t b = tid; b < HBINS; b += JT)
        if (s_hist[b]) atomicAdd(a.jhist + (size_t)it * HBINS + b, s_hist[b]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TJ_TMEM_COLS) : "memory");
}

// ---------------------------------------------------------------------------
namespace {

template <int KC, bool TAU, bool EPI>
cudaError_t run_join_tc(const MatchArgs* a, uint32_t grid, cudaStream_t s, uint32_t* occ, uint32_t na_max) {
  static int attr_dev = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (attr_dev != dev) {
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_join_tc<KC, TAU, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 2048);
    if (e == cudaSuccess)  // the largest shared-memory carveout, so that two CTAs fit an SM
      e = cudaFuncSetAttribute(k_join_tc<KC, TAU, EPI>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  const size_t smem = tj_smem_bytes(KC, na_max);
  if (occ) {  // resident CTAs per SM from the resources (at most 2: tensor memory)
    cudaFuncAttributes fa{};
    int sm_smem = 0;
    e = cudaFuncGetAttributes(&fa, k_join_tc<KC, TAU, EPI>);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e != cudaSuccess) return e;
    const size_t per_cta = smem + fa.sharedSizeBytes + 1024;  // + the 1 KB the system reserves per CTA
    const uint32_t by_smem = (uint32_t)((size_t)sm_smem / per_cta);
    const uint32_t by_regs = (uint32_t)(65536 / ((size_t)(fa.numRegs > 0 ? fa.numRegs : 1) * JT));
    uint32_t nb = by_smem < by_regs ? by_smem : by_regs;
    *occ = nb < 2 ? nb : 2;
    return cudaSuccess;
  }
  k_join_tc<KC, TAU, EPI><<<grid, JT, smem, s>>>(*a);
  return cudaGetLastError();
}

template <int KC>
cudaError_t run_join_tc_kc(const MatchArgs* a, bool tau, bool epi, uint32_t grid, cudaStream_t s, uint32_t* occ,
                           uint32_t na_max) {
  if (epi) return tau ? run_join_tc<KC, true, true>(a, grid, s, occ, na_max)
                      : run_join_tc<KC, false, true>(a, grid, s, occ, na_max);
  return tau ? run_join_tc<KC, true, false>(a, grid, s, occ, na_max)
             : run_join_tc<KC, false, false>(a, grid, s, occ, na_max);
}

cudaError_t join_tc_dispatch(uint32_t k, const MatchArgs* a, bool tau, bool epi, uint32_t grid, cudaStream_t s,
                             uint32_t* occ, uint32_t na_max) {
  if (k <= 4) return run_join_tc_kc<4>(a, tau, epi, grid, s, occ, na_max);
  if (k <= 8) return run_join_tc_kc<8>(a, tau, epi, grid, s, occ, na_max);
  if (k <= 10) return run_join_tc_kc<10>(a, tau, epi, grid, s, occ, na_max);
  if (k <= 16) return run_join_tc_kc<16>(a, tau, epi, grid, s, occ, na_max);
  return run_join_tc_kc<32>(a, tau, epi, grid, s, occ, na_max);
}

int kc_of_tc(uint32_t k) { return k <= 4 ? 4 : k <= 8 ? 8 : k <= 10 ? 10 : k <= 16 ? 16 : 32; }

}  // namespace

uint32_t join_tc_grid(const KParams& kp, uint32_t na_max, uint32_t n_items, uint32_t ctas_per_sm) {
  int dev = 0, nsm = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (tj_smem_bytes(kc_of_tc(kp.top_k), na_max) + 4096 > (size_t)optin) return 0;
  uint32_t occ = 0;
  if (join_tc_dispatch(kp.top_k, nullptr, kp.tau < kp.code_bits, kp.epi_px >= 0.0, 0, 0, &occ, na_max) !=
      cudaSuccess) {
    cudaGetLastError();
    occ = 0;
  }
  if (ctas_per_sm && ctas_per_sm < occ) occ = ctas_per_sm;
  const uint64_t gr = (uint64_t)nsm * occ;
  return (uint32_t)(n_items < gr ? n_items : gr);
}

cudaError_t launch_join_tc(const MatchArgs& a, uint32_t grid, cudaStream_t s) {
  if (a.n_items == 0 || grid == 0) return cudaSuccess;
  return join_tc_dispatch(a.kp.top_k, &a, a.kp.tau < a.kp.code_bits, a.kp.epi_px >= 0.0, grid, s, nullptr,
                          a.na_max);
}

}  // namespace chx
