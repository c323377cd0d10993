// Internal declarations of the CUDA Cascade Hashing library (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cashash.h"

namespace chx {

constexpr int DIM = 128;
constexpr int MAX_ROWS = 128 + CASHASH_MAX_TABLES * 8;  // projection rows: remap code + table bits
constexpr int JC = 3968;          // features of the candidate image per lookup-table chunk
                                  // (sized so that two 512-thread matching CTAs fit one SM)
constexpr int OFF_STRIDE = 264;   // uint16 bucket offsets per (chunk, table): 257 used, padded to 16 B
constexpr uint32_t NO_MATCH = 0xFFFFFFFFu;
constexpr uint32_t PENDING = 0xFFFFFFFEu;  // query left to the exact fallback kernel
constexpr uint32_t QCAP = 64;              // survivor-queue entries per query thread
constexpr uint32_t JSEG = 64;              // bucket join: survivor-list entries per query
constexpr uint32_t HBINS = 129;            // bucket join: per-pair histogram of k-th Hamming distances
constexpr uint32_t KEY_INF = 0xFFFFFFFFu;

// device status bits (ORed into the context's status word)
enum : uint32_t { DST_OVERFLOW = 1u, DST_INDEX = 2u };

// Bytes of one lookup-table chunk: T tables x (bucket offsets + local indices), uint16.
__host__ __device__ inline uint64_t chunk_bytes(uint32_t T) {
  return (uint64_t)T * (uint64_t)(OFF_STRIDE + JC) * 2u;
}

// Parameters passed to kernels by value.
struct KParams {
  uint32_t code_bits, n_tables, bits_per_table, top_k;
  uint32_t ratio_num, ratio_den, tau, rows;
  double epi_px;
  uint32_t flags, pad;
};

// One image pair of a plan.
struct PairInfo {
  uint64_t a0, b0;      // first feature of the query image / candidate image
  uint64_t qbase;       // offset of this pair's queries in the per-query result array
  uint32_t nA, nB;      // feature counts
  uint32_t bchunk0;     // first lookup-table chunk of the candidate image
  uint32_t pad;
  uint64_t ajoin, bjoin;  // byte offsets of the two images' bucket-sorted tables (join region)
};

// Bucket-sorted tables ("join" region of the table buffer), per image and
// table t, at join_base(image) + t * join_block(N):
//   uint32 off[260]   bucket v holds positions off[v] .. off[v+1]
//   uint32 idx[N4]    feature index within the image, ascending within a bucket
//   uint4  code[N]    the 128-bit code of that feature (inline copy)
__host__ __device__ inline uint64_t join_block(uint64_t n) {
  return 1040u + 4u * ((n + 3) / 4 * 4) + 16u * n;
}

// Bucket join with the band: per CTA, FP32 (a, b, c, w_lo) of each query's line, then w_hi.
__host__ __device__ inline uint64_t jline_stride(uint64_t na_max) { return na_max + (na_max + 3) / 4; }

// Per-row constants of the projection (Sec. 5.1) derived from R and the centre.
struct RowConst {
  float c32;     // fl32(c_b), c_b = sum_j R_bj mu_j
  float alpha;   // bound factor on ||x||_2 (FP32 form) or on ||x||_2 (BF16 form)
  float beta;    // additive bound term
  float pad;
};

constexpr int PT_ROWS_TC = 192;   // projection rows supported by the tensor-core form (padded to 16)

#ifdef __CUDACC__
// ---------------------------------------------------------------------------
// Shared epilogue: from the approximate projections of one feature, write its
// code words, bucket bytes and squared norm, and record flagged rows.
// sbits / sflag hold 192 bits per feature (rows 0..191).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t extract_bits(const uint32_t* w, uint32_t pos, uint32_t m) {
  if (m == 0) return 0;
  const uint32_t wi = pos >> 5, sh = pos & 31;
  uint64_t v = w[wi];
  if (wi + 1 < 6) v |= (uint64_t)w[wi + 1] << 32;
  return (uint32_t)(v >> sh) & ((1u << m) - 1u);
}

__device__ __forceinline__ void write_feature(uint64_t f, const uint32_t* bits, const uint32_t* flags,
                                              uint32_t sq, const KParams& kp, uint32_t* __restrict__ codes,
                                              uint8_t* __restrict__ buckets, uint32_t* __restrict__ sqnorm,
                                              uint32_t* __restrict__ flagmask, uint32_t* __restrict__ flaglist,
                                              unsigned long long* __restrict__ nflag_feat) {
  uint4 c;
  c.x = bits[0];
  c.y = kp.code_bits > 32 ? bits[1] : 0u;
  c.z = kp.code_bits > 64 ? bits[2] : 0u;
  c.w = kp.code_bits > 96 ? bits[3] : 0u;
  reinterpret_cast<uint4*>(codes)[f] = c;
  uint32_t b[8];
#pragma unroll
  for (int t = 0; t < 8; ++t)
    b[t] = ((uint32_t)t < kp.n_tables) ? extract_bits(bits, kp.code_bits + t * kp.bits_per_table, kp.bits_per_table) : 0u;
  uint2 bb;
  bb.x = b[0] | (b[1] << 8) | (b[2] << 16) | (b[3] << 24);
  bb.y = b[4] | (b[5] << 8) | (b[6] << 16) | (b[7] << 24);
  reinterpret_cast<uint2*>(buckets)[f] = bb;
  sqnorm[f] = sq;
  const uint32_t any = flags[0] | flags[1] | flags[2] | flags[3] | flags[4] | flags[5];
  if (any) {
#pragma unroll
    for (int k = 0; k < 6; ++k) flagmask[f * 6 + k] = flags[k];
    const unsigned long long slot = atomicAdd(nflag_feat, 1ull);
    flaglist[slot] = (uint32_t)f;  // features are < 2^32 per set (checked on the host)
  }
}

// Predicated 32-bit global store (one instruction, no branch): *p = v if c.
// Survivor appends use it: their conditions are data-dependent per lane.
__device__ __forceinline__ void st_global_if(uint32_t* p, uint32_t v, bool c) {
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.b32 q, %2, 0;\n @q st.global.u32 [%0], %1;\n}" ::"l"(__cvta_generic_to_global(p)),
      "r"(v), "r"((uint32_t)c)
      : "memory");
}

// Step 4 ratio test over nv ranked candidates with the two smallest squared
// distances d1 <= d2: den^2 d1 < num^2 d2 in 64-bit integers (strict, on
// distances); one ranked candidate matches only with CASHASH_FLAG_ACCEPT_SINGLE.
__device__ __forceinline__ bool ratio_ok(const KParams& kp, uint32_t nv, uint32_t d1, uint32_t d2) {
  if (nv == 1) return (kp.flags & CASHASH_FLAG_ACCEPT_SINGLE) != 0;
  return nv >= 2 && (uint64_t)kp.ratio_den * kp.ratio_den * d1 < (uint64_t)kp.ratio_num * kp.ratio_num * d2;
}

// ---------------------------------------------------------------------------
// Sec. 7.2 band test, shared by the matching kernels.
// ---------------------------------------------------------------------------
// The epipolar line of the query, l = F p_q, and d^2 (a^2 + b^2), in FP64.
__device__ __forceinline__ void epi_line(const double* F, float2 pq, double dd, double& la, double& lb, double& lc,
                                         double& rhs) {
  const double x = (double)pq.x, y = (double)pq.y;
  la = __dadd_rn(__dadd_rn(__dmul_rn(F[0], x), __dmul_rn(F[1], y)), F[2]);
  lb = __dadd_rn(__dadd_rn(__dmul_rn(F[3], x), __dmul_rn(F[4], y)), F[5]);
  lc = __dadd_rn(__dadd_rn(__dmul_rn(F[6], x), __dmul_rn(F[7], y)), F[8]);
  rhs = __dmul_rn(dd, __dadd_rn(__dmul_rn(la, la), __dmul_rn(lb, lb)));
}

// Eq. 1-2, squared: keep p' iff (a x' + b y' + c)^2 <= d^2 (a^2 + b^2).
__device__ __forceinline__ bool epi_keep(double la, double lb, double lc, double rhs, float2 pc) {
  const double num = __dadd_rn(__dadd_rn(__dmul_rn(la, (double)pc.x), __dmul_rn(lb, (double)pc.y)), lc);
  return __dmul_rn(num, num) <= rhs;
}

// The band test of one query: the FP64 line and right-hand side exactly as
// epi_line computes them, and their FP32 roundings.
struct EpiQ {
  double la, lb, lc, rhs;
  float a, b, c, r;
};

__device__ __forceinline__ EpiQ epi_query(const double* F, float2 pq, double dd) {
  EpiQ e;
  epi_line(F, pq, dd, e.la, e.lb, e.lc, e.rhs);
  e.a = __double2float_rn(e.la);
  e.b = __double2float_rn(e.lb);
  e.c = __double2float_rn(e.lc);
  e.r = __double2float_rn(e.rhs);
  return e;
}

// epi_keep decided in FP32 from the FP32 roundings (a, b, c, r) of the line
// and right-hand side: 1 keep, 0 drop, 2 undecided (decide in FP64).  The
// FP32 difference r - n^2 is trusted when it clears a bound on its distance
// from the FP64 difference.  With u = 2^-24: a, b, c carry one rounding each
// and n two FMA roundings, so |n32 - n64| <= 3.01 u S, S = |a x'| + |b y'| + |c|
// (the FP64 evaluation's own error, ~3 * 2^-53 S, is inside the slack); then
// |(r - n^2)32 - (rhs - num^2)64| <= 2u r + 3u n^2 + e_n (2|n| + e_n).  The
// margins below are 6.7u and 8.4u, plus an absolute 1e-30 for underflow;
// overflow or NaN fails both comparisons.
__device__ __forceinline__ int epi_test32(float a, float b, float c, float r, float2 pc) {
  const float n = fmaf(a, pc.x, fmaf(b, pc.y, c));
  const float S = fmaf(fabsf(a), fabsf(pc.x), fmaf(fabsf(b), fabsf(pc.y), fabsf(c)));
  const float lhs = n * n;
  const float diff = r - lhs;
  const float en = 4.0e-7f * S;
  const float err = fmaf(en, fmaf(2.0f, fabsf(n), en), fmaf(5.0e-7f, r + lhs, 1.0e-30f));
  if (diff > err) return 1;
  if (diff < -err) return 0;
  return 2;
}

// Thresholds on |n|, n = fl32(a x' + b y' + c) as two FMAs (a, b, c the FP32 roundings of the
// FP64 line), that decide epi_keep for every candidate of an image whose key-points satisfy
// |x'| <= mx and |y'| <= my: |n| <= w_lo keeps, |n| >= w_hi drops, anything between (or NaN) is
// left to the FP64 expression.  With u = 2^-24 and S = |a| mx + |b| my + |c|, the two FMA
// roundings and the roundings of a, b, c give |n - num| <= 3 u S (1 + u) + 3 * 2^-53 S, num the
// FP64 numerator; the FP64 square num^2 <= rhs holds whenever |num| <= sqrt(rhs) (1 - 2^-40) and
// fails whenever |num| >= sqrt(rhs) (1 + 2^-40), since the roundings of the square, of the root
// and of these bounds are all below 2^-50 relative.  The absolute 1e-30 covers FP32 underflow;
// lines that are not finite, or so large that n could overflow, leave every candidate to FP64.
__device__ __forceinline__ void band_thresholds(const EpiQ& e, float mx, float my, float& wlo, float& whi) {
  wlo = -INFINITY;
  whi = INFINITY;
  const double t = sqrt(e.rhs);
  const double S = fabs((double)e.a) * (double)mx + fabs((double)e.b) * (double)my + fabs((double)e.c);
  const double en = 3.02 * 0x1p-24 * S + 1e-30;
  const double lo = t * (1.0 - 0x1p-40) - en, hi = t * (1.0 + 0x1p-40) + en;
  if (S < 1e30 && isfinite(lo) && isfinite(hi)) {
    wlo = __double2float_rd(lo);
    whi = __double2float_ru(hi);
  }
}

// The FP64 decisions as real calls: inlined, the compiler may predicate them
// and run them for every candidate, which makes the FP64 pipe the limit.
static __device__ __noinline__ bool epi_keep_fp64(const EpiQ& e, float2 pc) {
  return epi_keep(e.la, e.lb, e.lc, e.rhs, pc);
}

static __device__ __noinline__ bool epi_keep_fp64_F(const double* F, float2 pq, double dd, float2 pc) {
  double la, lb, lc, rhs;
  epi_line(F, pq, dd, la, lb, lc, rhs);
  return epi_keep(la, lb, lc, rhs, pc);
}

__device__ __forceinline__ bool epi_keep_fast(const EpiQ& e, float2 pc) {
  const int d = epi_test32(e.a, e.b, e.c, e.r, pc);
  return d == 2 ? epi_keep_fp64(e, pc) : d == 1;
}

#endif

// 1 when every field of p is in the range the entry points accept (code
// bits, tables, bits per table, k, ratio, precision, schedule, flags, and a
// finite band width), else 0.
int params_ok(const cashash_params* p);

// ---- launchers (return cudaError_t of the launch) ----
// Column sums of n descriptors into sums[128] (zeroed first unless add).
cudaError_t launch_colsum(const uint8_t* desc, uint64_t n, unsigned long long* sums, cudaStream_t s,
                          bool add = false);
cudaError_t launch_row_consts(const unsigned long long* sums, uint64_t n, int have_mean, double* mu,
                              const double* R, const double* nrmR, uint32_t rows, float alpha_scale,
                              RowConst* rc, cudaStream_t s);
cudaError_t launch_project_fp32(const uint8_t* desc, uint64_t n, const float* R32T, const RowConst* rc,
                                const KParams& kp, uint32_t* codes, uint8_t* buckets, uint32_t* sqnorm,
                                uint32_t* flagmask, uint32_t* flaglist, unsigned long long* nflag_feat,
                                cudaStream_t s, float* dbg_x = nullptr, float* dbg_e = nullptr);
cudaError_t launch_project_bf16(const uint8_t* desc, uint64_t n, const void* Rbf, uint32_t NP, const RowConst* rc,
                                const KParams& kp, uint32_t* codes, uint8_t* buckets, uint32_t* sqnorm,
                                uint32_t* flagmask, uint32_t* flaglist, unsigned long long* nflag_feat,
                                uint32_t* status, cudaStream_t s, float* dbg_x = nullptr, float* dbg_e = nullptr);
// (dbg_x, dbg_e: when non-null, [n][rows] FP32 approximation v~ - c and bound E of
// every projection, for cashash_projection_bounds; null in the matching path.)
cudaError_t launch_fix_fp64(const uint8_t* desc, const double* mu, const double* R, const KParams& kp,
                            const uint32_t* flagmask, const uint32_t* flaglist,
                            const unsigned long long* nflag_feat, uint64_t max_feat, uint32_t* codes,
                            uint8_t* buckets, unsigned long long* n_reeval, cudaStream_t s);
cudaError_t launch_build_tables(const uint8_t* buckets, const uint64_t* chunk_feat0, const uint32_t* chunk_len,
                                uint32_t n_chunks, uint32_t n_tables, uint8_t* tables, cudaStream_t s);
cudaError_t launch_build_join(const uint8_t* buckets, const uint32_t* codes, const uint64_t* img_f0,
                              const uint32_t* img_n, const uint64_t* img_join, uint32_t n_images, uint32_t n_tables,
                              uint32_t n_max, uint8_t* join, cudaStream_t s);

struct MatchArgs {
  const uint8_t* desc;
  const uint32_t* codes;
  const uint8_t* buckets;
  const uint32_t* sqnorm;
  const uint8_t* tables;
  const float* kpts;
  const double* F;           // [P][9] or null
  const PairInfo* pairs;
  const uint2* items;        // (pair, first query) work items
  uint32_t n_items;
  uint32_t n_pairs;
  unsigned int* item_ctr;    // work-item counter of this launch
  uint32_t* res;             // per-query result (candidate index, NO_MATCH or PENDING)
  uint64_t n_res;
  unsigned long long* pair_cnt;
  uint32_t* status;
  uint32_t* queue;           // speculative form: [grid][TPB][QCAP] survivor queues
  uint32_t* tau_pair;        // speculative form, per pair: 0 = no guess yet, else (threshold + 1);
                             // learned as the largest k-th Hamming distance seen, kept across launches
  uint32_t tau_fixed;        // speculative form: do not learn (keep the values set by the host)
  uint32_t all_queries;      // exact warp-per-query kernel: every query, not only the PENDING ones
  const uint8_t* join;       // bucket join: table buffer holding the bucket-sorted tables
  uint32_t* jqueue;          // bucket join: [grid][na_max][JSEG] survivor lists
  uint32_t* jhist;           // bucket join: [P][HBINS] k-th Hamming distances seen per pair
  float4* jline;             // bucket join with the band: per CTA jline_stride(na_max) float4s of query lines
  uint32_t na_max;           // bucket join: largest query image of the plan
  KParams kp;
};
// Bucket-join matching (batched schedule): calibration of missing per-pair
// thresholds (launch_join_calibrate), then the join kernel over items = pairs.
cudaError_t launch_join_calibrate(const MatchArgs& a, cudaStream_t s);
// ntc: candidate tiles of 8 columns held in registers (2 or 4).
cudaError_t launch_join(const MatchArgs& a, uint32_t grid, uint32_t ntc, cudaStream_t s);
// Resident CTAs of the join for n_items pairs (at most ctas_per_sm per SM when
// non-zero); 0 when the join does not apply (the largest query image exceeds
// its shared memory).  The band form runs with 4 candidate tiles.
uint32_t join_grid(const KParams& kp, uint32_t na_max, uint32_t n_items, uint32_t ntc, uint32_t ctas_per_sm);
// The bucket join on tcgen05 tensor cores (same results as launch_join):
// resident CTAs for n_items pairs (at most 2 per SM, ctas_per_sm when
// non-zero and smaller), 0 when the largest query image exceeds its shared
// memory; and the launch.
uint32_t join_tc_grid(const KParams& kp, uint32_t na_max, uint32_t n_items, uint32_t ctas_per_sm);
cudaError_t launch_join_tc(const MatchArgs& a, uint32_t grid, cudaStream_t s);
// Matching kernel launch.  spec = 0: direct register top-k (one pair per
// launch); spec = 1: survivor queues with a speculative threshold (batched).
// tile: queries per CTA of the speculative form (256, or 512 when k <= 16; 0 = default).
cudaError_t launch_match(const MatchArgs& a, int spec, uint32_t grid, cudaStream_t s, uint32_t tile = 0);
// Largest useful grid (resident CTAs) for a launch over n_items items.
uint32_t match_grid(uint32_t top_k, int spec, bool epi, uint32_t n_tables, uint32_t n_items, uint32_t tile = 0);
// Queries per CTA (= per work item) of a form; tile 0 = default.
int match_tile_size(uint32_t top_k, int spec, uint32_t tile = 0);
// Exact re-matching of the queries the speculative kernel left PENDING.
cudaError_t launch_match_fallback(const MatchArgs& a, cudaStream_t s);
// Mutual check: F2 = (F, F^T) for the P pairs and their reversals; then the
// filter of the P forward pairs against the reverse results (pairs P..2P-1).
cudaError_t launch_mutual_F(const double* F, uint32_t P, double* F2, cudaStream_t s);
cudaError_t launch_mutual(const PairInfo* pairs, uint32_t P, uint32_t* res, unsigned long long* pair_cnt,
                          cudaStream_t s);
cudaError_t launch_scan_counts(const unsigned long long* pair_cnt, uint32_t P, uint64_t* match_off,
                               uint64_t cap, uint32_t* status, unsigned long long* total, cudaStream_t s);
cudaError_t launch_compact(const PairInfo* pairs, uint32_t P, const uint32_t* res, const uint64_t* match_off,
                           uint32_t* matches, uint64_t cap, cudaStream_t s);

}  // namespace chx
