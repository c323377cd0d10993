/*
 * cashash_oracle.h -- plain, slow, single-threaded CPU oracle for Cascade
 * Hashing (CasHash) image matching.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path
 * (the CUDA library under paper_1805_08995_gb300/) never links, loads or
 * calls it, and shares no source with it.
 *
 * What it computes follows the paper (Xu, Sun, Tao, "GPU Accelerated Cascade
 * Hashing Image Matching for Large Scale 3D Reconstruction"):
 *   Sec. 3.1 Step 1  hashing lookup with several tables of m-bit codes
 *   Sec. 3.1 Step 2  hashing remapping to n-bit codes, Hamming distance
 *   Sec. 3.1 Step 3  hashing ranking: keep the k smallest Hamming distances
 *   Sec. 3.1 Step 4  Euclidean distance on those k, Lowe's ratio test
 *   Sec. 5.1         hash bits are signs of inner products with random
 *                    vectors r_k (Charikar's sign LSH)
 *   Sec. 6           optional Hamming threshold tau before ranking
 *   Sec. 7.2 Eq. 1-2 optional epipolar band |dist(p', l_q)| <= d
 *
 * Readings where the paper is silent (documented beside each function):
 * descriptors are centred by their mean over the whole set given to one
 * code-building call; the projection is evaluated in IEEE double precision
 * in a fixed order with no fused multiply-add; sign at exactly zero is bit 0;
 * ties in the ranking are broken by the smaller candidate index; the ratio
 * test is strict on distances; a query needs two ranked candidates to match
 * (unless ORACLE_ACCEPT_SINGLE); the mutual check (ORACLE_MUTUAL) keeps (q, j)
 * of pair (A, B) only when matching j of B against A, by the same procedure
 * with F transposed, gives q.
 *
 * Parity pins (tests/test_oracle_*.py): exact rational arithmetic for the
 * mean and the projection sign, axis-aligned projections (closed form),
 * brute-force nearest neighbour when one bucket holds every point and k is
 * at least the image size, brute-force bucket-equality candidate sets,
 * independent sorting of (Hamming, index) keys, and structural invariants.
 */
#ifndef CASHASH_ORACLE_H
#define CASHASH_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_DIM 128        /* SIFT descriptor length d (Sec. 5.1: d = 128) */
#define ORACLE_MAX_TABLES 8
#define ORACLE_MAX_K 64

/* oracle_params.flags */
#define ORACLE_MUTUAL 1u         /* keep (q, j) only when the reverse match of j is q (oracle_match_pairs) */
#define ORACLE_ACCEPT_SINGLE 2u  /* a query with exactly one ranked candidate matches it */

typedef struct {
  uint32_t code_bits;       /* n of Step 2: length of the remapping code, 1..128 */
  uint32_t n_tables;        /* number of lookup tables of Step 1, 1..8 */
  uint32_t bits_per_table;  /* m of Step 1: bits of each short code, 0..8 */
  uint32_t top_k;           /* k of Step 3, 1..64 */
  uint32_t ratio_num;       /* Lowe ratio as a fraction num/den (0.8 = 4/5) */
  uint32_t ratio_den;
  uint32_t tau;             /* Sec. 6 threshold; >= code_bits means off */
  uint32_t flags;           /* ORACLE_MUTUAL | ORACLE_ACCEPT_SINGLE */
  double epi_px;            /* Sec. 7.2 threshold d in pixels; < 0 means off */
} oracle_params;

/* Per-query detail for invariant tests. */
typedef struct {
  uint32_t n_cand;          /* |C_q| after the epipolar band and tau */
  uint32_t n_top;           /* |T_q| = min(k, |C_q|) */
  uint32_t top_j[ORACLE_MAX_K];   /* T_q ordered by (Hamming, index) */
  uint32_t top_h[ORACLE_MAX_K];
  int32_t  top_d[ORACLE_MAX_K];   /* squared Euclidean distance of each */
  int32_t  match_j;         /* -1 if no match */
  int32_t  d1, d2;          /* smallest and second smallest squared distance, -1 if absent */
} oracle_query_detail;

/* Column means of n descriptors (reading: centring over the whole set). */
void oracle_mean(const uint8_t* desc, uint64_t n, double* mu /* [128] */);

/* One projection value v = sum_j R[b][j] * (x_j - mu_j), ordered double. */
double oracle_projection(const uint8_t* x /* [128] */, const double* mu, const double* Rrow);

/* Hash codes (Sec. 5.1 + Steps 1-2).  R has code_bits + n_tables*bits_per_table
 * rows of 128 doubles.  codes: [n][4] uint32, bit b of the remapping code in
 * word b/32 at bit b%32, unused bits zero.  buckets: [n][n_tables], bucket of
 * table t = sum_i bit(code_bits + t*m + i) << i. */
void oracle_hash(const uint8_t* desc, uint64_t n, const double* mu, const double* R,
                 const oracle_params* p, uint32_t* codes, uint8_t* buckets);

/* All projections of n features against rows 0..rows-1 of R: v is [n][rows],
 * each value the ordered double sum of oracle_projection. */
void oracle_projections(const uint8_t* desc, uint64_t n, const double* mu, const double* R, uint32_t rows,
                        double* v);

/* Match one image pair (I = A queries, J = B candidates).  match[q] is the
 * matched index in B or -1.  F (row-major 3x3, x_B^T F x_A = 0) and the
 * key-points ([n][2] float x,y) are used only when p->epi_px >= 0.
 * detail may be NULL; otherwise it receives nA entries.  Returns the number
 * of matches, or -1 on bad arguments. */
int64_t oracle_match_pair(const uint8_t* descA, const uint32_t* codesA, const uint8_t* bucketsA, uint32_t nA,
                          const uint8_t* descB, const uint32_t* codesB, const uint8_t* bucketsB, uint32_t nB,
                          const oracle_params* p, const double* F, const float* kptsA, const float* kptsB,
                          int32_t* match, oracle_query_detail* detail);

/* Many pairs over an image set stored back to back (img_off[i]..img_off[i+1]),
 * split across n_threads POSIX threads (pairs are independent, Sec. 1).
 * With ORACLE_MUTUAL each pair (A, B) is also matched as (B, A) with F
 * transposed (x_A^T F^T x_B = 0), and (q, j) is kept only if the reverse
 * match of j is q.
 * Output: match_off[P+1] (prefix of per-pair counts) and matches[...][2] =
 * (query index in A, index in B) ascending in the query index; matches may be
 * NULL to only count.  F is [P][9] or NULL; kpts is [n_total][2] or NULL.
 * Returns total matches, or -1 on bad arguments / capacity exceeded
 * (cap = capacity of matches in entries). */
int64_t oracle_match_pairs(const uint8_t* desc, const uint64_t* img_off, uint32_t n_images,
                           const uint32_t* codes, const uint8_t* buckets,
                           const uint32_t* pairs, uint32_t P, const oracle_params* p,
                           const double* F, const float* kpts,
                           uint64_t* match_off, uint32_t* matches, uint64_t cap, int n_threads);

/* Epipolar predicate of Eq. 1-2 for one (query, candidate) pair: the line
 * l = F p_q in image B, keep p' iff (l . p')^2 <= d^2 (a^2 + b^2). */
int oracle_epipolar_keep(const double* F, float xq, float yq, float xc, float yc, double d);

#ifdef __cplusplus
}
#endif
#endif
