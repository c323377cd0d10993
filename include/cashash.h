/*
 * cashash.h -- C-ABI of the GB300 (sm_103a) Cascade Hashing image matcher.
 *
 * The library implements Cascade Hashing (CasHash) SIFT matching between
 * image pairs as described in Xu, Sun and Tao, "GPU Accelerated Cascade
 * Hashing Image Matching for Large Scale 3D Reconstruction":
 *   Sec. 3.1 ("Review of Cascade Hashing")
 *            Step 1  lookup in several tables of m-bit short codes
 *            Step 2  remapping to an n-bit code, Hamming distance
 *            Step 3  ranking: the k candidates of smallest Hamming distance
 *            Step 4  squared Euclidean distance on those k, Lowe's ratio test
 *   Sec. 5.1 ("The Improved Parallel Calculation of Hashing Code")
 *                    hash bit = sign of the inner product with a random vector
 *   Sec. 5.2 ("Improved Parallel Euclidean Distance Calculation") Step 4 on the GPU
 *   Sec. 6   ("Improved Parallel Hashing Ranking") optional Hamming threshold
 *                    tau before ranking
 *   Sec. 7.1 ("First Stage of Image Matching") Ga-CasHash: top-scale subsets, F
 *   Sec. 7.2 ("Second Stage of Guided Matching"), Eq. 1-2: optional epipolar
 *                    band before ranking
 *   Sec. 4   ("Three-Level Data Scheduling Strategy") is replaced by resident
 *                    device sets and pinned, chunked host staging (cashash_run_host)
 *
 * Results are defined exactly (bit-exact, not approximately):
 *   - descriptors are centred by the mean over every descriptor of the set
 *     passed to cashash_build_codes (or by a caller-given mean);
 *   - bit b of a feature is [v_b > 0] where v_b is the projection
 *     sum_j R[b][j] * (x_j - mu_j) evaluated in IEEE double, j ascending,
 *     each difference, product and sum rounded to nearest (no fused
 *     multiply-add); the GPU computes a cheaper bounded approximation and,
 *     whenever the approximation is within its rounding bound of zero,
 *     decides the sign of exactly that double sequence (from a tree sum of
 *     the same rounded products with a bound on its distance from the
 *     sequence, or from the sequence itself inside that bound);
 *   - the candidate set of a query is the set of points of the other image
 *     that share its bucket in at least one table (each point once);
 *   - ranking orders candidates by (Hamming distance, candidate index);
 *   - squared distances are exact integers; the nearest candidate (smaller
 *     index on equal distance) matches when den^2 * d1 < num^2 * d2 and at
 *     least two candidates were ranked.
 *
 * Conventions for every entry point:
 *   - "DEVICE" pointers are CUDA device memory of the current device,
 *     owned by the caller and left untouched by the library beyond what the
 *     call documents; "HOST" pointers are ordinary host memory.
 *   - Calls that take a cudaStream_t are asynchronous with respect to the
 *     host and ordered on that stream (0 = legacy default stream).  Device
 *     side errors (capacity exceeded, bad index) are recorded in a status
 *     word of the context and returned by cashash_sync_status().
 *   - Every entry point returns a cashash_status; nothing aborts, traps or
 *     throws across the boundary.
 *   - A context is not thread-safe: use one per host thread.
 */
#ifndef CASHASH_H
#define CASHASH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* cashash_stream_t; /* ABI-identical to cudaStream_t */
typedef struct cashash_ctx cashash_ctx;          /* opaque context */

typedef enum {
  CASHASH_OK = 0,
  CASHASH_EINVAL = 1,     /* bad argument (null pointer, size out of range, bad parameter) */
  CASHASH_ENOMEM = 2,     /* device or pinned host allocation failed */
  CASHASH_ECUDA = 3,      /* a CUDA runtime call failed */
  CASHASH_EOVERFLOW = 4,  /* match capacity too small; match_off[P] holds the total needed */
  CASHASH_EDEVICE = 5,    /* a kernel recorded an internal error (index out of range) */
  CASHASH_ETIMEOUT = 6,   /* a bounded device or staging wait ran out */
  CASHASH_ENOTSUP = 7     /* parameter combination the library does not support */
} cashash_status;

enum { CASHASH_FP32 = 0, CASHASH_BF16 = 1 };                          /* projection precision form */
enum { CASHASH_SCHED_PER_PAIR = 0, CASHASH_SCHED_PERSISTENT = 1 };   /* matching schedule */

#define CASHASH_DIM 128          /* SIFT descriptor length d (Sec. 5.1) */
#define CASHASH_MAX_TABLES 8
#define CASHASH_MAX_K 32
#define CASHASH_MAX_IMAGE 16777215u   /* features per image (24-bit candidate index) */

/* Method parameters.  The paper fixes none of m, n, the number of tables, k
 * or the ratio; defaults used by the benchmarks are given in brackets. */
typedef struct {
  uint32_t code_bits;       /* n of Step 2: 32, 64, 96 or 128 [128] */
  uint32_t n_tables;        /* lookup tables of Step 1: 1..8 [6] */
  uint32_t bits_per_table;  /* m of Step 1: 0..8 [8] (0 = one bucket) */
  uint32_t top_k;           /* k of Step 3: 1..32 [10] */
  uint32_t ratio_num;       /* Lowe ratio num/den [4/5] */
  uint32_t ratio_den;
  uint32_t tau;             /* Sec. 6 threshold: candidates with Hamming > tau are dropped;
                               tau >= code_bits turns it off [code_bits] */
  uint32_t precision;       /* CASHASH_FP32 (CUDA-core projection) or CASHASH_BF16 (tensor cores) */
  uint32_t schedule;        /* CASHASH_SCHED_PER_PAIR (one launch per pair) or
                               CASHASH_SCHED_PERSISTENT (one launch over the whole pair list) */
  uint32_t flags;           /* CASHASH_FLAG_* below, ORed [0] */
  double epi_px;            /* Sec. 7.2 threshold d in pixels; < 0 turns the band off [-1] */
} cashash_params;

/* cashash_params.flags (readings beyond the paper, off by default):
 * CASHASH_FLAG_MUTUAL: a match (q, j) of pair (A, B) is kept only when matching
 *   j of B against A by the same procedure (Steps 1-4, tau, the band with F
 *   transposed) gives q; every pair is matched in both directions.
 * CASHASH_FLAG_ACCEPT_SINGLE: a query with exactly one ranked candidate
 *   matches it (by default the ratio test needs a second neighbour). */
#define CASHASH_FLAG_MUTUAL 1u
#define CASHASH_FLAG_ACCEPT_SINGLE 2u

/* Fills p with the defaults listed above. */
void cashash_default_params(cashash_params* p);

/* An image set: images stored back to back.  Feature f of image i is row
 * img_off[i] + f.  All DEVICE arrays are caller-allocated. */
typedef struct {
  uint32_t n_images;
  uint32_t reserved;
  uint64_t n_features;       /* = img_off[n_images] */
  const uint64_t* img_off;   /* HOST [n_images + 1], non-decreasing, img_off[0] = 0;
                                every image has at most CASHASH_MAX_IMAGE features */
  const uint8_t* desc;       /* DEVICE [n_features][128] uint8 descriptors, 16-byte aligned */
  uint32_t* codes;           /* DEVICE [n_features][4] out: n-bit remapping code, bit b in
                                word b/32 at bit b%32, unused bits 0 (Step 2) */
  uint8_t* buckets;          /* DEVICE [n_features][8] out: byte t = short code of table t
                                (Step 1), bit i from projection row code_bits + t*m + i;
                                bytes >= n_tables are 0 */
  uint32_t* sqnorm;          /* DEVICE [n_features] out: sum_j x_j^2 (used by Step 4) */
  uint8_t* tables;           /* DEVICE out: lookup tables of Step 1, cashash_tables_bytes()
                                bytes, 16-byte aligned; layout private to the library */
  const float* kpts;         /* DEVICE [n_features][2] key-point (x, y) in pixels, or NULL;
                                needed only when epi_px >= 0 */
} cashash_set;

/* Bytes of the lookup-table buffer for a set (HOST img_off).  0 on bad input. */
uint64_t cashash_tables_bytes(const cashash_params* p, const uint64_t* img_off, uint32_t n_images);

/* Creates a context on the current CUDA device.  R_host is the matrix of
 * random vectors r_k of Sec. 5.1: [code_bits + n_tables * bits_per_table]
 * rows of 128 doubles, row-major; rows 0..code_bits-1 give the remapping
 * code, row code_bits + t*m + i gives bit i of table t.  The context copies
 * R and owns its device workspace.  Errors: EINVAL, ENOTSUP, ENOMEM, ECUDA. */
int cashash_create(cashash_ctx** out, const cashash_params* p, const double* R_host);

/* Releases the context and its workspace (after synchronising its work). */
void cashash_destroy(cashash_ctx* ctx);

/* Sec. 5.1 + Steps 1-2: hash codes and lookup tables for every feature of
 * the set.  mean_host: HOST [128] caller-given centre, or NULL to use the
 * mean over every descriptor of the set (computed exactly from integer
 * column sums, one correctly rounded division).  Writes set->codes,
 * set->buckets, set->sqnorm and set->tables.  Asynchronous on `stream`.
 * With mean_host NULL, a second and later call for the same set (the same
 * struct contents and image offsets) under the same profiling setting
 * replays the launch sequence as one CUDA graph captured on that second
 * call; it reads the buffers' current contents.  Calls on one context must
 * not overlap.  Errors: EINVAL (null pointer, bad offsets), ENOMEM, ECUDA. */
int cashash_build_codes(cashash_ctx* ctx, const cashash_set* set, const double* mean_host,
                        cashash_stream_t stream);

/* Diagnostic of the rounding bound of the projection (Sec. 5.1; not needed
 * for matching).  For features [first, first + count) of `set`, runs the
 * context's projection form (precision FP32 or BF16) with the centre and row
 * constants of the last cashash_build_codes on this context, and writes, row-
 * major [count][rows] with rows = code_bits + n_tables * bits_per_table:
 *   approx: the FP32 approximation v~_b - c_b of each projection
 *           v_b = sum_j R_bj (x_j - mu_j), as the kernel computed it;
 *   bound:  the bound E_b the kernel compares |approx| with (a projection with
 *           |approx| <= E_b is re-evaluated exactly in double, any other takes
 *           the sign of approx), valid when |approx - v_b| <= E_b.
 * approx, bound: DEVICE, caller-allocated, 4-byte aligned.  The set's codes
 * and tables are not written (the kernels' other outputs go to scratch that
 * the call allocates and frees).  Synchronous on `stream`.
 * Errors: EINVAL (no cashash_build_codes yet, bad range), ENOMEM, ECUDA. */
int cashash_projection_bounds(cashash_ctx* ctx, const cashash_set* set, uint64_t first, uint64_t count,
                              float* approx, float* bound, cashash_stream_t stream);

/* The centre used by the last cashash_build_codes (HOST [128] out).
 * Synchronises the context's stream.  Errors: EINVAL, ECUDA. */
int cashash_get_mean(cashash_ctx* ctx, double* mean_out);

/* A pair list prepared for matching (work items, per-pair offsets). */
typedef struct cashash_plan cashash_plan;

/* Prepares pairs_host (HOST [P][2] uint32: query image, candidate image)
 * for matching against `set`.  The plan keeps copies; it is valid while the
 * set's device buffers are.  Errors: EINVAL (image index out of range),
 * ENOMEM, ECUDA. */
int cashash_plan_create(cashash_ctx* ctx, const cashash_set* set, const uint32_t* pairs_host, uint32_t P,
                        cashash_plan** out);
void cashash_plan_destroy(cashash_plan* plan);

/* Steps 1-4 (+ Sec. 6 tau, + Sec. 7.2 epipolar band when epi_px >= 0) for
 * every pair of the plan.  Outputs (DEVICE, caller-allocated):
 *   match_off [P + 1] uint64: matches of pair i are entries
 *                             match_off[i] .. match_off[i+1]-1;
 *   matches   [cap][2] uint32: (query feature index in the query image,
 *                             candidate feature index in the other image),
 *                             ascending query index within each pair.
 * F_dev: DEVICE [P][9] row-major fundamental matrices (x_cand^T F x_query = 0)
 * when epi_px >= 0, else ignored (may be NULL).  When the total exceeds cap,
 * match_off is still complete, nothing beyond cap is written and
 * cashash_sync_status() returns EOVERFLOW.  Asynchronous on `stream`.
 * With the persistent schedule all pairs are matched by one batched kernel:
 * by default a bucket join whose Hamming distances come from the tensor cores
 * when every query image fits its shared-memory counters (at least 40,000
 * features), else a speculative per-query kernel (cashash_plan_autotune may
 * choose otherwise); the launch sequence
 * is captured once as a CUDA graph (per set of output pointers, F and
 * profiling setting) and replayed on `stream`; calls on the same plan must
 * not overlap.
 * Errors: EINVAL, ECUDA. */
int cashash_match_plan(cashash_ctx* ctx, cashash_plan* plan, const double* F_dev, uint64_t* match_off,
                       uint32_t* matches, uint64_t cap, cashash_stream_t stream);

/* Performance hint for the batched (persistent) schedule: the Hamming
 * distance at or below which candidates are kept for ranking when matching
 * starts.  The kernels then adapt it per pair to the k-th ranked distances
 * they observe (unless `fixed` is non-zero).  Results never depend on it: a
 * query for which the hint turns away candidates it needed is re-matched
 * exactly.  hamming >= code_bits disables the speculation.
 * Errors: EINVAL, ECUDA. */
int cashash_plan_set_threshold_hint(cashash_plan* plan, uint32_t hamming, int fixed);

/* Kernel configuration of a batched (persistent) plan.  Every configuration
 * gives the same, exact results; they differ in speed only.  The paper has no
 * counterpart (it runs one kernel shape). */
enum { CASHASH_KERNEL_JOIN = 1, CASHASH_KERNEL_QUERY = 2, CASHASH_KERNEL_JOIN_TC = 3, CASHASH_KERNEL_WARP = 4 };
typedef struct {
  uint32_t kernel;       /* CASHASH_KERNEL_JOIN: bucket join with warp-level (mma.sync) tensor-core
                            Hamming distances (query images that fit its shared-memory counters);
                            CASHASH_KERNEL_JOIN_TC: the same join with tcgen05 MMAs into tensor
                            memory, 128 query rows per tile (same limit);
                            CASHASH_KERNEL_QUERY: per-query speculative kernel over shared-memory
                            staged table chunks;
                            CASHASH_KERNEL_WARP: one warp per query, exact without a threshold guess
                            (no calibration; the fit for a few pairs, where the other kernels leave
                            most SMs idle) */
  uint32_t tile;         /* JOIN: candidate tiles of 8 columns held in registers (2 or 4; 4 with
                            the band); JOIN_TC, WARP: ignored (0);
                            QUERY: queries per CTA (256, or 512 when top_k <= 16) */
  uint32_t ctas_per_sm;  /* JOIN, JOIN_TC: resident CTAs per SM, 0 = as many as fit (JOIN_TC: at most
                            2); QUERY, WARP: ignored */
  uint32_t reserved;
  double ms_sample;      /* set by cashash_plan_autotune: matching time (ms) of its sample with
                            this configuration; -1 otherwise */
} cashash_tuning;

/* The configuration a plan matches with (chosen at creation: the join when it
 * applies, else the per-query kernel).  Errors: EINVAL. */
int cashash_plan_get_tuning(const cashash_plan* plan, cashash_tuning* out);

/* Forces a configuration (fields normalised to supported values; the plan's
 * captured graph is dropped).  Errors: EINVAL (not a batched plan),
 * ENOTSUP (the join does not apply to this plan: a query image exceeds its
 * shared-memory counters), ENOMEM, ECUDA. */
int cashash_plan_set_tuning(cashash_plan* plan, const cashash_tuning* t);

/* Autotuner: times every applicable configuration (three runs after two
 * untimed ones, in two interleaved rounds; a configuration more than 25 %
 * behind after the first round is not timed again; each keeps its minimum) and
 * keeps the plan's default configuration unless another is more than 3 %
 * faster (then the fastest).  max_pairs == 0 (or >= the plan's
 * pairs): on the plan itself, which is exact about locality and tails but
 * costs up to about 60 plan runs; else on a sample of the plan's pairs spread over
 * their N_A * N_B cost order, max(max_pairs, 16 per SM) pairs so that the
 * tails of the persistent kernels weigh roughly as in the full run.  F_dev as
 * for cashash_match_plan.  Call it after cashash_build_codes for the plan's
 * set: the timed runs match the set's current codes.  Synchronises `stream`;
 * allocates temporary device buffers (outputs of the timed runs); the plan's
 * thresholds start afresh.  Errors: EINVAL, ENOMEM, ECUDA. */
int cashash_plan_autotune(cashash_ctx* ctx, cashash_plan* plan, const double* F_dev, uint32_t max_pairs,
                          cashash_stream_t stream);

/* Convenience: plan + match + plan release in one call (same outputs). */
int cashash_match_pairs(cashash_ctx* ctx, const cashash_set* set, const uint32_t* pairs_host, uint32_t P,
                        const double* F_dev, uint64_t* match_off, uint32_t* matches, uint64_t cap,
                        cashash_stream_t stream);

/* Synchronises `stream` and returns (then clears) the first device-side
 * error recorded since the last call: OK, EOVERFLOW or EDEVICE. */
int cashash_sync_status(cashash_ctx* ctx, cashash_stream_t stream);

/* End-to-end from HOST buffers: stages descriptors host -> device through
 * pinned buffers on a side stream (chunks of at most stage_bytes, 0 = 4 GiB),
 * builds codes and tables, matches every pair, and copies match_off and the
 * matches back.  The column sums of the centre are taken block by block (at
 * most 256 MiB) as each block lands, overlapping the rest of the copy; the
 * projections wait for the whole set (their centre is its mean).  With
 * profiling on, the copies are timed as stages H2D and D2H.  desc_host: HOST [img_off[n_images]][128]; kpts_host /
 * F_host may be NULL unless epi_px >= 0.  match_off_host: HOST [P + 1];
 * matches_host: HOST [cap][2].  Synchronous.  Errors: EINVAL, ENOMEM, ECUDA,
 * EOVERFLOW (match_off_host complete, matches truncated to cap), EDEVICE. */
int cashash_run_host(cashash_ctx* ctx, const uint8_t* desc_host, const uint64_t* img_off, uint32_t n_images,
                     const float* kpts_host, const uint32_t* pairs_host, uint32_t P, const double* F_host,
                     uint64_t* match_off_host, uint32_t* matches_host, uint64_t cap, uint64_t stage_bytes);

/* Kernel configuration of the plans cashash_run_host and
 * cashash_match_chunked build for batched contexts (t: kernel JOIN or QUERY,
 * tile and ctas_per_sm as for cashash_plan_set_tuning, e.g. the result of
 * cashash_plan_autotune on the same workload), or NULL for the default
 * choice.  Drops run_host's cached plan.  Where the join does not apply the
 * default stays.  Errors: EINVAL. */
int cashash_set_host_tuning(cashash_ctx* ctx, const cashash_tuning* t);

/* The configuration set by cashash_set_host_tuning (HOST out; kernel 0 when
 * none is set).  Errors: EINVAL. */
int cashash_get_host_tuning(const cashash_ctx* ctx, cashash_tuning* out);

/* Largest query image (features) that cashash_match_pair_noalloc accepts. */
#define CASHASH_NOALLOC_MAX_QUERIES 65536u

/* Allocation-free matching of one image pair.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc at the
 * moment they need a match -- a real-time pipeline that must not allocate or
 * implicitly synchronise the device after start-up, a host that gives all
 * device memory to its own pool allocator, or a caller whose device memory is
 * already committed.  It needs no context and allocates nothing: its scratch
 * (pair record, work items, per-query results, match counter, status word)
 * is one fixed, file-scope device array of about 260 KB that every GPU
 * loading this library holds until the process exits.
 *
 * Computes for pair (image_a queries, image_b candidates) of `set` the same
 * matches as cashash_match_pairs would for that single pair with the same
 * parameters (p->precision and p->schedule are ignored: the codes and lookup
 * tables of `set` must already have been built, e.g. by cashash_build_codes).
 * p->code_bits, p->n_tables and p->bits_per_table must be the values the
 * set's codes and tables were built with: the set does not record them, and
 * other values make the kernel read the tables with the wrong layout.
 *   match_off: DEVICE [2] uint64 out: 0 and the number of matches;
 *   matches:   DEVICE [cap][2] uint32 out: (query index, candidate index),
 *              ascending query index; entries beyond cap are not written, so
 *              match_off[1] > cap means the list was truncated.
 *   F_dev:     DEVICE [9] fundamental matrix when p->epi_px >= 0, else NULL.
 * Asynchronous on `stream`.  Every call looks up the scratch array's device
 * address in the current device's context (this allocates nothing, and stays
 * right after cudaDeviceReset); the first call on a device may load the
 * library's device code, so make it before any stream capture.  Every call
 * shares the one array: calls that overlap on the GPU (other streams, other
 * host threads) race and must be serialised by the caller.  Device-side
 * errors (a truncated list, an index out of range) are ORed into the array's
 * status word by every call and reported by cashash_noalloc_status.
 * Errors: EINVAL (bad parameters or set, image index out of range, or
 * image_a larger than CASHASH_NOALLOC_MAX_QUERIES features), ENOTSUP
 * (CASHASH_FLAG_MUTUAL: the reverse match would need a second scratch),
 * ECUDA. */
int cashash_match_pair_noalloc(const cashash_params* p, const cashash_set* set, uint32_t image_a,
                               uint32_t image_b, const double* F_dev, uint64_t* match_off, uint32_t* matches,
                               uint64_t cap, cashash_stream_t stream);

/* Device-side status of the allocation-free calls on the current device:
 * synchronises `stream` (which must order after those calls), reads the
 * status word of the shared scratch array and clears it.  Allocates nothing.
 * Returns OK, EDEVICE (a kernel recorded an index out of range) or EOVERFLOW
 * (a list was longer than its cap; match_off[1] holds its length), for every
 * cashash_match_pair_noalloc call since the last cashash_noalloc_status;
 * ECUDA when a CUDA call fails. */
int cashash_noalloc_status(cashash_stream_t stream);

/* Resumable chunked matching of long pair lists (out-of-core outputs; the
 * paper has no counterpart, its loader streams inputs).  The callback of one
 * chunk: pairs [first, first + count) of the caller's list were matched;
 * match_off (HOST [count + 1], starting at 0 for this chunk) and matches
 * (HOST [match_off[count]][2], as in cashash_match_plan) are valid during the
 * call only.  Return 0 to continue, non-zero to stop after this chunk. */
typedef int (*cashash_chunk_fn)(void* user, uint64_t first, uint32_t count, const uint64_t* match_off,
                                const uint32_t* matches);

/* Matches pairs_host[*cursor .. P) (HOST [P][2]) against the resident set
 * `set` in chunks of chunk_pairs pairs (one plan per chunk, with the context's
 * schedule), copies each chunk's lists to pinned host buffers and calls fn.
 * *cursor advances past every chunk whose callback has returned, so a run
 * stopped by the callback, or failed, resumes by calling again with the same
 * cursor.  F_dev: DEVICE [P][9] for the whole list when epi_px >= 0, else
 * NULL.  Synchronous on `stream`.  Returns OK when the list is done or the
 * callback stopped it (then *cursor < P).  Errors: EINVAL (cursor > P, bad
 * pair, chunk_pairs 0, NULL callback), ENOMEM, ECUDA, EDEVICE; the cursor then
 * still points at the chunk that failed. */
int cashash_match_chunked(cashash_ctx* ctx, const cashash_set* set, const uint32_t* pairs_host, uint64_t P,
                          const double* F_dev, uint32_t chunk_pairs, uint64_t* cursor, cashash_chunk_fn fn,
                          void* user, cashash_stream_t stream);

/* Stage ids of cashash_stats.ms_stage. */
enum {
  CASHASH_STAGE_CENTRE = 0,     /* column sums, centre and per-row constants */
  CASHASH_STAGE_PROJECT = 1,    /* projection, signs, rounding-bound test */
  CASHASH_STAGE_REEVAL = 2,     /* exact double re-evaluation of flagged projections */
  CASHASH_STAGE_TABLES = 3,     /* lookup tables of Step 1 */
  CASHASH_STAGE_MATCH = 4,      /* matching kernel(s): Steps 1-4 */
  CASHASH_STAGE_COMPACT = 5,    /* per-pair offsets and compaction of the match lists */
  CASHASH_STAGE_CALIBRATE = 6,  /* batched schedule: per-pair Hamming threshold guesses */
  CASHASH_STAGE_FALLBACK = 7,   /* batched schedule: exact re-matching of the queries left pending */
  CASHASH_STAGE_H2D = 8,        /* cashash_run_host: host -> device copies of the inputs (copy stream) */
  CASHASH_STAGE_D2H = 9,        /* cashash_run_host: device -> host copies of the match lists */
  CASHASH_N_STAGES = 10
};

/* Counters of the last build/match calls (host copies after the call's stream sync). */
typedef struct {
  uint64_t n_features;        /* features hashed by the last build */
  uint64_t n_reevaluated;     /* projections re-evaluated in double (|approx| under the bound) */
  uint64_t n_pairs;           /* pairs in the last match */
  uint64_t n_matches;         /* matches found by the last match */
  uint64_t n_work_items;      /* (pair, query tile) items of the last match */
  uint64_t n_launches;        /* kernels launched by this context since it was created */
  double ms_stage[CASHASH_N_STAGES];  /* with profiling on: device milliseconds of each stage of
                                         the last build/match (CUDA events recorded on the
                                         launching stream); -1 when not measured */
} cashash_stats;

/* Turns per-stage CUDA-event timing on (1) or off (0).  Off by default. */
int cashash_set_profiling(cashash_ctx* ctx, int on);

/* Synchronises the context's last stream and fills *out.  Errors: EINVAL, ECUDA. */
int cashash_get_stats(cashash_ctx* ctx, cashash_stats* out);

/* Static text for a status code. */
const char* cashash_strerror(int status);

/* ------------------------------------------------------------------------
 * Ga-CasHash, first stage (Sec. 7.1).  The top 20 % of each image's features
 * by SIFT scale are matched exhaustively with CasHash; a pair with at least
 * 16 matches gets a fundamental matrix from the GPU, and goes on to the
 * guided matching of Sec. 7.2 (the band, epi_px >= 0, with that F) when at
 * least 2/3 of its matches are inliers.  The paper names no estimator: this
 * is the normalised 8-point algorithm (Hartley 1997) inside RANSAC (Fischler
 * and Bolles 1981) with the squared Sampson distance as the inlier test and a
 * least-squares refit on the best hypothesis' inliers (at least 8), all in
 * FP64.  The random draws are caller-given: word k (k = 0..7) of hypothesis h
 * of pair p, u = words[(p * n_hyp + h) * 8 + k], picks r = floor(u (m - k) /
 * 2^32), the r-th smallest of the m match indices not drawn before.
 * Convention: x_B^T F x_A = 0 for the pair (A, B).  F is returned with unit
 * Frobenius norm and its largest-magnitude entry (first on ties) positive.
 * ------------------------------------------------------------------------ */
#define CASHASH_GA_MAX_HYP 4096u

typedef struct {
  uint32_t top_pct;      /* 20: each image keeps ceil(n * top_pct / 100) features (1..100) */
  uint32_t min_matches;  /* 16: pairs with fewer stage-1 matches get no F (>= 8) */
  uint32_t n_hyp;        /* 256: at most this many RANSAC hypotheses per pair (1..CASHASH_GA_MAX_HYP) */
  uint32_t inlier_num;   /* 2 */
  uint32_t inlier_den;   /* 3: accepted when inlier_den * inliers >= inlier_num * matches */
  uint32_t kernel;       /* 0: matching kernel of the subsets chosen by their size (the per-query
                            kernel when the mean subset image has fewer than 4096 features, else
                            the join); CASHASH_KERNEL_JOIN / CASHASH_KERNEL_QUERY force one */
  double thresh_px;      /* 3.0: inlier when the Sampson distance is <= thresh_px pixels */
  double confidence;     /* 0.99: hypotheses run in batches of 32; after a batch RANSAC stops when
                            (1 - w^8)^N <= 1 - confidence (Hartley and Zisserman, Algorithm 4.5;
                            N hypotheses done, w the best inlier fraction so far, each step one
                            correctly rounded double operation); >= 1: all n_hyp run */
} cashash_ga_params;

typedef struct {
  uint32_t n_matches;    /* stage-1 matches of the pair */
  uint32_t n_inliers;    /* inliers of the returned F (0 when there is none) */
  uint32_t best_hyp;     /* winning hypothesis, or 0xFFFFFFFF */
  uint32_t accepted;     /* 1: the pair goes on to guided matching with F */
  uint32_t n_evaluated;  /* hypotheses run (a multiple of 32, or n_hyp) */
  uint32_t reserved[3];
} cashash_ga_info;

/* Fills gp with the defaults listed above. */
void cashash_ga_default_params(cashash_ga_params* gp);

/* The parameters a context was created with (HOST out).  Errors: EINVAL. */
int cashash_get_params(const cashash_ctx* ctx, cashash_params* out);

/* HOST sub_off [n_images + 1] out: offsets of the selected subsets
 * (image i keeps ceil(n_i * top_pct / 100) features).  Errors: EINVAL. */
int cashash_ga_subset_offsets(const uint64_t* img_off, uint32_t n_images, uint32_t top_pct, uint64_t* sub_off);

/* Selection by scale: DEVICE scale [n_features] (finite; -0 counts as 0),
 * HOST img_off; DEVICE sel out [sub_off[n_images]]: the global indices of
 * each image's ceil(n * top_pct / 100) features of largest scale (ties to the
 * lower index), ascending within the image.  Sets of fewer than 2^32
 * features.  Asynchronous on `stream`.  Errors: EINVAL, ENOMEM, ECUDA. */
int cashash_ga_select(const float* scale, const uint64_t* img_off, uint32_t n_images, uint32_t top_pct,
                      uint32_t* sel, cashash_stream_t stream);

/* RANSAC F estimation for every pair from its match list: DEVICE kpts
 * [N][2] (HOST img_off gives the images), HOST pairs [P][2], DEVICE
 * match_off [P + 1] and matches [.][2] (query, candidate) local indices as
 * written by cashash_match_plan, DEVICE words [P][n_hyp][8]; DEVICE out
 * F [P][9] (row-major; zeros without an estimate) and info [P].  Reads
 * match_off[P] on the host (synchronises `stream` once); the rest is
 * asynchronous.  Errors: EINVAL, ENOMEM, ECUDA. */
int cashash_estimate_F(const float* kpts, const uint64_t* img_off, uint32_t n_images, const uint32_t* pairs,
                       uint32_t P, const uint64_t* match_off, const uint32_t* matches, const cashash_ga_params* gp,
                       const uint32_t* words, double* F, cashash_ga_info* info, cashash_stream_t stream);

/* The whole first stage for the pairs of `set` (its desc and kpts; codes,
 * tables etc. are not used): selection, the subsets' codes with the caller's
 * centre mean_host (HOST [128]: the full set's, e.g. from cashash_get_mean,
 * so stage-1 codes are the full set's codes of the selected features),
 * CasHash matching of the subsets with ctx (which must have epi_px < 0), then
 * cashash_estimate_F.  Work buffers are allocated and released inside
 * (stream-ordered); the call synchronises `stream` after the subset matching,
 * and F / info are written asynchronously on it after that.  Errors: EINVAL,
 * ENOMEM, ECUDA, EDEVICE. */
int cashash_ga_stage1(cashash_ctx* ctx, const cashash_set* set, const float* scale, const double* mean_host,
                      const uint32_t* pairs, uint32_t P, const cashash_ga_params* gp, const uint32_t* words,
                      double* F, cashash_ga_info* info, cashash_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif
