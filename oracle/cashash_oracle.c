/*
 * cashash_oracle.c -- plain CPU oracle for Cascade Hashing image matching.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product library.
 *
 * Built with -ffp-contract=off so that every double operation below is one
 * IEEE round-to-nearest operation in the order written.
 *
 * Each function names the passage of the paper it follows; the readings
 * taken where the paper is silent are stated where they are used.
 */
#include "cashash_oracle.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ------------------------------------------------------------------------ */
/* Centring (the paper is silent; reading: one mean over the whole set of    */
/* descriptors passed to one code-building call, so that the hyperplanes of  */
/* Sec. 5.1 are the same for every image).                                   */
/* ------------------------------------------------------------------------ */
void oracle_mean(const uint8_t* desc, uint64_t n, double* mu) {
  uint64_t s[ORACLE_DIM];
  memset(s, 0, sizeof s);
  for (uint64_t f = 0; f < n; ++f)
    for (int j = 0; j < ORACLE_DIM; ++j) s[j] += desc[f * ORACLE_DIM + j];
  for (int j = 0; j < ORACLE_DIM; ++j)
    mu[j] = (n == 0) ? 0.0 : (double)s[j] / (double)n;
}

/* ------------------------------------------------------------------------ */
/* Sec. 5.1: a hash bit is the sign of the inner product of the (centred)    */
/* descriptor with a random vector r_k.  Reading: double precision, terms    */
/* taken in index order j = 0..127, each term (x_j - mu_j) * r_kj rounded,   */
/* accumulated left to right; no fused multiply-add.                        */
/* ------------------------------------------------------------------------ */
double oracle_projection(const uint8_t* x, const double* mu, const double* Rrow) {
  double s = 0.0;
  for (int j = 0; j < ORACLE_DIM; ++j) {
    double t = (double)x[j] - mu[j];
    double p = Rrow[j] * t;
    s = s + p;
  }
  return s;
}

static int params_ok(const oracle_params* p) {
  return p && p->code_bits >= 1 && p->code_bits <= 128 && p->n_tables >= 1 &&
         p->n_tables <= ORACLE_MAX_TABLES && p->bits_per_table <= 8 && p->top_k >= 1 &&
         p->top_k <= ORACLE_MAX_K && p->ratio_den > 0;
}

/* Steps 1 and 2 of Sec. 3.1 with the hash functions of Sec. 5.1.  Rows
 * 0..n-1 of R give the n-bit remapping code (Step 2); rows n + t*m + i give
 * bit i of the m-bit short code of lookup table t (Step 1).  Sign at exactly
 * zero is bit 0 (reading: the strict test v > 0). */
void oracle_hash(const uint8_t* desc, uint64_t n, const double* mu, const double* R,
                 const oracle_params* p, uint32_t* codes, uint8_t* buckets) {
  const uint32_t nb = p->code_bits, m = p->bits_per_table, T = p->n_tables;
  for (uint64_t f = 0; f < n; ++f) {
    const uint8_t* x = desc + f * ORACLE_DIM;
    uint32_t* c = codes + f * 4;
    c[0] = c[1] = c[2] = c[3] = 0;
    for (uint32_t b = 0; b < nb; ++b) {
      double v = oracle_projection(x, mu, R + (uint64_t)b * ORACLE_DIM);
      if (v > 0.0) c[b >> 5] |= 1u << (b & 31);
    }
    for (uint32_t t = 0; t < T; ++t) {
      uint32_t id = 0;
      for (uint32_t i = 0; i < m; ++i) {
        double v = oracle_projection(x, mu, R + (uint64_t)(nb + t * m + i) * ORACLE_DIM);
        if (v > 0.0) id |= 1u << i;
      }
      buckets[f * T + t] = (uint8_t)id;
    }
  }
}

/* Every projection of a block of features, v[f][b] = oracle_projection of
 * feature f with row b of R, b < rows (the values whose signs oracle_hash
 * takes); used to measure the GPU's rounding bounds. */
void oracle_projections(const uint8_t* desc, uint64_t n, const double* mu, const double* R, uint32_t rows,
                        double* v) {
  for (uint64_t f = 0; f < n; ++f)
    for (uint32_t b = 0; b < rows; ++b)
      v[f * rows + b] = oracle_projection(desc + f * ORACLE_DIM, mu, R + (uint64_t)b * ORACLE_DIM);
}

/* Sec. 7.2, Eq. 1-2: the epipolar line of the query is l_q = F p_q with
 * p_q = (x, y, 1); a candidate p' = (x', y', 1) is kept when its distance to
 * l_q is at most d.  Eq. 2 as printed has no absolute value; the distance of
 * a point to a line is meant, so the test is |a x' + b y' + c| <= d sqrt(a^2+b^2),
 * evaluated squared to avoid the square root:
 *   (a x' + b y' + c)^2 <= d^2 (a^2 + b^2).
 * All in double, left to right, no fused multiply-add. */
int oracle_epipolar_keep(const double* F, float xq, float yq, float xc, float yc, double d) {
  const double x = (double)xq, y = (double)yq, xp = (double)xc, yp = (double)yc;
  const double a = (F[0] * x + F[1] * y) + F[2];
  const double b = (F[3] * x + F[4] * y) + F[5];
  const double c = (F[6] * x + F[7] * y) + F[8];
  const double num = (a * xp + b * yp) + c;
  return num * num <= (d * d) * (a * a + b * b);
}

typedef struct {
  uint32_t h, j;
} hk;

static int cmp_hk(const void* pa, const void* pb) {
  const hk* a = (const hk*)pa;
  const hk* b = (const hk*)pb;
  if (a->h != b->h) return a->h < b->h ? -1 : 1;
  if (a->j != b->j) return a->j < b->j ? -1 : 1;
  return 0;
}

typedef struct {
  int32_t d;
  uint32_t j;
} dk;

static int cmp_dk(const void* pa, const void* pb) {
  const dk* a = (const dk*)pa;
  const dk* b = (const dk*)pb;
  if (a->d != b->d) return a->d < b->d ? -1 : 1;
  if (a->j != b->j) return a->j < b->j ? -1 : 1;
  return 0;
}

static uint32_t hamming(const uint32_t* a, const uint32_t* b) {
  return (uint32_t)(__builtin_popcount(a[0] ^ b[0]) + __builtin_popcount(a[1] ^ b[1]) +
                    __builtin_popcount(a[2] ^ b[2]) + __builtin_popcount(a[3] ^ b[3]));
}

static int32_t sqdist(const uint8_t* a, const uint8_t* b) {
  int32_t s = 0;
  for (int k = 0; k < ORACLE_DIM; ++k) {
    int32_t e = (int32_t)a[k] - (int32_t)b[k];
    s += e * e;
  }
  return s;
}

/* One image pair, Sec. 3.1 Steps 1-4 (and Sec. 7.2 steps 1-5 when the
 * epipolar band is on). */
int64_t oracle_match_pair(const uint8_t* descA, const uint32_t* codesA, const uint8_t* bucketsA, uint32_t nA,
                          const uint8_t* descB, const uint32_t* codesB, const uint8_t* bucketsB, uint32_t nB,
                          const oracle_params* p, const double* F, const float* kptsA, const float* kptsB,
                          int32_t* match, oracle_query_detail* detail) {
  if (!params_ok(p)) return -1;
  const int epi = p->epi_px >= 0.0;
  if (epi && (!F || !kptsA || !kptsB)) return -1;
  const uint32_t T = p->n_tables, nbk = 1u << p->bits_per_table, K = p->top_k;

  /* Step 1: the lookup tables of image J -- for table t and short code
   * value v, the list of points of J whose code in table t is v, in index
   * order (a counting sort by code value). */
  uint32_t* off = (uint32_t*)calloc((size_t)T * (nbk + 1), sizeof(uint32_t));
  uint32_t* lst = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)T * nB + 1));
  uint32_t* seen = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)nB + 1));
  hk* cand = (hk*)malloc(sizeof(hk) * ((size_t)nB + 1));
  if (!off || !lst || !seen || !cand) {
    free(off); free(lst); free(seen); free(cand);
    return -1;
  }
  for (uint32_t t = 0; t < T; ++t) {
    uint32_t* o = off + (size_t)t * (nbk + 1);
    for (uint32_t j = 0; j < nB; ++j) o[bucketsB[(size_t)j * T + t] + 1]++;
    for (uint32_t v = 0; v < nbk; ++v) o[v + 1] += o[v];
    uint32_t* cur = (uint32_t*)malloc(sizeof(uint32_t) * nbk);
    memcpy(cur, o, sizeof(uint32_t) * nbk);
    for (uint32_t j = 0; j < nB; ++j) lst[(size_t)t * nB + cur[bucketsB[(size_t)j * T + t]]++] = j;
    free(cur);
  }
  for (uint32_t j = 0; j < nB; ++j) seen[j] = 0xFFFFFFFFu;

  int64_t nmatch = 0;
  for (uint32_t q = 0; q < nA; ++q) {
    /* Step 1: every point of J sharing the query's bucket in any table is a
     * candidate; the candidate set is a set (each point once). */
    uint32_t nc = 0;
    for (uint32_t t = 0; t < T; ++t) {
      const uint32_t v = bucketsA[(size_t)q * T + t];
      const uint32_t* o = off + (size_t)t * (nbk + 1);
      for (uint32_t e = o[v]; e < o[v + 1]; ++e) {
        const uint32_t j = lst[(size_t)t * nB + e];
        if (seen[j] == q) continue;
        seen[j] = q;
        cand[nc].j = j;
        cand[nc].h = 0;
        nc++;
      }
    }
    /* Sec. 7.2 step 3: the epipolar band removes candidates before ranking. */
    if (epi) {
      uint32_t w = 0;
      for (uint32_t e = 0; e < nc; ++e) {
        const uint32_t j = cand[e].j;
        if (oracle_epipolar_keep(F, kptsA[2 * (size_t)q], kptsA[2 * (size_t)q + 1], kptsB[2 * (size_t)j],
                                 kptsB[2 * (size_t)j + 1], p->epi_px))
          cand[w++] = cand[e];
      }
      nc = w;
    }
    /* Step 2: Hamming distance between the n-bit remapping codes. */
    for (uint32_t e = 0; e < nc; ++e) cand[e].h = hamming(codesA + (size_t)q * 4, codesB + (size_t)cand[e].j * 4);
    /* Sec. 6: candidates farther than tau are discarded (off when tau >= n). */
    if (p->tau < p->code_bits) {
      uint32_t w = 0;
      for (uint32_t e = 0; e < nc; ++e)
        if (cand[e].h <= p->tau) cand[w++] = cand[e];
      nc = w;
    }
    /* Step 3: rank by Hamming distance, keep the k smallest; equal
     * distances are ordered by candidate index (reading). */
    qsort(cand, nc, sizeof(hk), cmp_hk);
    const uint32_t ntop = nc < K ? nc : K;
    /* Step 4: exact squared Euclidean distances of the k, the nearest one
     * (smaller index on equal distance) matches if Lowe's ratio test holds:
     * sqrt(d1) < (num/den) sqrt(d2)  <=>  den^2 d1 < num^2 d2. */
    dk dd[ORACLE_MAX_K];
    for (uint32_t e = 0; e < ntop; ++e) {
      dd[e].j = cand[e].j;
      dd[e].d = sqdist(descA + (size_t)q * ORACLE_DIM, descB + (size_t)cand[e].j * ORACLE_DIM);
    }
    if (detail) {
      oracle_query_detail* D = detail + q;
      D->n_cand = nc;
      D->n_top = ntop;
      for (uint32_t e = 0; e < ntop; ++e) {
        D->top_j[e] = cand[e].j;
        D->top_h[e] = cand[e].h;
        D->top_d[e] = dd[e].d;
      }
    }
    qsort(dd, ntop, sizeof(dk), cmp_dk);
    int32_t mj = -1;
    if (ntop >= 2) {
      const int64_t lhs = (int64_t)p->ratio_den * p->ratio_den * dd[0].d;
      const int64_t rhs = (int64_t)p->ratio_num * p->ratio_num * dd[1].d;
      if (lhs < rhs) mj = (int32_t)dd[0].j;
    } else if (ntop == 1 && (p->flags & ORACLE_ACCEPT_SINGLE)) {
      mj = (int32_t)dd[0].j;  /* the single-candidate reading, when asked for */
    }
    if (detail) {
      detail[q].match_j = mj;
      detail[q].d1 = ntop >= 1 ? dd[0].d : -1;
      detail[q].d2 = ntop >= 2 ? dd[1].d : -1;
    }
    if (match) match[q] = mj;
    if (mj >= 0) nmatch++;
  }
  free(off);
  free(lst);
  free(seen);
  free(cand);
  return nmatch;
}

/* ------------------------------------------------------------------------ */
/* Many pairs: plain parallel loop over independent pairs (Sec. 1 notes the  */
/* matching of different image pairs is independent).                        */
/* ------------------------------------------------------------------------ */
typedef struct {
  const uint8_t* desc;
  const uint64_t* img_off;
  const uint32_t* codes;
  const uint8_t* buckets;
  const uint32_t* pairs;
  uint32_t P;
  const oracle_params* p;
  const double* F;
  const float* kpts;
  uint32_t** res;      /* per pair: compact (q, j) list */
  uint64_t* cnt;       /* per pair count */
  int64_t err;
  uint32_t next;
  pthread_mutex_t mu;
} job_t;

static void* worker(void* arg) {
  job_t* J = (job_t*)arg;
  const uint32_t T = J->p->n_tables;
  for (;;) {
    pthread_mutex_lock(&J->mu);
    const uint32_t i = J->next++;
    pthread_mutex_unlock(&J->mu);
    if (i >= J->P) break;
    const uint32_t a = J->pairs[2 * (size_t)i], b = J->pairs[2 * (size_t)i + 1];
    const uint64_t oa = J->img_off[a], ob = J->img_off[b];
    const uint32_t nA = (uint32_t)(J->img_off[a + 1] - oa), nB = (uint32_t)(J->img_off[b + 1] - ob);
    int32_t* m = (int32_t*)malloc(sizeof(int32_t) * ((size_t)nA + 1));
    int64_t r = oracle_match_pair(J->desc + oa * ORACLE_DIM, J->codes + oa * 4, J->buckets + oa * T, nA,
                                  J->desc + ob * ORACLE_DIM, J->codes + ob * 4, J->buckets + ob * T, nB, J->p,
                                  J->F ? J->F + 9 * (size_t)i : NULL, J->kpts ? J->kpts + 2 * oa : NULL,
                                  J->kpts ? J->kpts + 2 * ob : NULL, m, NULL);
    if (r >= 0 && (J->p->flags & ORACLE_MUTUAL)) {
      /* the reverse match: queries of B against candidates of A, F transposed */
      double Ft[9];
      if (J->F)
        for (int u = 0; u < 3; ++u)
          for (int v = 0; v < 3; ++v) Ft[3 * u + v] = J->F[9 * (size_t)i + 3 * v + u];
      int32_t* mr = (int32_t*)malloc(sizeof(int32_t) * ((size_t)nB + 1));
      const int64_t rr = oracle_match_pair(J->desc + ob * ORACLE_DIM, J->codes + ob * 4, J->buckets + ob * T, nB,
                                           J->desc + oa * ORACLE_DIM, J->codes + oa * 4, J->buckets + oa * T, nA,
                                           J->p, J->F ? Ft : NULL, J->kpts ? J->kpts + 2 * ob : NULL,
                                           J->kpts ? J->kpts + 2 * oa : NULL, mr, NULL);
      if (rr < 0) {
        r = -1;
      } else {
        r = 0;
        for (uint32_t q = 0; q < nA; ++q) {
          if (m[q] >= 0 && mr[m[q]] != (int32_t)q) m[q] = -1;
          if (m[q] >= 0) r++;
        }
      }
      free(mr);
    }
    if (r < 0) {
      pthread_mutex_lock(&J->mu);
      J->err = -1;
      pthread_mutex_unlock(&J->mu);
      free(m);
      continue;
    }
    uint32_t* l = (uint32_t*)malloc(sizeof(uint32_t) * 2 * ((size_t)r + 1));
    uint64_t c = 0;
    for (uint32_t q = 0; q < nA; ++q)
      if (m[q] >= 0) {
        l[2 * c] = q;
        l[2 * c + 1] = (uint32_t)m[q];
        c++;
      }
    free(m);
    J->res[i] = l;
    J->cnt[i] = c;
  }
  return NULL;
}

int64_t oracle_match_pairs(const uint8_t* desc, const uint64_t* img_off, uint32_t n_images,
                           const uint32_t* codes, const uint8_t* buckets,
                           const uint32_t* pairs, uint32_t P, const oracle_params* p,
                           const double* F, const float* kpts,
                           uint64_t* match_off, uint32_t* matches, uint64_t cap, int n_threads) {
  if (!params_ok(p) || !match_off) return -1;
  for (uint32_t i = 0; i < P; ++i)
    if (pairs[2 * (size_t)i] >= n_images || pairs[2 * (size_t)i + 1] >= n_images) return -1;
  job_t J;
  memset(&J, 0, sizeof J);
  J.desc = desc; J.img_off = img_off; J.codes = codes; J.buckets = buckets; J.pairs = pairs; J.P = P;
  J.p = p; J.F = F; J.kpts = kpts;
  J.res = (uint32_t**)calloc((size_t)P + 1, sizeof(uint32_t*));
  J.cnt = (uint64_t*)calloc((size_t)P + 1, sizeof(uint64_t));
  pthread_mutex_init(&J.mu, NULL);
  if (n_threads <= 0) n_threads = (int)sysconf(_SC_NPROCESSORS_ONLN);
  if (n_threads < 1) n_threads = 1;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)n_threads);
  for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, worker, &J);
  for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  free(th);
  pthread_mutex_destroy(&J.mu);
  int64_t total = 0;
  match_off[0] = 0;
  for (uint32_t i = 0; i < P; ++i) {
    match_off[i + 1] = match_off[i] + J.cnt[i];
    total += (int64_t)J.cnt[i];
  }
  if (J.err == 0 && matches) {
    if ((uint64_t)total > cap) {
      J.err = -1;
    } else {
      for (uint32_t i = 0; i < P; ++i)
        memcpy(matches + 2 * match_off[i], J.res[i], sizeof(uint32_t) * 2 * J.cnt[i]);
    }
  }
  for (uint32_t i = 0; i < P; ++i) free(J.res[i]);
  free(J.res);
  free(J.cnt);
  return J.err ? -1 : total;
}
