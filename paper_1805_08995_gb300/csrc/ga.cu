// First stage of Ga-CasHash (Sec. 7.1): the top 20 % of each image's
// features by SIFT scale are matched exhaustively with CasHash; a pair with
// at least 16 matches gets a fundamental matrix estimated on the GPU, and it
// goes on to the guided matching of Sec. 7.2 when at least 2/3 of its matches
// are inliers of that F.
//
// The paper names no estimator.  Here: the normalised 8-point algorithm
// (Hartley 1997) inside RANSAC (Fischler and Bolles 1981), the squared
// Sampson distance (Hartley and Zisserman, Multiple View Geometry, 2nd ed.,
// Sec. 11.4.3) as the inlier test, and a least-squares refit on the winning
// hypothesis' inliers.  All geometry is FP64.  The random draws of RANSAC are
// caller-given uint32 words; word k of a hypothesis picks r_k = floor(u_k (m -
// k) / 2^32), the r_k-th smallest match index not drawn before.
//
// Kernels:
//   k_ga_select   one CTA per image: radix select of the k-th largest scale
//                 key (4 passes of 8 bits), then a stable compaction in
//                 feature order (ties to the lower index);
//   k_ga_gather   subset descriptors and key-points;
//   k_ga_ransac   one warp per pair: Hartley normalisation (warp sums),
//                 hypotheses in batches of 32, one per lane (8 x 9
//                 elimination with partial pivoting for the null vector, rank
//                 2 by a one-sided Jacobi SVD of the 3 x 3, inlier count),
//                 warp argmax, the adaptive stop after each batch, refit from
//                 the 9 x 9 normal matrix (inverse iteration on its Cholesky
//                 factor), final count.  The
//                 inlier test runs in FP32 with a rounding bound and falls
//                 back to FP64 only near the threshold, so every decision is
//                 the FP64 one.
#include <algorithm>
#include <vector>

#include "internal.h"

namespace chx {

constexpr int GA_T = 256;
constexpr uint32_t GA_NONE = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------
// selection by scale
// ---------------------------------------------------------------------------

// Order-preserving uint32 key of a float (total order on finite values; -0 as +0).
__device__ __forceinline__ uint32_t scale_key(float s) {
  uint32_t b = __float_as_uint(s);
  if (b == 0x80000000u) b = 0u;
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Exclusive rank of this thread's flag among the CTA's flags, and the total.
__device__ __forceinline__ uint32_t cta_scan(bool f, uint32_t* s_w, uint32_t& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t bal = __ballot_sync(0xFFFFFFFFu, f);
  if (lane == 0) s_w[w] = __popc(bal);
  __syncthreads();
  uint32_t before = 0, tot = 0;
  for (int k = 0; k < GA_T / 32; ++k) {
    const uint32_t c = s_w[k];
    if (k < w) before += c;
    tot += c;
  }
  __syncthreads();
  total = tot;
  return before + __popc(bal & ((1u << lane) - 1u));
}

__global__ void __launch_bounds__(GA_T) k_ga_select(const float* __restrict__ scale, const uint64_t* __restrict__ off,
                                                    const uint64_t* __restrict__ sub_off, uint32_t* __restrict__ sel) {
  __shared__ uint32_t hist[256];
  __shared__ uint32_t s_w[GA_T / 32];
  __shared__ uint32_t s_digit, s_above;
  const uint32_t i = blockIdx.x, tid = threadIdx.x;
  const uint64_t a = off[i];
  const uint32_t n = (uint32_t)(off[i + 1] - a);
  const uint32_t k = (uint32_t)(sub_off[i + 1] - sub_off[i]);
  uint32_t* out = sel + sub_off[i];
  if (k == 0) return;
  // the k-th largest key: thr; need = how many keys equal to thr are taken
  uint32_t thr = 0, need = k;
  if (k < n) {
    uint32_t prefix = 0, pmask = 0;
    for (int pass = 0; pass < 4; ++pass) {
      const int shift = 24 - 8 * pass;
      for (uint32_t d = tid; d < 256; d += GA_T) hist[d] = 0;
      __syncthreads();
      for (uint32_t j = tid; j < n; j += GA_T) {
        const uint32_t key = scale_key(scale[a + j]);
        if ((key & pmask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
      }
      __syncthreads();
      if (tid == 0) {
        uint32_t above = 0, d = 255;
        for (;; --d) {
          if (above + hist[d] >= need || d == 0) break;
          above += hist[d];
        }
        s_digit = d;
        s_above = above;
      }
      __syncthreads();
      prefix |= s_digit << shift;
      pmask |= 0xFFu << shift;
      need -= s_above;
      __syncthreads();
    }
    thr = prefix;
  }
  // stable compaction in feature order
  uint32_t eq_before = 0, out_before = 0;
  for (uint32_t j0 = 0; j0 < n; j0 += GA_T) {
    const uint32_t j = j0 + tid;
    const uint32_t key = j < n ? scale_key(scale[a + j]) : 0u;
    const bool gt = j < n && (k == n || key > thr);
    const bool eq = j < n && k < n && key == thr;
    uint32_t eq_tot;
    const uint32_t eq_rank = cta_scan(eq, s_w, eq_tot);
    const bool take = gt || (eq && eq_before + eq_rank < need);
    uint32_t tk_tot;
    const uint32_t pos = cta_scan(take, s_w, tk_tot);
    if (take && out_before + pos < k) out[out_before + pos] = (uint32_t)(a + j);
    eq_before += eq_tot;
    out_before += tk_tot;
  }
}

__global__ void k_ga_gather(const uint32_t* __restrict__ sel, uint64_t n_sub, const uint8_t* __restrict__ desc,
                            const float2* __restrict__ kpts, uint8_t* __restrict__ desc_sub,
                            float2* __restrict__ kpts_sub) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_sub * 8;
       e += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t r = e >> 3, c = e & 7;
    const uint64_t f = sel[r];
    reinterpret_cast<uint4*>(desc_sub)[r * 8 + c] = reinterpret_cast<const uint4*>(desc)[f * 8 + c];
    if (c == 0) kpts_sub[r] = kpts[f];
  }
}

// ---------------------------------------------------------------------------
// fundamental matrix
// ---------------------------------------------------------------------------

// One correspondence: key-point of the query (x, y) and of the candidate (z, w).
struct alignas(32) GaPt {
  double x, y, z, w;
};

struct GaArgs {
  const float2* kpts;      // [N][2]
  const uint64_t* img_off; // [n_images + 1]
  const uint32_t* pairs;   // [P][2]
  const uint64_t* moff;    // [P + 1]
  const uint32_t* mt;      // [.][2] (q, j) local
  const uint32_t* words;   // [P][n_hyp][8]
  GaPt* pts;            // [total matches] scratch: (xa, ya, xb, yb)
  float4* pts32;        // the same in FP32 (exact: key-points are FP32)
  uint8_t* inl;            // [total matches] scratch
  double* F;               // [P][9] out
  uint4* info;             // [P][2] out: (matches, inliers, best, accepted), (evaluated, 0, 0, 0)
  uint32_t P, n_hyp, min_matches, num, den;
  double t2, thresh, conf;
};


// Squared Sampson distance <= t2 (x_B^T F x_A = 0).
__host__ __device__ __forceinline__ bool ga_inlier(const double* F, const GaPt p, double t2) {
  const double fx0 = F[0] * p.x + F[1] * p.y + F[2];
  const double fx1 = F[3] * p.x + F[4] * p.y + F[5];
  const double fx2 = F[6] * p.x + F[7] * p.y + F[8];
  const double ft0 = F[0] * p.z + F[3] * p.w + F[6];
  const double ft1 = F[1] * p.z + F[4] * p.w + F[7];
  const double r = p.z * fx0 + p.w * fx1 + fx2;
  const double e = (r * r) / (fx0 * fx0 + fx1 * fx1 + ft0 * ft0 + ft1 * ft1);
  return e <= t2;
}

// The same decision from an FP32 evaluation with a rounding bound; returns 1
// (inlier) or 0 (outlier) when the bound decides, else the FP64 test.  With
// u = 2^-24, F' = fl32(F) (F scaled as above), a = (xa, ya, 1), b = (xb, yb, 1), the FP32 values
// (nested fmaf) satisfy |r32 - r| <= 6u sum_ij |b_i||F_ij||a_j| for r =
// b^T F a, and each of F a and F^T b (first two rows) is off by at most
// 3.1u sum |F||a| (resp. |F^T||b|) per component, so the norm g of the
// Sampson denominator is off by at most 3.1u (S0 + S1 + T0 + T1) plus 3u g
// for its own evaluation.  The test |r| <= t g (e = r^2 / g^2 <= t^2) is
// decided when |r32| +- Er clears t (g32 -+ Eg) with margins 8u / 4u.
// The Sampson distance does not depend on the scale of F, so F is scaled to
// max |F_ij| = 1 before rounding (no overflow; entries that round as
// subnormals lose at most 2^-149 each, covered by the absolute term of the
// bounds).  A zero or non-finite F gives NaN values, which send every test to
// FP64.
struct GaF32 {
  float f[9], a[9];     // fl32(F / max |F|) and its absolute values
  float t_lo, t_hi;     // thresh rounded down / up
};

__device__ __forceinline__ void ga_f32(const double* F, double thresh, GaF32& g) {
  double mx = 0.0;
  for (int e = 0; e < 9; ++e) mx = fmax(mx, fabs(F[e]));
  const double sc = (mx > 0.0 && mx < 1e308) ? 1.0 / mx : __longlong_as_double(0x7FF8000000000000LL);
  for (int e = 0; e < 9; ++e) {
    g.f[e] = __double2float_rn(F[e] * sc);
    g.a[e] = fabsf(g.f[e]);
  }
  g.t_lo = __double2float_rd(thresh);
  g.t_hi = __double2float_ru(thresh);
}

__device__ __forceinline__ bool ga_inlier_fast(const GaF32& g, const float4 q, const double* F, const GaPt p,
                                               double t2) {
  const float u = 5.9604645e-08f;  // 2^-24
  const float* f = g.f;
  const float* a = g.a;
  const float fx0 = fmaf(f[0], q.x, fmaf(f[1], q.y, f[2]));
  const float fx1 = fmaf(f[3], q.x, fmaf(f[4], q.y, f[5]));
  const float fx2 = fmaf(f[6], q.x, fmaf(f[7], q.y, f[8]));
  const float ft0 = fmaf(f[0], q.z, fmaf(f[3], q.w, f[6]));
  const float ft1 = fmaf(f[1], q.z, fmaf(f[4], q.w, f[7]));
  const float r = fmaf(q.z, fx0, fmaf(q.w, fx1, fx2));
  const float ax = fabsf(q.x), ay = fabsf(q.y), bx = fabsf(q.z), by = fabsf(q.w);
  const float S0 = fmaf(a[0], ax, fmaf(a[1], ay, a[2]));
  const float S1 = fmaf(a[3], ax, fmaf(a[4], ay, a[5]));
  const float S2 = fmaf(a[6], ax, fmaf(a[7], ay, a[8]));
  const float T0 = fmaf(a[0], bx, fmaf(a[3], by, a[6]));
  const float T1 = fmaf(a[1], bx, fmaf(a[4], by, a[7]));
  const float Sr = fmaf(bx, S0, fmaf(by, S1, S2));
  const float gg = sqrtf(fmaf(fx0, fx0, fmaf(fx1, fx1, fmaf(ft0, ft0, ft1 * ft1))));
  const float ea = 1.f + ax + ay, eb = 1.f + bx + by;  // subnormal rounding: 1e-36 per unit of |a| |b|
  const float Er = fmaf(8.f * u, Sr, 1e-36f * ea * eb);
  const float Eg = fmaf(4.f * u, S0 + S1 + T0 + T1 + gg, 1e-36f * (ea + eb));
  const float ar = fabsf(r);
  if (ar + Er < g.t_lo * (gg - Eg) * (1.f - 4.f * u)) return true;
  if (ar - Er > g.t_hi * (gg + Eg) * (1.f + 4.f * u)) return false;
  return ga_inlier(F, p, t2);
}

// One-sided Jacobi SVD of a 3 x 3 (columns orthogonalised); returns the right
// singular vector of the smallest singular value in v.
__host__ __device__ void smallest_right_sv3(const double* Fm, double* v) {
  double U[9], V[9];
  for (int e = 0; e < 9; ++e) {
    U[e] = Fm[e];
    V[e] = (e % 4 == 0) ? 1.0 : 0.0;
  }
  for (int sweep = 0; sweep < 30; ++sweep) {
    bool rot = false;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int r = 0; r < 3; ++r) {
          al += U[3 * r + p] * U[3 * r + p];
          be += U[3 * r + q] * U[3 * r + q];
          ga += U[3 * r + p] * U[3 * r + q];
        }
        if (fabs(ga) <= 1e-300 || fabs(ga) <= 1e-15 * sqrt(al * be)) continue;
        rot = true;
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        for (int r = 0; r < 3; ++r) {
          const double up = U[3 * r + p], uq = U[3 * r + q];
          U[3 * r + p] = c * up - s * uq;
          U[3 * r + q] = s * up + c * uq;
          const double vp = V[3 * r + p], vq = V[3 * r + q];
          V[3 * r + p] = c * vp - s * vq;
          V[3 * r + q] = s * vp + c * vq;
        }
      }
    if (!rot) break;
  }
  int best = 0;
  double bn = 0.0;
  for (int col = 0; col < 3; ++col) {
    const double nn = U[col] * U[col] + U[3 + col] * U[3 + col] + U[6 + col] * U[6 + col];
    if (col == 0 || nn < bn) {
      bn = nn;
      best = col;
    }
  }
  for (int r = 0; r < 3; ++r) v[r] = V[3 * r + best];
}

// F := F - (F v)(v^T) for the smallest right singular vector v (closest rank 2).
__host__ __device__ void rank2(double* Fm) {
  double v[3];
  smallest_right_sv3(Fm, v);
  for (int r = 0; r < 3; ++r) {
    const double fv = Fm[3 * r] * v[0] + Fm[3 * r + 1] * v[1] + Fm[3 * r + 2] * v[2];
    for (int c = 0; c < 3; ++c) Fm[3 * r + c] -= fv * v[c];
  }
}

// F = Tb^T Fn Ta for T = [[s, 0, -s cx], [0, s, -s cy], [0, 0, 1]].
__host__ __device__ void denormalise(const double* Fn, const double* Ta, const double* Tb, double* F) {
  double G[9];  // Fn Ta
  for (int r = 0; r < 3; ++r) {
    G[3 * r + 0] = Fn[3 * r] * Ta[0];
    G[3 * r + 1] = Fn[3 * r + 1] * Ta[0];
    G[3 * r + 2] = Fn[3 * r] * Ta[1] + Fn[3 * r + 1] * Ta[2] + Fn[3 * r + 2];
  }
  for (int c = 0; c < 3; ++c) {
    F[c] = Tb[0] * G[c];
    F[3 + c] = Tb[0] * G[3 + c];
    F[6 + c] = Tb[1] * G[c] + Tb[2] * G[3 + c] + G[6 + c];
  }
}

// The design row of x_B^T F x_A = 0 (f = F row-major) in normalised coordinates.
__host__ __device__ __forceinline__ void design_row(const GaPt p, const double* Ta, const double* Tb, double* row) {
  const double xa = Ta[0] * p.x + Ta[1], ya = Ta[0] * p.y + Ta[2];
  const double xb = Tb[0] * p.z + Tb[1], yb = Tb[0] * p.w + Tb[2];
  row[0] = xb * xa;
  row[1] = xb * ya;
  row[2] = xb;
  row[3] = yb * xa;
  row[4] = yb * ya;
  row[5] = yb;
  row[6] = xa;
  row[7] = ya;
  row[8] = 1.0;
}

// Hypothesis h of the pair: 8 distinct matches from the words, the null vector
// of the 8 x 9 system (partial pivoting, f_8 = 1), rank 2, denormalised.
// false when the sample is degenerate or the result is not finite.
__host__ __device__ bool hypothesis(const GaPt* pts, uint32_t m, const uint32_t* w, const double* Ta, const double* Tb,
                                    double* F, double* fnull) {
  uint32_t idx[8];
  for (int k = 0; k < 8; ++k) {
    uint32_t v = (uint32_t)(((uint64_t)w[k] * (uint64_t)(m - k)) >> 32);
    // walk the earlier picks in ascending order
    uint32_t sorted[8];
    for (int t = 0; t < k; ++t) sorted[t] = idx[t];
    for (int t = 1; t < k; ++t)
      for (int u = t; u > 0 && sorted[u - 1] > sorted[u]; --u) {
        const uint32_t x = sorted[u];
        sorted[u] = sorted[u - 1];
        sorted[u - 1] = x;
      }
    for (int t = 0; t < k; ++t)
      if (sorted[t] <= v) ++v;
    idx[k] = v;
  }
  double A[8][9];
  for (int r = 0; r < 8; ++r) design_row(pts[idx[r]], Ta, Tb, A[r]);
  for (int c = 0; c < 8; ++c) {
    int piv = c;
    double pm = fabs(A[c][c]);
    for (int r = c + 1; r < 8; ++r)
      if (fabs(A[r][c]) > pm) {
        pm = fabs(A[r][c]);
        piv = r;
      }
    if (!(pm > 0.0)) return false;
    if (piv != c)
      for (int e = 0; e < 9; ++e) {
        const double x = A[c][e];
        A[c][e] = A[piv][e];
        A[piv][e] = x;
      }
    for (int r = c + 1; r < 8; ++r) {
      const double l = A[r][c] / A[c][c];
      for (int e = c; e < 9; ++e) A[r][e] -= l * A[c][e];
    }
  }
  double f[9];
  f[8] = 1.0;
  for (int c = 7; c >= 0; --c) {
    double s = 0.0;
    for (int e = c + 1; e < 9; ++e) s += A[c][e] * f[e];
    f[c] = -s / A[c][c];
  }
  for (int e = 0; e < 9; ++e) fnull[e] = f[e];
  rank2(f);
  denormalise(f, Ta, Tb, F);
  for (int e = 0; e < 9; ++e)
    if (!isfinite(F[e])) return false;
  return true;
}

// Eigenvector of the smallest eigenvalue of the symmetric positive
// semi-definite 9 x 9 M (the refit's normal matrix), by inverse iteration
// (Wilkinson; Golub and Van Loan, Sec. 7.6.1) on the Cholesky factor of
// M + delta I, delta = 1e-14 trace M (a shift leaves the eigenvectors as they
// are and keeps the factor finite when the fit is exact), started from x.
// Stops when an iterate moves by less than 1e-15 (max-norm) or after 100
// iterations.  x is overwritten with the unit eigenvector.  M (row-major, 81)
// and L (81) are in shared memory in the kernel.
__host__ __device__ void smallest_eigvec9(const double* M, double* L, double* x) {
  double tr = 0.0;
  for (int i = 0; i < 9; ++i) tr += M[10 * i];
  const double delta = 1e-14 * tr + 1e-300;
  for (int j = 0; j < 9; ++j) {  // L L^T = M + delta I, lower triangle of L
    double d = M[10 * j] + delta;
    for (int k = 0; k < j; ++k) d -= L[9 * j + k] * L[9 * j + k];
    d = sqrt(d > 0.0 ? d : 1e-300);
    L[10 * j] = d;
    for (int i = j + 1; i < 9; ++i) {
      double v = M[9 * i + j];
      for (int k = 0; k < j; ++k) v -= L[9 * i + k] * L[9 * j + k];
      L[9 * i + j] = v / d;
    }
  }
  double n0 = 0.0;
  for (int i = 0; i < 9; ++i) n0 += x[i] * x[i];
  n0 = 1.0 / sqrt(n0);
  for (int i = 0; i < 9; ++i) x[i] *= n0;
  for (int it = 0; it < 100; ++it) {
    double y[9];
    for (int i = 0; i < 9; ++i) {  // L y = x
      double v = x[i];
      for (int k = 0; k < i; ++k) v -= L[9 * i + k] * y[k];
      y[i] = v / L[10 * i];
    }
    for (int i = 8; i >= 0; --i) {  // L^T z = y
      double v = y[i];
      for (int k = i + 1; k < 9; ++k) v -= L[9 * k + i] * y[k];
      y[i] = v / L[10 * i];
    }
    double nn = 0.0, dot = 0.0;
    for (int i = 0; i < 9; ++i) {
      nn += y[i] * y[i];
      dot += y[i] * x[i];
    }
    const double sc = (dot >= 0.0 ? 1.0 : -1.0) / sqrt(nn);
    double mv = 0.0;
    for (int i = 0; i < 9; ++i) {
      const double z = y[i] * sc;
      mv = fmax(mv, fabs(z - x[i]));
      x[i] = z;
    }
    if (mv < 1e-15) break;
  }
}

constexpr uint32_t GA_BATCH = 32;  // hypotheses per check of the adaptive stop: one per lane

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

// Adaptive stop (Hartley and Zisserman, Algorithm 4.5): (1 - w^8)^done <=
// 1 - confidence with w = best / m, every step one correctly rounded double
// operation in a fixed order (three squarings, binary exponentiation), so the
// decision is the same wherever it is evaluated.  confidence >= 1: never.
__device__ bool ga_stop(uint32_t best, uint32_t m, uint32_t done, double conf) {
  if (!(conf < 1.0)) return false;
  const double w = __ddiv_rn((double)best, (double)m);
  const double w2 = __dmul_rn(w, w), w4 = __dmul_rn(w2, w2);
  double base = __dsub_rn(1.0, __dmul_rn(w4, w4)), r = 1.0;
  for (uint32_t e = done; e; e >>= 1) {
    if (e & 1u) r = __dmul_rn(r, base);
    base = __dmul_rn(base, base);
  }
  return r <= __dsub_rn(1.0, conf);
}

__device__ __forceinline__ void ga_write_info(const GaArgs& a, uint32_t p, uint32_t m, uint32_t n_in, uint32_t bh,
                                              uint32_t acc, uint32_t done) {
  a.info[2 * (size_t)p] = make_uint4(m, n_in, bh, acc);
  a.info[2 * (size_t)p + 1] = make_uint4(done, 0u, 0u, 0u);
}

// One warp per pair: hypotheses in batches of 32 (one per lane) until the
// adaptive stop holds or n_hyp are done; the most inliers win, ties to the
// lower hypothesis (a later batch replaces the best only with more inliers).
__global__ void __launch_bounds__(32, 16) k_ga_ransac(GaArgs a) {
  __shared__ double s_hF[32][9], s_hf[32][9];  // the batch's hypotheses: F and the null vector
  __shared__ double s_F[9], s_x[9], s_M[45], s_Mf[81], s_L[81];
  const uint32_t p = blockIdx.x, lane = threadIdx.x;
  const uint64_t m0 = a.moff[p];
  const uint32_t m = (uint32_t)(a.moff[p + 1] - m0);
  double* Fout = a.F + 9 * (size_t)p;
  if (m < a.min_matches) {
    if (lane < 9) Fout[lane] = 0.0;
    if (lane == 0) ga_write_info(a, p, m, 0u, GA_NONE, 0u, 0u);
    return;
  }
  const uint32_t ia = a.pairs[2 * p], ib = a.pairs[2 * p + 1];
  const uint64_t A0 = a.img_off[ia], B0 = a.img_off[ib];
  const uint32_t nA = (uint32_t)(a.img_off[ia + 1] - A0), nB = (uint32_t)(a.img_off[ib + 1] - B0);
  GaPt* pts = a.pts + m0;
  float4* pts32 = a.pts32 + m0;
  uint8_t* inl = a.inl + m0;
  double sxa = 0.0, sya = 0.0, sxb = 0.0, syb = 0.0;
  for (uint32_t i = lane; i < m; i += 32) {
    const uint32_t qa = a.mt[2 * (m0 + i)], jb = a.mt[2 * (m0 + i) + 1];
    // indices outside the images (never written by the matcher) read as (0, 0)
    const float2 pa = qa < nA ? a.kpts[A0 + qa] : make_float2(0.f, 0.f);
    const float2 pb = jb < nB ? a.kpts[B0 + jb] : make_float2(0.f, 0.f);
    const GaPt q = {(double)pa.x, (double)pa.y, (double)pb.x, (double)pb.y};
    pts[i] = q;
    pts32[i] = make_float4(pa.x, pa.y, pb.x, pb.y);
    sxa += q.x;
    sya += q.y;
    sxb += q.z;
    syb += q.w;
  }
  const double cxa = warp_sum(sxa) / m, cya = warp_sum(sya) / m;
  const double cxb = warp_sum(sxb) / m, cyb = warp_sum(syb) / m;
  __syncwarp();  // pts visible to the whole warp
  double da = 0.0, db = 0.0;
  for (uint32_t i = lane; i < m; i += 32) {
    const GaPt q = pts[i];
    da += sqrt((q.x - cxa) * (q.x - cxa) + (q.y - cya) * (q.y - cya));
    db += sqrt((q.z - cxb) * (q.z - cxb) + (q.w - cyb) * (q.w - cyb));
  }
  const double sa = sqrt(2.0) / (warp_sum(da) / m), sb = sqrt(2.0) / (warp_sum(db) / m);
  const double Ta[3] = {sa, -sa * cxa, -sa * cya}, Tb[3] = {sb, -sb * cxb, -sb * cyb};  // s, -s cx, -s cy

  uint32_t best_c = 0, best_h = GA_NONE, done = 0;  // warp-uniform
  while (done < a.n_hyp) {
    const uint32_t h = done + lane;
    uint32_t c = 0, bh = GA_NONE;
    if (h < a.n_hyp) {
      double F[9], fn[9];
      if (hypothesis(pts, m, a.words + ((size_t)p * a.n_hyp + h) * 8, Ta, Tb, F, fn)) {
        GaF32 g;
        ga_f32(F, a.thresh, g);
        for (uint32_t i = 0; i < m; ++i) c += ga_inlier_fast(g, pts32[i], F, pts[i], a.t2) ? 1u : 0u;
        for (int e = 0; e < 9; ++e) {
          s_hF[lane][e] = F[e];
          s_hf[lane][e] = fn[e];
        }
        bh = h;
      }
    }
    // the batch's winner (a total order: valid first, more inliers, lower h), on every lane
    uint32_t bc = c;
    for (int o = 16; o > 0; o >>= 1) {
      const uint32_t oc = __shfl_xor_sync(0xFFFFFFFFu, bc, o), oh = __shfl_xor_sync(0xFFFFFFFFu, bh, o);
      if (oh != GA_NONE && (bh == GA_NONE || oc > bc || (oc == bc && oh < bh))) {
        bc = oc;
        bh = oh;
      }
    }
    __syncwarp();  // the batch's hypotheses are in shared memory
    if (bh != GA_NONE && (best_h == GA_NONE || bc > best_c)) {
      best_c = bc;
      best_h = bh;
      if (lane < 9) {
        s_F[lane] = s_hF[bh - done][lane];
        s_x[lane] = s_hf[bh - done][lane];
      }
    }
    __syncwarp();
    done = min(done + GA_BATCH, a.n_hyp);
    if (best_h != GA_NONE && ga_stop(best_c, m, done, a.conf)) break;
  }
  if (best_h == GA_NONE) {
    if (lane < 9) Fout[lane] = 0.0;
    if (lane == 0) ga_write_info(a, p, m, 0u, GA_NONE, 0u, done);
    return;
  }
  double F[9];
  for (int e = 0; e < 9; ++e) F[e] = s_F[e];
  uint32_t cnt_local = 0;
  GaF32 g;
  ga_f32(F, a.thresh, g);
  for (uint32_t i = lane; i < m; i += 32) {
    const bool in = ga_inlier_fast(g, pts32[i], F, pts[i], a.t2);
    inl[i] = in ? 1 : 0;
    cnt_local += in ? 1u : 0u;
  }
  const uint32_t n_best = __reduce_add_sync(0xFFFFFFFFu, cnt_local);
  __syncwarp();  // inlier flags visible
  if (n_best >= 8) {
    // normal matrix of the inliers' design rows: lane l sums entries l and l + 32 ((r, c), r <= c,
    // row-major over the upper triangle) over the matches in order
    for (uint32_t ent = lane; ent < 45; ent += 32) {
      uint32_t r = 0, t = ent;
      while (t >= 9 - r) {
        t -= 9 - r;
        ++r;
      }
      const uint32_t c = r + t;
      double sum = 0.0;
      for (uint32_t i = 0; i < m; ++i) {
        if (!inl[i]) continue;
        double row[9];
        design_row(pts[i], Ta, Tb, row);
        sum += row[r] * row[c];
      }
      s_M[ent] = sum;
    }
    __syncwarp();
    if (lane == 0) {
      double f[9];
      for (uint32_t r = 0, e = 0; r < 9; ++r)
        for (uint32_t c = r; c < 9; ++c, ++e) s_Mf[9 * r + c] = s_Mf[9 * c + r] = s_M[e];
      for (int e = 0; e < 9; ++e) f[e] = s_x[e];  // start: the winning sample's null vector
      smallest_eigvec9(s_Mf, s_L, f);
      rank2(f);
      denormalise(f, Ta, Tb, s_F);
    }
    __syncwarp();
    for (int e = 0; e < 9; ++e) F[e] = s_F[e];
  }
  // unit Frobenius norm, largest-magnitude entry (first on ties) positive
  double nn = 0.0, big = 0.0;
  int bi = 0;
  for (int e = 0; e < 9; ++e) {
    nn += F[e] * F[e];
    if (fabs(F[e]) > big) {
      big = fabs(F[e]);
      bi = e;
    }
  }
  const double sc = (F[bi] > 0.0 ? 1.0 : -1.0) / sqrt(nn);
  for (int e = 0; e < 9; ++e) F[e] *= sc;
  uint32_t c2 = 0;
  ga_f32(F, a.thresh, g);
  for (uint32_t i = lane; i < m; i += 32) c2 += ga_inlier_fast(g, pts32[i], F, pts[i], a.t2) ? 1u : 0u;
  const uint32_t n_in = __reduce_add_sync(0xFFFFFFFFu, c2);
  if (lane < 9) Fout[lane] = F[lane];
  if (lane == 0) ga_write_info(a, p, m, n_in, best_h, (uint64_t)a.den * n_in >= (uint64_t)a.num * m ? 1u : 0u, done);
}

}  // namespace chx

using namespace chx;

namespace {

int err_of(cudaError_t e) {
  if (e == cudaSuccess) return CASHASH_OK;
  return e == cudaErrorMemoryAllocation ? CASHASH_ENOMEM : CASHASH_ECUDA;
}

bool ga_params_ok(const cashash_ga_params* gp) {
  return gp && gp->top_pct >= 1 && gp->top_pct <= 100 && gp->min_matches >= 8 && gp->n_hyp >= 1 &&
         gp->n_hyp <= CASHASH_GA_MAX_HYP && gp->inlier_den >= 1 && gp->inlier_num <= gp->inlier_den &&
         gp->thresh_px > 0.0 && gp->thresh_px < 1e150 && gp->kernel <= CASHASH_KERNEL_QUERY &&
         gp->confidence >= 0.0;
}

// Device scratch released at the end of a call (stream-ordered).
struct Scratch {
  cudaStream_t s;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t st) : s(st) {}
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
  template <class T>
  int get(T*& out, uint64_t n) {
    void* p = nullptr;
    const int st = err_of(cudaMallocAsync(&p, std::max<uint64_t>(n, 1) * sizeof(T), s));
    if (st != CASHASH_OK) return st;
    ptrs.push_back(p);
    out = static_cast<T*>(p);
    return CASHASH_OK;
  }
};

}  // namespace

extern "C" void cashash_ga_default_params(cashash_ga_params* gp) {
  if (!gp) return;
  gp->top_pct = 20;
  gp->min_matches = 16;
  gp->n_hyp = 256;
  gp->inlier_num = 2;
  gp->inlier_den = 3;
  gp->kernel = 0;
  gp->thresh_px = 3.0;
  gp->confidence = 0.99;
}

extern "C" int cashash_ga_subset_offsets(const uint64_t* img_off, uint32_t n_images, uint32_t top_pct,
                                         uint64_t* sub_off) {
  if ((n_images > 0 && !img_off) || !sub_off || top_pct < 1 || top_pct > 100) return CASHASH_EINVAL;
  sub_off[0] = 0;
  for (uint32_t i = 0; i < n_images; ++i) {
    if (img_off[i + 1] < img_off[i]) return CASHASH_EINVAL;
    const uint64_t n = img_off[i + 1] - img_off[i];
    sub_off[i + 1] = sub_off[i] + (n * top_pct + 99) / 100;
  }
  return CASHASH_OK;
}

extern "C" int cashash_ga_select(const float* scale, const uint64_t* img_off, uint32_t n_images, uint32_t top_pct,
                                 uint32_t* sel, cashash_stream_t stream_) {
  if ((n_images > 0 && !img_off) || top_pct < 1 || top_pct > 100) return CASHASH_EINVAL;
  if (n_images == 0) return CASHASH_OK;
  const uint64_t N = img_off[n_images];
  if (N >= (1ull << 32) || (N > 0 && (!scale || !sel))) return CASHASH_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
  std::vector<uint64_t> sub(n_images + 1);
  int st = cashash_ga_subset_offsets(img_off, n_images, top_pct, sub.data());
  if (st != CASHASH_OK) return st;
  if (sub[n_images] == 0) return CASHASH_OK;
  Scratch sc(s);
  uint64_t *d_off = nullptr, *d_sub = nullptr;
  if ((st = sc.get(d_off, n_images + 1)) != CASHASH_OK || (st = sc.get(d_sub, n_images + 1)) != CASHASH_OK) return st;
  if ((st = err_of(cudaMemcpyAsync(d_off, img_off, (n_images + 1) * 8ull, cudaMemcpyHostToDevice, s))) != CASHASH_OK)
    return st;
  if ((st = err_of(cudaMemcpyAsync(d_sub, sub.data(), (n_images + 1) * 8ull, cudaMemcpyHostToDevice, s))) !=
      CASHASH_OK)
    return st;
  if (n_images > 0x7FFFFFFFu) return CASHASH_EINVAL;  // one CTA per image
  k_ga_select<<<n_images, GA_T, 0, s>>>(scale, d_off, d_sub, sel);
  return err_of(cudaGetLastError());
}

extern "C" int cashash_estimate_F(const float* kpts, const uint64_t* img_off, uint32_t n_images,
                                  const uint32_t* pairs_host, uint32_t P, const uint64_t* match_off,
                                  const uint32_t* matches, const cashash_ga_params* gp, const uint32_t* words,
                                  double* F_out, cashash_ga_info* info_out, cashash_stream_t stream_) {
  if (!ga_params_ok(gp) || (n_images > 0 && !img_off) || (P > 0 && (!pairs_host || !match_off || !F_out ||
                                                                    !info_out || !words || !kpts)))
    return CASHASH_EINVAL;
  if (P == 0) return CASHASH_OK;
  if (P > 0x7FFFFFFFu) return CASHASH_EINVAL;  // one CTA per pair
  for (uint64_t i = 0; i < 2ull * P; ++i)
    if (pairs_host[i] >= n_images) return CASHASH_EINVAL;
  for (uint32_t i = 0; i < n_images; ++i)
    if (img_off[i + 1] < img_off[i]) return CASHASH_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
  uint64_t total = 0;
  int st = err_of(cudaMemcpyAsync(&total, match_off + P, sizeof total, cudaMemcpyDeviceToHost, s));
  if (st == CASHASH_OK) st = err_of(cudaStreamSynchronize(s));
  if (st != CASHASH_OK) return st;
  if (total > 0 && !matches) return CASHASH_EINVAL;
  Scratch sc(s);
  uint64_t* d_off = nullptr;
  uint32_t* d_pairs = nullptr;
  GaPt* d_pts = nullptr;
  uint8_t* d_inl = nullptr;
  float4* d_pts32 = nullptr;
  if ((st = sc.get(d_off, n_images + 1)) != CASHASH_OK || (st = sc.get(d_pairs, 2ull * P)) != CASHASH_OK ||
      (st = sc.get(d_pts, total)) != CASHASH_OK || (st = sc.get(d_inl, total)) != CASHASH_OK ||
      (st = sc.get(d_pts32, total)) != CASHASH_OK)
    return st;
  if ((st = err_of(cudaMemcpyAsync(d_off, img_off, (n_images + 1) * 8ull, cudaMemcpyHostToDevice, s))) != CASHASH_OK)
    return st;
  if ((st = err_of(cudaMemcpyAsync(d_pairs, pairs_host, 8ull * P, cudaMemcpyHostToDevice, s))) != CASHASH_OK)
    return st;
  GaArgs a{};
  a.kpts = reinterpret_cast<const float2*>(kpts);
  a.img_off = d_off;
  a.pairs = d_pairs;
  a.moff = match_off;
  a.mt = matches;
  a.words = words;
  a.pts = d_pts;
  a.pts32 = d_pts32;
  a.inl = d_inl;
  a.F = F_out;
  a.info = reinterpret_cast<uint4*>(info_out);
  a.P = P;
  a.n_hyp = gp->n_hyp;
  a.min_matches = gp->min_matches;
  a.num = gp->inlier_num;
  a.den = gp->inlier_den;
  a.t2 = gp->thresh_px * gp->thresh_px;
  a.thresh = gp->thresh_px;
  a.conf = gp->confidence;
  k_ga_ransac<<<P, 32, 0, s>>>(a);
  return err_of(cudaGetLastError());
}

extern "C" int cashash_ga_stage1(cashash_ctx* ctx, const cashash_set* set, const float* scale,
                                 const double* mean_host, const uint32_t* pairs_host, uint32_t P,
                                 const cashash_ga_params* gp, const uint32_t* words, double* F_out,
                                 cashash_ga_info* info_out, cashash_stream_t stream_) {
  cashash_params cp;
  if (!ctx || !set || !mean_host || !ga_params_ok(gp) || cashash_get_params(ctx, &cp) != CASHASH_OK)
    return CASHASH_EINVAL;
  if (cp.epi_px >= 0.0) return CASHASH_EINVAL;  // stage 1 runs without a band
  const uint32_t n_images = set->n_images;
  if ((n_images > 0 && !set->img_off) || (set->n_features > 0 && (!set->desc || !set->kpts || !scale)))
    return CASHASH_EINVAL;
  if (P > 0 && (!pairs_host || !words || !F_out || !info_out)) return CASHASH_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
  std::vector<uint64_t> sub(n_images + 1, 0);
  int st = cashash_ga_subset_offsets(set->img_off, n_images, gp->top_pct, sub.data());
  if (st != CASHASH_OK) return st;
  const uint64_t N = sub[n_images];
  uint64_t cap = 0;
  for (uint32_t i = 0; i < P; ++i) {
    if (pairs_host[2 * (size_t)i] >= n_images || pairs_host[2 * (size_t)i + 1] >= n_images) return CASHASH_EINVAL;
    cap += sub[pairs_host[2 * (size_t)i] + 1] - sub[pairs_host[2 * (size_t)i]];
  }
  Scratch sc(s);
  uint32_t *sel = nullptr, *codes = nullptr, *sq = nullptr, *mt = nullptr;
  uint8_t *desc = nullptr, *buckets = nullptr, *tables = nullptr;
  float* kp = nullptr;
  uint64_t* moff = nullptr;
  const uint64_t tb = cashash_tables_bytes(&cp, sub.data(), n_images);
  if ((st = sc.get(sel, N)) != CASHASH_OK || (st = sc.get(desc, N * 128)) != CASHASH_OK ||
      (st = sc.get(kp, N * 2)) != CASHASH_OK || (st = sc.get(codes, N * 4)) != CASHASH_OK ||
      (st = sc.get(buckets, N * 8)) != CASHASH_OK || (st = sc.get(sq, N)) != CASHASH_OK ||
      (st = sc.get(tables, tb)) != CASHASH_OK || (st = sc.get(moff, (uint64_t)P + 1)) != CASHASH_OK ||
      (st = sc.get(mt, 2 * std::max<uint64_t>(cap, 1))) != CASHASH_OK)
    return st;
  if ((st = cashash_ga_select(scale, set->img_off, n_images, gp->top_pct, sel, stream_)) != CASHASH_OK) return st;
  if (N > 0) {
    const uint64_t work = N * 8;
    const unsigned grid = (unsigned)std::min<uint64_t>((work + 255) / 256, 65535);
    k_ga_gather<<<grid, 256, 0, s>>>(sel, N, set->desc, reinterpret_cast<const float2*>(set->kpts), desc,
                                     reinterpret_cast<float2*>(kp));
    if ((st = err_of(cudaGetLastError())) != CASHASH_OK) return st;
  }
  cashash_set S{};
  S.n_images = n_images;
  S.n_features = N;
  S.img_off = sub.data();
  S.desc = desc;
  S.codes = codes;
  S.buckets = buckets;
  S.sqnorm = sq;
  S.tables = tables;
  S.kpts = kp;
  if ((st = cashash_build_codes(ctx, &S, mean_host, stream_)) != CASHASH_OK) return st;
  if (P == 0) return err_of(cudaStreamSynchronize(s));
  cashash_plan* pl = nullptr;
  if ((st = cashash_plan_create(ctx, &S, pairs_host, P, &pl)) != CASHASH_OK) return st;
  cashash_tuning tu{};
  if (cashash_plan_get_tuning(pl, &tu) == CASHASH_OK && tu.kernel != 0) {  // batched plans only
    uint32_t want = gp->kernel;
    if (want == 0) want = N < 4096ull * std::max<uint32_t>(n_images, 1) ? CASHASH_KERNEL_QUERY : CASHASH_KERNEL_JOIN;
    if (want != tu.kernel) {
      cashash_tuning t2{};
      t2.kernel = want;
      st = cashash_plan_set_tuning(pl, &t2);
      if (st == CASHASH_ENOTSUP) st = CASHASH_OK;  // the join does not apply: keep the plan's kernel
    }
  }
  if (st == CASHASH_OK) st = cashash_match_plan(ctx, pl, nullptr, moff, mt, cap, stream_);
  if (st == CASHASH_OK) st = cashash_sync_status(ctx, stream_);
  cashash_plan_destroy(pl);
  if (st != CASHASH_OK) return st;
  return cashash_estimate_F(kp, sub.data(), n_images, pairs_host, P, moff, mt, gp, words, F_out, info_out, stream_);
}
