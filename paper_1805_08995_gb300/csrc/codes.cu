// Hash codes of Sec. 5.1 / Steps 1-2 (Sec. 3.1): centring, projection, signs.
//
// A feature's bit b is the sign of v_b = sum_j R_bj (x_j - mu_j) evaluated in
// IEEE double, j ascending, every difference, product and sum rounded to
// nearest.  The fast kernels compute an approximation v~ with a rigorous
// per-(feature, row) bound E on |v~ - v_double|; when |v~| > E the sign of v~
// is the sign of v_double.  Otherwise the (feature, row) is flagged and
// k_fix_fp64 evaluates the exact double sequence.
#include "internal.h"

namespace chx {

// ---------------------------------------------------------------------------
// Column sums of the descriptors (the centre is the set mean; the paper is
// silent on centring).  Integer sums are exact and order independent.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_colsum(const uint8_t* __restrict__ desc, uint64_t n,
                                                unsigned long long* __restrict__ sums) {
  __shared__ uint32_t part[32][129];
  const int g = threadIdx.x & 7;    // 16-column group
  const int rl = threadIdx.x >> 3;  // row lane
  uint32_t acc[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) acc[k] = 0;
  const uint4* d4 = reinterpret_cast<const uint4*>(desc);
  for (uint64_t r = (uint64_t)blockIdx.x * 32 + rl; r < n; r += (uint64_t)gridDim.x * 32) {
    const uint4 v = __ldg(&d4[r * 8 + g]);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      acc[4 * k + 0] += w[k] & 0xFFu;
      acc[4 * k + 1] += (w[k] >> 8) & 0xFFu;
      acc[4 * k + 2] += (w[k] >> 16) & 0xFFu;
      acc[4 * k + 3] += w[k] >> 24;
    }
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) part[rl][16 * g + k] = acc[k];
  __syncthreads();
  if (threadIdx.x < DIM) {
    unsigned long long s = 0;
    for (int r = 0; r < 32; ++r) s += part[r][threadIdx.x];
    atomicAdd(&sums[threadIdx.x], s);
  }
}

cudaError_t launch_colsum(const uint8_t* desc, uint64_t n, unsigned long long* sums, cudaStream_t s, bool add) {
  cudaError_t e = add ? cudaSuccess : cudaMemsetAsync(sums, 0, DIM * sizeof(unsigned long long), s);
  if (e != cudaSuccess || n == 0) return e;
  uint64_t want = (n + 32 * 8 - 1) / (32 * 8);  // about 8 rows of 16-byte loads per thread
  int grid = (int)(want < 1216 ? want : 1216);
  k_colsum<<<grid, 256, 0, s>>>(desc, n, sums);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Centre and per-row constants.  mu_j = S_j / N (one correctly rounded double
// division).  c_b = sum_j R_bj mu_j is needed only by the approximation, so
// its summation order is free; its error enters the bound.
//   FP32 form bound (see the header comment of this file):
//     |v~ - v_double| <= alpha_b ||x||_2 + beta_b,
//     alpha_b = alpha_scale * ||R_b||_2,
//     beta_b  = 2^-23 |c_b| + 2^-40 ||R_b||_2 (||mu||_2 + 1).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_row_consts(const unsigned long long* __restrict__ sums, uint64_t n,
                                                    int have_mean, double* __restrict__ mu,
                                                    const double* __restrict__ R, const double* __restrict__ nrmR,
                                                    uint32_t rows, float alpha_scale, RowConst* __restrict__ rc) {
  __shared__ double mu_s[DIM];
  __shared__ double nmu_s;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t < DIM) {
    double m;
    if (have_mean) {
      m = mu[t];
    } else {
      m = (n == 0) ? 0.0 : __ddiv_rn((double)sums[t], (double)n);
    }
    mu_s[t] = m;
  }
  __syncthreads();
  if (!have_mean && blockIdx.x == 0 && t < DIM) mu[t] = mu_s[t];  // (every CTA reads the sums, one writes mu)
  // ||mu|| and c_b = sum_j R_bj mu_j by warp reductions: only the approximation
  // uses them and the bound covers their rounding, so the order is free.  ||mu||
  // enters the bound only, as an upper bound: FP32 with every step rounded up.
  if (warp == 0) {
    float s = 0.f;
    for (int j = lane; j < DIM; j += 32) {
      const float m = __double2float_ru(fabs(mu_s[j]));
      s = __fmaf_ru(m, m, s);
    }
    for (int o = 16; o > 0; o >>= 1) s = __fadd_ru(s, __shfl_xor_sync(0xFFFFFFFFu, s, o));
    if (lane == 0) nmu_s = (double)__fsqrt_ru(s);
  }
  __syncthreads();
  for (uint32_t b = blockIdx.x * (blockDim.x / 32) + warp; b < rows; b += gridDim.x * (blockDim.x / 32)) {
    double c = 0.0;
    for (int j = lane; j < DIM; j += 32) c += R[(size_t)b * DIM + j] * mu_s[j];
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    if (lane == 0) {
      RowConst r;
      r.c32 = (float)c;
      r.alpha = (float)(alpha_scale * nrmR[b] * (1.0 + 0x1p-20));
      r.beta = (float)((0x1p-23 * fabs(c) + 0x1p-40 * nrmR[b] * (nmu_s + 1.0)) * (1.0 + 0x1p-20) + 0x1p-60);
      r.pad = 0.f;
      rc[b] = r;
    }
  }
}

cudaError_t launch_row_consts(const unsigned long long* sums, uint64_t n, int have_mean, double* mu,
                              const double* R, const double* nrmR, uint32_t rows, float alpha_scale,
                              RowConst* rc, cudaStream_t s) {
  // one warp per row, the rows spread over CTAs (each CTA derives the centre itself)
  k_row_consts<<<(rows + 7) / 8, 256, 0, s>>>(sums, n, have_mean, mu, R, nrmR, rows, alpha_scale, rc);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP32 CUDA-core projection.  Tile: 64 features x 192 rows per CTA of 256
// threads; thread (fg, rg) owns features 4fg..4fg+3 and rows 12rg..12rg+11.
// Each accumulator is one sequential FMA chain over j = 0..127, which the
// bound alpha_scale = 2^-16 covers (gamma_256 for FP32 with margin).
// ---------------------------------------------------------------------------
constexpr int PT_F = 64;     // features per tile
constexpr int PT_R = 192;    // rows per tile (padded)

__global__ void __launch_bounds__(256, 1) k_project_fp32(const uint8_t* __restrict__ desc, uint64_t n,
                                                         const float* __restrict__ R32T,
                                                         const RowConst* __restrict__ rcg, KParams kp,
                                                         uint32_t* __restrict__ codes, uint8_t* __restrict__ buckets,
                                                         uint32_t* __restrict__ sqnorm,
                                                         uint32_t* __restrict__ flagmask,
                                                         uint32_t* __restrict__ flaglist,
                                                         unsigned long long* __restrict__ nflag_feat,
                                                         float* __restrict__ dbg_x, float* __restrict__ dbg_e) {
  extern __shared__ __align__(16) float psm[];
  float* Rs = psm;                       // [128][192]  R32 transposed (j-major)
  float* xs = Rs + DIM * PT_R;           // [128][64]   x as float (j-major)
  __shared__ RowConst rc[PT_R];
  __shared__ float nx_s[PT_F];
  __shared__ uint32_t sq_s[PT_F];
  __shared__ uint32_t sbits[PT_F][6];
  __shared__ uint32_t sflag[PT_F][6];

  const int tid = threadIdx.x;
  for (int i = tid; i < DIM * PT_R / 4; i += 256)
    reinterpret_cast<float4*>(Rs)[i] = __ldg(reinterpret_cast<const float4*>(R32T) + i);
  for (int i = tid; i < PT_R; i += 256) {
    if ((uint32_t)i < kp.rows) rc[i] = rcg[i];
    else { RowConst z; z.c32 = 0.f; z.alpha = 0.f; z.beta = 0.f; z.pad = 0.f; rc[i] = z; }
  }
  const int fg = tid & 15, rg = tid >> 4;
  const uint64_t ntiles = (n + PT_F - 1) / PT_F;
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint64_t f0 = tile * PT_F;
    __syncthreads();
    // load 64 descriptors: thread -> feature tid>>2, bytes 32*(tid&3) .. +31
    {
      const int fl = tid >> 2, qq = tid & 3;
      const uint64_t f = f0 + fl;
      uint4 v0 = make_uint4(0, 0, 0, 0), v1 = v0;
      if (f < n) {
        const uint4* row = reinterpret_cast<const uint4*>(desc + f * DIM) + 2 * qq;
        v0 = __ldg(row);
        v1 = __ldg(row + 1);
      }
      const uint32_t w[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
      uint32_t sq = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        sq = __dp4a(w[k], w[k], sq);
#pragma unroll
        for (int b = 0; b < 4; ++b) xs[(32 * qq + 4 * k + b) * PT_F + fl] = (float)((w[k] >> (8 * b)) & 0xFFu);
      }
      sq += __shfl_xor_sync(0xFFFFFFFFu, sq, 1);
      sq += __shfl_xor_sync(0xFFFFFFFFu, sq, 2);
      if (qq == 0) {
        sq_s[fl] = sq;
        nx_s[fl] = sqrtf((float)sq);
      }
      if (tid < PT_F * 6) {
        (&sbits[0][0])[tid] = 0u;
        (&sflag[0][0])[tid] = 0u;
      }
      if (tid + 256 < PT_F * 6) {
        (&sbits[0][0])[tid + 256] = 0u;
        (&sflag[0][0])[tid + 256] = 0u;
      }
    }
    __syncthreads();
    float acc[4][12];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 12; ++b) acc[a][b] = 0.f;
#pragma unroll 4
    for (int j = 0; j < DIM; ++j) {
      const float4 xv = *reinterpret_cast<const float4*>(xs + j * PT_F + 4 * fg);
      const float4 r0 = *reinterpret_cast<const float4*>(Rs + j * PT_R + 12 * rg);
      const float4 r1 = *reinterpret_cast<const float4*>(Rs + j * PT_R + 12 * rg + 4);
      const float4 r2 = *reinterpret_cast<const float4*>(Rs + j * PT_R + 12 * rg + 8);
      const float xa[4] = {xv.x, xv.y, xv.z, xv.w};
      const float ra[12] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w, r2.x, r2.y, r2.z, r2.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 12; ++b) acc[a][b] = __fmaf_rn(ra[b], xa[a], acc[a][b]);
    }
    // signs, bound test, flags
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int fl = 4 * fg + a;
      const float nx = nx_s[fl];
#pragma unroll
      for (int b = 0; b < 12; ++b) {
        const int row = 12 * rg + b;
        if ((uint32_t)row < kp.rows) {
          const RowConst r = rc[row];
          const float v = acc[a][b] - r.c32;
          const float E = __fmaf_ru(r.alpha, nx, r.beta);
          if (dbg_x && f0 + fl < n) {  // diagnostic of the bound (cashash_projection_bounds)
            dbg_x[(f0 + fl) * kp.rows + row] = v;
            dbg_e[(f0 + fl) * kp.rows + row] = E;
          }
          if (fabsf(v) <= E) atomicOr(&sflag[fl][row >> 5], 1u << (row & 31));
          else if (v > 0.f) atomicOr(&sbits[fl][row >> 5], 1u << (row & 31));
        }
      }
    }
    __syncthreads();
    if (tid < PT_F && f0 + tid < n)
      write_feature(f0 + tid, sbits[tid], sflag[tid], sq_s[tid], kp, codes, buckets, sqnorm, flagmask, flaglist,
                    nflag_feat);
  }
}

cudaError_t launch_project_fp32(const uint8_t* desc, uint64_t n, const float* R32T, const RowConst* rc,
                                const KParams& kp, uint32_t* codes, uint8_t* buckets, uint32_t* sqnorm,
                                uint32_t* flagmask, uint32_t* flaglist, unsigned long long* nflag_feat,
                                cudaStream_t s, float* dbg_x, float* dbg_e) {
  if (n == 0) return cudaSuccess;
  const size_t smem = (size_t)DIM * PT_R * 4 + (size_t)DIM * PT_F * 4;
  cudaError_t e = cudaFuncSetAttribute(k_project_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t ntiles = (n + PT_F - 1) / PT_F;
  const int grid = (int)(ntiles < (uint64_t)nsm ? ntiles : (uint64_t)nsm);
  k_project_fp32<<<grid, 256, smem, s>>>(desc, n, R32T, rc, kp, codes, buckets, sqnorm, flagmask, flaglist,
                                         nflag_feat, dbg_x, dbg_e);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Exact re-evaluation of flagged (feature, row) projections: the sign of the
// double sequence t = x_j - mu_j, p = R_bj * t, s = s + p for j = 0..127, each
// rounded to nearest (explicit _rn intrinsics, so no contraction).  One warp
// per flagged feature: the lanes form the t_j and p_j of four columns each and
// the warp sums them as a tree, which fixes the sign of the ordered sum unless
// the tree sum lies within a bound of zero (then the warp runs the ordered
// additions themselves).  The 128 dependent additions of the ordered sum, slow
// on the narrow FP64 pipe, run only for such rounding-noise projections.  Bits
// that come out 1 are ORed into the codes / bucket bytes (they were written as 0).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_fix_fp64(const uint8_t* __restrict__ desc, const double* __restrict__ mu,
                                                  const double* __restrict__ R, KParams kp,
                                                  const uint32_t* __restrict__ flagmask,
                                                  const uint32_t* __restrict__ flaglist,
                                                  const unsigned long long* __restrict__ nflag_feat,
                                                  uint64_t max_feat, uint32_t* __restrict__ codes,
                                                  uint8_t* __restrict__ buckets,
                                                  unsigned long long* __restrict__ n_reeval) {
  __shared__ double mu_s[DIM];
  for (int i = threadIdx.x; i < DIM; i += blockDim.x) mu_s[i] = mu[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  uint64_t nf = *nflag_feat;
  if (nf > max_feat) nf = max_feat;
  // one warp per flagged feature, warps numbered across CTAs first, so that a
  // short flagged list spreads over the SMs (the FP64 pipe of one SM is narrow)
  const uint64_t warp = (uint64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  const uint64_t nwarp = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long done = 0;
  for (uint64_t i = warp; i < nf; i += nwarp) {
    const uint32_t f = flaglist[i];
    // lane l holds columns 4 l .. 4 l + 3: t_j = x_j - mu_j exactly as the ordered sequence has it
    const uint32_t xw = __ldg(reinterpret_cast<const uint32_t*>(desc + (uint64_t)f * DIM) + lane);
    double t[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) t[e] = __dsub_rn((double)((xw >> (8 * e)) & 0xFFu), mu_s[4 * lane + e]);
    for (int w = 0; w < 6; ++w) {
      uint32_t mw = flagmask[(uint64_t)f * 6 + w];  // the same word in every lane
      while (mw) {
        const uint32_t row = 32u * w + (uint32_t)(__ffs(mw) - 1);
        mw &= mw - 1u;
        const double2* Rr = reinterpret_cast<const double2*>(R + (size_t)row * DIM + 4 * lane);
        const double2 r01 = __ldg(Rr), r23 = __ldg(Rr + 1);
        const double p[4] = {__dmul_rn(r01.x, t[0]), __dmul_rn(r01.y, t[1]), __dmul_rn(r23.x, t[2]),
                             __dmul_rn(r23.y, t[3])};
        // The ordered sum s_ord = (..((p_0 + p_1) + p_2) ..) + p_127 has |s_ord - sum p| <=
        // gamma_127 sum |p| (gamma_n = n u / (1 - n u), u = 2^-53); this warp's tree sum s (every
        // p_j through at most 8 additions) has |s - sum p| <= gamma_8 sum |p|, and the tree sum A
        // of the |p_j| is at least (1 - gamma_8) sum |p|.  So |s| > 1.6e-14 A (> (gamma_127 +
        // gamma_8) A / (1 - gamma_8), roundings of the test included) fixes the sign of sum p and
        // therefore of s_ord (which cannot be 0 then); the absolute term covers underflow.
        // Otherwise the ordered sequence itself is evaluated.
        double sp = __dadd_rn(__dadd_rn(__dadd_rn(p[0], p[1]), p[2]), p[3]);
        double ap = __dadd_rn(__dadd_rn(__dadd_rn(fabs(p[0]), fabs(p[1])), fabs(p[2])), fabs(p[3]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          sp = __dadd_rn(sp, __shfl_xor_sync(0xFFFFFFFFu, sp, o));
          ap = __dadd_rn(ap, __shfl_xor_sync(0xFFFFFFFFu, ap, o));
        }
        bool pos;
        if (fabs(sp) > __dadd_rn(__dmul_rn(1.6e-14, ap), 1e-290)) {  // warp-uniform
          pos = sp > 0.0;
        } else {
          double so = 0.0;
          for (int j = 0; j < DIM; ++j) {
            const int e = j & 3;
            const double mine = e == 0 ? p[0] : e == 1 ? p[1] : e == 2 ? p[2] : p[3];
            so = __dadd_rn(so, __shfl_sync(0xFFFFFFFFu, mine, j >> 2));
          }
          pos = so > 0.0;
        }
        if (lane == 0) {
          ++done;
          if (pos) {
            if (row < kp.code_bits) {
              atomicOr(&codes[(uint64_t)f * 4 + (row >> 5)], 1u << (row & 31));
            } else {
              const uint32_t rt = row - kp.code_bits;
              const uint32_t tt = rt / kp.bits_per_table, bi = rt % kp.bits_per_table;
              const uint64_t byte = (uint64_t)f * 8 + tt;
              atomicOr(reinterpret_cast<uint32_t*>(buckets) + (byte >> 2), 1u << (8 * (byte & 3) + bi));
            }
          }
        }
      }
    }
  }
  // one counter update per warp
  if (lane == 0 && done) atomicAdd(n_reeval, done);
}

cudaError_t launch_fix_fp64(const uint8_t* desc, const double* mu, const double* R, const KParams& kp,
                            const uint32_t* flagmask, const uint32_t* flaglist,
                            const unsigned long long* nflag_feat, uint64_t max_feat, uint32_t* codes,
                            uint8_t* buckets, unsigned long long* n_reeval, cudaStream_t s) {
  if (max_feat == 0) return cudaSuccess;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  k_fix_fp64<<<nsm * 8, 256, 0, s>>>(desc, mu, R, kp, flagmask, flaglist, nflag_feat, max_feat, codes, buckets,
                                     n_reeval);
  return cudaGetLastError();
}

}  // namespace chx
