// BF16 tensor-core form of the projection of Sec. 5.1 (tcgen05 + TMEM, sm_103a).
//
// v_fb = sum_j R_bj x_fj - c_b is computed as a GEMM D[128 features x N rows]
// = X (uint8 -> bf16, exact) times [Rhi | Rlo]^T, where Rhi = bf16(R) and
// Rlo = bf16(R - Rhi) (both round-to-nearest, so |R - Rhi - Rlo| <= 2^-16 |R|),
// accumulated in FP32 in tensor memory: K = 128 for Rhi, then K = 128 for Rlo
// into the same accumulator.  Products of 8-bit integers and 8-bit-significand
// bf16 values are exact in FP32.  For the accumulation the bound assumes a
// pessimistic adder (every step truncates, no guard bits), which gives at most
// 33 * 2^-23 * sum |terms| <= 2^-18 * 1.01 ||R_b|| ||x||; with the split
// residual the error is below 1.26 * 2^-16 ||R_b|| ||x||, and the flag test
// uses alpha = 2^-15 ||R_b||.  Everything under the bound is re-evaluated
// exactly in double by k_fix_fp64, so the signs equal the double definition.
//
// Shared-memory operands use the canonical K-major layout without swizzle:
// 8-row x 16-byte core matrices of 128 contiguous bytes; core matrix (r8, k8)
// sits at (r8 * 16 + k8) * 128 bytes, so the leading-dimension offset (next
// core matrix along K) is 128 B and the stride offset (next 8 rows) is 2 KB.
//
// One CTA of 512 threads per SM, persistent over tiles of 128 features, with
// two tiles in flight (two groups of 8 warps, each with its own A buffer,
// TMEM accumulator and mbarrier; the R operands are shared).  Feature row r of
// a group's tile is TMEM lane r; the two warps of a group that may access that
// lane each convert half of the row's descriptor and read back half of its
// accumulator columns with tcgen05.ld.  Every wait on an MMA mbarrier is
// bounded; on timeout the group records an error and stops issuing work, and
// the CTA still releases its tensor memory.
#include "tc_common.cuh"

namespace chx {

constexpr int TC_M = 128;
constexpr int TC_K = 128;
constexpr uint32_t TC_TMEM_COLS = 512;  // two accumulators of up to 192 columns
constexpr int PT_THREADS = 512;          // two groups of 8 warps
__device__ __forceinline__ uint32_t bf16x2_of_bytes(uint32_t w, int half) {
  // two bytes of w (half 0: bytes 0,1; half 1: bytes 2,3) as bf16x2, exact
  const float a = (float)((w >> (16 * half)) & 0xFFu);
  const float b = (float)((w >> (16 * half + 8)) & 0xFFu);
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
  return r;
}

// Named barrier of one 256-thread feature group (ids 1 and 2; __syncthreads
// uses 0).
__device__ __forceinline__ void group_sync(uint32_t id) { asm volatile("bar.sync %0, 256;" ::"r"(id) : "memory"); }

// The same barrier, returning whether any thread of the group passed x = true.
__device__ __forceinline__ bool group_any(uint32_t id, bool x) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred p, %2, 256, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)x), "r"(id)
      : "memory");
  return r != 0;
}

// Tile of 128 features: A = [16 row groups][16 k groups][128 B]; B = hi then
// lo, each [NP/8 row groups][16 k groups][128 B].  Two groups of 8 warps work
// on alternate tiles, each with its own A buffer, TMEM accumulator (columns
// 0 and 256) and mbarrier, so one group's loads, MMAs and epilogue overlap the
// other's.  In a group, warps 0-3 and 4-7 split every feature row: half h
// converts descriptor bytes 64 h .. 64 h + 63 and reads accumulator columns
// 96 h .. 96 h + 95 (rows 32 (w % 4) + lane of TMEM, the lanes warp w may
// access); half 1 hands its code / flag words to half 0, which writes the
// feature.
__global__ void __launch_bounds__(PT_THREADS, 1) k_project_bf16(const uint8_t* __restrict__ desc, uint64_t n,
                                                                const uint4* __restrict__ Rbf, uint32_t NP,
                                                                const RowConst* __restrict__ rcg, KParams kp,
                                                                uint32_t* __restrict__ codes,
                                                                uint8_t* __restrict__ buckets,
                                                                uint32_t* __restrict__ sqnorm,
                                                                uint32_t* __restrict__ flagmask,
                                                                uint32_t* __restrict__ flaglist,
                                                                unsigned long long* __restrict__ nflag_feat,
                                                                uint32_t* __restrict__ status,
                                                                float* __restrict__ dbg_x,
                                                                float* __restrict__ dbg_e) {
  extern __shared__ __align__(1024) uint8_t tsm[];
  __shared__ __align__(8) uint64_t s_mbar[2];
  __shared__ uint32_t s_tmem;
  __shared__ RowConst rc[PT_ROWS_TC];
  __shared__ uint32_t s_sq[2][2][TC_M];  // [group][half][row]: partial squared norms
  __shared__ uint32_t s_hi[2][6][TC_M];  // [group][word][row]: code words 3..5, then flag words 3..5
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int grp = warp >> 3, half = (warp >> 2) & 1, quarter = warp & 3;
  const uint32_t r = (uint32_t)(quarter * 32 + lane);  // feature row in the tile = TMEM lane
  const int leader = grp * 256;                        // issues the group's MMAs
  uint8_t* As = tsm + grp * (TC_M * TC_K * 2);         // 32 KB per group
  uint8_t* Bs = tsm + 2 * (TC_M * TC_K * 2);           // 2 x NP x 256 B
  const uint32_t bbytes = NP * TC_K * 2;               // one of hi / lo

  // operands of R (hi and lo) and the row constants, once per CTA
  for (uint32_t i = tid; i < 2 * bbytes / 16; i += PT_THREADS) reinterpret_cast<uint4*>(Bs)[i] = __ldg(Rbf + i);
  for (int i = tid; i < PT_ROWS_TC; i += PT_THREADS) {
    if ((uint32_t)i < kp.rows) rc[i] = rcg[i];
    else { RowConst z; z.c32 = 0.f; z.alpha = 0.f; z.beta = 0.f; z.pad = 0.f; rc[i] = z; }
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mbar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem + (uint32_t)grp * 256u;  // this group's accumulator columns
  const uint32_t mbar = smem_u32(&s_mbar[grp]);
  const uint32_t bar_id = 1u + (uint32_t)grp;
  const uint32_t idesc = tc_idesc(TC_M, NP);
  const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;

  const uint64_t ntiles = (n + TC_M - 1) / TC_M;
  const uint64_t stride = 2ull * gridDim.x;
  uint64_t tile = 2ull * blockIdx.x + (uint64_t)grp;
  // this thread's half row of a tile: 16-byte chunks 4 half .. 4 half + 3 (zeros beyond n)
  uint4 v[4];
  auto load_half = [&](uint64_t t) {
    const uint64_t f = t * TC_M + r;
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] = make_uint4(0u, 0u, 0u, 0u);
    if (t < ntiles && f < n) {
      const uint4* src = reinterpret_cast<const uint4*>(desc + f * DIM) + 4 * half;
#pragma unroll
      for (int c = 0; c < 4; ++c) v[c] = __ldg(src + c);
    }
  };
  load_half(tile);
  uint32_t phase = 0;
  for (; tile < ntiles; tile += stride) {
    const uint64_t f = tile * TC_M + r;
    {  // descriptor bytes -> bf16 A rows, partial squared norm
      uint8_t* rowbase = As + (r >> 3) * 2048 + (r & 7) * 16;
      uint32_t sq = 0;
#pragma unroll
      for (int c = 0; c < 4; ++c) {  // 16 bytes = 16 elements = two k groups
        const int kc = 4 * half + c;
        sq = __dp4a(v[c].x, v[c].x, sq);
        sq = __dp4a(v[c].y, v[c].y, sq);
        sq = __dp4a(v[c].z, v[c].z, sq);
        sq = __dp4a(v[c].w, v[c].w, sq);
        uint4 lo8, hi8;
        lo8.x = bf16x2_of_bytes(v[c].x, 0);
        lo8.y = bf16x2_of_bytes(v[c].x, 1);
        lo8.z = bf16x2_of_bytes(v[c].y, 0);
        lo8.w = bf16x2_of_bytes(v[c].y, 1);
        hi8.x = bf16x2_of_bytes(v[c].z, 0);
        hi8.y = bf16x2_of_bytes(v[c].z, 1);
        hi8.z = bf16x2_of_bytes(v[c].w, 0);
        hi8.w = bf16x2_of_bytes(v[c].w, 1);
        *reinterpret_cast<uint4*>(rowbase + (2 * kc) * 128) = lo8;
        *reinterpret_cast<uint4*>(rowbase + (2 * kc + 1) * 128) = hi8;
      }
      s_sq[grp][half][r] = sq;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    group_sync(bar_id);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == leader) {
      const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll
      for (int part = 0; part < 2; ++part) {  // Rhi, then Rlo
#pragma unroll
        for (int kk = 0; kk < TC_K / 16; ++kk) {
          const uint64_t ad = tc_desc(a0 + kk * 256, 128, 2048);
          const uint64_t bd = tc_desc(b0 + part * bbytes + kk * 256, 128, 2048);
          tc_mma(tmem, ad, bd, idesc, (part | kk) ? 1u : 0u);
        }
      }
      tc_commit(mbar);
    }
    load_half(tile + stride);  // the next tile's bytes are in flight during the MMAs and the epilogue
    const bool waited = mbar_wait(mbar, phase);
    if (group_any(bar_id, !waited)) {  // never expected: record it, let in-flight MMAs drain, stop
      if (tid == leader) atomicOr(status, DST_INDEX);
      mbar_wait(mbar, phase);
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // epilogue: this thread's 96 accumulator columns, 16 at a time
    const uint32_t sq = s_sq[grp][0][r] + s_sq[grp][1][r];
    const float nx = sqrtf((float)sq);
    uint32_t bits[3] = {0u, 0u, 0u}, flags[3] = {0u, 0u, 0u};  // rows 96 half + 32 k + bit
#pragma unroll
    for (int b = 0; b < 2; ++b) {  // three 16-column loads in flight
      uint32_t r3[3][16];
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const uint32_t col = (uint32_t)(96 * half + (3 * b + u) * 16);
        if (col < NP) tmem_ld16_nowait(tmem + lane_base + col, r3[u]);
      }
      tmem_wait_ld();
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        if ((uint32_t)(96 * half + (3 * b + u) * 16) >= NP) continue;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int lr = (3 * b + u) * 16 + i;  // row within the half
          const uint32_t row = (uint32_t)(96 * half + lr);
          if (row < kp.rows) {
            const RowConst rw = rc[row];
            const float x = __uint_as_float(r3[u][i]) - rw.c32;
            const float E = __fmaf_ru(rw.alpha, nx, rw.beta);
            if (dbg_x && f < n) {  // diagnostic of the bound (cashash_projection_bounds)
              dbg_x[f * kp.rows + row] = x;
              dbg_e[f * kp.rows + row] = E;
            }
            if (fabsf(x) <= E) flags[lr >> 5] |= 1u << (lr & 31);
            else if (x > 0.f) bits[lr >> 5] |= 1u << (lr & 31);
          }
        }
      }
    }
    if (half == 1) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        s_hi[grp][k][r] = bits[k];
        s_hi[grp][3 + k][r] = flags[k];
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    group_sync(bar_id);
    if (half == 0 && f < n) {
      const uint32_t b6[6] = {bits[0], bits[1], bits[2], s_hi[grp][0][r], s_hi[grp][1][r], s_hi[grp][2][r]};
      const uint32_t f6[6] = {flags[0], flags[1], flags[2], s_hi[grp][3][r], s_hi[grp][4][r], s_hi[grp][5][r]};
      write_feature(f, b6, f6, sq, kp, codes, buckets, sqnorm, flagmask, flaglist, nflag_feat);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem), "r"(TC_TMEM_COLS) : "memory");
}

cudaError_t launch_project_bf16(const uint8_t* desc, uint64_t n, const void* Rbf, uint32_t NP, const RowConst* rc,
                                const KParams& kp, uint32_t* codes, uint8_t* buckets, uint32_t* sqnorm,
                                uint32_t* flagmask, uint32_t* flaglist, unsigned long long* nflag_feat,
                                uint32_t* status, cudaStream_t s, float* dbg_x, float* dbg_e) {
  if (n == 0) return cudaSuccess;
  if (NP % 16 || NP < 16 || NP > PT_ROWS_TC) return cudaErrorInvalidValue;
  const size_t smem = 2 * (size_t)TC_M * TC_K * 2 + 2 * (size_t)NP * TC_K * 2;
  static int attr_dev = -1;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (attr_dev != dev) {
    e = cudaFuncSetAttribute(k_project_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(2 * TC_M * TC_K * 2 + 2 * PT_ROWS_TC * TC_K * 2));
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t ntiles = (n + TC_M - 1) / TC_M, pairs = (ntiles + 1) / 2;  // two tiles in flight per CTA
  const int grid = (int)(pairs < (uint64_t)nsm ? pairs : (uint64_t)nsm);
  k_project_bf16<<<grid, PT_THREADS, smem, s>>>(desc, n, reinterpret_cast<const uint4*>(Rbf), NP, rc, kp, codes,
                                                buckets, sqnorm, flagmask, flaglist, nflag_feat, status, dbg_x,
                                                dbg_e);
  return cudaGetLastError();
}

}  // namespace chx
