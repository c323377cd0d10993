// BF16 tensor-core form of the projection of Sec. 4.1 (tcgen05 + TMEM, sm_103a).
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
// One CTA of 128 threads (one warpgroup) per SM, persistent over tiles of 128
// features.  Thread t of warp w owns feature row 32 w + t: it converts the
// descriptor into the A tile, and after the MMAs reads its accumulator row
// back from TMEM lane 32 w + t with tcgen05.ld.  Every wait on the MMA
// mbarrier is bounded; on timeout the kernel records an error, stops issuing
// work, and still releases its tensor memory.
#include "internal.h"

namespace chx {

constexpr int TC_M = 128;
constexpr int TC_K = 128;
constexpr uint32_t TC_TMEM_COLS = 256;
constexpr uint32_t TC_SPIN_LIMIT = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// tcgen05 shared-memory matrix descriptor, K-major, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  // base offset 0, LBO mode 0, layout type 0 (no swizzle)
  return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: D = F32, A = B = BF16,
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t tc_idesc(uint32_t M, uint32_t N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (uint32_t i = 0; i < TC_SPIN_LIMIT; ++i) {
    uint32_t done = 0;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 16 consecutive accumulator columns of this thread's TMEM lane; no wait here
// (several loads are issued back to back, then one tcgen05.wait::ld).
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t bf16x2_of_bytes(uint32_t w, int half) {
  // two bytes of w (half 0: bytes 0,1; half 1: bytes 2,3) as bf16x2, exact
  const float a = (float)((w >> (16 * half)) & 0xFFu);
  const float b = (float)((w >> (16 * half + 8)) & 0xFFu);
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
  return r;
}

// Tile of 128 features: A = [16 row groups][16 k groups][128 B]; B = hi then
// lo, each [NP/8 row groups][16 k groups][128 B].
__global__ void __launch_bounds__(128, 1) k_project_bf16(const uint8_t* __restrict__ desc, uint64_t n,
                                                         const uint4* __restrict__ Rbf, uint32_t NP,
                                                         const RowConst* __restrict__ rcg, KParams kp,
                                                         uint32_t* __restrict__ codes, uint8_t* __restrict__ buckets,
                                                         uint32_t* __restrict__ sqnorm,
                                                         uint32_t* __restrict__ flagmask,
                                                         uint32_t* __restrict__ flaglist,
                                                         unsigned long long* __restrict__ nflag_feat,
                                                         uint32_t* __restrict__ status) {
  extern __shared__ __align__(1024) uint8_t tsm[];
  __shared__ __align__(8) uint64_t s_mbar;
  __shared__ uint32_t s_tmem;
  __shared__ RowConst rc[PT_ROWS_TC];
  uint8_t* As = tsm;                                   // 32 KB
  uint8_t* Bs = tsm + TC_M * TC_K * 2;                 // 2 x NP x 256 B
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bbytes = NP * TC_K * 2;               // one of hi / lo

  // operands of R (hi and lo) and the row constants, once per CTA
  for (uint32_t i = tid; i < 2 * bbytes / 16; i += 128) reinterpret_cast<uint4*>(Bs)[i] = __ldg(Rbf + i);
  for (int i = tid; i < PT_ROWS_TC; i += 128) {
    if ((uint32_t)i < kp.rows) rc[i] = rcg[i];
    else { RowConst z; z.c32 = 0.f; z.alpha = 0.f; z.beta = 0.f; z.pad = 0.f; rc[i] = z; }
  }
  const uint32_t mbar = smem_u32(&s_mbar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
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
  const uint32_t tmem = s_tmem;
  const uint32_t idesc = tc_idesc(TC_M, NP);
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  bool ok = true;

  const uint64_t ntiles = (n + TC_M - 1) / TC_M;
  uint32_t phase = 0;
  for (uint64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const uint64_t f = tile * TC_M + tid;
    // descriptor -> bf16 A rows (zeros beyond n), squared norm
    uint32_t sq = 0;
    {
      const uint32_t r = tid;                     // row in the tile
      uint8_t* rowbase = As + (r >> 3) * 2048 + (r & 7) * 16;
#pragma unroll
      for (int c = 0; c < 8; ++c) {               // 16 bytes = 16 elements = two k groups
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (f < n) v = __ldg(reinterpret_cast<const uint4*>(desc + f * DIM) + c);
        sq = __dp4a(v.x, v.x, sq);
        sq = __dp4a(v.y, v.y, sq);
        sq = __dp4a(v.z, v.z, sq);
        sq = __dp4a(v.w, v.w, sq);
        uint4 lo8, hi8;
        lo8.x = bf16x2_of_bytes(v.x, 0);
        lo8.y = bf16x2_of_bytes(v.x, 1);
        lo8.z = bf16x2_of_bytes(v.y, 0);
        lo8.w = bf16x2_of_bytes(v.y, 1);
        hi8.x = bf16x2_of_bytes(v.z, 0);
        hi8.y = bf16x2_of_bytes(v.z, 1);
        hi8.z = bf16x2_of_bytes(v.w, 0);
        hi8.w = bf16x2_of_bytes(v.w, 1);
        *reinterpret_cast<uint4*>(rowbase + (2 * c) * 128) = lo8;
        *reinterpret_cast<uint4*>(rowbase + (2 * c + 1) * 128) = hi8;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll
      for (int part = 0; part < 2; ++part) {      // Rhi, then Rlo
#pragma unroll
        for (int kk = 0; kk < TC_K / 16; ++kk) {
          const uint64_t ad = tc_desc(a0 + kk * 256, 128, 2048);
          const uint64_t bd = tc_desc(b0 + part * bbytes + kk * 256, 128, 2048);
          tc_mma(tmem, ad, bd, idesc, (part | kk) ? 1u : 0u);
        }
      }
      tc_commit(mbar);
    }
    if (!mbar_wait(mbar, phase)) {  // never expected: record it, let in-flight MMAs drain, stop
      ok = false;
      if (tid == 0) atomicOr(status, DST_INDEX);
      mbar_wait(mbar, phase);
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // epilogue: this thread's accumulator row, 16 columns at a time
    const float nx = sqrtf((float)sq);
    uint32_t bits[6] = {0u, 0u, 0u, 0u, 0u, 0u}, flags[6] = {0u, 0u, 0u, 0u, 0u, 0u};
#pragma unroll
    for (int cg0 = 0; cg0 < PT_ROWS_TC / 16; cg0 += 3) {  // three 16-column loads in flight
      uint32_t r3[3][16];
#pragma unroll
      for (int u = 0; u < 3; ++u)
        if ((uint32_t)((cg0 + u) * 16) < NP) tmem_ld16_nowait(tmem + lane_base + (uint32_t)((cg0 + u) * 16), r3[u]);
      tmem_wait_ld();
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        if ((uint32_t)((cg0 + u) * 16) >= NP) continue;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int row = (cg0 + u) * 16 + i;
          if ((uint32_t)row < kp.rows) {
            const RowConst r = rc[row];
            const float x = __uint_as_float(r3[u][i]) - r.c32;
            const float E = __fmaf_ru(r.alpha, nx, r.beta);
            if (fabsf(x) <= E) flags[row >> 5] |= 1u << (row & 31);
            else if (x > 0.f) bits[row >> 5] |= 1u << (row & 31);
          }
        }
      }
    }
    if (f < n) write_feature(f, bits, flags, sq, kp, codes, buckets, sqnorm, flagmask, flaglist, nflag_feat);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  (void)lane;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
}

cudaError_t launch_project_bf16(const uint8_t* desc, uint64_t n, const void* Rbf, uint32_t NP, const RowConst* rc,
                                const KParams& kp, uint32_t* codes, uint8_t* buckets, uint32_t* sqnorm,
                                uint32_t* flagmask, uint32_t* flaglist, unsigned long long* nflag_feat,
                                uint32_t* status, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (NP % 16 || NP < 16 || NP > PT_ROWS_TC) return cudaErrorInvalidValue;
  const size_t smem = (size_t)TC_M * TC_K * 2 + 2 * (size_t)NP * TC_K * 2;
  static int attr_dev = -1;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (attr_dev != dev) {
    e = cudaFuncSetAttribute(k_project_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(TC_M * TC_K * 2 +
                                                                                                  2 * PT_ROWS_TC * TC_K * 2));
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t ntiles = (n + TC_M - 1) / TC_M;
  const int grid = (int)(ntiles < (uint64_t)nsm ? ntiles : (uint64_t)nsm);
  k_project_bf16<<<grid, 128, smem, s>>>(desc, n, reinterpret_cast<const uint4*>(Rbf), NP, rc, kp, codes, buckets,
                                         sqnorm, flagmask, flaglist, nflag_feat, status);
  return cudaGetLastError();
}

}  // namespace chx
