// Allocation-free matching of one image pair.
//
// Some callers cannot call cudaMalloc when they want a match: a real-time
// pipeline that must not allocate (or implicitly synchronise the device)
// after start-up, a host that hands all device memory to its own pool
// allocator, or a caller whose device heap is already committed.  This entry
// point gives them the per-pair matcher with every piece of scratch memory
// (the pair record, its work items, the per-query results, the match counter
// and the status word) taken from one file-scope device array of fixed size.
// The caller still provides the inputs (an image set whose codes and lookup
// tables were built) and the outputs (match offsets and the match list).
//
// The scratch array is a static __device__ object: every GPU that loads this
// library holds it until the process exits, and every call shares it.  In
// host code its name is only a host-side stand-in, so every call looks up its
// device address with cudaGetSymbolAddress on the current device (a lookup
// that allocates nothing).  Looking it up per call, rather than caching it
// per device number, keeps the address right when the device's primary
// context is torn down and created again (cudaDeviceReset), which can load
// the array at a new address.  Calls that overlap on the GPU (on different
// streams, or from different host threads) race on the array.
#include "internal.h"

namespace chx {

struct NoAllocScratch {
  PairInfo pair;                                   // the one pair of a call
  unsigned long long count;                        // its number of matches (cleared per call)
  unsigned long long total;                        // scan output (= count)
  unsigned int item_ctr;                           // tile counter of the per-pair matching kernel (every
                                                   // tile is claimed through it): cleared before each launch
  uint32_t status;                                 // device status bits, ORed by every call until
                                                   // cashash_noalloc_status reads and clears them
  uint32_t pad[4];
  uint2 items[CASHASH_NOALLOC_MAX_QUERIES / 256];  // (pair 0, first query) per 256-query tile
  uint32_t res[CASHASH_NOALLOC_MAX_QUERIES];       // per-query result
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Writes the pair record and its work items and clears what must start at
// zero (the match counter and the tile counter); everything comes from kernel
// arguments, so no host copy is needed.  The status word is left alone: it
// collects the errors of every call until the caller reads it.
__global__ void k_noalloc_setup(NoAllocScratch* sc, PairInfo pi, uint32_t n_items, uint32_t tile) {
  for (uint32_t i = threadIdx.x; i < n_items; i += blockDim.x) sc->items[i] = make_uint2(0u, i * tile);
  if (threadIdx.x == 0) {
    sc->pair = pi;
    sc->count = 0ull;
    sc->total = 0ull;
    sc->item_ctr = 0u;
  }
}

namespace {
// The device address of the scratch array in the current device's context.
int scratch_ptr(NoAllocScratch** out) {
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess || !ptr) {
    cudaGetLastError();
    return CASHASH_ECUDA;
  }
  *out = static_cast<NoAllocScratch*>(ptr);
  return CASHASH_OK;
}
}  // namespace

}  // namespace chx

using namespace chx;

extern "C" int cashash_match_pair_noalloc(const cashash_params* p, const cashash_set* s, uint32_t image_a,
                                          uint32_t image_b, const double* F_dev, uint64_t* match_off,
                                          uint32_t* matches, uint64_t cap, cashash_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (!p || !s || !match_off || (cap > 0 && !matches)) return CASHASH_EINVAL;
  {
    cashash_params q = *p;  // precision and schedule do not apply here
    q.precision = CASHASH_FP32;
    q.schedule = CASHASH_SCHED_PER_PAIR;
    if (!params_ok(&q)) return CASHASH_EINVAL;
  }
  if (p->flags & CASHASH_FLAG_MUTUAL) return CASHASH_ENOTSUP;  // would need scratch for the reverse pair
  if (!s->img_off || image_a >= s->n_images || image_b >= s->n_images) return CASHASH_EINVAL;
  if (s->img_off[0] != 0 || s->img_off[s->n_images] != s->n_features) return CASHASH_EINVAL;
  const bool epi = p->epi_px >= 0.0;
  if (epi && (!F_dev || !s->kpts)) return CASHASH_EINVAL;
  if ((reinterpret_cast<uintptr_t>(match_off) & 7) || (reinterpret_cast<uintptr_t>(matches) & 3))
    return CASHASH_EINVAL;
  // candidate-image chunk index and sizes from the host offsets
  uint32_t bchunk0 = 0;
  for (uint32_t i = 0; i < s->n_images; ++i) {
    if (s->img_off[i + 1] < s->img_off[i] || s->img_off[i + 1] - s->img_off[i] > CASHASH_MAX_IMAGE)
      return CASHASH_EINVAL;
    if (i < image_b) bchunk0 += (uint32_t)((s->img_off[i + 1] - s->img_off[i] + JC - 1) / JC);
  }
  const uint64_t nA = s->img_off[image_a + 1] - s->img_off[image_a];
  const uint64_t nB = s->img_off[image_b + 1] - s->img_off[image_b];
  if (nA > CASHASH_NOALLOC_MAX_QUERIES) return CASHASH_EINVAL;  // beyond the fixed scratch
  if ((nA > 0 || nB > 0) && (!s->desc || !s->codes || !s->buckets || !s->sqnorm || !s->tables))
    return CASHASH_EINVAL;

  NoAllocScratch* sc = nullptr;
  if (scratch_ptr(&sc) != CASHASH_OK) return CASHASH_ECUDA;

  KParams kp{};
  kp.code_bits = p->code_bits;
  kp.n_tables = p->n_tables;
  kp.bits_per_table = p->bits_per_table;
  kp.top_k = p->top_k;
  kp.ratio_num = p->ratio_num;
  kp.ratio_den = p->ratio_den;
  kp.tau = p->tau < p->code_bits ? p->tau : p->code_bits;
  kp.rows = p->code_bits + p->n_tables * p->bits_per_table;
  kp.epi_px = p->epi_px;
  kp.flags = p->flags;

  PairInfo pi{};
  pi.a0 = s->img_off[image_a];
  pi.b0 = s->img_off[image_b];
  pi.qbase = 0;
  pi.nA = (uint32_t)nA;
  pi.nB = (uint32_t)nB;
  pi.bchunk0 = bchunk0;
  const uint32_t tile = (uint32_t)match_tile_size(p->top_k, 0);
  const uint32_t n_items = (uint32_t)((nA + tile - 1) / tile);
  if (n_items > CASHASH_NOALLOC_MAX_QUERIES / 256) return CASHASH_EINVAL;

  k_noalloc_setup<<<1, 256, 0, stream>>>(sc, pi, n_items, tile);
  if (cudaGetLastError() != cudaSuccess) return CASHASH_ECUDA;
  MatchArgs a{};
  a.desc = s->desc;
  a.codes = s->codes;
  a.buckets = s->buckets;
  a.sqnorm = s->sqnorm;
  a.tables = s->tables;
  a.kpts = s->kpts;
  a.F = epi ? F_dev : nullptr;
  a.pairs = &sc->pair;
  a.n_pairs = 1;
  a.n_res = nA;
  a.items = sc->items;
  a.n_items = n_items;
  a.item_ctr = &sc->item_ctr;
  a.res = sc->res;
  a.pair_cnt = &sc->count;
  a.status = &sc->status;
  a.kp = kp;
  if (launch_match(a, 0, n_items, stream) != cudaSuccess) return CASHASH_ECUDA;
  if (launch_scan_counts(&sc->count, 1, match_off, cap, &sc->status, &sc->total, stream) != cudaSuccess)
    return CASHASH_ECUDA;
  if (launch_compact(&sc->pair, 1, sc->res, match_off, matches, cap, stream) != cudaSuccess) return CASHASH_ECUDA;
  return CASHASH_OK;
}

extern "C" int cashash_noalloc_status(cashash_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  NoAllocScratch* sc = nullptr;
  if (scratch_ptr(&sc) != CASHASH_OK) return CASHASH_ECUDA;
  uint32_t st = 0;
  if (cudaMemcpyAsync(&st, &sc->status, sizeof st, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaMemsetAsync(&sc->status, 0, sizeof(uint32_t), stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess) {
    cudaGetLastError();
    return CASHASH_ECUDA;
  }
  if (st & DST_INDEX) return CASHASH_EDEVICE;
  if (st & DST_OVERFLOW) return CASHASH_EOVERFLOW;
  return CASHASH_OK;
}
