// Resumable chunked matching of a long pair list (the paper has no
// counterpart; its Disk-Memory-GPU loader streams data, not results): the
// caller's pairs are matched a chunk at a time against a resident image set,
// each chunk's match lists are copied to pinned host buffers and handed to a
// callback, and a cursor past the last flushed chunk lets a stopped or failed
// run resume where it left off.  Host code only; the matching itself is the
// plan / match_plan path.
#include <algorithm>
#include <vector>

#include "internal.h"

using namespace chx;

namespace {

int err_of(cudaError_t e) {
  if (e == cudaSuccess) return CASHASH_OK;
  return e == cudaErrorMemoryAllocation ? CASHASH_ENOMEM : CASHASH_ECUDA;
}

// Device and pinned host buffers of one call, grown to the largest chunk.
struct ChunkBuffers {
  uint64_t* moff_d = nullptr;
  uint32_t* mt_d = nullptr;
  uint64_t* moff_h = nullptr;
  uint32_t* mt_h = nullptr;
  uint64_t cap_off = 0, cap_mt = 0;
  ~ChunkBuffers() {
    if (moff_d) cudaFree(moff_d);
    if (mt_d) cudaFree(mt_d);
    if (moff_h) cudaFreeHost(moff_h);
    if (mt_h) cudaFreeHost(mt_h);
  }
  int reserve(uint64_t n_off, uint64_t n_mt) {
    if (n_off > cap_off) {
      if (moff_d) cudaFree(moff_d);
      if (moff_h) cudaFreeHost(moff_h);
      moff_d = nullptr;
      moff_h = nullptr;
      cap_off = 0;
      int st = err_of(cudaMalloc(reinterpret_cast<void**>(&moff_d), n_off * sizeof(uint64_t)));
      if (st == CASHASH_OK) st = err_of(cudaMallocHost(reinterpret_cast<void**>(&moff_h), n_off * sizeof(uint64_t)));
      if (st != CASHASH_OK) return st;
      cap_off = n_off;
    }
    if (n_mt > cap_mt) {
      if (mt_d) cudaFree(mt_d);
      if (mt_h) cudaFreeHost(mt_h);
      mt_d = nullptr;
      mt_h = nullptr;
      cap_mt = 0;
      int st = err_of(cudaMalloc(reinterpret_cast<void**>(&mt_d), n_mt * 2 * sizeof(uint32_t)));
      if (st == CASHASH_OK) st = err_of(cudaMallocHost(reinterpret_cast<void**>(&mt_h), n_mt * 2 * sizeof(uint32_t)));
      if (st != CASHASH_OK) return st;
      cap_mt = n_mt;
    }
    return CASHASH_OK;
  }
};

}  // namespace

extern "C" int cashash_match_chunked(cashash_ctx* c, const cashash_set* s, const uint32_t* pairs_host, uint64_t P,
                                     const double* F_dev, uint32_t chunk_pairs, uint64_t* cursor,
                                     cashash_chunk_fn fn, void* user, cashash_stream_t stream_) {
  if (!c || !s || !cursor || !fn || chunk_pairs == 0 || (P > 0 && !pairs_host) || *cursor > P) return CASHASH_EINVAL;
  if (!s->img_off && s->n_images > 0) return CASHASH_EINVAL;
  for (uint64_t i = *cursor; i < P; ++i)
    if (pairs_host[2 * i] >= s->n_images || pairs_host[2 * i + 1] >= s->n_images) return CASHASH_EINVAL;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  ChunkBuffers buf;
  while (*cursor < P) {
    const uint64_t first = *cursor;
    const uint32_t count = (uint32_t)std::min<uint64_t>(chunk_pairs, P - first);
    const uint32_t* pr = pairs_host + 2 * first;
    uint64_t cap = 0;  // at most one match per query of the chunk
    for (uint32_t i = 0; i < count; ++i) cap += s->img_off[pr[2 * (size_t)i] + 1] - s->img_off[pr[2 * (size_t)i]];
    int st = buf.reserve((uint64_t)count + 1, std::max<uint64_t>(cap, 1));
    if (st != CASHASH_OK) return st;
    cashash_plan* pl = nullptr;
    st = cashash_plan_create(c, s, pr, count, &pl);
    if (st != CASHASH_OK) return st;
    cashash_tuning want{}, cur{};
    if (cashash_get_host_tuning(c, &want) == CASHASH_OK && want.kernel != 0 &&
        cashash_plan_get_tuning(pl, &cur) == CASHASH_OK && cur.kernel != 0) {  // batched plans only
      st = cashash_plan_set_tuning(pl, &want);
      if (st == CASHASH_ENOTSUP) st = CASHASH_OK;  // the join does not apply to this chunk
    }
    if (st == CASHASH_OK)
      st = cashash_match_plan(c, pl, F_dev ? F_dev + 9 * first : nullptr, buf.moff_d, buf.mt_d, cap, stream_);
    if (st == CASHASH_OK) st = cashash_sync_status(c, stream_);
    if (st == CASHASH_OK)
      st = err_of(cudaMemcpyAsync(buf.moff_h, buf.moff_d, ((uint64_t)count + 1) * sizeof(uint64_t),
                                  cudaMemcpyDeviceToHost, stream));
    if (st == CASHASH_OK) st = err_of(cudaStreamSynchronize(stream));
    const uint64_t total = st == CASHASH_OK ? std::min<uint64_t>(buf.moff_h[count], cap) : 0;
    if (st == CASHASH_OK && total)
      st = err_of(cudaMemcpyAsync(buf.mt_h, buf.mt_d, total * 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, stream));
    if (st == CASHASH_OK) st = err_of(cudaStreamSynchronize(stream));
    cashash_plan_destroy(pl);
    if (st != CASHASH_OK) return st;  // the cursor still points at this chunk
    const int stop = fn(user, first, count, buf.moff_h, buf.mt_h);
    *cursor = first + count;
    if (stop) break;
  }
  return CASHASH_OK;
}
