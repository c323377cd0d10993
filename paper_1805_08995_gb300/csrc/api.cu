// Host runtime behind the C-ABI of include/cashash.h: argument checks, the
// context (projection matrix, centre, workspace), pair plans, the launch
// sequences of cashash_build_codes / cashash_match_plan, and the end-to-end
// host path with pinned staging on a side stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

using namespace chx;

namespace {

struct HostWS {  // device buffers of the end-to-end host path, grown on demand
  uint8_t* desc = nullptr;       uint64_t cap_desc = 0;
  uint32_t* codes = nullptr;     uint64_t cap_codes = 0;
  uint8_t* buckets = nullptr;    uint64_t cap_buckets = 0;
  uint32_t* sqnorm = nullptr;    uint64_t cap_sq = 0;
  uint8_t* tables = nullptr;     uint64_t cap_tables = 0;
  float* kpts = nullptr;         uint64_t cap_kpts = 0;
  double* F = nullptr;           uint64_t cap_F = 0;
  uint64_t* moff = nullptr;      uint64_t cap_moff = 0;
  uint32_t* matches = nullptr;   uint64_t cap_matches = 0;
  uint8_t* pin[2] = {nullptr, nullptr};
  uint64_t pin_cap = 0;
  cudaStream_t copy = nullptr, comp = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaEvent_t staged = nullptr;
  std::vector<uint32_t> plan_pairs;  // pair list of the cached plan
  std::vector<uint64_t> plan_off;    // image offsets of the cached plan
  cashash_plan* plan = nullptr;
  cashash_tuning tune{};             // configuration for the host path's plans, when has_tune
  bool has_tune = false;
};

}  // namespace

struct cashash_ctx {
  cashash_params p{};
  KParams kp{};
  int device = 0;
  int nsm = 0;
  uint32_t rows = 0;
  double* d_R = nullptr;        // [rows][128]
  double* d_nrmR = nullptr;     // [rows]
  float* d_R32T = nullptr;      // [128][192] FP32 R, transposed, zero padded
  void* d_Rbf = nullptr;        // BF16 form operands: R hi and lo, core-matrix layout
  uint32_t np_tc = 0;           // BF16 form: rows padded to a multiple of 16
  double* d_mu = nullptr;       // [128]
  RowConst* d_rc = nullptr;     // [192]
  unsigned long long* d_colsum = nullptr;  // [128]
  unsigned long long* d_cnt = nullptr;     // [0] flagged features [1] re-evaluated rows [2] matches
  uint32_t* d_status = nullptr;
  uint32_t* d_flagmask = nullptr;   // [n][6] rows flagged for re-evaluation
  uint32_t* d_flaglist = nullptr;   // [n] features with flagged rows
  uint64_t cap_flagmask = 0, cap_flaglist = 0;
  uint64_t* d_chunk_feat0 = nullptr;
  uint32_t* d_chunk_len = nullptr;
  uint64_t cap_cf0 = 0, cap_clen = 0;
  uint64_t* d_img_f0 = nullptr;     // per image: first feature, feature count, join-table base
  uint32_t* d_img_n = nullptr;
  uint64_t* d_img_join = nullptr;
  uint64_t cap_if0 = 0, cap_in = 0, cap_ij = 0;
  cudaStream_t last_stream = nullptr;
  uint64_t last_n_features = 0;
  int built = 0;                       // cashash_build_codes has run (centre and row constants set)
  std::vector<uint64_t> layout_off;    // image offsets of the uploaded layout arrays
  const void* layout_bufs[5] = {};     // the buffers they were uploaded to
  bool layout_ok = false;
  cudaEvent_t layout_ev = nullptr;     // recorded after the last upload
  // cashash_build_codes as a CUDA graph: captured on the second call with the same set, layout,
  // scratch buffers and profiling setting, replayed while they stay the same
  cashash_set bg_set{};
  std::vector<uint64_t> bg_off;
  const void* bg_scratch[8] = {};
  int bg_prof = -1;
  int bg_seen = 0;                     // calls with the current key (the first runs eagerly)
  cudaStream_t bg_stream = nullptr;
  cudaGraphExec_t bg_exec = nullptr;
  uint64_t last_pairs = 0;
  uint64_t last_items = 0;
  uint64_t n_launches = 0;
  int profiling = 0;
  cudaEvent_t ev[CASHASH_N_STAGES][2] = {};
  int ev_used[CASHASH_N_STAGES] = {};
  HostWS hw;
};

struct cashash_plan {
  cashash_ctx* ctx = nullptr;
  uint32_t P = 0;                      // pairs matched (with the mutual check: the user's pairs, then their reversals)
  uint32_t P_out = 0;                  // pairs reported (the user's)
  double* d_F2 = nullptr;              // mutual check with the band: F of every matched pair (F, then F^T)
  uint64_t cap_F2 = 0;
  int persistent = 0;
  PairInfo* d_pairs = nullptr;
  uint2* d_items = nullptr;
  uint32_t n_items = 0;
  uint32_t* d_res = nullptr;
  uint64_t n_res = 0;
  unsigned long long* d_pair_cnt = nullptr;
  unsigned int* d_item_ctr = nullptr;  // [P + 1]: per-pair launches, then the persistent launch
  uint32_t* d_queue = nullptr;         // survivor queues of the persistent (speculative) kernel
  uint32_t* d_tau = nullptr;           // per pair: learned Hamming threshold + 1 (0 = none yet)
  uint32_t grid = 0;                   // persistent grid (resident CTAs)
  uint32_t tau_fixed = 0;              // keep the Hamming threshold hint fixed
  uint32_t occ_grid = 0;               // per-pair launches: resident CTAs
  bool join = false;                   // persistent schedule: bucket join (else speculative kernel)
  cashash_tuning tune{};               // persistent schedule: kernel configuration
  uint32_t na_max = 1;                 // largest query image (bucket-join scratch)
  uint32_t* d_jhist = nullptr;         // bucket join: per-pair histogram of k-th Hamming distances
  float4* d_jline = nullptr;           // bucket join with the band: per-CTA query lines
  uint64_t cap_items = 0, cap_queue = 0, cap_jline = 0;
  std::vector<uint32_t> first, count;  // per-pair item ranges (per-pair schedule)
  std::vector<PairInfo> info;          // host copies: pair records, pair list, the set and its offsets
  std::vector<uint32_t> pairs_h;
  std::vector<uint64_t> img_off_h;
  cashash_set set{};
  // persistent schedule: the launch sequence captured as a CUDA graph, replayed
  // while the outputs, F and the profiling setting stay the same
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const double* g_F = nullptr;
  uint64_t* g_moff = nullptr;
  uint32_t* g_mt = nullptr;
  uint64_t g_cap = 0;
  int g_prof = -1;
  const uint8_t* desc = nullptr;
  const uint32_t* codes = nullptr;
  const uint8_t* buckets = nullptr;
  const uint32_t* sqnorm = nullptr;
  const uint8_t* tables = nullptr;
  const float* kpts = nullptr;
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
// Parameter ranges every entry point accepts (declared in internal.h).
int chx::params_ok(const cashash_params* p) {
  if (!p) return 0;
  if (p->code_bits != 32 && p->code_bits != 64 && p->code_bits != 96 && p->code_bits != 128) return 0;
  if (p->n_tables < 1 || p->n_tables > CASHASH_MAX_TABLES) return 0;
  if (p->bits_per_table > 8) return 0;
  if (p->top_k < 1 || p->top_k > CASHASH_MAX_K) return 0;
  if (p->ratio_den < 1 || p->ratio_den > 65535 || p->ratio_num > 65535) return 0;
  if (p->precision > CASHASH_BF16 || p->schedule > CASHASH_SCHED_PERSISTENT) return 0;
  if (p->flags & ~(CASHASH_FLAG_MUTUAL | CASHASH_FLAG_ACCEPT_SINGLE)) return 0;
  if (std::isnan(p->epi_px) || std::isinf(p->epi_px)) return 0;
  return 1;
}

namespace {

int cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return CASHASH_OK;
  if (e == cudaErrorMemoryAllocation) return CASHASH_ENOMEM;
  return CASHASH_ECUDA;
}

#define CK(x)                              \
  do {                                     \
    const int _st = cuda_err((x));         \
    if (_st != CASHASH_OK) return _st;     \
  } while (0)


template <class T>
int grow(T*& ptr, uint64_t& cap, uint64_t need) {
  if (need <= cap && ptr) return CASHASH_OK;
  if (ptr) {
    cudaDeviceSynchronize();
    cudaFree(ptr);
  }
  ptr = nullptr;
  cap = 0;
  if (need == 0) need = 1;
  if (cudaMalloc(reinterpret_cast<void**>(&ptr), need * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    ptr = nullptr;
    return CASHASH_ENOMEM;
  }
  cap = need;
  return CASHASH_OK;
}

template <class T>
void dfree(T*& ptr) {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
}

// Round-to-nearest-even of a double to bfloat16 (8-bit significand), bits.
uint16_t bf16_rn(double x) {
  if (x == 0.0 || !std::isfinite(x)) return std::signbit(x) ? 0x8000u : 0u;
  int e = 0;
  const double m = std::frexp(std::fabs(x), &e);  // |x| = m 2^e, m in [0.5, 1)
  double M = std::nearbyint(std::ldexp(m, 8));     // 8 significant bits, ties to even
  if (M == 256.0) {
    M = 128.0;
    e += 1;
  }
  const float v = (float)std::ldexp(M, e - 8);     // exact: at most 8 significant bits
  uint32_t u;
  std::memcpy(&u, &v, sizeof u);
  if (x < 0) u |= 0x80000000u;
  return (uint16_t)(u >> 16);
}

double bf16_to_double(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, sizeof f);
  return (double)f;
}

// Validates a set; returns number of lookup-table chunks through *n_chunks.
int set_ok(const cashash_set* s, uint64_t* n_chunks) {
  if (!s || (s->n_images > 0 && !s->img_off)) return 0;
  if (s->n_images == 0) {
    if (n_chunks) *n_chunks = 0;
    return s->n_features == 0;
  }
  if (s->img_off[0] != 0 || s->img_off[s->n_images] != s->n_features) return 0;
  if (s->n_features >= (1ull << 32)) return 0;
  uint64_t ch = 0;
  for (uint32_t i = 0; i < s->n_images; ++i) {
    if (s->img_off[i + 1] < s->img_off[i]) return 0;
    const uint64_t n = s->img_off[i + 1] - s->img_off[i];
    if (n > CASHASH_MAX_IMAGE) return 0;
    ch += (n + JC - 1) / JC;
  }
  if (s->n_features > 0) {
    if (!s->desc || !s->codes || !s->buckets || !s->sqnorm || !s->tables) return 0;
    if ((reinterpret_cast<uintptr_t>(s->desc) & 15) || (reinterpret_cast<uintptr_t>(s->codes) & 15) ||
        (reinterpret_cast<uintptr_t>(s->buckets) & 7) || (reinterpret_cast<uintptr_t>(s->sqnorm) & 3) ||
        (reinterpret_cast<uintptr_t>(s->tables) & 15) || (reinterpret_cast<uintptr_t>(s->kpts) & 7))
      return 0;
  }
  if (n_chunks) *n_chunks = ch;
  return 1;
}

void chunk_layout(const uint64_t* img_off, uint32_t n_images, std::vector<uint64_t>& f0, std::vector<uint32_t>& len,
                  std::vector<uint32_t>* first_chunk) {
  f0.clear();
  len.clear();
  if (first_chunk) first_chunk->assign(n_images, 0);
  for (uint32_t i = 0; i < n_images; ++i) {
    if (first_chunk) (*first_chunk)[i] = (uint32_t)f0.size();
    const uint64_t n = img_off[i + 1] - img_off[i];
    for (uint64_t c = 0; c * JC < n; ++c) {
      f0.push_back(img_off[i] + c * JC);
      len.push_back((uint32_t)std::min<uint64_t>(JC, n - c * JC));
    }
  }
}

// Stage timing: events recorded on the launching stream around a stage.
struct StageTimer {
  cashash_ctx* c;
  int id;
  cudaStream_t s;
  unsigned flags;  // cudaEventRecordExternal while capturing a graph
  StageTimer(cashash_ctx* c_, int id_, cudaStream_t s_, bool capturing = false)
      : c(c_), id(id_), s(s_), flags(capturing ? cudaEventRecordExternal : 0u) {
    if (c->profiling && c->ev[id][0]) cudaEventRecordWithFlags(c->ev[id][0], s, flags);
  }
  ~StageTimer() {
    if (c->profiling && c->ev[id][1]) {
      cudaEventRecordWithFlags(c->ev[id][1], s, flags);
      c->ev_used[id] = 1;
    }
  }
};

// Byte offsets of every image's bucket-sorted tables in the table buffer
// (after the chunked lookup tables).
void join_layout(const uint64_t* img_off, uint32_t n_images, uint32_t T, std::vector<uint64_t>& base) {
  uint64_t ch = 0;
  for (uint32_t i = 0; i < n_images; ++i) ch += (img_off[i + 1] - img_off[i] + JC - 1) / JC;
  uint64_t o = std::max<uint64_t>(ch, 1) * chunk_bytes(T);
  base.resize(n_images);
  for (uint32_t i = 0; i < n_images; ++i) {
    base[i] = o;
    o += (uint64_t)T * join_block(img_off[i + 1] - img_off[i]);
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// C-ABI
// ---------------------------------------------------------------------------
namespace {
// cashash_build_codes; sums_ready: the column sums of the set are already in
// c->d_colsum (taken block by block while the host path stages the set).
int build_codes_impl(cashash_ctx* c, const cashash_set* s, const double* mean_host, cudaStream_t stream,
                     bool sums_ready) {
  uint64_t n_chunks = 0;
  if (!c || !set_ok(s, &n_chunks)) return CASHASH_EINVAL;
  if (mean_host)
    for (int j = 0; j < DIM; ++j)
      if (!std::isfinite(mean_host[j])) return CASHASH_EINVAL;
  const uint64_t n = s->n_features;
  CK(cudaSetDevice(c->device));
  int st = grow(c->d_flagmask, c->cap_flagmask, std::max<uint64_t>(n, 1) * 6);
  if (st == CASHASH_OK) st = grow(c->d_flaglist, c->cap_flaglist, std::max<uint64_t>(n, 1));
  if (st == CASHASH_OK) st = grow(c->d_chunk_feat0, c->cap_cf0, std::max<uint64_t>(n_chunks, 1));
  if (st == CASHASH_OK) st = grow(c->d_chunk_len, c->cap_clen, std::max<uint64_t>(n_chunks, 1));
  const uint64_t ni = std::max<uint32_t>(s->n_images, 1);
  if (st == CASHASH_OK) st = grow(c->d_img_f0, c->cap_if0, ni);
  if (st == CASHASH_OK) st = grow(c->d_img_n, c->cap_in, ni);
  if (st == CASHASH_OK) st = grow(c->d_img_join, c->cap_ij, ni);
  if (st != CASHASH_OK) return st;
  std::vector<uint32_t> inn(s->n_images);
  for (uint32_t i = 0; i < s->n_images; ++i) inn[i] = (uint32_t)(s->img_off[i + 1] - s->img_off[i]);
  // Layout arrays of the set (image and chunk offsets, table bases): uploaded
  // again only when the image offsets (or the buffers holding them) changed.
  const void* bufs[5] = {c->d_img_f0, c->d_img_n, c->d_img_join, c->d_chunk_feat0, c->d_chunk_len};
  const bool same_layout = c->layout_ok && c->layout_off.size() == (size_t)s->n_images + 1 &&
                           std::memcmp(c->layout_off.data(), s->img_off, 8 * ((size_t)s->n_images + 1)) == 0 &&
                           std::memcmp(c->layout_bufs, bufs, sizeof bufs) == 0;
  if (same_layout) {
    CK(cudaStreamWaitEvent(stream, c->layout_ev, 0));  // the uploads, if another stream made them
  } else {
    c->layout_ok = false;
    std::vector<uint64_t> jbase, if0(s->img_off, s->img_off + s->n_images);
    join_layout(s->img_off, s->n_images, c->p.n_tables, jbase);
    if (s->n_images) {
      CK(cudaMemcpyAsync(c->d_img_f0, if0.data(), s->n_images * sizeof(uint64_t), cudaMemcpyHostToDevice, stream));
      CK(cudaMemcpyAsync(c->d_img_n, inn.data(), s->n_images * sizeof(uint32_t), cudaMemcpyHostToDevice, stream));
      CK(cudaMemcpyAsync(c->d_img_join, jbase.data(), s->n_images * sizeof(uint64_t), cudaMemcpyHostToDevice,
                         stream));
    }
    std::vector<uint64_t> f0;
    std::vector<uint32_t> len;
    chunk_layout(s->img_off, s->n_images, f0, len, nullptr);
    if (n_chunks) {
      CK(cudaMemcpyAsync(c->d_chunk_feat0, f0.data(), n_chunks * sizeof(uint64_t), cudaMemcpyHostToDevice, stream));
      CK(cudaMemcpyAsync(c->d_chunk_len, len.data(), n_chunks * sizeof(uint32_t), cudaMemcpyHostToDevice, stream));
    }
    if (!c->layout_ev) CK(cudaEventCreateWithFlags(&c->layout_ev, cudaEventDisableTiming));
    CK(cudaEventRecord(c->layout_ev, stream));
    c->layout_off.assign(s->img_off, s->img_off + s->n_images + 1);
    std::memcpy(c->layout_bufs, bufs, sizeof bufs);
    c->layout_ok = true;
  }
  for (int i = 0; i < 4; ++i) c->ev_used[i] = 0;
  const uint32_t n_max = inn.empty() ? 0u : *std::max_element(inn.begin(), inn.end());
  // the stages, on `st` (capturing: while a graph is being captured)
  auto enqueue = [&](cudaStream_t st, bool capturing) -> int {
    {  // centre (reading: mean over the whole set) and per-row constants
      StageTimer tm(c, CASHASH_STAGE_CENTRE, st, capturing);
      if (mean_host) {
        CK(cudaMemcpyAsync(c->d_mu, mean_host, DIM * sizeof(double), cudaMemcpyHostToDevice, st));
      } else if (!sums_ready) {
        CK(launch_colsum(s->desc, n, c->d_colsum, st));
      }
      // bound factor on ||R_b|| ||x||: FP32 FMA chains (2^-16), BF16 tensor cores (2^-15)
      const float alpha_scale = c->p.precision == CASHASH_BF16 ? 0x1p-15f : 0x1p-16f;
      CK(launch_row_consts(c->d_colsum, n, mean_host ? 1 : 0, c->d_mu, c->d_R, c->d_nrmR, c->rows, alpha_scale,
                           c->d_rc, st));
      CK(cudaMemsetAsync(c->d_cnt, 0, 2 * sizeof(unsigned long long), st));
    }
    if (n) {
      {
        StageTimer tm(c, CASHASH_STAGE_PROJECT, st, capturing);
        if (c->p.precision == CASHASH_BF16)
          CK(launch_project_bf16(s->desc, n, c->d_Rbf, c->np_tc, c->d_rc, c->kp, s->codes, s->buckets, s->sqnorm,
                                 c->d_flagmask, c->d_flaglist, c->d_cnt + 0, c->d_status, st));
        else
          CK(launch_project_fp32(s->desc, n, c->d_R32T, c->d_rc, c->kp, s->codes, s->buckets, s->sqnorm,
                                 c->d_flagmask, c->d_flaglist, c->d_cnt + 0, st));
      }
      {
        StageTimer tm(c, CASHASH_STAGE_REEVAL, st, capturing);
        CK(launch_fix_fp64(s->desc, c->d_mu, c->d_R, c->kp, c->d_flagmask, c->d_flaglist, c->d_cnt + 0, n, s->codes,
                           s->buckets, c->d_cnt + 1, st));
      }
      {
        StageTimer tm(c, CASHASH_STAGE_TABLES, st, capturing);
        CK(launch_build_tables(s->buckets, c->d_chunk_feat0, c->d_chunk_len, (uint32_t)n_chunks, c->p.n_tables,
                               s->tables, st));
        CK(launch_build_join(s->buckets, s->codes, c->d_img_f0, c->d_img_n, c->d_img_join, s->n_images,
                             c->p.n_tables, n_max, s->tables, st));
      }
    }
    return CASHASH_OK;
  };
  c->n_launches += (!mean_host && !sums_ready && n ? 1 : 0) + 1 + (n ? 4 : 0);
  // A repeated build of the same set (same buffers, layout and scratch, the centre computed here)
  // replays one captured graph: the stages are a dozen short launches whose gaps would otherwise
  // show on small sets.
  const void* scratch[8] = {c->d_flagmask, c->d_flaglist, c->d_chunk_feat0, c->d_chunk_len,
                            c->d_img_f0,   c->d_img_n,    c->d_img_join,    c->d_colsum};
  const bool graphable = !mean_host && !sums_ready && n > 0;
  const bool same_key = graphable && std::memcmp(&c->bg_set, s, sizeof *s) == 0 && c->bg_prof == c->profiling &&
                        std::memcmp(c->bg_scratch, scratch, sizeof scratch) == 0 &&
                        c->bg_off.size() == (size_t)s->n_images + 1 &&
                        std::memcmp(c->bg_off.data(), s->img_off, 8 * ((size_t)s->n_images + 1)) == 0;
  if (!same_key) {
    if (c->bg_exec) cudaGraphExecDestroy(c->bg_exec);
    c->bg_exec = nullptr;
    c->bg_seen = 0;
    if (graphable) {
      c->bg_set = *s;
      c->bg_off.assign(s->img_off, s->img_off + s->n_images + 1);
      std::memcpy(c->bg_scratch, scratch, sizeof scratch);
      c->bg_prof = c->profiling;
    } else {
      c->bg_prof = -1;
    }
  }
  if (graphable && ++c->bg_seen >= 2) {
    if (!c->bg_exec) {
      if (!c->bg_stream) CK(cudaStreamCreateWithFlags(&c->bg_stream, cudaStreamNonBlocking));
      CK(cudaStreamBeginCapture(c->bg_stream, cudaStreamCaptureModeThreadLocal));
      const int es = enqueue(c->bg_stream, true);
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(c->bg_stream, &g);
      if (es != CASHASH_OK) {
        if (g) cudaGraphDestroy(g);
        return es;
      }
      CK(e);
      const cudaError_t ei = cudaGraphInstantiate(&c->bg_exec, g, 0);
      cudaGraphDestroy(g);
      CK(ei);
    }
    CK(cudaGraphLaunch(c->bg_exec, stream));
    if (c->profiling)  // the graph holds the stage events as external event-record nodes
      for (int i = 0; i < 4; ++i) c->ev_used[i] = 1;
  } else {
    const int es = enqueue(stream, false);
    if (es != CASHASH_OK) return es;
  }
  c->last_stream = stream;
  c->last_n_features = n;
  c->built = 1;
  return CASHASH_OK;
}
}  // namespace

extern "C" {

const char* cashash_strerror(int st) {
  switch (st) {
    case CASHASH_OK: return "ok";
    case CASHASH_EINVAL: return "invalid argument";
    case CASHASH_ENOMEM: return "out of memory";
    case CASHASH_ECUDA: return "CUDA runtime error";
    case CASHASH_EOVERFLOW: return "match capacity exceeded";
    case CASHASH_EDEVICE: return "device-side error recorded";
    case CASHASH_ETIMEOUT: return "bounded wait timed out";
    case CASHASH_ENOTSUP: return "not supported by the library";
    default: return "unknown status";
  }
}

void cashash_default_params(cashash_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->code_bits = 128;
  p->n_tables = 6;
  p->bits_per_table = 8;
  p->top_k = 10;
  p->ratio_num = 4;
  p->ratio_den = 5;
  p->tau = 128;
  p->precision = CASHASH_FP32;
  p->schedule = CASHASH_SCHED_PERSISTENT;
  p->epi_px = -1.0;
}

uint64_t cashash_tables_bytes(const cashash_params* p, const uint64_t* img_off, uint32_t n_images) {
  if (!params_ok(p) || (n_images > 0 && !img_off)) return 0;
  uint64_t ch = 0, jb = 0;
  for (uint32_t i = 0; i < n_images; ++i) {
    if (img_off[i + 1] < img_off[i]) return 0;
    const uint64_t n = img_off[i + 1] - img_off[i];
    ch += (n + JC - 1) / JC;
    jb += (uint64_t)p->n_tables * join_block(n);
  }
  return std::max<uint64_t>(ch, 1) * chunk_bytes(p->n_tables) + jb;
}

int cashash_get_params(const cashash_ctx* c, cashash_params* out) {
  if (!c || !out) return CASHASH_EINVAL;
  *out = c->p;
  return CASHASH_OK;
}

void cashash_destroy(cashash_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  if (c->hw.plan) cashash_plan_destroy(c->hw.plan);
  HostWS& h = c->hw;
  dfree(h.desc); dfree(h.codes); dfree(h.buckets); dfree(h.sqnorm); dfree(h.tables); dfree(h.kpts);
  dfree(h.F); dfree(h.moff); dfree(h.matches);
  for (int i = 0; i < 2; ++i) {
    if (h.pin[i]) cudaFreeHost(h.pin[i]);
    if (h.ev[i]) cudaEventDestroy(h.ev[i]);
  }
  if (h.staged) cudaEventDestroy(h.staged);
  if (c->layout_ev) cudaEventDestroy(c->layout_ev);
  if (c->bg_exec) cudaGraphExecDestroy(c->bg_exec);
  if (c->bg_stream) cudaStreamDestroy(c->bg_stream);
  if (h.copy) cudaStreamDestroy(h.copy);
  if (h.comp) cudaStreamDestroy(h.comp);
  dfree(c->d_R); dfree(c->d_nrmR); dfree(c->d_R32T); dfree(c->d_Rbf); dfree(c->d_mu); dfree(c->d_rc);
  dfree(c->d_colsum); dfree(c->d_cnt); dfree(c->d_status); dfree(c->d_flagmask); dfree(c->d_flaglist);
  dfree(c->d_chunk_feat0); dfree(c->d_chunk_len);
  dfree(c->d_img_f0); dfree(c->d_img_n); dfree(c->d_img_join);
  for (int i = 0; i < CASHASH_N_STAGES; ++i)
    for (int k = 0; k < 2; ++k)
      if (c->ev[i][k]) cudaEventDestroy(c->ev[i][k]);
  delete c;
}

int cashash_create(cashash_ctx** out, const cashash_params* p, const double* R_host) {
  if (!out || !params_ok(p) || !R_host) return CASHASH_EINVAL;
  *out = nullptr;
  const uint32_t rows = p->code_bits + p->n_tables * p->bits_per_table;
  for (uint64_t i = 0; i < (uint64_t)rows * DIM; ++i)
    if (!std::isfinite(R_host[i])) return CASHASH_EINVAL;
  cashash_ctx* c = new (std::nothrow) cashash_ctx();
  if (!c) return CASHASH_ENOMEM;
  c->p = *p;
  c->rows = rows;
  c->kp.code_bits = p->code_bits;
  c->kp.n_tables = p->n_tables;
  c->kp.bits_per_table = p->bits_per_table;
  c->kp.top_k = p->top_k;
  c->kp.ratio_num = p->ratio_num;
  c->kp.ratio_den = p->ratio_den;
  c->kp.tau = std::min(p->tau, p->code_bits);
  c->kp.rows = rows;
  c->kp.epi_px = p->epi_px;
  c->kp.flags = p->flags;
  int st = cuda_err(cudaGetDevice(&c->device));
  if (st == CASHASH_OK) st = cuda_err(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device));
  // host-side constants: FP32 transposed copy of R and row norms (rounded up)
  std::vector<float> r32t((size_t)DIM * 192, 0.f);
  std::vector<double> nrm(rows, 0.0);
  for (uint32_t b = 0; b < rows; ++b) {
    long double s = 0.0L;
    for (int j = 0; j < DIM; ++j) {
      const double v = R_host[(size_t)b * DIM + j];
      r32t[(size_t)j * 192 + b] = (float)v;
      s += (long double)v * (long double)v;
    }
    nrm[b] = (double)sqrtl(s) * (1.0 + 1e-12);
  }
  uint64_t cap = 0;
  if (st == CASHASH_OK) st = grow(c->d_R, cap, (uint64_t)rows * DIM);
  cap = 0;
  if (st == CASHASH_OK) st = grow(c->d_nrmR, cap, rows);
  cap = 0;
  if (st == CASHASH_OK) st = grow(c->d_R32T, cap, (uint64_t)DIM * 192);
  cap = 0;
  if (st == CASHASH_OK) st = grow(c->d_mu, cap, DIM);
  cap = 0;
  if (st == CASHASH_OK) st = grow(c->d_rc, cap, 192);
  cap = 0;
  if (st == CASHASH_OK) st = grow(c->d_colsum, cap, DIM);
  cap = 0;
  if (st == CASHASH_OK) st = grow(c->d_cnt, cap, 8);
  cap = 0;
  if (st == CASHASH_OK) st = grow(c->d_status, cap, 1);
  if (st == CASHASH_OK) st = cuda_err(cudaMemcpy(c->d_R, R_host, sizeof(double) * rows * DIM, cudaMemcpyHostToDevice));
  if (st == CASHASH_OK) st = cuda_err(cudaMemcpy(c->d_nrmR, nrm.data(), sizeof(double) * rows, cudaMemcpyHostToDevice));
  if (st == CASHASH_OK)
    st = cuda_err(cudaMemcpy(c->d_R32T, r32t.data(), sizeof(float) * r32t.size(), cudaMemcpyHostToDevice));
  if (st == CASHASH_OK && p->precision == CASHASH_BF16) {
    // R = hi + lo + r with hi = bf16(R), lo = bf16(R - hi) (R - hi is exact by Sterbenz), |r| <= 2^-16 |R|;
    // laid out as K-major core matrices: (row group, k group) at ((r8 * 16 + k8) * 64) elements
    const uint32_t NP = (rows + 15) / 16 * 16;
    c->np_tc = NP;
    std::vector<uint16_t> hb((size_t)2 * NP * DIM, 0);
    for (uint32_t b = 0; b < rows; ++b)
      for (int j = 0; j < DIM; ++j) {
        const double v = R_host[(size_t)b * DIM + j];
        const uint16_t hi = bf16_rn(v);
        const uint16_t lo = bf16_rn(v - bf16_to_double(hi));
        const size_t off = ((size_t)(b >> 3) * 16 + (j >> 3)) * 64 + (b & 7) * 8 + (j & 7);
        hb[off] = hi;
        hb[(size_t)NP * DIM + off] = lo;
      }
    cap = 0;
    uint16_t* d = nullptr;
    st = grow(d, cap, hb.size());
    c->d_Rbf = d;
    if (st == CASHASH_OK)
      st = cuda_err(cudaMemcpy(c->d_Rbf, hb.data(), hb.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
  }
  if (st == CASHASH_OK) st = cuda_err(cudaMemset(c->d_cnt, 0, 8 * sizeof(unsigned long long)));
  if (st == CASHASH_OK) st = cuda_err(cudaMemset(c->d_status, 0, sizeof(uint32_t)));
  if (st == CASHASH_OK) st = cuda_err(cudaMemset(c->d_mu, 0, DIM * sizeof(double)));
  if (st != CASHASH_OK) {
    cashash_destroy(c);
    return st;
  }
  *out = c;
  return CASHASH_OK;
}

int cashash_build_codes(cashash_ctx* c, const cashash_set* s, const double* mean_host, cashash_stream_t stream_) {
  return build_codes_impl(c, s, mean_host, reinterpret_cast<cudaStream_t>(stream_), false);
}


int cashash_projection_bounds(cashash_ctx* c, const cashash_set* s, uint64_t first, uint64_t count,
                              float* approx, float* bound, cashash_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  uint64_t n_chunks = 0;
  if (!c || !set_ok(s, &n_chunks) || !approx || !bound || !c->built) return CASHASH_EINVAL;
  if (first > s->n_features || count > s->n_features - first) return CASHASH_EINVAL;
  if ((reinterpret_cast<uintptr_t>(approx) & 3) || (reinterpret_cast<uintptr_t>(bound) & 3)) return CASHASH_EINVAL;
  if (count == 0) return CASHASH_OK;
  CK(cudaSetDevice(c->device));
  // the projection kernels' other outputs go to scratch, so the set is not touched
  uint32_t *codes = nullptr, *sqn = nullptr, *fm = nullptr, *fl = nullptr;
  uint8_t* bk = nullptr;
  unsigned long long* cnt = nullptr;
  uint64_t c1 = 0, c2 = 0, c3 = 0, c4 = 0, c5 = 0, c6 = 0;
  int st = grow(codes, c1, 4 * count);
  if (st == CASHASH_OK) st = grow(bk, c2, 8 * count);
  if (st == CASHASH_OK) st = grow(sqn, c3, count);
  if (st == CASHASH_OK) st = grow(fm, c4, 6 * count);
  if (st == CASHASH_OK) st = grow(fl, c5, count);
  if (st == CASHASH_OK) st = grow(cnt, c6, 2);
  if (st == CASHASH_OK) st = cuda_err(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), stream));
  const uint8_t* d = s->desc + first * DIM;
  if (st == CASHASH_OK) {
    if (c->p.precision == CASHASH_BF16)
      st = cuda_err(launch_project_bf16(d, count, c->d_Rbf, c->np_tc, c->d_rc, c->kp, codes, bk, sqn, fm, fl, cnt,
                                        c->d_status, stream, approx, bound));
    else
      st = cuda_err(launch_project_fp32(d, count, c->d_R32T, c->d_rc, c->kp, codes, bk, sqn, fm, fl, cnt, stream,
                                        approx, bound));
  }
  if (st == CASHASH_OK) st = cuda_err(cudaStreamSynchronize(stream));
  dfree(codes);
  dfree(bk);
  dfree(sqn);
  dfree(fm);
  dfree(fl);
  dfree(cnt);
  return st;
}

int cashash_get_mean(cashash_ctx* c, double* mean_out) {
  if (!c || !mean_out) return CASHASH_EINVAL;
  CK(cudaSetDevice(c->device));
  CK(cudaStreamSynchronize(c->last_stream));
  CK(cudaMemcpy(mean_out, c->d_mu, DIM * sizeof(double), cudaMemcpyDeviceToHost));
  return CASHASH_OK;
}

void cashash_plan_destroy(cashash_plan* pl) {
  if (!pl) return;
  cudaDeviceSynchronize();
  dfree(pl->d_pairs);
  dfree(pl->d_items);
  dfree(pl->d_res);
  dfree(pl->d_pair_cnt);
  dfree(pl->d_item_ctr);
  dfree(pl->d_queue);
  dfree(pl->d_tau);
  dfree(pl->d_jhist);
  dfree(pl->d_jline);
  dfree(pl->d_F2);
  if (pl->gexec) cudaGraphExecDestroy(pl->gexec);
  if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
  delete pl;
}

namespace {

// Work items, grid and scratch of a plan for configuration t (persistent
// schedule), or for the per-pair schedule.  Drops the captured graph.
int plan_configure(cashash_plan* pl, cashash_tuning t) {
  cashash_ctx* c = pl->ctx;
  const uint32_t P = pl->P;
  const std::vector<PairInfo>& info = pl->info;
  const bool epi = c->p.epi_px >= 0.0;
  if (pl->gexec) {
    cudaGraphExecDestroy(pl->gexec);
    pl->gexec = nullptr;
  }
  std::vector<uint2> items;
  bool join = false;
  uint32_t grid = 0;
  if (!pl->persistent) {
    const uint32_t tile = (uint32_t)match_tile_size(c->p.top_k, 0);
    for (uint32_t i = 0; i < P; ++i) {
      pl->first[i] = (uint32_t)items.size();
      for (uint32_t q0 = 0; q0 < info[i].nA; q0 += tile) items.push_back(make_uint2(i, q0));
      pl->count[i] = (uint32_t)items.size() - pl->first[i];
    }
    pl->occ_grid = match_grid(c->p.top_k, 0, epi, c->p.n_tables, 0xFFFFFFFFu);
    t = cashash_tuning{};
  } else if (t.kernel == CASHASH_KERNEL_JOIN || t.kernel == CASHASH_KERNEL_JOIN_TC) {
    if (t.kernel == CASHASH_KERNEL_JOIN) {
      t.tile = (t.tile <= 2 && !epi) ? 2u : 4u;  // the band form has 4 candidate tiles only
      grid = join_grid(c->kp, pl->na_max, P, t.tile, t.ctas_per_sm);
    } else {
      t.tile = 0;
      t.ctas_per_sm = t.ctas_per_sm > 2 ? 0u : t.ctas_per_sm;
      grid = join_tc_grid(c->kp, pl->na_max, P, t.ctas_per_sm);
    }
    if (P && !grid) return CASHASH_ENOTSUP;
    join = true;
    // One item per pair.  The resident CTAs take consecutive items, so the
    // pairs are grouped by candidate image: the pairs in flight then share
    // their candidate images, whose descriptors and tables stay in L2 (on an
    // all-pairs set as fast as tiles of images, on a sparse neighbour graph
    // clearly faster).  Within a group the largest (N_A * N_B) pairs come first.
    std::vector<uint32_t> order(P);
    for (uint32_t i = 0; i < P; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
      const uint32_t bx = pl->pairs_h[2 * (size_t)x + 1], by = pl->pairs_h[2 * (size_t)y + 1];
      if (bx != by) return bx < by;
      return (uint64_t)info[x].nA * info[x].nB > (uint64_t)info[y].nA * info[y].nB;
    });
    for (uint32_t i : order) items.push_back(make_uint2(i, 0u));
  } else if (t.kernel == CASHASH_KERNEL_QUERY) {
    t.tile = (uint32_t)match_tile_size(c->p.top_k, 1, t.tile);
    t.ctas_per_sm = 0;
    // tiles of queries, grouped by candidate image so that a candidate
    // image's chunks are reused from L2 by consecutive items
    std::vector<uint32_t> order(P);
    for (uint32_t i = 0; i < P; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
      return pl->pairs_h[2 * (size_t)x + 1] < pl->pairs_h[2 * (size_t)y + 1];
    });
    for (uint32_t i : order)
      for (uint32_t q0 = 0; q0 < info[i].nA; q0 += t.tile) items.push_back(make_uint2(i, q0));
    grid = match_grid(c->p.top_k, 1, epi, c->p.n_tables, (uint32_t)items.size(), t.tile);
  } else if (t.kernel == CASHASH_KERNEL_WARP) {
    t.tile = 0;  // no work items: the exact warp-per-query kernel walks the result array
    t.ctas_per_sm = 0;
  } else {
    return CASHASH_EINVAL;
  }
  int st = grow(pl->d_items, pl->cap_items, std::max<uint64_t>(items.size(), 1));
  if (st == CASHASH_OK && pl->persistent) {
    const uint64_t q = join ? (uint64_t)grid * pl->na_max * JSEG : (uint64_t)grid * t.tile * QCAP;
    st = grow(pl->d_queue, pl->cap_queue, std::max<uint64_t>(q, 1));
  }
  if (st == CASHASH_OK && join && epi)
    st = grow(pl->d_jline, pl->cap_jline, std::max<uint64_t>((uint64_t)grid * jline_stride(pl->na_max), 1));
  if (st == CASHASH_OK && join && !pl->d_jhist) {
    uint64_t cap = 0;
    st = grow(pl->d_jhist, cap, std::max<uint64_t>((uint64_t)P * HBINS, 1));
    if (st == CASHASH_OK)
      st = cuda_err(cudaMemset(pl->d_jhist, 0, sizeof(uint32_t) * std::max<uint64_t>((uint64_t)P * HBINS, 1)));
  }
  if (st == CASHASH_OK && !items.empty())
    st = cuda_err(cudaMemcpy(pl->d_items, items.data(), sizeof(uint2) * items.size(), cudaMemcpyHostToDevice));
  if (st != CASHASH_OK) return st;
  pl->n_items = (uint32_t)items.size();
  pl->join = join;
  pl->grid = grid;
  t.ms_sample = -1.0;
  t.reserved = 0;
  pl->tune = t;
  return CASHASH_OK;
}

}  // namespace

int cashash_plan_create(cashash_ctx* c, const cashash_set* s, const uint32_t* pairs_host, uint32_t P,
                        cashash_plan** out) {
  if (!c || !out || !set_ok(s, nullptr) || (P > 0 && !pairs_host)) return CASHASH_EINVAL;
  *out = nullptr;
  if (c->p.epi_px >= 0.0 && s->n_features > 0 && !s->kpts) return CASHASH_EINVAL;
  for (uint32_t i = 0; i < P; ++i)
    if (pairs_host[2 * (size_t)i] >= s->n_images || pairs_host[2 * (size_t)i + 1] >= s->n_images)
      return CASHASH_EINVAL;
  CK(cudaSetDevice(c->device));
  cashash_plan* pl = new (std::nothrow) cashash_plan();
  if (!pl) return CASHASH_ENOMEM;
  // mutual check: pairs P..2P-1 are the reversals of the user's pairs
  const uint32_t P_out = P;
  std::vector<uint32_t> pairs_int;
  if (c->p.flags & CASHASH_FLAG_MUTUAL) {
    if ((uint64_t)P * 2 > 0xFFFFFFFFull) {
      delete pl;
      return CASHASH_EINVAL;
    }
    pairs_int.assign(pairs_host, pairs_host + 2 * (size_t)P);
    for (uint32_t i = 0; i < P; ++i) {
      pairs_int.push_back(pairs_host[2 * (size_t)i + 1]);
      pairs_int.push_back(pairs_host[2 * (size_t)i]);
    }
    P = 2 * P;
    pairs_host = pairs_int.data();
  }
  pl->ctx = c;
  pl->P = P;
  pl->P_out = P_out;
  pl->persistent = c->p.schedule == CASHASH_SCHED_PERSISTENT;
  pl->desc = s->desc;
  pl->codes = s->codes;
  pl->buckets = s->buckets;
  pl->sqnorm = s->sqnorm;
  pl->tables = s->tables;
  pl->kpts = s->kpts;
  std::vector<uint64_t> f0;
  std::vector<uint32_t> len, firstc;
  chunk_layout(s->img_off, s->n_images, f0, len, &firstc);
  std::vector<PairInfo> info(P);
  std::vector<uint64_t> jbase;
  join_layout(s->img_off, s->n_images, c->p.n_tables, jbase);
  uint64_t qbase = 0;
  for (uint32_t i = 0; i < P; ++i) {
    const uint32_t a = pairs_host[2 * (size_t)i], b = pairs_host[2 * (size_t)i + 1];
    PairInfo& pi = info[i];
    pi.a0 = s->img_off[a];
    pi.b0 = s->img_off[b];
    pi.nA = (uint32_t)(s->img_off[a + 1] - s->img_off[a]);
    pi.nB = (uint32_t)(s->img_off[b + 1] - s->img_off[b]);
    pi.bchunk0 = firstc[b];
    pi.pad = 0;
    pi.ajoin = jbase[a];
    pi.bjoin = jbase[b];
    pi.qbase = qbase;
    qbase += pi.nA;
  }
  pl->n_res = qbase;
  uint32_t na_max = 0;
  for (uint32_t i = 0; i < P; ++i) na_max = std::max(na_max, info[i].nA);
  pl->na_max = std::max<uint32_t>(na_max, 1);
  pl->info = info;
  pl->pairs_h.assign(pairs_host, pairs_host + 2 * (size_t)P);
  pl->img_off_h.assign(s->img_off, s->img_off + (size_t)s->n_images + 1);
  pl->set = *s;
  pl->set.img_off = pl->img_off_h.data();
  pl->first.assign(P, 0);
  pl->count.assign(P, 0);
  uint64_t cap = 0;
  int st = grow(pl->d_pairs, cap, std::max<uint64_t>(P, 1));
  cap = 0;
  if (st == CASHASH_OK) st = grow(pl->d_res, cap, std::max<uint64_t>(qbase, 1));
  if (st == CASHASH_OK && P != P_out && c->p.epi_px >= 0.0)
    st = grow(pl->d_F2, pl->cap_F2, std::max<uint64_t>(9ull * P, 1));
  cap = 0;
  if (st == CASHASH_OK) st = grow(pl->d_pair_cnt, cap, std::max<uint64_t>(P, 1));
  cap = 0;
  if (st == CASHASH_OK) st = grow(pl->d_item_ctr, cap, (uint64_t)P + 1);
  cap = 0;
  if (st == CASHASH_OK) st = grow(pl->d_tau, cap, std::max<uint64_t>(P, 1));
  if (st == CASHASH_OK) st = cuda_err(cudaMemset(pl->d_tau, 0, sizeof(uint32_t) * std::max<uint64_t>(P, 1)));
  if (st == CASHASH_OK && P)
    st = cuda_err(cudaMemcpy(pl->d_pairs, info.data(), sizeof(PairInfo) * P, cudaMemcpyHostToDevice));
  if (st == CASHASH_OK) {
    if (pl->persistent) {
      cashash_tuning t{};  // the join when it applies, else the per-query kernel
      t.kernel = CASHASH_KERNEL_JOIN;
      t.tile = 4;
      st = plan_configure(pl, t);
      if (st == CASHASH_ENOTSUP) {
        t.kernel = CASHASH_KERNEL_QUERY;
        t.tile = 0;
        st = plan_configure(pl, t);
      }
    } else {
      st = plan_configure(pl, cashash_tuning{});
    }
  }
  if (st != CASHASH_OK) {
    cashash_plan_destroy(pl);
    return st;
  }
  *out = pl;
  return CASHASH_OK;
}

namespace {

// Enqueues the matching sequence of a plan on `stream`: counter resets, the
// matching kernel(s), the exact fallback (persistent form), offsets and
// compaction.  `capturing` marks a graph capture (events become external nodes).
int enqueue_match(cashash_ctx* c, cashash_plan* pl, const double* F_dev, uint64_t* match_off, uint32_t* matches,
                  uint64_t cap, cudaStream_t stream, bool capturing) {
  const uint32_t P = pl->P;
  const bool mutual = pl->P_out != pl->P;
  if (P) CK(cudaMemsetAsync(pl->d_pair_cnt, 0, sizeof(unsigned long long) * P, stream));
  if (mutual && c->p.epi_px >= 0.0 && F_dev) {  // F of the reverse pairs: transposed
    CK(launch_mutual_F(F_dev, pl->P_out, pl->d_F2, stream));
    F_dev = pl->d_F2;
  }
  MatchArgs a{};
  a.desc = pl->desc;
  a.codes = pl->codes;
  a.buckets = pl->buckets;
  a.sqnorm = pl->sqnorm;
  a.tables = pl->tables;
  a.kpts = pl->kpts;
  a.F = c->p.epi_px >= 0.0 ? F_dev : nullptr;
  a.pairs = pl->d_pairs;
  a.n_pairs = P;
  a.res = pl->d_res;
  a.n_res = pl->n_res;
  a.pair_cnt = pl->d_pair_cnt;
  a.status = c->d_status;
  a.queue = pl->d_queue;
  a.tau_pair = pl->d_tau;
  a.tau_fixed = pl->tau_fixed;
  const bool warp_only = pl->persistent && pl->tune.kernel == CASHASH_KERNEL_WARP;
  a.all_queries = warp_only ? 1u : 0u;
  a.join = pl->tables;
  a.jqueue = pl->d_queue;
  a.jhist = pl->d_jhist;
  a.jline = pl->d_jline;
  a.na_max = pl->na_max;
  a.kp = c->kp;
  CK(cudaMemsetAsync(pl->d_item_ctr, 0, sizeof(unsigned int) * ((size_t)P + 1), stream));
  if (pl->persistent) {
    a.items = pl->d_items;
    a.n_items = pl->n_items;
    a.item_ctr = pl->d_item_ctr + P;
    if (c->p.epi_px < 0.0 && !warp_only) {  // threshold guesses for pairs without one (either kernel)
      StageTimer tm(c, CASHASH_STAGE_CALIBRATE, stream, capturing);
      CK(launch_join_calibrate(a, stream));
    }
    if (!warp_only) {
      StageTimer tm(c, CASHASH_STAGE_MATCH, stream, capturing);
      if (pl->join && pl->tune.kernel == CASHASH_KERNEL_JOIN_TC) CK(launch_join_tc(a, pl->grid, stream));
      else if (pl->join) CK(launch_join(a, pl->grid, pl->tune.tile, stream));
      else CK(launch_match(a, 1, pl->grid, stream, pl->tune.tile));
    }
    {
      StageTimer tm(c, CASHASH_STAGE_FALLBACK, stream, capturing);
      CK(launch_match_fallback(a, stream));
    }
  } else {
    StageTimer tm(c, CASHASH_STAGE_MATCH, stream, capturing);
    for (uint32_t i = 0; i < P; ++i) {
      if (!pl->count[i]) continue;
      a.items = pl->d_items + pl->first[i];
      a.n_items = pl->count[i];
      a.item_ctr = pl->d_item_ctr + i;
      CK(launch_match(a, 0, std::min(pl->count[i], pl->occ_grid), stream));
    }
  }
  {
    StageTimer tm(c, CASHASH_STAGE_COMPACT, stream, capturing);
    if (mutual) CK(launch_mutual(pl->d_pairs, pl->P_out, pl->d_res, pl->d_pair_cnt, stream));
    CK(launch_scan_counts(pl->d_pair_cnt, pl->P_out, match_off, cap, c->d_status, c->d_cnt + 2, stream));
    CK(launch_compact(pl->d_pairs, pl->P_out, pl->d_res, match_off, matches, cap, stream));
  }
  return CASHASH_OK;
}

uint64_t match_launches(const cashash_plan* pl) {
  uint64_t n = pl->P ? 2 : 1;  // scan + compaction
  if (pl->P_out != pl->P) n += 1 + (pl->ctx->p.epi_px >= 0.0 ? 1 : 0);  // mutual filter (+ transposed F)
  if (pl->persistent) {
    // calibration (not with the band), the join or the speculative kernel, then the fallback
    const bool cal = pl->ctx->p.epi_px < 0.0 && pl->P;
    n += (pl->grid ? (cal ? 2 : 1) : 0) + (pl->n_res ? 1 : 0);
  } else {
    for (uint32_t i = 0; i < pl->P; ++i) n += pl->count[i] ? 1 : 0;
  }
  return n;
}

}  // namespace

int cashash_match_plan(cashash_ctx* c, cashash_plan* pl, const double* F_dev, uint64_t* match_off,
                       uint32_t* matches, uint64_t cap, cashash_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (!c || !pl || pl->ctx != c || !match_off || (cap > 0 && !matches)) return CASHASH_EINVAL;
  if (c->p.epi_px >= 0.0 && pl->P > 0 && !F_dev) return CASHASH_EINVAL;
  if ((reinterpret_cast<uintptr_t>(match_off) & 7) || (reinterpret_cast<uintptr_t>(matches) & 3)) return CASHASH_EINVAL;
  CK(cudaSetDevice(c->device));
  c->ev_used[CASHASH_STAGE_MATCH] = c->ev_used[CASHASH_STAGE_COMPACT] = 0;
  c->ev_used[CASHASH_STAGE_CALIBRATE] = c->ev_used[CASHASH_STAGE_FALLBACK] = 0;
  if (pl->persistent) {
    const bool same = pl->gexec && pl->g_F == F_dev && pl->g_moff == match_off && pl->g_mt == matches &&
                      pl->g_cap == cap && pl->g_prof == c->profiling;
    if (!same) {
      if (pl->gexec) cudaGraphExecDestroy(pl->gexec);
      pl->gexec = nullptr;
      if (!pl->cap_stream) CK(cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking));
      CK(cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeThreadLocal));
      const int st = enqueue_match(c, pl, F_dev, match_off, matches, cap, pl->cap_stream, true);
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(pl->cap_stream, &g);
      if (st != CASHASH_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      CK(e);
      const cudaError_t ei = cudaGraphInstantiate(&pl->gexec, g, 0);
      cudaGraphDestroy(g);
      CK(ei);
      pl->g_F = F_dev;
      pl->g_moff = match_off;
      pl->g_mt = matches;
      pl->g_cap = cap;
      pl->g_prof = c->profiling;
    }
    CK(cudaGraphLaunch(pl->gexec, stream));
    if (c->profiling) {  // the graph holds the stage events as external event-record nodes
      const bool warp_only = pl->tune.kernel == CASHASH_KERNEL_WARP;  // the fallback kernel alone
      c->ev_used[CASHASH_STAGE_COMPACT] = c->ev_used[CASHASH_STAGE_FALLBACK] = 1;
      if (!warp_only) c->ev_used[CASHASH_STAGE_MATCH] = 1;
      if (c->p.epi_px < 0.0 && !warp_only) c->ev_used[CASHASH_STAGE_CALIBRATE] = 1;
    }
  } else {
    const int st = enqueue_match(c, pl, F_dev, match_off, matches, cap, stream, false);
    if (st != CASHASH_OK) return st;
  }
  c->n_launches += match_launches(pl);
  c->last_stream = stream;
  c->last_pairs = pl->P;
  c->last_items = pl->n_items;
  return CASHASH_OK;
}

int cashash_plan_set_threshold_hint(cashash_plan* pl, uint32_t hamming, int fixed) {
  if (!pl || !pl->ctx || !pl->d_tau) return CASHASH_EINVAL;
  CK(cudaSetDevice(pl->ctx->device));
  const uint32_t v = hamming >= pl->ctx->p.code_bits ? 0u : hamming + 1u;
  std::vector<uint32_t> h(std::max<uint32_t>(pl->P, 1), v);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(pl->d_tau, h.data(), sizeof(uint32_t) * h.size(), cudaMemcpyHostToDevice));
  if (pl->d_jhist) CK(cudaMemset(pl->d_jhist, 0, sizeof(uint32_t) * (size_t)std::max<uint32_t>(pl->P, 1) * HBINS));
  pl->tau_fixed = fixed ? 1u : 0u;
  return CASHASH_OK;
}

int cashash_plan_get_tuning(const cashash_plan* pl, cashash_tuning* out) {
  if (!pl || !out) return CASHASH_EINVAL;
  *out = pl->tune;
  return CASHASH_OK;
}

int cashash_plan_set_tuning(cashash_plan* pl, const cashash_tuning* t) {
  if (!pl || !t || !pl->ctx || !pl->persistent) return CASHASH_EINVAL;
  CK(cudaSetDevice(pl->ctx->device));
  CK(cudaDeviceSynchronize());
  const cashash_tuning keep = pl->tune;
  const int st = plan_configure(pl, *t);
  if (st != CASHASH_OK && plan_configure(pl, keep) != CASHASH_OK) return CASHASH_ECUDA;
  return st;
}

int cashash_plan_autotune(cashash_ctx* c, cashash_plan* pl, const double* F_dev, uint32_t max_pairs,
                          cashash_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (!c || !pl || pl->ctx != c) return CASHASH_EINVAL;
  if (c->p.epi_px >= 0.0 && pl->P > 0 && !F_dev) return CASHASH_EINVAL;
  if (!pl->persistent || pl->P == 0) return CASHASH_OK;
  CK(cudaSetDevice(c->device));
  CK(cudaStreamSynchronize(stream));
  const uint32_t P = pl->P_out;  // the user's pairs (a mutual plan matches them twice internally)
  // max_pairs == 0 (or >= P): the candidates run on the plan itself.  Else on a
  // sample spread over the plan's cost order, with enough pairs per SM that the
  // persistent kernels' tails weigh as in the full run (a join item is a pair).
  const bool whole = max_pairs == 0 || max_pairs >= P;
  int nsm = 0;
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
  const uint32_t S = whole ? P : std::min<uint32_t>(P, std::max<uint32_t>(max_pairs, 16u * (uint32_t)nsm));
  std::vector<uint32_t> pick;
  uint64_t cap = 0;
  cashash_plan* sp = pl;
  int st = CASHASH_OK;
  if (!whole) {
    std::vector<uint32_t> order(P);
    for (uint32_t i = 0; i < P; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
      return (uint64_t)pl->info[x].nA * pl->info[x].nB > (uint64_t)pl->info[y].nA * pl->info[y].nB;
    });
    pick.resize(S);
    std::vector<uint32_t> sub(2 * (size_t)S);
    for (uint32_t i = 0; i < S; ++i) {
      pick[i] = order[(uint32_t)(((uint64_t)i * P) / S)];
      sub[2 * (size_t)i] = pl->pairs_h[2 * (size_t)pick[i]];
      sub[2 * (size_t)i + 1] = pl->pairs_h[2 * (size_t)pick[i] + 1];
      cap += pl->info[pick[i]].nA;
    }
    sp = nullptr;
    st = cashash_plan_create(c, &pl->set, sub.data(), S, &sp);
    if (st != CASHASH_OK) return st;
  } else {
    cap = pl->n_res;
  }
  double* dF = nullptr;
  uint64_t* dmo = nullptr;
  uint32_t* dmt = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  uint64_t c1 = 0, c2 = 0, c3 = 0;
  st = grow(dmo, c1, (uint64_t)S + 1);
  if (st == CASHASH_OK) st = grow(dmt, c2, 2 * std::max<uint64_t>(cap, 1));
  const double* Fs = whole ? F_dev : nullptr;
  if (!whole && st == CASHASH_OK && F_dev && c->p.epi_px >= 0.0) {
    st = grow(dF, c3, 9 * (uint64_t)S);
    for (uint32_t i = 0; st == CASHASH_OK && i < S; ++i)
      st = cuda_err(cudaMemcpyAsync(dF + 9 * (size_t)i, F_dev + 9 * (size_t)pick[i], 9 * sizeof(double),
                                    cudaMemcpyDeviceToDevice, stream));
    Fs = dF;
  }
  if (st == CASHASH_OK) st = cuda_err(cudaEventCreate(&e0));
  if (st == CASHASH_OK) st = cuda_err(cudaEventCreate(&e1));
  const int prof = c->profiling;
  c->profiling = 0;
  std::vector<cashash_tuning> cand;
  for (uint32_t ctas : {0u, 1u})
    for (uint32_t tile : {4u, 2u}) {
      cashash_tuning t{};
      t.kernel = CASHASH_KERNEL_JOIN;
      t.tile = tile;
      t.ctas_per_sm = ctas;
      cand.push_back(t);
    }
  for (uint32_t ctas : {0u, 1u}) {
    cashash_tuning t{};
    t.kernel = CASHASH_KERNEL_JOIN_TC;
    t.ctas_per_sm = ctas;
    cand.push_back(t);
  }
  for (uint32_t tile : {512u, 256u}) {
    cashash_tuning t{};
    t.kernel = CASHASH_KERNEL_QUERY;
    t.tile = tile;
    cand.push_back(t);
  }
  {
    cashash_tuning t{};
    t.kernel = CASHASH_KERNEL_WARP;
    cand.push_back(t);
  }
  // Two interleaved rounds (so that clock and cache drift hit every candidate),
  // each candidate's time the minimum of its rounds; a candidate more than 25 %
  // behind the best after the first round is not timed again.  The first
  // applicable candidate is the plan's default; another replaces it only when
  // it is more than 3 % faster.
  const size_t nc = cand.size();
  std::vector<double> tbest(nc, -1.0);
  std::vector<cashash_tuning> tnorm(nc);
  for (int round = 0; round < 2 && st == CASHASH_OK; ++round) {
    double lead = -1.0;
    for (size_t ci = 0; ci < nc && round == 1; ++ci)
      if (tbest[ci] >= 0.0 && (lead < 0.0 || tbest[ci] < lead)) lead = tbest[ci];
    for (size_t ci = 0; ci < nc; ++ci) {
      if (st != CASHASH_OK) break;
      if (round == 1 && (tbest[ci] < 0.0 || tbest[ci] > 1.25 * lead)) continue;
      const cashash_tuning& t0 = cand[ci];
      const int cs = plan_configure(sp, t0);
      if (cs == CASHASH_ENOTSUP) continue;
      if (cs != CASHASH_OK) {
        st = cs;
        break;
      }
      if (t0.kernel == CASHASH_KERNEL_QUERY && sp->tune.tile != t0.tile) continue;  // normalised to another one
      // fresh thresholds: two untimed runs calibrate them, three timed runs follow
      st = cuda_err(cudaMemsetAsync(sp->d_tau, 0, sizeof(uint32_t) * sp->P, stream));
      if (st == CASHASH_OK && sp->d_jhist)
        st = cuda_err(cudaMemsetAsync(sp->d_jhist, 0, sizeof(uint32_t) * (size_t)sp->P * HBINS, stream));
      float ms = 0.f;
      for (int r = 0; r < 5 && st == CASHASH_OK; ++r) {
        if (r == 2) st = cuda_err(cudaEventRecord(e0, stream));
        if (st == CASHASH_OK) st = enqueue_match(c, sp, Fs, dmo, dmt, cap, stream, false);
      }
      if (st == CASHASH_OK) st = cuda_err(cudaEventRecord(e1, stream));
      if (st == CASHASH_OK) st = cuda_err(cudaEventSynchronize(e1));
      if (st == CASHASH_OK) st = cuda_err(cudaEventElapsedTime(&ms, e0, e1));
      if (st != CASHASH_OK) break;
      const double t_ms = ms / 3.0;
      tnorm[ci] = sp->tune;
      if (tbest[ci] < 0.0 || t_ms < tbest[ci]) tbest[ci] = t_ms;
    }
  }
  cashash_tuning best{};
  double best_ms = -1.0, def_ms = -1.0;
  for (size_t ci = 0; ci < nc; ++ci) {
    if (tbest[ci] < 0.0) continue;
    if (def_ms < 0.0) {
      def_ms = best_ms = tbest[ci];
      best = tnorm[ci];
    } else if (tbest[ci] < 0.97 * def_ms && tbest[ci] < best_ms) {
      best_ms = tbest[ci];
      best = tnorm[ci];
    }
  }
  c->profiling = prof;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  dfree(dF);
  dfree(dmo);
  dfree(dmt);
  if (!whole) cashash_plan_destroy(sp);
  if (st != CASHASH_OK) return st;
  if (best_ms < 0.0) return CASHASH_OK;
  st = plan_configure(pl, best);
  if (st == CASHASH_OK) pl->tune.ms_sample = best_ms;
  if (st == CASHASH_OK && whole) {  // thresholds are learned afresh by the chosen kernel
    st = cuda_err(cudaMemset(pl->d_tau, 0, sizeof(uint32_t) * pl->P));
    if (st == CASHASH_OK && pl->d_jhist)
      st = cuda_err(cudaMemset(pl->d_jhist, 0, sizeof(uint32_t) * (size_t)pl->P * HBINS));
  }
  return st;
}

int cashash_match_pairs(cashash_ctx* c, const cashash_set* s, const uint32_t* pairs_host, uint32_t P,
                        const double* F_dev, uint64_t* match_off, uint32_t* matches, uint64_t cap,
                        cashash_stream_t stream) {
  cashash_plan* pl = nullptr;
  int st = cashash_plan_create(c, s, pairs_host, P, &pl);
  if (st != CASHASH_OK) return st;
  st = cashash_match_plan(c, pl, F_dev, match_off, matches, cap, stream);
  if (st == CASHASH_OK) st = cuda_err(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
  cashash_plan_destroy(pl);
  return st;
}

int cashash_sync_status(cashash_ctx* c, cashash_stream_t stream) {
  if (!c) return CASHASH_EINVAL;
  CK(cudaSetDevice(c->device));
  CK(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
  uint32_t s = 0;
  CK(cudaMemcpy(&s, c->d_status, sizeof s, cudaMemcpyDeviceToHost));
  CK(cudaMemset(c->d_status, 0, sizeof(uint32_t)));
  if (s & DST_INDEX) return CASHASH_EDEVICE;
  if (s & DST_OVERFLOW) return CASHASH_EOVERFLOW;
  return CASHASH_OK;
}

int cashash_set_profiling(cashash_ctx* c, int on) {
  if (!c) return CASHASH_EINVAL;
  CK(cudaSetDevice(c->device));
  if (on && !c->ev[0][0]) {
    for (int i = 0; i < CASHASH_N_STAGES; ++i)
      for (int k = 0; k < 2; ++k) CK(cudaEventCreate(&c->ev[i][k]));
  }
  c->profiling = on ? 1 : 0;
  return CASHASH_OK;
}

int cashash_get_stats(cashash_ctx* c, cashash_stats* out) {
  if (!c || !out) return CASHASH_EINVAL;
  CK(cudaSetDevice(c->device));
  CK(cudaStreamSynchronize(c->last_stream));
  unsigned long long h[8];
  CK(cudaMemcpy(h, c->d_cnt, sizeof h, cudaMemcpyDeviceToHost));
  out->n_features = c->last_n_features;
  out->n_reevaluated = h[1];
  out->n_pairs = c->last_pairs;
  out->n_matches = h[2];
  out->n_work_items = c->last_items;
  out->n_launches = c->n_launches;
  for (int i = 0; i < CASHASH_N_STAGES; ++i) {
    out->ms_stage[i] = -1.0;
    if (c->ev_used[i] && c->ev[i][0]) {
      float ms = 0.f;
      CK(cudaEventSynchronize(c->ev[i][1]));
      CK(cudaEventElapsedTime(&ms, c->ev[i][0], c->ev[i][1]));
      out->ms_stage[i] = ms;
    }
  }
  return CASHASH_OK;
}

int cashash_set_host_tuning(cashash_ctx* c, const cashash_tuning* t) {
  if (!c) return CASHASH_EINVAL;
  if (t && t->kernel != CASHASH_KERNEL_JOIN && t->kernel != CASHASH_KERNEL_JOIN_TC &&
      t->kernel != CASHASH_KERNEL_QUERY && t->kernel != CASHASH_KERNEL_WARP)
    return CASHASH_EINVAL;
  HostWS& h = c->hw;
  h.has_tune = t != nullptr;
  if (t) h.tune = *t;
  if (h.plan) {  // the next call builds its plan with the new configuration
    cashash_plan_destroy(h.plan);
    h.plan = nullptr;
    h.plan_pairs.clear();
    h.plan_off.clear();
  }
  return CASHASH_OK;
}

int cashash_get_host_tuning(const cashash_ctx* c, cashash_tuning* out) {
  if (!c || !out) return CASHASH_EINVAL;
  if (c->hw.has_tune) {
    *out = c->hw.tune;
  } else {
    *out = cashash_tuning{};
    out->ms_sample = -1.0;
  }
  return CASHASH_OK;
}

int cashash_run_host(cashash_ctx* c, const uint8_t* desc_host, const uint64_t* img_off, uint32_t n_images,
                     const float* kpts_host, const uint32_t* pairs_host, uint32_t P, const double* F_host,
                     uint64_t* match_off_host, uint32_t* matches_host, uint64_t cap, uint64_t stage_bytes) {
  if (!c || (n_images > 0 && !img_off) || !match_off_host || (cap > 0 && !matches_host)) return CASHASH_EINVAL;
  const uint64_t N = n_images ? img_off[n_images] : 0;
  if (N > 0 && !desc_host) return CASHASH_EINVAL;
  const bool epi = c->p.epi_px >= 0.0;
  if (epi && ((N > 0 && !kpts_host) || (P > 0 && !F_host))) return CASHASH_EINVAL;
  if (stage_bytes == 0) stage_bytes = 4ull << 30;
  stage_bytes = std::max<uint64_t>(stage_bytes & ~(uint64_t)15, 1u << 20);
  CK(cudaSetDevice(c->device));
  HostWS& h = c->hw;
  if (!h.copy) {
    CK(cudaStreamCreateWithFlags(&h.copy, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&h.comp, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h.ev[0], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h.ev[1], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h.staged, cudaEventDisableTiming));
  }
  int st = CASHASH_OK;
  cashash_params pp = c->p;
  const uint64_t tb = cashash_tables_bytes(&pp, img_off, n_images);
  if ((st = grow(h.desc, h.cap_desc, std::max<uint64_t>(N, 1) * DIM)) != CASHASH_OK) return st;
  if ((st = grow(h.codes, h.cap_codes, std::max<uint64_t>(N, 1) * 4)) != CASHASH_OK) return st;
  if ((st = grow(h.buckets, h.cap_buckets, std::max<uint64_t>(N, 1) * 8)) != CASHASH_OK) return st;
  if ((st = grow(h.sqnorm, h.cap_sq, std::max<uint64_t>(N, 1))) != CASHASH_OK) return st;
  if ((st = grow(h.tables, h.cap_tables, tb)) != CASHASH_OK) return st;
  if ((st = grow(h.moff, h.cap_moff, (uint64_t)P + 1)) != CASHASH_OK) return st;
  if (epi) {
    if ((st = grow(h.kpts, h.cap_kpts, std::max<uint64_t>(N, 1) * 2)) != CASHASH_OK) return st;
    if ((st = grow(h.F, h.cap_F, std::max<uint64_t>(P, 1) * 9)) != CASHASH_OK) return st;
  }
  // Inputs host -> device on the copy stream: key-points and F first, then the
  // descriptors in blocks of at most 256 MiB (pinned sources directly,
  // pageable ones through two pinned bounce buffers of at most stage_bytes).
  // The compute stream takes each block's column sums as soon as it lands;
  // the projections wait for the whole set, whose mean is their centre.
  for (int i = 0; i < CASHASH_STAGE_H2D; ++i) c->ev_used[i] = 0;
  c->ev_used[CASHASH_STAGE_H2D] = c->ev_used[CASHASH_STAGE_D2H] = 0;
  const uint64_t bytes = N * DIM;
  const uint64_t blk = std::min<uint64_t>(stage_bytes, 256ull << 20) & ~(uint64_t)(DIM * 16 - 1);
  CK(cudaMemsetAsync(c->d_colsum, 0, DIM * sizeof(unsigned long long), h.comp));
  CK(cudaEventRecord(h.staged, h.comp));      // the colsum buffer is cleared before any block adds to it
  CK(cudaStreamWaitEvent(h.copy, h.staged, 0));
  {
    StageTimer tm(c, CASHASH_STAGE_H2D, h.copy);
    if (epi) {
      if (N) CK(cudaMemcpyAsync(h.kpts, kpts_host, N * 2 * sizeof(float), cudaMemcpyHostToDevice, h.copy));
      if (P) CK(cudaMemcpyAsync(h.F, F_host, (uint64_t)P * 9 * sizeof(double), cudaMemcpyHostToDevice, h.copy));
    }
    // one block landed: its column sums on the compute stream
    auto landed = [&](uint64_t o, uint64_t l) -> int {
      CK(cudaEventRecord(h.staged, h.copy));
      CK(cudaStreamWaitEvent(h.comp, h.staged, 0));
      CK(launch_colsum(h.desc + o, l / DIM, c->d_colsum, h.comp, true));
      c->n_launches += 1;
      return CASHASH_OK;
    };
    if (bytes) {
      cudaPointerAttributes attr{};
      bool pinned = false;
      if (cudaPointerGetAttributes(&attr, desc_host) == cudaSuccess)
        pinned = attr.type == cudaMemoryTypeHost;
      else
        cudaGetLastError();
      if (pinned) {
        for (uint64_t o = 0; o < bytes; o += blk) {
          const uint64_t l = std::min(blk, bytes - o);
          CK(cudaMemcpyAsync(h.desc + o, desc_host + o, l, cudaMemcpyHostToDevice, h.copy));
          if ((st = landed(o, l)) != CASHASH_OK) return st;
        }
      } else {
        const uint64_t chunk = std::min(blk, bytes);
        if (h.pin_cap < chunk) {
          for (int i = 0; i < 2; ++i) {
            if (h.pin[i]) cudaFreeHost(h.pin[i]);
            h.pin[i] = nullptr;
          }
          h.pin_cap = 0;
          for (int i = 0; i < 2; ++i)
            if (cudaHostAlloc(reinterpret_cast<void**>(&h.pin[i]), chunk, cudaHostAllocDefault) != cudaSuccess) {
              cudaGetLastError();
              return CASHASH_ENOMEM;
            }
          h.pin_cap = chunk;
        }
        uint64_t k = 0;
        for (uint64_t o = 0; o < bytes; o += chunk, ++k) {
          const int b = (int)(k & 1);
          if (k >= 2) CK(cudaEventSynchronize(h.ev[b]));
          const uint64_t l = std::min(chunk, bytes - o);
          std::memcpy(h.pin[b], desc_host + o, l);
          CK(cudaMemcpyAsync(h.desc + o, h.pin[b], l, cudaMemcpyHostToDevice, h.copy));
          CK(cudaEventRecord(h.ev[b], h.copy));
          if ((st = landed(o, l)) != CASHASH_OK) return st;
        }
      }
    }
  }
  CK(cudaEventRecord(h.staged, h.copy));  // key-points, F and every block
  CK(cudaStreamWaitEvent(h.comp, h.staged, 0));
  cashash_set S{};
  S.n_images = n_images;
  S.n_features = N;
  S.img_off = img_off;
  S.desc = h.desc;
  S.codes = h.codes;
  S.buckets = h.buckets;
  S.sqnorm = h.sqnorm;
  S.tables = h.tables;
  S.kpts = epi ? h.kpts : nullptr;
  st = build_codes_impl(c, &S, nullptr, h.comp, true);
  if (st != CASHASH_OK) return st;
  // plan: reused while the pair list and image sizes are unchanged
  const bool same = h.plan && h.plan_pairs.size() == 2 * (size_t)P && h.plan_off.size() == (size_t)n_images + 1 &&
                    (P == 0 || std::memcmp(h.plan_pairs.data(), pairs_host, 8 * (size_t)P) == 0) &&
                    std::memcmp(h.plan_off.data(), img_off, 8 * ((size_t)n_images + 1)) == 0 &&
                    h.plan->desc == h.desc && h.plan->tables == h.tables && h.plan->kpts == S.kpts;
  if (!same) {
    if (h.plan) cashash_plan_destroy(h.plan);
    h.plan = nullptr;
    st = cashash_plan_create(c, &S, pairs_host, P, &h.plan);
    if (st != CASHASH_OK) return st;
    cashash_tuning cur{};
    if (h.has_tune && cashash_plan_get_tuning(h.plan, &cur) == CASHASH_OK && cur.kernel != 0) {
      st = cashash_plan_set_tuning(h.plan, &h.tune);
      if (st == CASHASH_ENOTSUP) st = CASHASH_OK;  // the join does not apply here: keep the default
      if (st != CASHASH_OK) return st;
    }
    h.plan_pairs.assign(pairs_host, pairs_host + 2 * (size_t)P);
    h.plan_off.assign(img_off, img_off + n_images + 1);
  }
  const uint64_t mcap = std::min<uint64_t>(cap, std::max<uint64_t>(h.plan->n_res, 1));
  if ((st = grow(h.matches, h.cap_matches, std::max<uint64_t>(mcap, 1) * 2)) != CASHASH_OK) return st;
  st = cashash_match_plan(c, h.plan, epi ? h.F : nullptr, h.moff, h.matches, mcap,
                          reinterpret_cast<cashash_stream_t>(h.comp));
  if (st != CASHASH_OK) return st;
  {
    StageTimer tm(c, CASHASH_STAGE_D2H, h.comp);
    CK(cudaMemcpyAsync(match_off_host, h.moff, ((uint64_t)P + 1) * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                       h.comp));
    CK(cudaStreamSynchronize(h.comp));
    const uint64_t total = match_off_host[P];
    const uint64_t ncopy = std::min(total, mcap);
    if (ncopy)
      CK(cudaMemcpyAsync(matches_host, h.matches, ncopy * 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, h.comp));
  }
  const uint64_t total = match_off_host[P];
  st = cashash_sync_status(c, reinterpret_cast<cashash_stream_t>(h.comp));
  if (st == CASHASH_OK && total > cap) st = CASHASH_EOVERFLOW;
  return st;
}

}  // extern "C"
