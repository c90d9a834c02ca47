// api.cu -- the C ABI of libwfa_gpu.so (declared in include/wfa_gpu.h):
// argument checks, device buffers, host<->device staging, and the order of
// kernel launches for one batch of read pairs (the paper's host flow,
// Sec. I: inputs distributed to the processing units, pairs aligned
// independently, results gathered back).
#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "internal.h"
#include "launch.h"
#include "wfa_gpu.h"

namespace {

template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t cap = 0;
  // grow to at least n elements (contents are not kept)
  cudaError_t ensure(size_t n) {
    if (n <= cap && p) return cudaSuccess;
    // geometric growth: few reallocations (each cudaFree synchronises the
    // device) when batch sizes creep up
    const size_t want = std::max<size_t>(std::max(n + n / 2, 2 * cap), 64);
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p), want * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    cap = want;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

// Page-locked host staging, grown geometrically, contents not kept.
template <class T>
struct HostBuf {
  T* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t n) {
    if (n <= cap && p) return cudaSuccess;
    const size_t want = std::max<size_t>(std::max(n + n / 2, 2 * cap), 64);
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&p), want * sizeof(T), cudaHostAllocDefault);
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    cap = want;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
  }
};

int gcd(int a, int b) {
  while (b) {
    const int t = a % b;
    a = b;
    b = t;
  }
  return a;
}

bool pen_ok(const wfa_gpu_penalties& p) {
  return p.x >= 1 && p.o >= 0 && p.e >= 1 && p.x <= WFA_GPU_MAX_PENALTY && p.o <= WFA_GPU_MAX_PENALTY &&
         p.e <= WFA_GPU_MAX_PENALTY;
}

constexpr int kEvents = 6;  // start, inputs, align, general, cigar, end
constexpr int kRing = 3;    // ring slots of streamed inputs: copies run two chunks ahead
constexpr int64_t kPoolInitWords = 1 << 22;

}  // namespace

struct wfa_gpu_ctx {
  int device = 0;
  // where the CIGAR words of a host-pointer call go when set: asked for once
  // their total is known (merged server calls size their staging with it)
  wfa::CigarSink cig_sink = nullptr;
  void* cig_sink_user = nullptr;
  // ends-free alignment: free pattern begin / end, text begin / end lengths
  int32_t ends_free[4] = {0, 0, 0, 0};
  cudaStream_t own_stream = nullptr;
  // chunked host-pointer calls: output copies of one chunk overlap the next
  // chunk's work (stream and events of the context)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_chunk = nullptr, ev_copied = nullptr;
  // chunked calls with page-locked, back-to-back host sequences: chunk c's
  // bases go to ring slot c % kRing (patterns, then texts) on in_stream
  // while the chunks before compute; ev_in[s]: slot s filled, ev_free[s]:
  // its last reader done
  cudaStream_t in_stream = nullptr;
  cudaEvent_t ev_in[kRing] = {}, ev_free[kRing] = {};
  cudaStream_t stream = nullptr;
  int32_t* arena = nullptr;
  size_t arena_bytes = 0;
  int32_t* own_arena = nullptr;  // the context's own allocation (arena may be borrowed)
  size_t own_arena_bytes = 0;
  int occ_medium = 16, occ_long = 2, occ_narrow = 4;  // arena teams per SM
  int nsm = 1;
  int teams_medium = 1;  // one-warp arena teams
  int teams_long = 1;    // one-CTA arena teams of kLongTeamWide warps
  int teams_narrow = 1;  // one-CTA arena teams of kLongTeamNarrow warps
  wfa::ShortPlan plan{};
  // short-kernel variants (indices into plan.v), per penalty model (0
  // gap-affine, 1 gap-linear): candidates for sequences <= 127 bases,
  // smallest store first, chosen per batch from a sampled score
  // distribution (the largest store scores the sample); for <= 255 bases an
  // int16 variant
  int variants_small[2][3] = {{7, 4, 1}, {8, 9, 9}};
  int variant_big[2] = {1, 9};
  int variant_mid[2] = {6, 10};
  // ends-free calls, per model: <= 127 bases and <= 255 bases
  int variant_ef[2] = {11, 13};
  int variant_ef_mid[2] = {12, 14};
  // lane-per-pair variants (gap-affine, global), smallest store first: any
  // penalties, and for scaled penalties 2/4/1 the small stores with their
  // geometry compiled in (per-score code: for the large stores its size
  // costs more in instruction fetch than the constants save)
  int lane_variants[4] = {15, 16, 17, 18};
  int lane_ct_variants[4] = {19, 20, 17, 18};
  bool lane_on = true;      // WFA_GPU_LANE=0 turns them off (comparisons)
  // the lane kernel's pairs sorted by estimated score in groups (default
  // path; WFA_GPU_LANE_ORDER=0: call order), and the ordering's buffers
  bool lane_order = true;
  int lane_sort_min = 12;        // the ordering sorts for stores of scores 0-12 and up (WFA_GPU_LANE_SORT_MIN)
  int64_t pipe_chunk = 1 << 19;  // pairs per chunk of a pipelined host call (WFA_GPU_PIPE_CHUNK)
  DevBuf<uint32_t> lane_words;
  DevBuf<int2> lane_slots;
  int variant_forced = -1;  // tuning override (WFA_GPU_SHORT_VARIANT)
  int last_variant = -1;
  wfa::Ctrl* ctrl = nullptr;    // device
  wfa::Ctrl* h_ctrl = nullptr;  // pinned host mirror
  int64_t* h_total = nullptr;   // pinned host scalar
  // device addresses of h_ctrl and h_total (kernels write them)
  wfa::Ctrl* h_ctrl_dev = nullptr;
  int64_t* h_total_dev = nullptr;
  cudaEvent_t ev[kEvents] = {};
  wfa_gpu_timing last{};
  // inputs staged from host memory, and computed offsets
  DevBuf<char> pat, txt;
  DevBuf<int32_t> plen, tlen;
  DevBuf<int64_t> poff, toff;
  // outputs staged for host memory: device buffers, and page-locked host
  // staging for callers' pageable buffers
  DevBuf<int32_t> score;
  DevBuf<int8_t> status;
  DevBuf<int64_t> cig_off;
  DevBuf<uint32_t> cig;
  // page-locked staging of pageable host outputs (bytes)
  HostBuf<unsigned char> h_score, h_status, h_off, h_cig;
  // streamed inputs: the device ring and the chunks' first offsets
  DevBuf<char> ring;
  HostBuf<int64_t> h_bounds;
  // internal
  DevBuf<int32_t> nruns, defer, defer_long, overflow;
  DevBuf<int32_t> sorted, sorted_long, sort_aux;  // longest-first work lists (batched path)
  DevBuf<int64_t> run_src, scan_tmp;
  DevBuf<uint32_t> runs, pool;
  int64_t pool_words = kPoolInitWords;  // CIGAR words the arena pool holds
  // autotuner sample outputs
  DevBuf<int32_t> tune_score, tune_aux;
  DevBuf<int8_t> tune_status;
  DevBuf<int64_t> tune_src;
  int32_t* h_tune = nullptr;  // pinned [kTuneSample]
  // captured device work of repeated WFA_GPU_GRAPH calls (a few kinds of
  // call, replaced round robin)
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    uint64_t key[40] = {};
    int key_len = 0;
    int variant = -1;
    int launches = 0;  // kernels captured
  };
  static constexpr int kGraphs = 4;
  Graph graphs[kGraphs];
  int graph_next = 0;
};

void wfa::set_cigar_sink(wfa_gpu_ctx* ctx, wfa::CigarSink sink, void* user) {
  if (!ctx) return;
  ctx->cig_sink = sink;
  ctx->cig_sink_user = user;
}

namespace {

// Arena teams for the context's arena: as many as fit on the GPU at once,
// each with a slice of at least 256 KiB (one-warp teams), 4 MiB (wide
// one-CTA teams) or 8 MiB (narrow ones, which run many more pairs at once:
// smaller slices sent pairs of a few kbp to the retries); pairs that
// outgrow their slice are retried with larger ones.
void size_teams(wfa_gpu_ctx* c) {
  const long arena_b = (long)c->arena_bytes;
  c->teams_medium = (int)std::max(1L, std::min((long)c->nsm * c->occ_medium, arena_b / (256L << 10)));
  c->teams_long = (int)std::max(1L, std::min((long)c->nsm * c->occ_long, arena_b / (4L << 20)));
  c->teams_narrow = (int)std::max(1L, std::min((long)c->nsm * c->occ_narrow, arena_b / (8L << 20)));
}

}  // namespace

void wfa::set_arena(wfa_gpu_ctx* ctx, void* arena, size_t bytes) {
  if (!ctx) return;
  if (arena && bytes >= 4096) {
    ctx->arena = static_cast<int32_t*>(arena);
    ctx->arena_bytes = bytes & ~(size_t)255;
  } else {
    ctx->arena = ctx->own_arena;
    ctx->arena_bytes = ctx->own_arena_bytes;
  }
  size_teams(ctx);
}

namespace {

struct Call {
  wfa_gpu_ctx* c;
  bool timing;
  int launches = 0;
  cudaError_t err = cudaSuccess;
  void rec(int i) {
    if (timing && err == cudaSuccess) err = cudaEventRecord(c->ev[i], c->stream);
  }
  bool ok(cudaError_t e) {
    if (err == cudaSuccess) err = e;
    return err == cudaSuccess;
  }
  bool launched(cudaError_t e, int nk = 1) {
    launches += nk;
    return ok(e);
  }
};

int fail_cuda(Call& k) {
  (void)k;
  return WFA_GPU_ECUDA;
}

// The control block and the CIGAR word total to their page-locked host
// mirrors, and a control block to the device, as one-block kernels rather
// than copies: on a host-pointer call the copy engines may be busy with
// bulk copies of other streams or contexts (launch_put_ctrl says why).
bool ctrl_to_host(Call& k, cudaStream_t st) {
  return k.launched(wfa::launch_copy_small(k.c->h_ctrl_dev, k.c->ctrl, sizeof(wfa::Ctrl), st));
}
bool total_to_host(Call& k, const int64_t* src, cudaStream_t st) {
  return k.launched(wfa::launch_copy_small(k.c->h_total_dev, src, sizeof(int64_t), st));
}
bool ctrl_to_device(Call& k, wfa::Ctrl* dst, const wfa::Ctrl& v, cudaStream_t st) {
  return k.launched(wfa::launch_put_ctrl(dst, v, st));
}

int map_alloc(cudaError_t e) { return e == cudaErrorMemoryAllocation ? WFA_GPU_ENOMEM : WFA_GPU_ECUDA; }

float elapsed(wfa_gpu_ctx* c, int a, int b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, c->ev[a], c->ev[b]) != cudaSuccess) {
    cudaGetLastError();  // not a failure of the call: leave no error behind
    return 0.f;
  }
  return ms;
}

cudaError_t h2d(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (!bytes) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
}

cudaError_t d2h(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (!bytes) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st);
}

// Device address through which kernels can read the host range
// [p, p + bytes), or nullptr when that range is not page-locked, mapped
// memory of one allocation (then it is copied instead).  On a Grace-Blackwell
// node such reads travel over NVLink-C2C while the kernel runs, so page-locked
// inputs need no staging copy.
const void* mapped_range(const void* p, size_t bytes) {
  if (!p || !bytes) return nullptr;
  cudaPointerAttributes a0{}, a1{};
  if (cudaPointerGetAttributes(&a0, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a0.type != cudaMemoryTypeHost || !a0.devicePointer) return nullptr;
  const char* last = static_cast<const char*>(p) + bytes - 1;
  if (cudaPointerGetAttributes(&a1, last) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a1.type != cudaMemoryTypeHost || !a1.devicePointer) return nullptr;
  if (static_cast<const char*>(a1.devicePointer) != static_cast<const char*>(a0.devicePointer) + (bytes - 1))
    return nullptr;
  return a0.devicePointer;
}

// Lengths, offsets and sequences on the device (or mapped from page-locked
// host memory); validates them.  Returns 0 or a negative WFA_GPU_* code.
int stage_inputs(wfa_gpu_ctx* c, Call& k, int64_t n, bool dev, const char* pat, const int64_t* poff,
                 const int32_t* plen, const char* txt, const int64_t* toff, const int32_t* tlen,
                 const char** d_pat, const int64_t** d_poff, const int32_t** d_plen, const char** d_txt,
                 const int64_t** d_toff, const int32_t** d_tlen, bool* host_seqs = nullptr) {
  cudaStream_t st = c->stream;
  cudaError_t e;
  if (dev) {
    *d_plen = plen;
    *d_tlen = tlen;
  } else {
    // host lengths: one bulk copy each, also from page-locked memory (the
    // offset scans read them twice, and the kernels again: in place over
    // the link that costs several times the copy)
    if ((e = c->plen.ensure(n)) || (e = c->tlen.ensure(n))) return map_alloc(e);
    if (!k.ok(h2d(c->plen.p, plen, n * sizeof(int32_t), st)) || !k.ok(h2d(c->tlen.p, tlen, n * sizeof(int32_t), st)))
      return WFA_GPU_ECUDA;
    *d_plen = c->plen.p;
    *d_tlen = c->tlen.p;
  }
  if ((e = c->scan_tmp.ensure(wfa::scan_tmp_elems(n)))) return map_alloc(e);
  bool validated = false;
  if (!poff && !toff) {
    // back-to-back sequences: both offset scans and the checks in one pass
    if ((e = c->poff.ensure(n + 1)) || (e = c->toff.ensure(n + 1))) return map_alloc(e);
    if (!ctrl_to_device(k, c->ctrl, wfa::Ctrl{}, st) ||
        !k.launched(wfa::launch_offsets_validate(*d_plen, *d_tlen, n, c->poff.p, c->toff.p, c->scan_tmp.p, c->ctrl,
                                                 st), 3))
      return WFA_GPU_ECUDA;
    *d_poff = c->poff.p;
    *d_toff = c->toff.p;
    validated = true;
  }
  // offsets: caller's (staged if host) or the exclusive scan of the lengths
  const void* mpo = (poff && !dev) ? mapped_range(poff, n * sizeof(int64_t)) : nullptr;
  const void* mto = (toff && !dev) ? mapped_range(toff, n * sizeof(int64_t)) : nullptr;
  if (validated) {
  } else if (poff && dev) {
    *d_poff = poff;
  } else if (mpo) {
    *d_poff = static_cast<const int64_t*>(mpo);
  } else {
    if ((e = c->poff.ensure(n + 1))) return map_alloc(e);
    if (poff) {
      if (!k.ok(h2d(c->poff.p, poff, n * sizeof(int64_t), st))) return WFA_GPU_ECUDA;
    } else if (!k.launched(wfa::launch_scan(*d_plen, n, 0, c->poff.p, c->scan_tmp.p, st), 3)) {
      return WFA_GPU_ECUDA;
    }
    *d_poff = c->poff.p;
  }
  if (validated) {
  } else if (toff && dev) {
    *d_toff = toff;
  } else if (mto) {
    *d_toff = static_cast<const int64_t*>(mto);
  } else {
    if ((e = c->toff.ensure(n + 1))) return map_alloc(e);
    if (toff) {
      if (!k.ok(h2d(c->toff.p, toff, n * sizeof(int64_t), st))) return WFA_GPU_ECUDA;
    } else if (!k.launched(wfa::launch_scan(*d_tlen, n, 0, c->toff.p, c->scan_tmp.p, st), 3)) {
      return WFA_GPU_ECUDA;
    }
    *d_toff = c->toff.p;
  }
  if (!validated && (!ctrl_to_device(k, c->ctrl, wfa::Ctrl{}, st) ||
                     !k.launched(wfa::launch_validate(n, *d_poff, *d_plen, *d_toff, *d_tlen, c->ctrl, st))))
    return WFA_GPU_ECUDA;
  if (!ctrl_to_host(k, st) || !k.ok(cudaStreamSynchronize(st))) return WFA_GPU_ECUDA;
  if (c->h_ctrl->bad_input) return WFA_GPU_EINVAL;
  if (dev) {
    *d_pat = pat;
    *d_txt = txt;
  } else {
    const size_t pe = (size_t)c->h_ctrl->pat_extent, te = (size_t)c->h_ctrl->txt_extent;
    const void* mp = mapped_range(pat, pe);
    const void* mt = mapped_range(txt, te);
    if (host_seqs) *host_seqs = mp || mt;
    if (mp || pe == 0) {
      *d_pat = mp ? static_cast<const char*>(mp) : pat;
    } else {
      if ((e = c->pat.ensure(pe + 16))) return map_alloc(e);
      if (!k.ok(h2d(c->pat.p, pat, pe, st))) return WFA_GPU_ECUDA;
      *d_pat = c->pat.p;
    }
    if (mt || te == 0) {
      *d_txt = mt ? static_cast<const char*>(mt) : txt;
    } else {
      if ((e = c->txt.ensure(te + 16))) return map_alloc(e);
      if (!k.ok(h2d(c->txt.p, txt, te, st))) return WFA_GPU_ECUDA;
      *d_txt = c->txt.p;
    }
  }
  return 0;
}

int run_retries(wfa_gpu_ctx* c, Call& k, wfa::AlignArgs& a);

// Long pairs go to narrow one-CTA teams when there are more than this many.
// A narrow team has half the threads: about 1.2x the wide teams' throughput
// over many pairs, but each pair takes about 1.65x longer, and a call ends
// with its last pairs; past about four waves of wide teams the throughput
// wins.  Never when the arena gives no more narrow teams than wide ones.
int narrow_above(const wfa_gpu_ctx* c) {
  return c->teams_narrow > c->teams_long ? 4 * c->teams_long : INT32_MAX;
}

// The arena kernels over the pairs the short kernel deferred (medium pairs
// on one-warp teams, long ones on one-CTA teams), then retries of the pairs
// that did not fit: fewer, larger arena slices on one-CTA teams, or a larger
// CIGAR pool.  A pair that does not fit the whole arena gives ENOMEM.
int run_arena(wfa_gpu_ctx* c, Call& k, wfa::AlignArgs& a, bool longest_first) {
  cudaStream_t st = c->stream;
  wfa::Ctrl* hc = c->h_ctrl;
  wfa::Ctrl* dc = c->ctrl;
  const long arena = (long)c->arena_bytes;
  // batched path: the longest pairs first, so that the last pairs a team
  // takes are short ones (a shorter tail)
  const int32_t* medium = a.defer_list;
  const int32_t* lng = a.defer_long_list;
  if (longest_first && hc->defer_count > 1) {
    if (!k.launched(wfa::launch_sort_longest_first(a, a.defer_list, &dc->defer_count, hc->defer_count,
                                                   c->sort_aux.p, c->sorted.p, st), 3))
      return WFA_GPU_ECUDA;
    medium = c->sorted.p;
  }
  if (longest_first && hc->defer_long_count > 1) {
    if (!k.launched(wfa::launch_sort_longest_first(a, a.defer_long_list, &dc->defer_long_count,
                                                   hc->defer_long_count, c->sort_aux.p, c->sorted_long.p, st), 3))
      return WFA_GPU_ECUDA;
    lng = c->sorted_long.p;
  }
  // no more teams than pairs: small batches leave the GPU to concurrent work
  // and get larger arena slices
  const int tm = std::min<int>(c->teams_medium, hc->defer_count);
  const bool narrow = hc->defer_long_count > narrow_above(c);
  const int tl = std::min<int>(narrow ? c->teams_narrow : c->teams_long, hc->defer_long_count);
  if (tm > 0 && !k.launched(wfa::launch_arena(1, a, medium, &dc->defer_count, &dc->next_medium,
                                              &dc->overflow_count, reinterpret_cast<unsigned char*>(c->arena),
                                              (arena / tm) & ~255L, tm, st)))
    return WFA_GPU_ECUDA;
  if (tl > 0 && !k.launched(wfa::launch_arena(narrow ? wfa::kLongTeamNarrow : wfa::kLongTeamWide, a, lng, &dc->defer_long_count, &dc->next_long,
                                              &dc->overflow_count, reinterpret_cast<unsigned char*>(c->arena),
                                              (arena / tl) & ~255L, tl, st)))
    return WFA_GPU_ECUDA;
  if (!ctrl_to_host(k, st) || !k.ok(cudaStreamSynchronize(st))) return WFA_GPU_ECUDA;
  return run_retries(c, k, a);
}

// Retries of the pairs on the overflow list (h_ctrl mirrors the device
// control block on entry).
int run_retries(wfa_gpu_ctx* c, Call& k, wfa::AlignArgs& a) {
  cudaStream_t st = c->stream;
  wfa::Ctrl* hc = c->h_ctrl;
  wfa::Ctrl* dc = c->ctrl;
  const long arena = (long)c->arena_bytes;
  int teams = c->teams_long;
  int32_t* in = a.overflow_list;  // the pairs to retry
  int32_t* out = a.defer_list;    // free again: receives the next overflow
  while (hc->overflow_count > 0) {
    if (hc->pool_short) {
      // keep the runs already written, and at least double the pool
      const int64_t used = std::min<int64_t>((int64_t)hc->pool_top, (int64_t)c->pool.cap);
      const int64_t want = 2 * (int64_t)hc->pool_top + (1 << 22);
      uint32_t* nb = nullptr;
      cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&nb), (size_t)want * sizeof(uint32_t));
      if (e != cudaSuccess) return map_alloc(e);
      if (!k.ok(cudaMemcpyAsync(nb, c->pool.p, (size_t)used * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st)) ||
          !k.ok(cudaStreamSynchronize(st))) {
        cudaFree(nb);
        return WFA_GPU_ECUDA;
      }
      cudaFree(c->pool.p);
      c->pool.p = nb;
      c->pool.cap = (size_t)want;
      c->pool_words = want;
      a.pool = nb;
      a.pool_cap = want;
    } else {
      if (teams == 1) return WFA_GPU_ENOMEM;  // a pair needs more than the whole arena
      teams = std::max(1, std::min(teams, hc->overflow_count) / 8);
    }
    hc->retry_count = hc->overflow_count;
    hc->next_retry = 0;
    hc->overflow_count = 0;
    hc->pool_short = 0;
    if (!ctrl_to_device(k, dc, *hc, st)) return WFA_GPU_ECUDA;
    wfa::AlignArgs ar = a;
    ar.overflow_list = out;
    const int nt = std::max(1, std::min(teams, hc->retry_count));
    if (!k.launched(wfa::launch_arena(wfa::kLongTeamWide, ar, in, &dc->retry_count, &dc->next_retry, &dc->overflow_count,
                                      reinterpret_cast<unsigned char*>(c->arena), (arena / nt) & ~255L, nt, st)))
      return WFA_GPU_ECUDA;
    if (!ctrl_to_host(k, st) || !k.ok(cudaStreamSynchronize(st))) return WFA_GPU_ECUDA;
    std::swap(in, out);
  }
  return 0;
}

constexpr int64_t kTuneSample = 4096;

// The lane ordering's buffers for calls of up to n pairs: allocated here
// (eager calls), or only taken when already large enough (captured work,
// which must not allocate); left null when the context keeps call order.
cudaError_t lane_order_args(wfa_gpu_ctx* c, wfa::AlignArgs& a, int64_t n, bool may_alloc) {
  a.lane_words = nullptr;
  a.lane_slots = nullptr;
  if (!c->lane_order || n <= 0) return cudaSuccess;
  const int64_t slots = (n + wfa::kLaneGroup - 1) / wfa::kLaneGroup * wfa::kLaneGroup;
  const size_t words = (size_t)slots * 2 * wfa::kLaneNW;
  if (may_alloc) {
    cudaError_t e;
    if ((e = c->lane_words.ensure(words)) || (e = c->lane_slots.ensure((size_t)slots))) return e;
  } else if (c->lane_words.cap < words || c->lane_slots.cap < (size_t)slots) {
    return cudaSuccess;
  }
  a.lane_words = c->lane_words.p;
  a.lane_slots = c->lane_slots.p;
  a.lane_sort_min = c->lane_sort_min;
  return cudaSuccess;
}

// Pick the short-kernel variant for a batch of sequences <= 127 bases: the
// large-store variant scores the first kTuneSample pairs (score only); the
// smallest store that holds nearly all of them (more pairs resident per SM,
// and for the lane-per-pair kernel fewer lockstep cells) runs the batch.
// Gap-affine global calls use the lane-per-pair variants unless the context
// turned them off.  Returns the variant index, or -1 on a CUDA error.
int autotune_short(wfa_gpu_ctx* c, Call& k, const wfa::AlignArgs& a_in, int64_t n) {
  const int model = a_in.oes == a_in.es ? 1 : 0;  // o = 0: gap-linear
  if ((a_in.pb | a_in.pe | a_in.tb | a_in.te) != 0) return c->variant_ef[model];  // ends-free: one variant
  if (c->variant_forced >= 0) {
    const wfa::ShortVariant& f = c->plan.v[c->variant_forced];
    const bool ct_ok = f.ct_x == 0 || (f.ct_x == a_in.xs && f.ct_oe == a_in.oes && f.ct_e == a_in.es);
    if (f.linear == model && !f.ends_free && ct_ok) return c->variant_forced;
  }
  const wfa::ScaledPen pen{a_in.xs, a_in.oes, a_in.es};
  const bool lane = model == 0 && c->lane_on;
  const wfa::ShortVariant& ct = c->plan.v[c->lane_ct_variants[0]];
  const bool lane_ct = lane && ct.ct_x == a_in.xs && ct.ct_oe == a_in.oes && ct.ct_e == a_in.es;
  // (the compiled-in variants serve only their penalties: any other entry of
  // the list is a table-driven one)
  const int* cand = lane_ct ? c->lane_ct_variants : lane ? c->lane_variants : c->variants_small[model];
  const int ncand = lane ? 4 : 3;
  const int big = cand[ncand - 1];
  int s_store[4];
  for (int j = 0; j < ncand; ++j) {
    const wfa::ShortVariant& v = c->plan.v[cand[j]];
    if (v.kind == 1) {
      wfa::LaneGeo g;
      wfa::lane_geometry(a_in, v.cells, v.rw, &g);
      s_store[j] = g.s_store;
    } else {
      wfa::UGeo tab[64];
      s_store[j] = wfa::build_ugeo(tab, v.scap, v.cells, pen, 0, 0);
    }
  }
  const int64_t m = std::min(n, kTuneSample);
  cudaStream_t st = c->stream;
  if (c->tune_score.ensure(m) || c->tune_status.ensure(m) || c->tune_aux.ensure(m) || c->tune_src.ensure(m))
    return big;
  wfa::AlignArgs a = a_in;
  a.n = m;
  a.s_cap = std::min(a_in.s_cap, 1 << 20);
  a.score_only = 1;
  a.score = c->tune_score.p;
  a.status = c->tune_status.p;
  a.nruns = c->tune_aux.p;
  a.run_src = c->tune_src.p;
  a.defer_list = c->overflow.p;  // scratch: the sample's deferrals are discarded
  a.defer_long_list = c->overflow.p;
  a.ctrl = c->ctrl + 1;
  if (!k.ok(cudaMemsetAsync(a.ctrl, 0, sizeof(wfa::Ctrl), st))) return -1;
  // pairs the sample run defers keep score -1
  if (!k.ok(cudaMemsetAsync(a.score, 0xff, m * sizeof(int32_t), st))) return -1;
  if (!k.launched(wfa::launch_short(a, c->plan.v[big], st), wfa::short_launches(a, c->plan.v[big]))) return -1;
  if (!k.ok(d2h(c->h_tune, c->tune_score.p, m * sizeof(int32_t), st)) || !k.ok(cudaStreamSynchronize(st))) return -1;
  int64_t fit[4] = {0, 0, 0, 0}, tot = 0;
  for (int64_t i = 0; i < m; ++i) {
    const int sc = c->h_tune[i];
    if (sc < 0) continue;  // deferred, invalid or over the bound: not informative
    ++tot;
    for (int j = 0; j < ncand; ++j) fit[j] += (sc / a.g <= s_store[j]);
  }
  for (int j = 0; j < ncand; ++j)
    if (tot == 0 || fit[j] * 100 >= tot * 99) return cand[j];
  return big;
}

// The plain baseline's short-read variant: the largest store of the call's
// length class and penalty model, chosen without sampling.
int fixed_variant(const wfa_gpu_ctx* c, const wfa::AlignArgs& a, int max_len) {
  const int model = a.oes == a.es ? 1 : 0;
  const bool ef = (a.pb | a.pe | a.tb | a.te) != 0;
  if (max_len > 127) return ef ? c->variant_ef_mid[model] : c->variant_mid[model];
  if (ef) return c->variant_ef[model];
  return model == 0 && c->lane_on ? c->lane_variants[3] : c->variant_big[model];
}

}  // namespace

extern "C" {

int wfa_gpu_create(wfa_gpu_ctx** out, int device, size_t scratch_bytes) {
  if (!out) return WFA_GPU_EINVAL;
  *out = nullptr;
  if (device < 0) return WFA_GPU_EINVAL;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device >= count) return WFA_GPU_ECUDA;
  if (cudaSetDevice(device) != cudaSuccess) return WFA_GPU_ECUDA;
  wfa_gpu_ctx* c = new (std::nothrow) wfa_gpu_ctx();
  if (!c) return WFA_GPU_ENOMEM;
  c->device = device;
  int rc = WFA_GPU_OK;
  do {
    if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) { rc = WFA_GPU_ECUDA; break; }
    if (cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_chunk, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_copied, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->in_stream, cudaStreamNonBlocking) != cudaSuccess) {
      rc = WFA_GPU_ECUDA;
      break;
    }
    for (int i = 0; i < kRing; ++i)
      if (cudaEventCreateWithFlags(&c->ev_in[i], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&c->ev_free[i], cudaEventDisableTiming) != cudaSuccess)
        rc = WFA_GPU_ECUDA;
    if (rc) break;
    c->stream = c->own_stream;
    for (int i = 0; i < kEvents; ++i)
      if (cudaEventCreate(&c->ev[i]) != cudaSuccess) { rc = WFA_GPU_ECUDA; break; }
    if (rc) break;
    if (cudaMalloc(reinterpret_cast<void**>(&c->ctrl), 2 * sizeof(wfa::Ctrl)) != cudaSuccess) { rc = WFA_GPU_ENOMEM; break; }
    if (cudaHostAlloc(reinterpret_cast<void**>(&c->h_tune), kTuneSample * sizeof(int32_t), cudaHostAllocDefault) !=
        cudaSuccess) {
      rc = WFA_GPU_ENOMEM;
      break;
    }
    if (cudaHostAlloc(reinterpret_cast<void**>(&c->h_ctrl), sizeof(wfa::Ctrl), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void**>(&c->h_total), sizeof(int64_t), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->h_ctrl_dev), c->h_ctrl, 0) != cudaSuccess ||
        cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->h_total_dev), c->h_total, 0) != cudaSuccess) {
      rc = WFA_GPU_ENOMEM;
      break;
    }
    c->arena_bytes = scratch_bytes ? scratch_bytes : ((size_t)1 << 30);
    c->arena_bytes &= ~(size_t)255;
    if (c->arena_bytes < 4096) { rc = WFA_GPU_EINVAL; break; }
    if (cudaMalloc(reinterpret_cast<void**>(&c->arena), c->arena_bytes) != cudaSuccess) { rc = WFA_GPU_ENOMEM; break; }
    c->own_arena = c->arena;
    c->own_arena_bytes = c->arena_bytes;
    if (wfa::short_plan(device, &c->plan) != cudaSuccess) { rc = WFA_GPU_ECUDA; break; }
    if (c->plan.count < 23 || c->plan.v[c->lane_variants[0]].kind != 1 || c->plan.v[c->lane_variants[3]].kind != 1 ||
        c->plan.v[c->lane_ct_variants[0]].ct_x == 0 || c->plan.v[c->lane_ct_variants[1]].ct_x == 0) {
      rc = WFA_GPU_ECUDA;
      break;
    }
    if (const char* ev = std::getenv("WFA_GPU_LANE")) c->lane_on = std::atoi(ev) != 0;
    if (const char* ev = std::getenv("WFA_GPU_LANE_ORDER")) c->lane_order = std::atoi(ev) != 0;
    if (const char* ev = std::getenv("WFA_GPU_LANE_SORT_MIN")) c->lane_sort_min = std::atoi(ev);
    if (const char* ev = std::getenv("WFA_GPU_PIPE_CHUNK")) {
      const long long v = std::atoll(ev);
      if (v >= (1 << 14) && v <= (1 << 24)) c->pipe_chunk = v;
    }
    // tuning override: WFA_GPU_SHORT_VARIANT=<index> for the <= 127-base case
    if (const char* ev = std::getenv("WFA_GPU_SHORT_VARIANT")) {
      const int v = std::atoi(ev);
      if (v >= 0 && v < c->plan.count && c->plan.v[v].max_len >= 127) c->variant_forced = v;
    }
    cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, device);
    if (wfa::arena_occupancy(1, &c->occ_medium) != cudaSuccess ||
        wfa::arena_occupancy(wfa::kLongTeamWide, &c->occ_long) != cudaSuccess ||
        wfa::arena_occupancy(wfa::kLongTeamNarrow, &c->occ_narrow) != cudaSuccess) {
      rc = WFA_GPU_ECUDA;
      break;
    }
    size_teams(c);
    if (const char* ev = std::getenv("WFA_GPU_TEAMS")) {  // tuning override: "<medium>,<wide>[,<narrow>]"
      int a = 0, b = 0, d = 0;
      const int got = std::sscanf(ev, "%d,%d,%d", &a, &b, &d);
      if (got >= 2 && a > 0 && b > 0) {
        c->teams_medium = a;
        c->teams_long = b;
        c->teams_narrow = got == 3 && d > 0 ? d : b;
      }
    }
  } while (0);
  if (rc) {
    wfa_gpu_destroy(c);
    return rc;
  }
  *out = c;
  return WFA_GPU_OK;
}

int wfa_gpu_set_stream(wfa_gpu_ctx* ctx, void* stream) {
  if (!ctx) return WFA_GPU_EINVAL;
  ctx->stream = stream ? static_cast<cudaStream_t>(stream) : ctx->own_stream;
  return WFA_GPU_OK;
}

}  // extern "C"

namespace {

// Host-pointer calls of at least kPipeMinPairs pairs whose outputs are
// page-locked run in chunks of pipe_chunk pairs (512K unless the
// WFA_GPU_PIPE_CHUNK tuning variable says otherwise; smaller chunks measured
// slower, the host's round trip per chunk outweighing a shorter fill and
// drain of the pipeline): each chunk goes through
// the whole device sequence (short kernel, arena kernels for its deferred
// pairs, CIGAR offset scan and compaction, its CIGAR offsets moved to the
// call's running word count), and its outputs are copied back on the
// context's copy stream while the next chunk computes.  Page-locked
// sequences stored back to back (offsets computed here) are streamed in the
// same way: the copy engine moves later chunks' bases into a device ring
// while this chunk computes (the link's rate is the same for both, but a
// kernel that reads host memory in place waits on every load it sends over
// the link, where the copy engine's transfers hold up no computation).
constexpr int64_t kPipeMinPairs = 1 << 21;

// Host sequences a chunked call streams chunk by chunk (the lengths are on
// the device already).
struct StreamIn {
  const char* pat;
  const char* txt;
};

// Waits for the input stream when a chunked call returns: no copy of the
// caller's buffers outlives the call, also when it fails.
struct InStreamDrain {
  cudaStream_t s;
  ~InStreamDrain() {
    if (s) cudaStreamSynchronize(s);
  }
};

// mode: 0 default (autotuned variant, longest-first arena lists), 1 plain
// (fixed variant, lists in pair order), 2 arena only.
int align_pipelined(wfa_gpu_ctx* ctx, Call& k, const wfa::AlignArgs& a, int64_t n, int mode,
                    wfa_gpu_penalties pen, int32_t* out_scores, int8_t* out_status, uint32_t* out_cigars,
                    int64_t cap, int64_t* out_off, const StreamIn* sin) {
  cudaStream_t st = ctx->stream, cs = ctx->copy_stream, is = ctx->in_stream;
  const bool score_only = a.score_only != 0;
  const int64_t kChunk = ctx->pipe_chunk;
  const int64_t nchunks = (n + kChunk - 1) / kChunk;
  cudaError_t e;
  if (!score_only && (e = ctx->cig_off.ensure(n + nchunks + 1))) return map_alloc(e);
  const wfa::Ctrl staged = *ctx->h_ctrl;  // the whole batch's validation: extents, longest sequence
  // each chunk's starting control block: counters zero, the batch's extents
  // and longest sequence kept
  wfa::Ctrl staged_zero{};
  staged_zero.pat_extent = staged.pat_extent;
  staged_zero.txt_extent = staged.txt_extent;
  staged_zero.max_len = staged.max_len;
  InStreamDrain drain{sin ? is : nullptr};
  // streamed inputs: each chunk's first pattern and text offsets (the
  // device scans'), the ring slot size, and the first chunk's copy
  // ring slot layout: pattern bases, then text bases (slot bytes each)
  const int64_t *hp = nullptr, *ht = nullptr;
  int64_t slot = 0;
  auto slot_at = [&](int64_t c) { return ctx->ring.p + (size_t)(c % kRing) * (size_t)(2 * slot); };
  auto copy_in = [&](int64_t c) -> bool {
    const int s2 = (int)(c % kRing);
    char* rp = slot_at(c);
    return k.ok(cudaStreamWaitEvent(is, ctx->ev_free[s2], 0)) &&
           k.ok(h2d(rp, sin->pat + hp[c], (size_t)(hp[c + 1] - hp[c]), is)) &&
           k.ok(h2d(rp + slot, sin->txt + ht[c], (size_t)(ht[c + 1] - ht[c]), is)) &&
           k.ok(cudaEventRecord(ctx->ev_in[s2], is));
  };
  if (sin) {
    if ((e = ctx->h_bounds.ensure((size_t)(2 * (nchunks + 1))))) return map_alloc(e);
    int64_t* hb = ctx->h_bounds.p;
    const size_t pitch = (size_t)kChunk * sizeof(int64_t);
    if (!k.ok(cudaMemcpy2DAsync(hb, sizeof(int64_t), a.poff, pitch, sizeof(int64_t), (size_t)nchunks,
                                cudaMemcpyDeviceToHost, st)) ||
        !k.ok(cudaMemcpy2DAsync(hb + nchunks + 1, sizeof(int64_t), a.toff, pitch, sizeof(int64_t),
                                (size_t)nchunks, cudaMemcpyDeviceToHost, st)) ||
        !k.ok(cudaStreamSynchronize(st)))
      return fail_cuda(k);
    // back to back: the scans' totals are the extents
    hb[nchunks] = staged.pat_extent;
    hb[2 * nchunks + 1] = staged.txt_extent;
    hp = hb;
    ht = hb + nchunks + 1;
    for (int64_t c = 0; c < nchunks; ++c) slot = std::max(slot, std::max(hp[c + 1] - hp[c], ht[c + 1] - ht[c]));
    // 16 bytes of slack: the packer reads whole aligned 16-byte chunks
    slot = (slot + 16 + 255) & ~(int64_t)255;
    if ((e = ctx->ring.ensure((size_t)(kRing * 2 * slot)))) return map_alloc(e);
    for (int64_t c = 0; c < std::min<int64_t>(kRing - 1, nchunks); ++c)
      if (!copy_in(c)) return fail_cuda(k);
  }
  int vi = -1;
  int64_t base = 0, deferred = 0;
  bool over = false;
  for (int64_t c = 0; c < nchunks; ++c) {
    const int64_t b = c * kChunk, m = std::min(kChunk, n - b);
    wfa::AlignArgs ac = a;
    ac.n = m;
    ac.poff = a.poff + b; ac.plen = a.plen + b;
    ac.toff = a.toff + b; ac.tlen = a.tlen + b;
    ac.score = a.score + b; ac.status = a.status + b;
    ac.nruns = a.nruns + b; ac.run_src = a.run_src + b;
    ac.runs = a.runs + (score_only ? 0 : b * wfa::kSlot);
    if (sin) {
      // the chunk's bases at ring slot c % kRing: base addresses moved back by
      // the chunk's first offsets (integer arithmetic; the kernels add the
      // pairs' offsets, which land inside the slot)
      const int s2 = (int)(c % kRing);
      char* sp = slot_at(c);
      const uintptr_t rp = reinterpret_cast<uintptr_t>(sp);
      ac.pat = reinterpret_cast<const char*>(rp - (uintptr_t)hp[c]);
      ac.txt = reinterpret_cast<const char*>(rp + (uintptr_t)slot - (uintptr_t)ht[c]);
      ac.host_seqs = 0;
      if (!k.ok(cudaStreamWaitEvent(st, ctx->ev_in[s2], 0))) return fail_cuda(k);
    }
    *ctx->h_ctrl = staged_zero;
    if (!ctrl_to_device(k, ctx->ctrl, staged_zero, st)) return fail_cuda(k);
    if (mode == 2) {
      if (!k.launched(wfa::launch_route_all(ac, st))) return fail_cuda(k);
    } else {
      if (vi < 0) {
        vi = fixed_variant(ctx, ac, staged.max_len);
        if (mode == 0 && staged.max_len <= 127) {
          vi = autotune_short(ctx, k, ac, m);
          if (vi < 0) return fail_cuda(k);
        }
        ctx->last_variant = vi;
      }
      if (!k.launched(wfa::launch_short(ac, ctx->plan.v[vi], st), wfa::short_launches(ac, ctx->plan.v[vi])))
        return fail_cuda(k);
    }
    // later chunks' bases move while this one computes
    if (sin && c + kRing - 1 < nchunks && !copy_in(c + kRing - 1)) return fail_cuda(k);
    if (c == nchunks - 1) k.rec(2);
    // chunk c's CIGAR offsets at [b + c, b + c + m]: apart from chunk c+1's,
    // which may be written while these are still being copied.  One host
    // wait per chunk: the control block and the CIGAR total come back
    // together; a chunk with deferred pairs runs the arena kernels and
    // scans again.
    int64_t* off_c = score_only ? nullptr : ctx->cig_off.p + b + c;
    auto scan = [&]() -> bool {
      return score_only || (k.launched(wfa::launch_scan(ac.nruns, m, 0, off_c, ctx->scan_tmp.p, st), 3) &&
                            total_to_host(k, off_c + m, st));
    };
    if (!ctrl_to_host(k, st) || !scan() || !k.ok(cudaStreamSynchronize(st))) return fail_cuda(k);
    const int64_t dc = (int64_t)ctx->h_ctrl->defer_count + ctx->h_ctrl->defer_long_count;
    deferred += dc;
    if (dc > 0) {
      const int rc = run_arena(ctx, k, ac, mode == 0);
      if (rc) return rc;
      if (!scan() || !k.ok(cudaStreamSynchronize(st))) return fail_cuda(k);
    }
    // the chunk's bases are read no more: its ring slot may be refilled
    if (sin && !k.ok(cudaEventRecord(ctx->ev_free[c % kRing], st))) return fail_cuda(k);
    if (ctx->h_ctrl->internal_error) return WFA_GPU_ECUDA;
    if (c == nchunks - 1) k.rec(3);
    int64_t tot = 0;
    bool copy_words = false;
    if (!score_only) {
      tot = *ctx->h_total;
      if (base > 0 && !k.launched(wfa::launch_add(off_c, m + 1, base, st))) return fail_cuda(k);
      over = over || base + tot > cap;
      copy_words = !over && tot > 0;
      if (copy_words) {
        if ((size_t)(base + tot) > ctx->cig.cap) {
          // the copies in flight read the old buffer: let them finish first
          if (!k.ok(cudaStreamSynchronize(cs))) return fail_cuda(k);
          if ((e = ctx->cig.ensure(base + tot))) return map_alloc(e);
        }
        if (!k.launched(wfa::launch_compact(m, ac.nruns, ac.run_src, ac.runs, ac.pool, off_c, ctx->cig.p, cap,
                                            ctx->ctrl, st)))
          return fail_cuda(k);
      }
    }
    if (c == nchunks - 1) k.rec(4);
    // this chunk's outputs go back while the next one computes
    if (!k.ok(cudaEventRecord(ctx->ev_chunk, st)) || !k.ok(cudaStreamWaitEvent(cs, ctx->ev_chunk, 0)))
      return fail_cuda(k);
    if (!k.ok(d2h(out_scores + b, ac.score, (size_t)m * sizeof(int32_t), cs)) ||
        !k.ok(d2h(out_status + b, ac.status, (size_t)m * sizeof(int8_t), cs)))
      return fail_cuda(k);
    if (!score_only) {
      const int64_t cnt = c == nchunks - 1 ? m + 1 : m;
      if (!k.ok(d2h(out_off + b, off_c, (size_t)cnt * sizeof(int64_t), cs))) return fail_cuda(k);
      if (copy_words && !k.ok(d2h(out_cigars + base, ctx->cig.p + base, (size_t)tot * sizeof(uint32_t), cs)))
        return fail_cuda(k);
    }
    base += tot;
  }
  if (!k.ok(cudaEventRecord(ctx->ev_copied, cs)) || !k.ok(cudaStreamWaitEvent(st, ctx->ev_copied, 0)))
    return fail_cuda(k);
  k.rec(5);
  if (!k.ok(cudaStreamSynchronize(st))) return fail_cuda(k);
  ctx->last.deferred_pairs = deferred;
  return over ? WFA_GPU_ECIGAR_CAPACITY : WFA_GPU_OK;
}

int align_eager(wfa_gpu_ctx* ctx, int64_t n, const char* patterns, const int64_t* pattern_offsets,
                const int32_t* pattern_lengths, const char* texts, const int64_t* text_offsets,
                const int32_t* text_lengths, wfa_gpu_penalties pen, int32_t max_score, uint32_t flags,
                int32_t* out_scores, int8_t* out_status, uint32_t* out_cigars, int64_t cap,
                int64_t* out_cigar_offsets) {
  if (!ctx || n < 0 || n > INT32_MAX || cap < 0 || !pen_ok(pen)) return WFA_GPU_EINVAL;
  if (flags & ~(uint32_t)(WFA_GPU_SCORE_ONLY | WFA_GPU_DEVICE_PTRS | WFA_GPU_TIMING | WFA_GPU_PLAIN |
                          WFA_GPU_ARENA_ONLY))
    return WFA_GPU_EINVAL;
  const bool arena_only = flags & WFA_GPU_ARENA_ONLY;
  const bool plain = !arena_only && (flags & WFA_GPU_PLAIN);
  const int mode = arena_only ? 2 : plain ? 1 : 0;
  const bool dev = flags & WFA_GPU_DEVICE_PTRS;
  const bool score_only = flags & WFA_GPU_SCORE_ONLY;
  if (n > 0 && (!patterns || !pattern_lengths || !texts || !text_lengths || !out_scores || !out_status))
    return WFA_GPU_EINVAL;
  if (!score_only && !out_cigar_offsets) return WFA_GPU_EINVAL;
  const bool sink = ctx->cig_sink && !dev && !score_only;
  if (!score_only && cap > 0 && !out_cigars && !sink) return WFA_GPU_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return WFA_GPU_ECUDA;
  std::memset(&ctx->last, 0, sizeof ctx->last);
  ctx->last_variant = -1;
  cudaStream_t st = ctx->stream;
  Call k{ctx, (flags & WFA_GPU_TIMING) != 0};
  if (n == 0) {
    if (!score_only) {
      const int64_t zero = 0;
      if (dev) {
        if (!k.ok(cudaMemcpyAsync(out_cigar_offsets, &zero, sizeof zero, cudaMemcpyHostToDevice, st)) ||
            !k.ok(cudaStreamSynchronize(st)))
          return WFA_GPU_ECUDA;
      } else {
        out_cigar_offsets[0] = 0;
      }
    }
    return WFA_GPU_OK;
  }

  const int g = gcd(pen.x, gcd(pen.o, pen.e));
  k.rec(0);
  const char *d_pat, *d_txt;
  const int64_t *d_poff, *d_toff;
  const int32_t *d_plen, *d_tlen;
  bool host_seqs = false;
  int rc = stage_inputs(ctx, k, n, dev, patterns, pattern_offsets, pattern_lengths, texts, text_offsets,
                        text_lengths, &d_pat, &d_poff, &d_plen, &d_txt, &d_toff, &d_tlen, &host_seqs);
  if (rc) return rc;
  k.rec(1);

  cudaError_t e;
  // host-pointer outputs come back through device buffers and one bulk copy
  // each (kernel stores straight into mapped host memory cross the C2C link
  // in small pieces and measured several times slower)
  int32_t* d_score = out_scores;
  int8_t* d_status = out_status;
  if (!dev) {
    if ((e = ctx->score.ensure(n)) || (e = ctx->status.ensure(n))) return map_alloc(e);
    d_score = ctx->score.p;
    d_status = ctx->status.p;
  }
  const int64_t slot_words = score_only ? 1 : n * (int64_t)wfa::kSlot;
  if ((e = ctx->nruns.ensure(n)) || (e = ctx->run_src.ensure(n)) || (e = ctx->defer.ensure(n)) ||
      (e = ctx->defer_long.ensure(n)) || (e = ctx->overflow.ensure(n)) || (e = ctx->sorted.ensure(n)) ||
      (e = ctx->sorted_long.ensure(n)) || (e = ctx->sort_aux.ensure(2 * wfa::kSortBuckets)) ||
      (e = ctx->runs.ensure(slot_words)) ||
      (e = ctx->pool.ensure(score_only ? 1 : ctx->pool_words)))
    return map_alloc(e);

  wfa::AlignArgs a{};
  a.n = n;
  a.pat = d_pat; a.poff = d_poff; a.plen = d_plen;
  a.txt = d_txt; a.toff = d_toff; a.tlen = d_tlen;
  a.g = g;
  a.xs = pen.x / g;
  a.es = pen.e / g;
  a.oes = (pen.o + pen.e) / g;
  a.s_cap = max_score > 0 ? max_score / g : INT_MAX;
  a.score_only = score_only ? 1 : 0;
  a.pb = ctx->ends_free[0];
  a.pe = ctx->ends_free[1];
  a.tb = ctx->ends_free[2];
  a.te = ctx->ends_free[3];
  a.host_seqs = host_seqs ? 1 : 0;
  a.score = d_score;
  a.status = d_status;
  a.nruns = ctx->nruns.p;
  a.run_src = ctx->run_src.p;
  a.runs = ctx->runs.p;
  a.pool = ctx->pool.p;
  a.pool_cap = score_only ? 0 : (int64_t)ctx->pool.cap;
  a.defer_list = ctx->defer.p;
  a.defer_long_list = ctx->defer_long.p;
  a.overflow_list = ctx->overflow.p;
  a.ctrl = ctx->ctrl;

  // large host-pointer call with page-locked outputs: chunked, with the
  // output copies overlapping the compute
  if (!dev && !sink && n >= kPipeMinPairs && mapped_range(out_scores, (size_t)n * sizeof(int32_t)) &&
      mapped_range(out_status, (size_t)n) &&
      (score_only || (mapped_range(out_cigar_offsets, (size_t)(n + 1) * sizeof(int64_t)) &&
                      (cap == 0 || mapped_range(out_cigars, (size_t)cap * sizeof(uint32_t)))))) {
    const size_t pe = (size_t)ctx->h_ctrl->pat_extent, te = (size_t)ctx->h_ctrl->txt_extent;
    // the lengths are on the device already (stage_inputs)
    const StreamIn sin{patterns, texts};
    const bool streamed = host_seqs && !pattern_offsets && !text_offsets && mapped_range(patterns, pe) &&
                          mapped_range(texts, te);
    if (mode == 0 && (e = lane_order_args(ctx, a, std::min(n, ctx->pipe_chunk), true))) return map_alloc(e);
    rc = align_pipelined(ctx, k, a, n, mode, pen, out_scores, out_status, out_cigars, cap, out_cigar_offsets,
                         streamed ? &sin : nullptr);
    if (rc < 0 && rc != WFA_GPU_ECIGAR_CAPACITY) return rc;
    ctx->last.kernel_launches = k.launches;
    ctx->last.short_variant = ctx->last_variant;
    if (k.timing) {
      ctx->last.h2d_ms = elapsed(ctx, 0, 1);
      ctx->last.align_ms = elapsed(ctx, 1, 2);
      ctx->last.general_ms = elapsed(ctx, 2, 3);
      ctx->last.cigar_ms = elapsed(ctx, 3, 4);
      ctx->last.d2h_ms = elapsed(ctx, 4, 5);
      ctx->last.total_ms = elapsed(ctx, 0, 5);
    }
    return rc;
  }

  if (arena_only) {
    if (!k.launched(wfa::launch_route_all(a, st))) return fail_cuda(k);
  } else {
    if (!plain && (e = lane_order_args(ctx, a, n, true))) return map_alloc(e);
    int vi = fixed_variant(ctx, a, ctx->h_ctrl->max_len);
    if (!plain && ctx->h_ctrl->max_len <= 127) {
      vi = autotune_short(ctx, k, a, n);
      if (vi < 0) return fail_cuda(k);
    }
    ctx->last_variant = vi;
    if (!k.launched(wfa::launch_short(a, ctx->plan.v[vi], st), wfa::short_launches(a, ctx->plan.v[vi])))
      return fail_cuda(k);
  }
  k.rec(2);
  if (!ctrl_to_host(k, st) || !k.ok(cudaStreamSynchronize(st))) return fail_cuda(k);
  ctx->last.deferred_pairs = (int64_t)ctx->h_ctrl->defer_count + ctx->h_ctrl->defer_long_count;
  if (ctx->last.deferred_pairs > 0) {
    rc = run_arena(ctx, k, a, mode == 0);
    if (rc) return rc;
  }
  if (ctx->h_ctrl->internal_error) return WFA_GPU_ECUDA;
  k.rec(3);

  int64_t total = 0;
  int64_t* d_off = out_cigar_offsets;
  uint32_t* d_cig = out_cigars;
  if (!score_only) {
    if (!dev) {
      if ((e = ctx->cig_off.ensure(n + 1))) return map_alloc(e);
      d_off = ctx->cig_off.p;
    }
    if (!k.launched(wfa::launch_scan(ctx->nruns.p, n, 0, d_off, ctx->scan_tmp.p, st), 3)) return fail_cuda(k);
    if (!total_to_host(k, d_off + n, st) || !k.ok(cudaStreamSynchronize(st))) return fail_cuda(k);
    total = *ctx->h_total;
    if (total <= cap && total > 0 && sink) {
      out_cigars = ctx->cig_sink(ctx->cig_sink_user, total);
      if (!out_cigars) return WFA_GPU_ENOMEM;
    }
    if (total <= cap && total > 0) {
      if (!dev) {
        if ((e = ctx->cig.ensure(total))) return map_alloc(e);
        d_cig = ctx->cig.p;
      }
      if (!k.launched(
              wfa::launch_compact(n, ctx->nruns.p, ctx->run_src.p, ctx->runs.p, ctx->pool.p, d_off, d_cig, cap,
                                  ctx->ctrl, st)))
        return fail_cuda(k);
    }
  }
  k.rec(4);
  // host outputs: one copy each, straight into a page-locked destination,
  // else into page-locked staging (fast DMA, no shared driver bounce buffer)
  // and a host copy after the sync
  struct Back {
    void* dst;
    const void* src;
    size_t bytes;
    HostBuf<unsigned char>* stage;
    bool later;
  };
  Back back[4] = {{out_scores, d_score, (size_t)n * sizeof(int32_t), &ctx->h_score, false},
                  {out_status, d_status, (size_t)n * sizeof(int8_t), &ctx->h_status, false},
                  {out_cigar_offsets, d_off, (size_t)(n + 1) * sizeof(int64_t), &ctx->h_off, false},
                  {out_cigars, d_cig, (size_t)total * sizeof(uint32_t), &ctx->h_cig, false}};
  const int nback = dev ? 0 : score_only ? 2 : (total <= cap && total > 0) ? 4 : 3;
  for (int j = 0; j < nback; ++j) {
    Back& b = back[j];
    void* to = b.dst;
    if (!mapped_range(b.dst, b.bytes)) {
      if ((e = b.stage->ensure(b.bytes))) return map_alloc(e);
      to = b.stage->p;
      b.later = true;
    }
    if (!k.ok(d2h(to, b.src, b.bytes, st))) return fail_cuda(k);
  }
  k.rec(5);
  if (!k.ok(cudaStreamSynchronize(st))) return fail_cuda(k);
  for (int j = 0; j < nback; ++j)
    if (back[j].later) std::memcpy(back[j].dst, back[j].stage->p, back[j].bytes);
  ctx->last.kernel_launches = k.launches;
  ctx->last.short_variant = ctx->last_variant;
  if (k.timing) {
    ctx->last.h2d_ms = elapsed(ctx, 0, 1);
    ctx->last.align_ms = elapsed(ctx, 1, 2);
    ctx->last.general_ms = elapsed(ctx, 2, 3);
    ctx->last.cigar_ms = elapsed(ctx, 3, 4);
    ctx->last.d2h_ms = elapsed(ctx, 4, 5);
    ctx->last.total_ms = elapsed(ctx, 0, 5);
  }
  return total > cap ? WFA_GPU_ECIGAR_CAPACITY : WFA_GPU_OK;
}

// The arguments the device work of a call runs with (device-pointer calls;
// the internal buffers must already be large enough).
wfa::AlignArgs device_args(wfa_gpu_ctx* c, int64_t n, const char* pat, const int64_t* poff, const int32_t* plen,
                           const char* txt, const int64_t* toff, const int32_t* tlen, wfa_gpu_penalties pen,
                           int32_t max_score, bool score_only, int32_t* out_scores, int8_t* out_status) {
  const int g = gcd(pen.x, gcd(pen.o, pen.e));
  wfa::AlignArgs a{};
  a.n = n;
  a.pat = pat; a.poff = poff; a.plen = plen;
  a.txt = txt; a.toff = toff; a.tlen = tlen;
  a.g = g;
  a.xs = pen.x / g;
  a.es = pen.e / g;
  a.oes = (pen.o + pen.e) / g;
  a.s_cap = max_score > 0 ? max_score / g : INT_MAX;
  a.score_only = score_only ? 1 : 0;
  a.pb = c->ends_free[0];
  a.pe = c->ends_free[1];
  a.tb = c->ends_free[2];
  a.te = c->ends_free[3];
  a.score = out_scores;
  a.status = out_status;
  a.nruns = c->nruns.p;
  a.run_src = c->run_src.p;
  a.runs = c->runs.p;
  a.pool = c->pool.p;
  a.pool_cap = score_only ? 0 : (int64_t)c->pool.cap;
  a.defer_list = c->defer.p;
  a.defer_long_list = c->defer_long.p;
  a.overflow_list = c->overflow.p;
  a.ctrl = c->ctrl;
  return a;
}

// Everything the device does for a device-pointer call, without a host
// synchronisation: what a CUDA graph captures.  The short-kernel variant is
// the one the preceding eager call chose.
int enqueue_device_work(wfa_gpu_ctx* c, Call& k, int64_t n, const char* pat, const int64_t* poff,
                        const int32_t* plen, const char* txt, const int64_t* toff, const int32_t* tlen,
                        wfa_gpu_penalties pen, int32_t max_score, uint32_t flags, int32_t* out_scores,
                        int8_t* out_status, uint32_t* out_cigars, int64_t cap, int64_t* out_off,
                        bool longest_first) {
  cudaStream_t st = c->stream;
  const bool score_only = flags & WFA_GPU_SCORE_ONLY;
  // external event records become graph nodes: replays time their phases
  if (!k.ok(cudaEventRecordWithFlags(c->ev[0], st, cudaEventRecordExternal))) return WFA_GPU_ECUDA;
  if (!k.ok(cudaMemsetAsync(c->ctrl, 0, sizeof(wfa::Ctrl), st))) return WFA_GPU_ECUDA;
  const int64_t* d_poff = poff;
  const int64_t* d_toff = toff;
  if (!poff && !toff) {
    if (!k.launched(wfa::launch_offsets_validate(plen, tlen, n, c->poff.p, c->toff.p, c->scan_tmp.p, c->ctrl, st),
                    3))
      return WFA_GPU_ECUDA;
    d_poff = c->poff.p;
    d_toff = c->toff.p;
  } else {
    if (!d_poff) {
      if (!k.launched(wfa::launch_scan(plen, n, 0, c->poff.p, c->scan_tmp.p, st), 3)) return WFA_GPU_ECUDA;
      d_poff = c->poff.p;
    }
    if (!d_toff) {
      if (!k.launched(wfa::launch_scan(tlen, n, 0, c->toff.p, c->scan_tmp.p, st), 3)) return WFA_GPU_ECUDA;
      d_toff = c->toff.p;
    }
    if (!k.launched(wfa::launch_validate(n, d_poff, plen, d_toff, tlen, c->ctrl, st))) return WFA_GPU_ECUDA;
  }
  if (!k.ok(cudaEventRecordWithFlags(c->ev[1], st, cudaEventRecordExternal))) return WFA_GPU_ECUDA;
  wfa::AlignArgs a = device_args(c, n, pat, d_poff, plen, txt, d_toff, tlen, pen, max_score, score_only,
                                 out_scores, out_status);
  if (c->last_variant < 0) return WFA_GPU_ECUDA;
  if (lane_order_args(c, a, n, false) != cudaSuccess) return WFA_GPU_ECUDA;
  if (!k.launched(wfa::launch_short(a, c->plan.v[c->last_variant], st),
                  wfa::short_launches(a, c->plan.v[c->last_variant])))
    return WFA_GPU_ECUDA;
  if (!k.ok(cudaEventRecordWithFlags(c->ev[2], st, cudaEventRecordExternal))) return WFA_GPU_ECUDA;
  const long arena = (long)c->arena_bytes;
  unsigned char* ab = reinterpret_cast<unsigned char*>(c->arena);
  wfa::Ctrl* dc = c->ctrl;
  const int32_t* medium = a.defer_list;
  const int32_t* lng = a.defer_long_list;
  if (longest_first) {  // batched path with many deferred pairs: longest first
    if (!k.launched(wfa::launch_sort_longest_first(a, a.defer_list, &dc->defer_count, n, c->sort_aux.p,
                                                   c->sorted.p, st), 3) ||
        !k.launched(wfa::launch_sort_longest_first(a, a.defer_long_list, &dc->defer_long_count, n, c->sort_aux.p,
                                                   c->sorted_long.p, st), 3))
      return WFA_GPU_ECUDA;
    medium = c->sorted.p;
    lng = c->sorted_long.p;
  }
  // both one-CTA widths: the deferred count picks one on the device
  const int32_t narrow_lo = narrow_above(c);
  if (!k.launched(wfa::launch_arena(1, a, medium, &dc->defer_count, &dc->next_medium, &dc->overflow_count,
                                    ab, (arena / c->teams_medium) & ~255L, c->teams_medium, st)) ||
      !k.launched(wfa::launch_arena(wfa::kLongTeamWide, a, lng, &dc->defer_long_count, &dc->next_long,
                                    &dc->overflow_count, ab, (arena / c->teams_long) & ~255L, c->teams_long, st, 0,
                                    narrow_lo)) ||
      (narrow_lo < INT32_MAX &&
       !k.launched(wfa::launch_arena(wfa::kLongTeamNarrow, a, lng, &dc->defer_long_count, &dc->next_long,
                                     &dc->overflow_count, ab, (arena / c->teams_narrow) & ~255L, c->teams_narrow, st,
                                     narrow_lo))))
    return WFA_GPU_ECUDA;
  if (!k.ok(cudaEventRecordWithFlags(c->ev[3], st, cudaEventRecordExternal))) return WFA_GPU_ECUDA;
  if (!score_only) {
    if (!k.launched(wfa::launch_scan(c->nruns.p, n, 0, out_off, c->scan_tmp.p, st), 3) ||
        !k.launched(wfa::launch_compact(n, c->nruns.p, c->run_src.p, c->runs.p, c->pool.p, out_off, out_cigars, cap,
                                        c->ctrl, st)))
      return WFA_GPU_ECUDA;
  }
  if (!k.ok(cudaEventRecordWithFlags(c->ev[4], st, cudaEventRecordExternal))) return WFA_GPU_ECUDA;
  return 0;
}

// Key of a graph: the call's arguments and every internal buffer the
// captured work uses (a reallocation forces a new capture).
int graph_key(wfa_gpu_ctx* c, uint64_t* key, int64_t n, const void* const* ptrs, int nptrs, wfa_gpu_penalties pen,
              int32_t max_score, uint32_t flags, int64_t cap) {
  int l = 0;
  key[l++] = (uint64_t)n;
  for (int i = 0; i < nptrs; ++i) key[l++] = (uint64_t)(uintptr_t)ptrs[i];
  key[l++] = ((uint64_t)(uint32_t)pen.x << 32) | (uint32_t)pen.o;
  key[l++] = ((uint64_t)(uint32_t)pen.e << 32) | (uint32_t)max_score;
  key[l++] = flags & ~(uint32_t)WFA_GPU_TIMING;
  key[l++] = (uint64_t)cap;
  key[l++] = (uint64_t)(uintptr_t)c->stream;
  const void* bufs[] = {c->ctrl, c->poff.p, c->toff.p, c->scan_tmp.p, c->nruns.p, c->run_src.p, c->runs.p,
                        c->pool.p, c->defer.p, c->defer_long.p, c->overflow.p, c->arena,
                        c->sorted.p, c->sorted_long.p, c->sort_aux.p, c->lane_words.p, c->lane_slots.p};
  for (const void* b : bufs) key[l++] = (uint64_t)(uintptr_t)b;
  key[l++] = c->pool.cap;
  key[l++] = ((uint64_t)(uint32_t)c->teams_medium << 32) | (uint32_t)c->teams_long;
  key[l++] = ((uint64_t)(uint32_t)c->ends_free[0] << 32) | (uint32_t)c->ends_free[1];
  key[l++] = ((uint64_t)(uint32_t)c->ends_free[2] << 32) | (uint32_t)c->ends_free[3];
  return l;
}

// WFA_GPU_GRAPH: the first call of a kind runs eagerly and then captures
// its device work; later identical calls replay the capture and check the
// outcome once (retrying overflowed pairs eagerly if any).
int align_graph(wfa_gpu_ctx* ctx, int64_t n, const char* pat, const int64_t* poff, const int32_t* plen,
                const char* txt, const int64_t* toff, const int32_t* tlen, wfa_gpu_penalties pen, int32_t max_score,
                uint32_t flags, int32_t* out_scores, int8_t* out_status, uint32_t* out_cigars, int64_t cap,
                int64_t* out_off) {
  const uint32_t base = flags & ~(uint32_t)WFA_GPU_GRAPH;
  if (!ctx || !(flags & WFA_GPU_DEVICE_PTRS)) return WFA_GPU_EINVAL;
  const bool score_only = flags & WFA_GPU_SCORE_ONLY;
  const void* ptrs[] = {pat, poff, plen, txt, toff, tlen, out_scores, out_status, out_cigars, out_off};
  uint64_t key[40];  // 37 entries
  int kl = graph_key(ctx, key, n, ptrs, 10, pen, max_score, flags, cap);
  wfa_gpu_ctx::Graph* hit = nullptr;
  for (auto& gr : ctx->graphs)
    if (gr.exec && n > 0 && kl == gr.key_len && std::memcmp(key, gr.key, kl * sizeof(uint64_t)) == 0) hit = &gr;
  if (!hit) {
    const int rc = align_eager(ctx, n, pat, poff, plen, txt, toff, tlen, pen, max_score, base, out_scores,
                               out_status, out_cigars, cap, out_off);
    if ((rc != WFA_GPU_OK && rc != WFA_GPU_ECIGAR_CAPACITY) || n == 0) return rc;
    wfa_gpu_ctx::Graph& slot = ctx->graphs[ctx->graph_next];
    ctx->graph_next = (ctx->graph_next + 1) % wfa_gpu_ctx::kGraphs;
    if (slot.exec) {
      cudaGraphExecDestroy(slot.exec);
      slot.exec = nullptr;
      slot.key_len = 0;
    }
    const wfa_gpu_timing eager_timing = ctx->last;
    cudaStream_t st = ctx->stream;
    Call k{ctx, false};
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return WFA_GPU_ECUDA;
    // the longest-first sorts only when the eager run deferred many pairs
    // (a pure scheduling choice: replays stay correct either way)
    const bool longest_first = eager_timing.deferred_pairs > 1024;
    const int erc = enqueue_device_work(ctx, k, n, pat, poff, plen, txt, toff, tlen, pen, max_score, base,
                                        out_scores, out_status, out_cigars, cap, out_off, longest_first);
    const cudaError_t ee = cudaStreamEndCapture(st, &g);
    if (erc || ee != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return WFA_GPU_ECUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return WFA_GPU_ECUDA;
    slot.exec = exec;
    slot.variant = ctx->last_variant;
    slot.launches = k.launches;
    kl = graph_key(ctx, key, n, ptrs, 10, pen, max_score, flags, cap);
    std::memcpy(slot.key, key, kl * sizeof(uint64_t));
    slot.key_len = kl;
    ctx->last = eager_timing;
    return rc;
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess) return WFA_GPU_ECUDA;
  std::memset(&ctx->last, 0, sizeof ctx->last);
  ctx->last_variant = hit->variant;
  cudaStream_t st = ctx->stream;
  Call k{ctx, (flags & WFA_GPU_TIMING) != 0};
  if (!k.ok(cudaGraphLaunch(hit->exec, st))) return WFA_GPU_ECUDA;
  k.launches += hit->launches;  // the kernels the graph holds
  int64_t total = 0;
  if (!k.ok(d2h(ctx->h_ctrl, ctx->ctrl, sizeof(wfa::Ctrl), st))) return WFA_GPU_ECUDA;
  if (!score_only && !k.ok(d2h(ctx->h_total, out_off + n, sizeof(int64_t), st))) return WFA_GPU_ECUDA;
  if (!k.ok(cudaStreamSynchronize(st))) return WFA_GPU_ECUDA;
  if (ctx->h_ctrl->bad_input) return WFA_GPU_EINVAL;
  ctx->last.deferred_pairs = (int64_t)ctx->h_ctrl->defer_count + ctx->h_ctrl->defer_long_count;
  if (ctx->h_ctrl->overflow_count > 0) {
    // rare: pairs that outgrew their arena slice, retried outside the graph
    const int64_t* d_poff = poff ? poff : ctx->poff.p;
    const int64_t* d_toff = toff ? toff : ctx->toff.p;
    wfa::AlignArgs a = device_args(ctx, n, pat, d_poff, plen, txt, d_toff, tlen, pen, max_score, score_only,
                                   out_scores, out_status);
    const int rc = run_retries(ctx, k, a);
    if (rc) return rc;
    if (!score_only) {
      if (!k.launched(wfa::launch_scan(ctx->nruns.p, n, 0, out_off, ctx->scan_tmp.p, st), 3) ||
          !k.launched(wfa::launch_compact(n, ctx->nruns.p, ctx->run_src.p, ctx->runs.p, ctx->pool.p, out_off,
                                          out_cigars, cap, ctx->ctrl, st)) ||
          !k.ok(d2h(ctx->h_total, out_off + n, sizeof(int64_t), st)))
        return WFA_GPU_ECUDA;
    }
    if (!k.ok(cudaStreamSynchronize(st))) return WFA_GPU_ECUDA;
  }
  if (ctx->h_ctrl->internal_error) return WFA_GPU_ECUDA;
  if (!score_only) total = *ctx->h_total;
  ctx->last.kernel_launches = k.launches;
  ctx->last.short_variant = ctx->last_variant;
  if (k.timing) {
    // events recorded by the graph itself
    ctx->last.align_ms = elapsed(ctx, 1, 2);
    ctx->last.general_ms = elapsed(ctx, 2, 3);
    ctx->last.cigar_ms = elapsed(ctx, 3, 4);
    ctx->last.total_ms = elapsed(ctx, 0, 4);
  }
  return total > cap ? WFA_GPU_ECIGAR_CAPACITY : WFA_GPU_OK;
}

}  // namespace

extern "C" {

int wfa_gpu_align_batch(wfa_gpu_ctx* ctx, int64_t n, const char* patterns, const int64_t* pattern_offsets,
                        const int32_t* pattern_lengths, const char* texts, const int64_t* text_offsets,
                        const int32_t* text_lengths, wfa_gpu_penalties pen, int32_t max_score, uint32_t flags,
                        int32_t* out_scores, int8_t* out_status, uint32_t* out_cigars, int64_t cap,
                        int64_t* out_cigar_offsets) {
  if ((flags & WFA_GPU_GRAPH) && !(flags & (WFA_GPU_PLAIN | WFA_GPU_ARENA_ONLY)))
    return align_graph(ctx, n, patterns, pattern_offsets, pattern_lengths, texts, text_offsets, text_lengths, pen,
                       max_score, flags, out_scores, out_status, out_cigars, cap, out_cigar_offsets);
  if ((flags & WFA_GPU_GRAPH) && !(flags & WFA_GPU_DEVICE_PTRS)) return WFA_GPU_EINVAL;
  return align_eager(ctx, n, patterns, pattern_offsets, pattern_lengths, texts, text_offsets, text_lengths, pen,
                     max_score, flags & ~(uint32_t)WFA_GPU_GRAPH, out_scores, out_status, out_cigars, cap,
                     out_cigar_offsets);
}

int wfa_gpu_set_ends_free(wfa_gpu_ctx* ctx, int32_t pattern_begin_free, int32_t pattern_end_free,
                          int32_t text_begin_free, int32_t text_end_free) {
  if (!ctx) return WFA_GPU_EINVAL;
  const int32_t v[4] = {pattern_begin_free, pattern_end_free, text_begin_free, text_end_free};
  for (int32_t x : v)
    if (x < 0 || x > WFA_GPU_MAX_SEQ_LEN) return WFA_GPU_EINVAL;
  std::memcpy(ctx->ends_free, v, sizeof v);
  return WFA_GPU_OK;
}

const char* wfa_gpu_short_variant_name(const wfa_gpu_ctx* ctx, int index) {
  if (!ctx || index < 0 || index >= ctx->plan.count) return nullptr;
  return ctx->plan.v[index].name;
}

int wfa_gpu_pack2bit(wfa_gpu_ctx* ctx, int64_t n, const char* seqs, const int64_t* offsets, const int32_t* lengths,
                     uint32_t flags, uint64_t* out_words, int64_t words_capacity, int64_t* out_word_offsets,
                     int8_t* out_invalid) {
  if (!ctx || n < 0 || n > INT32_MAX || words_capacity < 0 || !out_word_offsets) return WFA_GPU_EINVAL;
  if (flags & ~(uint32_t)(WFA_GPU_DEVICE_PTRS)) return WFA_GPU_EINVAL;
  if (n > 0 && (!seqs || !lengths || !out_invalid || (words_capacity > 0 && !out_words))) return WFA_GPU_EINVAL;
  const bool dev = flags & WFA_GPU_DEVICE_PTRS;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return WFA_GPU_ECUDA;
  cudaStream_t st = ctx->stream;
  Call k{ctx, false};
  if (n == 0) {
    const int64_t zero = 0;
    if (dev) {
      if (!k.ok(cudaMemcpyAsync(out_word_offsets, &zero, sizeof zero, cudaMemcpyHostToDevice, st)) ||
          !k.ok(cudaStreamSynchronize(st)))
        return WFA_GPU_ECUDA;
    } else {
      out_word_offsets[0] = 0;
    }
    return WFA_GPU_OK;
  }
  const char *d_seq, *d_seq2;
  const int64_t *d_off, *d_off2;
  const int32_t *d_len, *d_len2;
  // the same sequences stand in for both halves of a pair
  int rc = stage_inputs(ctx, k, n, dev, seqs, offsets, lengths, seqs, offsets, lengths, &d_seq, &d_off, &d_len,
                        &d_seq2, &d_off2, &d_len2);
  if (rc) return rc;
  cudaError_t e;
  int64_t* d_woff = out_word_offsets;
  if (!dev) {
    if ((e = ctx->cig_off.ensure(n + 1))) return map_alloc(e);
    d_woff = ctx->cig_off.p;
  }
  if (!k.launched(wfa::launch_scan(d_len, n, 1, d_woff, ctx->scan_tmp.p, st), 3)) return WFA_GPU_ECUDA;
  if (!k.ok(d2h(ctx->h_total, d_woff + n, sizeof(int64_t), st)) || !k.ok(cudaStreamSynchronize(st)))
    return WFA_GPU_ECUDA;
  const int64_t total = *ctx->h_total;
  uint64_t* d_words = out_words;
  int8_t* d_inv = out_invalid;
  if (!dev) {
    if ((e = ctx->status.ensure(n))) return map_alloc(e);
    d_inv = ctx->status.p;
  }
  if (total <= words_capacity) {
    DevBuf<uint64_t> tmp;
    if (!dev) {
      if ((e = tmp.ensure(total))) return map_alloc(e);
      d_words = tmp.p;
    }
    if (!k.launched(wfa::launch_pack(n, d_seq, d_off, d_len, d_woff, d_words, d_inv, st))) {
      tmp.release();
      return WFA_GPU_ECUDA;
    }
    if (!dev && (!k.ok(d2h(out_words, d_words, total * sizeof(uint64_t), st)) ||
                 !k.ok(d2h(out_invalid, d_inv, n, st)))) {
      tmp.release();
      return WFA_GPU_ECUDA;
    }
    if (!k.ok(cudaStreamSynchronize(st))) {
      tmp.release();
      return WFA_GPU_ECUDA;
    }
    tmp.release();
  }
  if (!dev && (!k.ok(d2h(out_word_offsets, d_woff, (n + 1) * sizeof(int64_t), st)) ||
               !k.ok(cudaStreamSynchronize(st))))
    return WFA_GPU_ECUDA;
  return total > words_capacity ? WFA_GPU_ECIGAR_CAPACITY : WFA_GPU_OK;
}

int64_t wfa_gpu_cigar_bound(int32_t plen, int32_t tlen, wfa_gpu_penalties pen, int32_t max_score) {
  if (plen < 0 || tlen < 0 || plen > WFA_GPU_MAX_SEQ_LEN || tlen > WFA_GPU_MAX_SEQ_LEN || !pen_ok(pen)) return -1;
  if (plen == 0 && tlen == 0) return 0;
  const int64_t cols = (int64_t)plen + tlen;
  const int64_t mn = std::min<int64_t>(pen.x, (int64_t)pen.o + pen.e);
  int64_t s;
  if (max_score > 0) {
    s = max_score;
  } else {
    // the optimum is at most the cost of either of two alignments: all
    // diagonal (mismatches) plus one gap for the length difference, or one
    // gap per sequence
    const int64_t lo = std::min(plen, tlen), d = std::abs((int64_t)plen - tlen);
    const int64_t a = pen.x * lo + (d ? pen.o + d * pen.e : 0);
    const int64_t b = (plen ? pen.o + (int64_t)plen * pen.e : 0) + (tlen ? pen.o + (int64_t)tlen * pen.e : 0);
    s = std::min(a, b);
  }
  return std::min(cols, 2 * (s / mn) + 1);
}

int wfa_gpu_last_timing(const wfa_gpu_ctx* ctx, wfa_gpu_timing* out) {
  if (!ctx || !out) return WFA_GPU_EINVAL;
  *out = ctx->last;
  return WFA_GPU_OK;
}

const char* wfa_gpu_strerror(int code) {
  switch (code) {
    case WFA_GPU_OK: return "ok";
    case WFA_GPU_EINVAL: return "invalid argument";
    case WFA_GPU_ENOMEM: return "out of memory (device, host, or scratch arena too small for a pair)";
    case WFA_GPU_ECUDA: return "CUDA runtime error";
    case WFA_GPU_ECIGAR_CAPACITY: return "CIGAR output capacity too small";
    case WFA_GPU_ETIMEOUT: return "device-side wait timed out";
    default: return "unknown error code";
  }
}

void wfa_gpu_destroy(wfa_gpu_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->own_stream) cudaStreamSynchronize(c->own_stream);
  if (c->stream && c->stream != c->own_stream) cudaStreamSynchronize(c->stream);
  c->pat.release(); c->txt.release(); c->plen.release(); c->tlen.release();
  c->poff.release(); c->toff.release(); c->score.release(); c->status.release();
  c->cig_off.release(); c->cig.release(); c->nruns.release(); c->defer.release();
  c->overflow.release(); c->run_src.release(); c->scan_tmp.release(); c->runs.release();
  c->sorted.release(); c->sorted_long.release(); c->sort_aux.release();
  c->defer_long.release(); c->pool.release();
  if (c->in_stream) cudaStreamSynchronize(c->in_stream);
  c->h_score.release(); c->h_status.release(); c->h_off.release(); c->h_cig.release();
  c->ring.release(); c->h_bounds.release();
  c->lane_words.release(); c->lane_slots.release();
  if (c->own_arena) cudaFree(c->own_arena);
  if (c->ctrl) cudaFree(c->ctrl);
  if (c->h_ctrl) cudaFreeHost(c->h_ctrl);
  if (c->h_total) cudaFreeHost(c->h_total);
  if (c->h_tune) cudaFreeHost(c->h_tune);
  for (auto& gr : c->graphs)
    if (gr.exec) cudaGraphExecDestroy(gr.exec);
  c->tune_score.release(); c->tune_aux.release(); c->tune_status.release(); c->tune_src.release();
  for (int i = 0; i < kEvents; ++i)
    if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  if (c->copy_stream) {
    cudaStreamSynchronize(c->copy_stream);
    cudaStreamDestroy(c->copy_stream);
  }
  if (c->ev_chunk) cudaEventDestroy(c->ev_chunk);
  if (c->ev_copied) cudaEventDestroy(c->ev_copied);
  if (c->in_stream) cudaStreamDestroy(c->in_stream);
  for (int i = 0; i < kRing; ++i) {
    if (c->ev_in[i]) cudaEventDestroy(c->ev_in[i]);
    if (c->ev_free[i]) cudaEventDestroy(c->ev_free[i]);
  }
  delete c;
}

}  // extern "C"
