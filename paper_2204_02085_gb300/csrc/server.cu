// server.cu -- continuous batching of alignment requests (the serving half
// of the C ABI in include/wfa_gpu.h): a queue, admission by free scratch
// arena, and worker slots that each own a context (stream, buffers).  A
// slot that frees up takes the oldest request that fits the free arena
// (a later one may pass a request that does not fit yet, until that one has
// waited kMaxWaitS), together with the requests queued behind it that share
// its parameters; it gathers their pairs into one batch (pairs are
// independent, paper Sec. I), copies it to the device, aligns it with one
// device-pointer call on a slice of the server's arena sized to the batch's
// estimated wavefront need, and scatters every request's results back into
// its own buffers.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"
#include "wfa_gpu.h"

namespace {

using Clock = std::chrono::steady_clock;

// A request passed over by later ones (it did not fit the free arena) is
// not passed any more once it has waited this long: the slots then drain
// until it fits.
constexpr double kMaxWaitS = 0.05;
// The smallest arena slice a call runs on (short pairs the short-read kernel
// defers go to the arena kernels too).
constexpr int64_t kMinSlice = 64ll << 20;
// Calls in flight at once, whatever the slots: two keep the GPU busy while
// one call's batch is gathered or scattered on the host; more only queued
// behind one another on the GPU, split the queue into smaller merged calls
// and lengthened every call (measured: 8 unlimited slots gave 28 % less
// throughput than 2, and 3 running calls half again the median latency).
// A third call starts only to let a small request pass an older one that
// waits for arena space.
constexpr int kMaxRunning = 2;
constexpr int kMaxRunningPassing = 3;

struct Request {
  int64_t id = 0;
  wfa_gpu_request r{};
  int64_t need_arena = 0;  // wavefront_bytes: the arena it is admitted by
  bool whole = false;      // rerun on the whole arena (a pair outgrew its slice)
  int64_t pat_bytes = 0;   // sum of pattern lengths
  int64_t txt_bytes = 0;   // sum of text lengths
  bool mergeable = false;  // well-formed: safe to gather
  wfa_gpu_request_stats st{};
  bool done = false;
};

// Page-locked, device-mapped host buffer that grows geometrically.
template <class T>
struct Pinned {
  T* p = nullptr;
  size_t cap = 0;
  bool ensure(size_t n) {
    if (n <= cap && p) return true;
    const size_t want = std::max<size_t>(std::max(n + n / 2, 2 * cap), 4096);
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    if (cudaHostAlloc(reinterpret_cast<void**>(&p), want * sizeof(T), cudaHostAllocPortable | cudaHostAllocMapped) !=
        cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return false;
    }
    cap = want;
    return true;
  }
  ~Pinned() {
    if (p) cudaFreeHost(p);
  }
};

// Device buffer that grows geometrically (contents not kept).
template <class T>
struct Dev {
  T* p = nullptr;
  size_t cap = 0;
  bool ensure(size_t n) {
    if (n <= cap && p) return true;
    const size_t want = std::max<size_t>(std::max(n + n / 2, 2 * cap), 4096);
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    if (cudaMalloc(reinterpret_cast<void**>(&p), want * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return false;
    }
    cap = want;
    return true;
  }
  ~Dev() {
    if (p) cudaFree(p);
  }
};

// A worker slot: its context and stream, the page-locked gather of merged
// batches and their device copies.
struct Slot {
  wfa_gpu_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  Pinned<char> pat, txt;
  Pinned<int64_t> off;
  Pinned<int32_t> plen, tlen, score;
  Pinned<int8_t> status;
  Pinned<uint32_t> cig;
  Dev<char> dpat, dtxt;
  Dev<int32_t> dplen, dtlen, dscore;
  Dev<int8_t> dstatus;
  Dev<int64_t> doff;
  Dev<uint32_t> dcig;
};

// Scratch-arena bytes a request's wavefronts hold at once.  Pairs longer than
// the short-read kernels take (127 bases) go to the arena kernels, which
// keep every score's M, I and D offsets (2 bytes each below 32,000 bases, 4
// above) over about (s'/e' + 1)^2 cells, s' the scaled score of
// WFA_GPU_SERVER_EDIT_RATE edits per base at the costliest edit
// (max(x, o + e) / g each), e' = e / g; at most kConcurrentTeams pairs are in
// flight at once, so the estimate sums the kConcurrentTeams largest.
constexpr int kConcurrentTeams = 4096;
int gcd2(int a, int b) {
  while (b) {
    const int t = a % b;
    a = b;
    b = t;
  }
  return a;
}
int64_t wavefront_bytes(const wfa_gpu_request& r) {
  if (r.n_pairs <= 0 || !r.pattern_lengths || !r.text_lengths) return 0;
  const int g = gcd2(gcd2(r.pen.x, r.pen.o), r.pen.e);
  if (g <= 0 || r.pen.e <= 0) return 0;
  const double cost = (double)std::max(r.pen.x, r.pen.o + r.pen.e) / g, es = (double)r.pen.e / g;
  std::vector<int64_t> per;
  for (int64_t i = 0; i < r.n_pairs; ++i) {
    const int64_t L = std::max<int64_t>(std::max(0, r.pattern_lengths[i]), std::max(0, r.text_lengths[i]));
    if (L <= 127) continue;
    const double sp = WFA_GPU_SERVER_EDIT_RATE * (double)L * cost;
    const double cells = (sp / es + 1.0) * (sp / es + 1.0);
    per.push_back((int64_t)(3.0 * (L < 32000 ? 2 : 4) * cells + 16.0 * (sp + 1)));
  }
  if ((int64_t)per.size() > kConcurrentTeams) {
    std::nth_element(per.begin(), per.begin() + kConcurrentTeams, per.end(), std::greater<int64_t>());
    per.resize(kConcurrentTeams);
  }
  int64_t sum = 0;
  for (int64_t v : per) sum += v;
  return sum;
}

// Host-side checks that make gathering a request's pairs safe; a request
// that fails them runs alone, and wfa_gpu_align_batch reports its error.
bool well_formed(const wfa_gpu_request& r, int64_t* pat_bytes, int64_t* txt_bytes) {
  *pat_bytes = *txt_bytes = 0;
  if (r.n_pairs < 0 || r.n_pairs > INT32_MAX || r.cigar_capacity_words < 0) return false;
  const bool so = r.flags & WFA_GPU_SCORE_ONLY;
  if (!so && (!r.out_cigar_offsets || (r.cigar_capacity_words > 0 && !r.out_cigars))) return false;
  if (r.n_pairs == 0) return true;
  if (!r.patterns || !r.texts || !r.pattern_lengths || !r.text_lengths || !r.out_scores || !r.out_status)
    return false;
  for (int64_t i = 0; i < r.n_pairs; ++i) {
    const int32_t lp = r.pattern_lengths[i], lt = r.text_lengths[i];
    if (lp < 0 || lt < 0 || lp > WFA_GPU_MAX_SEQ_LEN || lt > WFA_GPU_MAX_SEQ_LEN) return false;
    if ((r.pattern_offsets && r.pattern_offsets[i] < 0) || (r.text_offsets && r.text_offsets[i] < 0)) return false;
    *pat_bytes += lp;
    *txt_bytes += lt;
  }
  return true;
}

bool same_call(const wfa_gpu_request& a, const wfa_gpu_request& b) {
  return a.pen.x == b.pen.x && a.pen.o == b.pen.o && a.pen.e == b.pen.e && a.max_score == b.max_score &&
         a.flags == b.flags;
}

int run_alone(wfa_gpu_ctx* ctx, const wfa_gpu_request& r) {
  return wfa_gpu_align_batch(ctx, r.n_pairs, r.patterns, r.pattern_offsets, r.pattern_lengths, r.texts,
                             r.text_offsets, r.text_lengths, r.pen, r.max_score, r.flags, r.out_scores, r.out_status,
                             r.out_cigars, r.cigar_capacity_words, r.out_cigar_offsets);
}

// Align several well-formed requests of the same parameters as one batch on
// the device: their pairs gathered back to back into page-locked staging,
// copied to the slot's device buffers, aligned by one device-pointer call,
// and the outputs copied back and scattered.  Returns false when the merged
// call could not give every request the result it gets alone (out of
// memory, a failed call); the caller then runs them one by one.
bool run_merged(Slot& sl, std::vector<std::shared_ptr<Request>>& run) {
  const wfa_gpu_request& r0 = run[0]->r;
  const bool so = r0.flags & WFA_GPU_SCORE_ONLY;
  int64_t n = 0, pb = 0, tb = 0, cap = 0;
  for (auto& q : run) {
    n += q->r.n_pairs;
    pb += q->pat_bytes;
    tb += q->txt_bytes;
    if (!so) cap = std::min<int64_t>(cap + q->r.cigar_capacity_words, INT64_MAX / 8);
  }
  if (n > INT32_MAX) return false;
  if (!sl.pat.ensure(std::max<int64_t>(pb, 1)) || !sl.txt.ensure(std::max<int64_t>(tb, 1)) ||
      !sl.plen.ensure(n + 1) || !sl.tlen.ensure(n + 1) || !sl.score.ensure(n + 1) || !sl.status.ensure(n + 1) ||
      (!so && !sl.off.ensure(n + 1)))
    return false;
  if (!sl.dpat.ensure(std::max<int64_t>(pb, 1) + 16) || !sl.dtxt.ensure(std::max<int64_t>(tb, 1) + 16) ||
      !sl.dplen.ensure(n + 1) || !sl.dtlen.ensure(n + 1) || !sl.dscore.ensure(n + 1) ||
      !sl.dstatus.ensure(n + 1) || (!so && (!sl.doff.ensure(n + 1) || !sl.dcig.ensure(std::max<int64_t>(cap, 1)))))
    return false;
  // gather: sequences back to back in request order, then pair order
  int64_t k = 0, pc = 0, tc = 0;
  for (auto& q : run) {
    const wfa_gpu_request& r = q->r;
    int64_t pr = 0, tr = 0;  // running offsets of requests without offset arrays
    for (int64_t i = 0; i < r.n_pairs; ++i, ++k) {
      const int32_t lp = r.pattern_lengths[i], lt = r.text_lengths[i];
      const int64_t op = r.pattern_offsets ? r.pattern_offsets[i] : pr;
      const int64_t ot = r.text_offsets ? r.text_offsets[i] : tr;
      pr += lp;
      tr += lt;
      std::memcpy(sl.pat.p + pc, r.patterns + op, (size_t)lp);
      std::memcpy(sl.txt.p + tc, r.texts + ot, (size_t)lt);
      sl.plen.p[k] = lp;
      sl.tlen.p[k] = lt;
      pc += lp;
      tc += lt;
    }
  }
  cudaStream_t st = sl.stream;
  auto h2d = [&](void* d, const void* h, size_t b) {
    return !b || cudaMemcpyAsync(d, h, b, cudaMemcpyHostToDevice, st) == cudaSuccess;
  };
  auto d2h = [&](void* h, const void* d, size_t b) {
    return !b || cudaMemcpyAsync(h, d, b, cudaMemcpyDeviceToHost, st) == cudaSuccess;
  };
  if (!h2d(sl.dpat.p, sl.pat.p, (size_t)pb) || !h2d(sl.dtxt.p, sl.txt.p, (size_t)tb) ||
      !h2d(sl.dplen.p, sl.plen.p, (size_t)n * sizeof(int32_t)) ||
      !h2d(sl.dtlen.p, sl.tlen.p, (size_t)n * sizeof(int32_t)))
    return false;
  // the call runs on the same stream, after the copies
  const int rc = wfa_gpu_align_batch(sl.ctx, n, sl.dpat.p, nullptr, sl.dplen.p, sl.dtxt.p, nullptr, sl.dtlen.p,
                                     r0.pen, r0.max_score, r0.flags | WFA_GPU_DEVICE_PTRS, sl.dscore.p,
                                     sl.dstatus.p, so ? nullptr : sl.dcig.p, so ? 0 : cap,
                                     so ? nullptr : sl.doff.p);
  if (rc != WFA_GPU_OK) return false;
  if (!d2h(sl.score.p, sl.dscore.p, (size_t)n * sizeof(int32_t)) ||
      !d2h(sl.status.p, sl.dstatus.p, (size_t)n * sizeof(int8_t)) ||
      (!so && !d2h(sl.off.p, sl.doff.p, (size_t)(n + 1) * sizeof(int64_t))) ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return false;
  if (!so) {
    const int64_t words = sl.off.p[n];
    if (words > cap || !sl.cig.ensure((size_t)std::max<int64_t>(words, 1)) ||
        !d2h(sl.cig.p, sl.dcig.p, (size_t)words * sizeof(uint32_t)) || cudaStreamSynchronize(st) != cudaSuccess)
      return false;
  }
  // scatter: each request gets its slice, CIGAR offsets rebased to 0
  k = 0;
  for (auto& q : run) {
    const wfa_gpu_request& r = q->r;
    const int64_t m = r.n_pairs;
    int res = WFA_GPU_OK;
    if (m > 0) {
      std::memcpy(r.out_scores, sl.score.p + k, (size_t)m * sizeof(int32_t));
      std::memcpy(r.out_status, sl.status.p + k, (size_t)m * sizeof(int8_t));
    }
    if (!so) {
      const int64_t b = sl.off.p[k], used = sl.off.p[k + m] - b;
      for (int64_t i = 0; i <= m; ++i) r.out_cigar_offsets[i] = sl.off.p[k + i] - b;
      if (used > r.cigar_capacity_words)
        res = WFA_GPU_ECIGAR_CAPACITY;  // as alone: offsets valid, CIGAR buffer untouched
      else if (used > 0)
        std::memcpy(r.out_cigars, sl.cig.p + b, (size_t)used * sizeof(uint32_t));
    }
    q->st.result = res;
    k += m;
  }
  return true;
}

// First-fit allocator of arena slices (256-byte aligned), free ranges
// coalesced on release.
struct ArenaAlloc {
  std::map<int64_t, int64_t> free_;  // offset -> size
  int64_t total = 0;
  void init(int64_t bytes) {
    total = bytes & ~255ll;
    free_.clear();
    free_[0] = total;
  }
  bool fits(int64_t bytes) const {
    bytes = (bytes + 255) & ~255ll;
    for (const auto& f : free_)
      if (f.second >= bytes) return true;
    return false;
  }
  int64_t take(int64_t bytes) {  // offset, or -1
    bytes = (bytes + 255) & ~255ll;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const int64_t off = it->first, rest = it->second - bytes;
      free_.erase(it);
      if (rest) free_[off + bytes] = rest;
      return off;
    }
    return -1;
  }
  void give(int64_t off, int64_t bytes) {
    bytes = (bytes + 255) & ~255ll;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

}  // namespace

struct wfa_gpu_server {
  int device = 0;
  Clock::time_point t0;
  std::vector<std::unique_ptr<Slot>> slots;
  std::vector<std::thread> threads;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::unordered_map<int64_t, std::shared_ptr<Request>> live;
  int64_t next_id = 0;
  unsigned char* arena = nullptr;  // the scratch arena the calls share
  ArenaAlloc alloc;
  int running = 0;
  bool stop = false;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

  // The arena slice a call of estimated need runs on: the need, at least
  // kMinSlice and at most half the arena (the arena kernels fit a smaller
  // slice than the estimate by running fewer pairs at once, with larger
  // slices each), or the whole arena for a rerun.
  int64_t slice_for(int64_t need, bool whole) const {
    if (whole) return alloc.total;
    const int64_t mb = (int64_t)1 << 20;
    const int64_t cap = std::max<int64_t>(kMinSlice, (alloc.total / 2) & ~(mb - 1));
    const int64_t s = (std::max<int64_t>(need, kMinSlice) + mb - 1) & ~(mb - 1);
    return std::min<int64_t>(std::min<int64_t>(s, cap), alloc.total);
  }

  // Under the lock: the next call to run -- while fewer than kMaxRunning run,
  // or fewer than kMaxRunningPassing when the oldest request waits for arena
  // space and the call passes it -- the oldest request whose slice fits the
  // free arena (a later one only while the oldest has waited less
  // than kMaxWaitS), with the same-parameter requests queued right behind
  // it when their slice fits too -- taken off the queue; false if none.
  bool pick(std::vector<std::shared_ptr<Request>>* run, int64_t* slice, int64_t* off) {
    if (queue.empty() || running >= kMaxRunningPassing) return false;
    const bool may_pass = now() - queue.front()->st.submit_s < kMaxWaitS;
    // beyond kMaxRunning calls: only passing an oldest request that does not
    // fit (alone) the free arena
    const bool only_pass = running >= kMaxRunning;
    if (only_pass &&
        (!may_pass || alloc.fits(slice_for(queue.front()->need_arena, queue.front()->whole))))
      return false;
    const size_t limit = may_pass ? std::min<size_t>(queue.size(), 64) : 1;
    for (size_t i = only_pass ? 1 : 0; i < limit; ++i) {
      const Request& q = *queue[i];
      // the group: q and the requests right behind it that share its call
      size_t j = i + 1;
      int64_t pairs = q.r.n_pairs;
      while (q.mergeable && !q.whole && j < queue.size()) {
        const Request& t = *queue[j];
        if (!t.mergeable || t.whole || !same_call(t.r, q.r) || pairs + t.r.n_pairs > WFA_GPU_SERVER_MERGE_PAIRS)
          break;
        pairs += t.r.n_pairs;
        ++j;
      }
      for (size_t end : {j, i + 1}) {  // the group, else q alone
        int64_t nd = 0;
        for (size_t t = i; t < end; ++t) nd += queue[t]->need_arena;
        const int64_t sl = slice_for(nd, q.whole);
        const int64_t o = alloc.take(sl);
        if (o < 0) continue;
        run->assign(queue.begin() + (long)i, queue.begin() + (long)end);
        queue.erase(queue.begin() + (long)i, queue.begin() + (long)end);
        *slice = sl;
        *off = o;
        return true;
      }
    }
    return false;
  }

  void worker(int w) {
    Slot& sl = *slots[w];
    cudaSetDevice(device);
    for (;;) {
      std::vector<std::shared_ptr<Request>> run;
      int64_t slice = 0, off = -1;
      {
        std::unique_lock<std::mutex> lk(mu);
        // a request waiting for arena space is looked at again when a call
        // ends or when its passing time runs out
        while (!stop && !pick(&run, &slice, &off)) cv_work.wait_for(lk, std::chrono::milliseconds(5));
        if (stop) return;
        ++running;
        const double t = now();
        for (auto& q : run) {
          q->st.start_s = t;
          q->st.worker = w;
        }
      }
      cv_work.notify_all();  // another slot may admit the next request
      wfa::set_arena(sl.ctx, arena + off, (size_t)slice);
      if (!(run[0]->mergeable && run_merged(sl, run)))
        for (auto& q : run) q->st.result = run_alone(sl.ctx, q->r);
      wfa::set_arena(sl.ctx, nullptr, 0);
      {
        std::lock_guard<std::mutex> lk(mu);
        alloc.give(off, slice);
        const double t = now();
        for (auto it = run.rbegin(); it != run.rend(); ++it) {
          auto& q = *it;
          if (q->st.result == WFA_GPU_ENOMEM && slice < alloc.total && !q->whole) {
            // a pair outgrew its slice: once more on the whole arena, first
            q->whole = true;
            queue.push_front(q);
            continue;
          }
          q->st.end_s = t;
          q->done = true;
        }
        --running;
      }
      cv_done.notify_all();
      cv_work.notify_all();
    }
  }
};

extern "C" {

int64_t wfa_gpu_request_bytes(const wfa_gpu_request* r) {
  if (!r || r->n_pairs < 0 || (r->n_pairs > 0 && (!r->pattern_lengths || !r->text_lengths))) return -1;
  int64_t seq = 0;
  for (int64_t i = 0; i < r->n_pairs; ++i) seq += (int64_t)std::max(0, r->pattern_lengths[i]) +
                                                 std::max(0, r->text_lengths[i]);
  // ASCII staging, lengths/offsets, outputs, per-pair work buffers and CIGAR
  // slots (about 150 bytes a pair), the caller's CIGAR capacity, and the
  // wavefronts in the scratch arena
  return seq + 150 * r->n_pairs + 4 * std::max<int64_t>(0, r->cigar_capacity_words) + wavefront_bytes(*r);
}

int wfa_gpu_server_create(wfa_gpu_server** out, int device, int workers, size_t budget) {
  if (!out) return WFA_GPU_EINVAL;
  *out = nullptr;
  if (device < 0 || workers < 1 || workers > 64) return WFA_GPU_EINVAL;
  if (!budget) budget = (size_t)8 << 30;
  if (budget < (size_t)kMinSlice) return WFA_GPU_EINVAL;
  wfa_gpu_server* s = new (std::nothrow) wfa_gpu_server();
  if (!s) return WFA_GPU_ENOMEM;
  s->device = device;
  s->t0 = Clock::now();
  if (cudaSetDevice(device) != cudaSuccess) {
    delete s;
    return WFA_GPU_ECUDA;
  }
  if (cudaMalloc(reinterpret_cast<void**>(&s->arena), budget) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return WFA_GPU_ENOMEM;
  }
  s->alloc.init((int64_t)budget);
  for (int w = 0; w < workers; ++w) {
    std::unique_ptr<Slot> sl(new (std::nothrow) Slot());
    if (!sl) {
      wfa_gpu_server_destroy(s);
      return WFA_GPU_ENOMEM;
    }
    // each call borrows a slice of the shared arena; the context's own is
    // a minimal one
    const int rc = wfa_gpu_create(&sl->ctx, device, (size_t)4 << 20);
    if (rc != WFA_GPU_OK) {
      wfa_gpu_server_destroy(s);
      return rc;
    }
    if (cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess ||
        wfa_gpu_set_stream(sl->ctx, sl->stream) != WFA_GPU_OK) {
      s->slots.push_back(std::move(sl));
      wfa_gpu_server_destroy(s);
      return WFA_GPU_ECUDA;
    }
    s->slots.push_back(std::move(sl));
  }
  try {
    for (int w = 0; w < workers; ++w) s->threads.emplace_back([s, w] { s->worker(w); });
  } catch (...) {
    wfa_gpu_server_destroy(s);
    return WFA_GPU_ENOMEM;
  }
  *out = s;
  return WFA_GPU_OK;
}

int64_t wfa_gpu_server_submit(wfa_gpu_server* s, const wfa_gpu_request* r) {
  if (!s || !r) return WFA_GPU_EINVAL;
  if (r->flags & ~(uint32_t)(WFA_GPU_SCORE_ONLY | WFA_GPU_PLAIN | WFA_GPU_ARENA_ONLY)) return WFA_GPU_EINVAL;
  if (wfa_gpu_request_bytes(r) < 0) return WFA_GPU_EINVAL;
  auto req = std::make_shared<Request>();
  req->r = *r;
  req->need_arena = wavefront_bytes(*r);
  req->mergeable = well_formed(*r, &req->pat_bytes, &req->txt_bytes);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return WFA_GPU_EINVAL;
    req->id = s->next_id++;
    req->st.submit_s = s->now();
    s->live[req->id] = req;
    s->queue.push_back(req);
  }
  s->cv_work.notify_all();
  return req->id;
}

int wfa_gpu_server_wait(wfa_gpu_server* s, int64_t id, double timeout_s, wfa_gpu_request_stats* stats) {
  if (!s) return WFA_GPU_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->live.find(id);
  if (it == s->live.end()) return WFA_GPU_EINVAL;
  std::shared_ptr<Request> req = it->second;
  auto ready = [&] { return req->done; };
  if (timeout_s < 0) {
    s->cv_done.wait(lk, ready);
  } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
    return WFA_GPU_ETIMEOUT;
  }
  if (stats) *stats = req->st;
  s->live.erase(id);
  return req->st.result;
}

void wfa_gpu_server_destroy(wfa_gpu_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (auto& q : s->queue) {
      q->st.result = WFA_GPU_ECUDA;
      q->done = true;
    }
    s->queue.clear();
  }
  s->cv_work.notify_all();
  s->cv_done.notify_all();
  for (auto& t : s->threads)
    if (t.joinable()) t.join();
  for (auto& sl : s->slots) {
    if (sl->ctx) wfa_gpu_destroy(sl->ctx);
    sl->ctx = nullptr;
    if (sl->stream) cudaStreamDestroy(sl->stream);
    sl->stream = nullptr;
  }
  s->slots.clear();  // page-locked staging and device buffers freed here
  if (s->arena) cudaFree(s->arena);
  delete s;
}

}  // extern "C"
