// server.cu -- continuous batching of alignment requests (the serving half
// of the C ABI in include/wfa_gpu.h): a FIFO queue, admission by free device
// memory, and worker slots that each own a context (stream, buffers, arena).
// A slot that frees up takes the oldest request together with the requests
// queued behind it that share its parameters, gathers their pairs into one
// batch (pairs are independent, paper Sec. I), aligns it with one call and
// scatters every request's results back into its own buffers.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <cstring>
#include <deque>
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

struct Request {
  int64_t id = 0;
  wfa_gpu_request r{};
  int64_t need = 0;        // wfa_gpu_request_bytes
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

// A worker slot: its context and the staging of merged batches.
struct Slot {
  wfa_gpu_ctx* ctx = nullptr;
  Pinned<char> pat, txt;
  Pinned<int64_t> poff, toff, off;
  Pinned<int32_t> plen, tlen, score;
  Pinned<int8_t> status;
  Pinned<uint32_t> cig;
};

uint32_t* cigar_sink(void* user, int64_t words) {
  Slot* s = static_cast<Slot*>(user);
  return s->cig.ensure((size_t)words) ? s->cig.p : nullptr;
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

// Align several well-formed requests of the same parameters as one batch.
// Returns false when the merged call could not give every request the
// result it gets alone (staging out of memory, a failed call); the caller
// then runs them one by one.
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
      !sl.poff.ensure(n + 1) || !sl.toff.ensure(n + 1) || !sl.plen.ensure(n + 1) || !sl.tlen.ensure(n + 1) ||
      !sl.score.ensure(n + 1) || !sl.status.ensure(n + 1) || (!so && !sl.off.ensure(n + 1)))
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
      sl.poff.p[k] = pc;
      sl.toff.p[k] = tc;
      sl.plen.p[k] = lp;
      sl.tlen.p[k] = lt;
      pc += lp;
      tc += lt;
    }
  }
  if (!so) wfa::set_cigar_sink(sl.ctx, cigar_sink, &sl);
  const int rc = wfa_gpu_align_batch(sl.ctx, n, sl.pat.p, sl.poff.p, sl.plen.p, sl.txt.p, sl.toff.p, sl.tlen.p,
                                     r0.pen, r0.max_score, r0.flags, sl.score.p, sl.status.p,
                                     so ? nullptr : sl.cig.p, so ? 0 : cap, so ? nullptr : sl.off.p);
  wfa::set_cigar_sink(sl.ctx, nullptr, nullptr);
  if (rc != WFA_GPU_OK) return false;
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
  int64_t budget = 0;     // admission budget, bytes
  int64_t in_flight = 0;  // estimated bytes of the admitted requests
  int running = 0;
  bool stop = false;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

  void worker(int w) {
    Slot& sl = *slots[w];
    cudaSetDevice(device);
    for (;;) {
      std::vector<std::shared_ptr<Request>> run;
      int64_t need = 0;
      {
        std::unique_lock<std::mutex> lk(mu);
        // FIFO: the oldest request goes first, when it fits the budget (or
        // nothing else is running, so that any request can make progress)
        cv_work.wait(lk, [&] {
          return stop || (!queue.empty() && (running == 0 || in_flight + queue.front()->need <= budget));
        });
        if (stop) return;
        run.push_back(queue.front());
        queue.pop_front();
        need = run[0]->need;
        int64_t pairs = run[0]->r.n_pairs;
        // the requests queued right behind it join when they share its
        // parameters and fit the merge limit and the budget
        while (run[0]->mergeable && !queue.empty()) {
          const Request& q = *queue.front();
          if (!q.mergeable || !same_call(q.r, run[0]->r) || pairs + q.r.n_pairs > WFA_GPU_SERVER_MERGE_PAIRS ||
              in_flight + need + q.need > budget)
            break;
          pairs += q.r.n_pairs;
          need += q.need;
          run.push_back(queue.front());
          queue.pop_front();
        }
        in_flight += need;
        ++running;
        const double t = now();
        for (auto& q : run) {
          q->st.start_s = t;
          q->st.worker = w;
        }
      }
      cv_work.notify_all();  // another slot may admit the next request
      if (run.size() == 1 || !run_merged(sl, run))
        for (auto& q : run) q->st.result = run_alone(sl.ctx, q->r);
      {
        std::lock_guard<std::mutex> lk(mu);
        const double t = now();
        for (auto& q : run) {
          q->st.end_s = t;
          q->done = true;
        }
        in_flight -= need;
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
  // slots (about 150 bytes a pair), the caller's CIGAR capacity
  return seq + 150 * r->n_pairs + 4 * std::max<int64_t>(0, r->cigar_capacity_words);
}

int wfa_gpu_server_create(wfa_gpu_server** out, int device, int workers, size_t budget) {
  if (!out) return WFA_GPU_EINVAL;
  *out = nullptr;
  if (device < 0 || workers < 1 || workers > 64) return WFA_GPU_EINVAL;
  if (!budget) budget = (size_t)8 << 30;
  wfa_gpu_server* s = new (std::nothrow) wfa_gpu_server();
  if (!s) return WFA_GPU_ENOMEM;
  s->device = device;
  s->t0 = Clock::now();
  s->budget = (int64_t)(budget / 2);
  const size_t arena = std::max<size_t>((budget / 2) / (size_t)workers, (size_t)64 << 20);
  for (int w = 0; w < workers; ++w) {
    std::unique_ptr<Slot> sl(new (std::nothrow) Slot());
    if (!sl) {
      wfa_gpu_server_destroy(s);
      return WFA_GPU_ENOMEM;
    }
    const int rc = wfa_gpu_create(&sl->ctx, device, arena);
    if (rc != WFA_GPU_OK) {
      wfa_gpu_server_destroy(s);
      return rc;
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
  const int64_t need = wfa_gpu_request_bytes(r);
  if (need < 0) return WFA_GPU_EINVAL;
  auto req = std::make_shared<Request>();
  req->r = *r;
  req->need = need;
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
  }
  s->slots.clear();  // page-locked staging freed here
  delete s;
}

}  // extern "C"
