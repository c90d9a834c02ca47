// arena_path.cuh -- the gap-affine WFA for pairs that do not fit the
// short-read kernel: medium and long reads, or high scores.
//
// A team -- one warp, or a whole CTA of WPP warps for long reads -- owns one
// pair at a time; its threads stride over the diagonals of each wavefront.
// Both sequences are packed (2 bits per base) into the team's shared memory
// when they fit, else into its slice of the global scratch arena.  The
// wavefronts live in that slice: every score's M/I/D block (int16 offsets
// when both sequences are shorter than 32,767, else int32) for score +
// CIGAR, or only a ring of the last max(x, o+e, e) + 1 scores when just the
// score is wanted (memory linear in the wavefront width).  Pairs come from
// a device work queue (an atomic counter over a list of pair indices).
#pragma once

#include "launch.h"
#include "short_path.cuh"
#include "wfa_device.cuh"

namespace wfa {

// Threads that work on one pair: a warp (WPP == 1) or a CTA of WPP warps.
template <int WPP>
struct Team {
  static constexpr int kSize = 32 * WPP;
  __device__ static int rank() { return WPP == 1 ? (int)(threadIdx.x & 31) : (int)threadIdx.x; }
  __device__ static void sync() {
    if (WPP == 1) __syncwarp();
    else __syncthreads();
  }
  // OR of `bits` over the team; a barrier for the team as well.  `flags`
  // points at the team's three rotating shared words; `round` counts calls.
  __device__ static int reduce_or(int bits, int* flags, int& round) {
    if (WPP == 1) {
      __syncwarp();  // orders the team's memory writes before its next reads
      return __reduce_or_sync(0xffffffffu, bits);
    }
    const int w = __reduce_or_sync(0xffffffffu, bits);
    volatile int* f = flags + (round % 3);
    if ((threadIdx.x & 31) == 0 && w) atomicOr(flags + (round % 3), w);
    if (threadIdx.x == 0) flags[(round + 1) % 3] = 0;
    ++round;
    __syncthreads();
    return *f;
  }
  // rank 0's value of v, for every member
  __device__ static int broadcast(int v, int* slot) {
    if (WPP == 1) return __shfl_sync(0xffffffffu, v, 0);
    if (threadIdx.x == 0) *slot = v;
    __syncthreads();
    const int r = *(volatile int*)slot;
    __syncthreads();
    return r;
  }
};

// Every score's wavefront kept in an arena slice.  Per-score metadata (4
// ints: lo, hi, base, exist bits) grows up from `meta`; each block
// [M w][I w][D w] of Off grows down from `end`; `base` counts elements from
// `end` to the block start.  Metadata and blocks meet at cap_bytes.
template <typename OffT>
struct ArenaViewT {
  using Off = OffT;
  int32_t* meta;
  OffT* end;
  long cap_bytes;

  __device__ __forceinline__ int lo_of(int s) const { return meta[4 * s]; }
  __device__ __forceinline__ int hi_of(int s) const { return meta[4 * s + 1]; }
  __device__ __forceinline__ int base_of(int s) const { return meta[4 * s + 2]; }
  __device__ __forceinline__ int ex_of(int s) const { return meta[4 * s + 3]; }
  __device__ __forceinline__ void set_meta(int s, int l, int h, int b, int e) {
    meta[4 * s] = l; meta[4 * s + 1] = h; meta[4 * s + 2] = b; meta[4 * s + 3] = e;
  }
  __device__ __forceinline__ void set_absent(int s) { meta[4 * s + 3] = 0; }
  __device__ __forceinline__ bool score_ok(int s, int top) const {
    return 16L * (s + 1) + (long)top * (long)sizeof(OffT) <= cap_bytes;
  }
  __device__ __forceinline__ bool alloc(int s, int w, int& top, int& b) const {
    const long elems = (long)top + 3L * w;
    if (16L * (s + 1) + elems * (long)sizeof(OffT) > cap_bytes || elems > INT_MAX) return false;
    top = (int)elems;
    b = top;
    return true;
  }
  __device__ __forceinline__ void release(int b, int& top) const {
    (void)b;
    (void)top;
  }
  __device__ __forceinline__ const OffT* blk(const Geo& g) const { return end - g.base; }
  // first cell of component c (0 M, 1 I, 2 D) of a stored wavefront
  __device__ __forceinline__ const OffT* comp(const Geo& g, int c) const { return end - g.base + c * g.w; }
  __device__ __forceinline__ int getM(const Geo& g, int i) const { return blk(g)[i]; }
  __device__ __forceinline__ int getI(const Geo& g, int i) const { return blk(g)[g.w + i]; }
  __device__ __forceinline__ int getD(const Geo& g, int i) const { return blk(g)[2 * g.w + i]; }
  __device__ __forceinline__ void put(int b, int w, int i, int mv, int iv, int dv) {
    OffT* q = end - b;
    q[i] = (OffT)mv; q[w + i] = (OffT)iv; q[2 * w + i] = (OffT)dv;
  }
};

// geo_of for the arena store: the score's metadata in one 16-byte load (the
// metadata of a slice starts 16-byte aligned).
template <typename OffT>
__device__ __forceinline__ Geo geo_of(const ArenaViewT<OffT>& view, int s, int bit) {
  Geo g{0, 0, 0};
  if (s >= 0) {
    const int4 t = *reinterpret_cast<const int4*>(view.meta + 4 * s);  // lo, hi, base, exist bits
    if (t.w & bit) {
      g.lo = t.x;
      g.w = t.y - t.x + 1;
      g.base = t.z;
    }
  }
  return g;
}

// Only the last R scores: score s lives in ring slot s % R, a block
// [M W][I W][D W] with W the widest possible wavefront; metadata likewise in
// a ring.  Enough for the recurrences, not for a backtrace.
template <typename OffT>
struct RingView {
  using Off = OffT;
  int32_t* meta;  // 4 ints per ring slot
  OffT* cells;    // R blocks of 3 W
  int R, W;

  __device__ __forceinline__ int slot(int s) const { return s % R; }
  __device__ __forceinline__ int lo_of(int s) const { return meta[4 * slot(s)]; }
  __device__ __forceinline__ int hi_of(int s) const { return meta[4 * slot(s) + 1]; }
  __device__ __forceinline__ int base_of(int s) const { return meta[4 * slot(s) + 2]; }
  __device__ __forceinline__ int ex_of(int s) const { return meta[4 * slot(s) + 3]; }
  __device__ __forceinline__ void set_meta(int s, int l, int h, int b, int e) {
    const int r = 4 * slot(s);
    meta[r] = l; meta[r + 1] = h; meta[r + 2] = b; meta[r + 3] = e;
  }
  __device__ __forceinline__ void set_absent(int s) { meta[4 * slot(s) + 3] = 0; }
  __device__ __forceinline__ bool score_ok(int s, int top) const {
    (void)s;
    (void)top;
    return true;
  }
  __device__ __forceinline__ bool alloc(int s, int w, int& top, int& b) const {
    (void)top;
    if (w > W) return false;
    b = slot(s) * 3 * W;
    return true;
  }
  __device__ __forceinline__ void release(int b, int& top) const {
    (void)b;
    (void)top;
  }
  __device__ __forceinline__ const OffT* comp(const Geo& g, int c) const { return cells + g.base + c * W; }
  __device__ __forceinline__ int getM(const Geo& g, int i) const { return cells[g.base + i]; }
  __device__ __forceinline__ int getI(const Geo& g, int i) const { return cells[g.base + W + i]; }
  __device__ __forceinline__ int getD(const Geo& g, int i) const { return cells[g.base + 2 * W + i]; }
  __device__ __forceinline__ void put(int b, int w, int i, int mv, int iv, int dv) {
    (void)w;
    cells[b + i] = (OffT)mv; cells[b + W + i] = (OffT)iv; cells[b + 2 * W + i] = (OffT)dv;
  }
};

// One source of the recurrences for a step: cells of one component of one
// stored wavefront, diagonals [lo, lo + w) (w == 0: absent).
template <typename OffT>
struct Src {
  const OffT* p;
  int lo;
  unsigned w;
  __device__ __forceinline__ int at(int k, int null_v) const {
    const unsigned i = (unsigned)(k - lo);
    return i < w ? (int)p[i] : null_v;
  }
};

template <class V>
__device__ __forceinline__ Src<typename V::Off> src_of(const V& view, const Geo& g, int c) {
  return Src<typename V::Off>{g.w ? view.comp(g, c) : nullptr, g.lo, (unsigned)g.w};
}

// The score loop for one pair on a team (the recurrences, range rules and
// outcomes of the short kernel's loop, with per-score ranges from the stored
// metadata).  Metadata of each score is written by every warp's lane 0
// (identical values), so each warp reads its own writes.  Packed sequences
// are 32-bit words (16 bases).
template <int WPP, class V>
__device__ int team_forward(V& view, const uint32_t* pw, const uint32_t* tw, int n, int m, ScaledPen p, int s_cap,
                            const AlignArgs& a, int* flags, int& round, int* s_out, int* k_out, int* h_out) {
  using Off = typename V::Off;
  using T = Team<WPP>;
  constexpr int NUL = NullOf<Off>::value;
  const int r = T::rank();
  const bool leader = (threadIdx.x & 31) == 0;
  const int kf = m - n;
  // End test of a score on diagonals [lo, lo + w) at block b (every member,
  // the same answer): the diagonal nearest kf reaching an end cell -- text
  // end (M == m) on kf .. kf + pe, pattern end (M == n + k) on kf - te ..
  // kf - 1 -- the larger k on a tie; kf alone for a global alignment.
  auto reaches_end = [&](int lo, int w, int b) -> bool {
    const int dmax = max(a.pe, a.te);
    for (int d = 0; d <= dmax; ++d) {
      if (d <= a.pe && kf + d >= lo && kf + d < lo + w && view.getM(Geo{lo, w, b}, kf + d - lo) == m) {
        *k_out = kf + d;
        *h_out = m;
        return true;
      }
      if (d > 0 && d <= a.te && kf - d >= lo && kf - d < lo + w && view.getM(Geo{lo, w, b}, kf - d - lo) == m - d) {
        *k_out = kf - d;
        *h_out = m - d;
        return true;
      }
    }
    return false;
  };
  // score 0: the free starts, diagonals -min(pb, n) .. min(tb, m) (0 alone
  // for a global alignment), M_0[k] = extend(max(k, 0))
  const int lo0 = -min(a.pb, n), hi0 = min(a.tb, m), w0 = hi0 - lo0 + 1;
  int top = 0, b0 = 0;
  if (!view.alloc(0, w0, top, b0)) return kFwdOverflow;
  for (int k = lo0 + r; k <= hi0; k += T::kSize)
    view.put(b0, w0, k - lo0, extend_diag32(pw, tw, n, m, k, k > 0 ? k : 0, 1), NUL, NUL);
  if (leader) view.set_meta(0, lo0, hi0, b0, 1);
  T::sync();
  if (reaches_end(lo0, w0, b0)) {
    *s_out = 0;
    return kFwdOk;
  }
  for (int s = 1;; ++s) {
    if (s > s_cap) return kFwdLimit;
    if (!view.score_ok(s, top)) return kFwdOverflow;
    const Geo gx = geo_of(view, s - p.x, 1);
    const Geo go = geo_of(view, s - p.oe, 1);
    const Geo gi = geo_of(view, s - p.e, 2);
    const Geo gd = geo_of(view, s - p.e, 4);
    int lo = INT_MAX, hi = INT_MIN;
    if (gx.w) { lo = min(lo, gx.lo); hi = max(hi, gx.lo + gx.w - 1); }
    if (go.w) { lo = min(lo, go.lo - 1); hi = max(hi, go.lo + go.w); }
    if (gi.w) { lo = min(lo, gi.lo - 1); hi = max(hi, gi.lo + gi.w); }
    if (gd.w) { lo = min(lo, gd.lo - 1); hi = max(hi, gd.lo + gd.w); }
    lo = max(lo, -n);
    hi = min(hi, m);
    if (lo > hi) {
      if (leader) view.set_absent(s);
      __syncwarp();
      continue;
    }
    const int w = hi - lo + 1;
    int b = 0;
    if (!view.alloc(s, w, top, b)) return kFwdOverflow;
    int bits = 0;
    const Src<Off> sx = src_of(view, gx, 0), so = src_of(view, go, 0);
    const Src<Off> si = src_of(view, gi, 1), sd = src_of(view, gd, 2);
    // two diagonals per thread and round: the ten source loads (previous
    // wavefronts, mostly from L2) are all issued before either cell is
    // computed; they never alias this score's block
    auto cell = [&](int k, int mx, int ml, int mr, int il, int dr) {
      int iv = max(ml, il) + 1;
      if (iv < 0 || iv > m) iv = NUL;
      int dv = max(mr, dr);
      if (dv < 0 || dv - k > n) dv = NUL;
      int xv = mx + 1;
      if (mx < 0 || xv > m || xv - k > n) xv = NUL;
      int mv = max(xv, max(iv, dv));
      if (mv >= 0) {
        mv = extend_diag32(pw, tw, n, m, k, mv, 1);
        bits |= 1;
      } else {
        mv = NUL;
      }
      bits |= (iv >= 0 ? 2 : 0) | (dv >= 0 ? 4 : 0);
      view.put(b, w, k - lo, mv, iv, dv);
    };
    for (int k = lo + r; k <= hi; k += 2 * T::kSize) {
      const int k2 = k + T::kSize;
      const int mx = sx.at(k, NUL), ml = so.at(k - 1, NUL), mr = so.at(k + 1, NUL);
      const int il = si.at(k - 1, NUL), dr = sd.at(k + 1, NUL);
      int mx2 = NUL, ml2 = NUL, mr2 = NUL, il2 = NUL, dr2 = NUL;
      if (k2 <= hi) {
        mx2 = sx.at(k2, NUL); ml2 = so.at(k2 - 1, NUL); mr2 = so.at(k2 + 1, NUL);
        il2 = si.at(k2 - 1, NUL); dr2 = sd.at(k2 + 1, NUL);
      }
      cell(k, mx, ml, mr, il, dr);
      if (k2 <= hi) cell(k2, mx2, ml2, mr2, il2, dr2);
    }
    const int exbits = T::reduce_or(bits, flags, round);  // also the barrier after the writes
    if (exbits == 0) view.release(b, top);
    if (leader) view.set_meta(s, lo, hi, b, exbits);
    __syncwarp();
    if ((exbits & 1) && reaches_end(lo, w, b)) {
      *s_out = s;
      return kFwdOk;
    }
  }
}

// Team packing of one sequence into out[0 .. ceil(len/16)] (32-bit words of
// 16 bases, first base in the top bits, last word zero); each word reads the
// one or two aligned 16-byte chunks holding its bases.  Returns, for every
// member, whether every byte is A/C/G/T.
template <int WPP>
__device__ __forceinline__ bool team_pack32(const char* __restrict__ seq, int len, uint32_t* out, int* flags,
                                            int& round) {
  const int nw = (len + 15) >> 4;
  const unsigned long long a = reinterpret_cast<uintptr_t>(seq);
  bool bad = false;
  for (int j = Team<WPP>::rank(); j <= nw; j += Team<WPP>::kSize) {
    uint32_t word = 0u;
    if (j < nw) {
      const unsigned long long w0 = a + 16ull * j, b0 = w0 & ~15ull;
      const int h = (int)(w0 - b0), rem = min(16, len - 16 * j);
      uint32_t m0, m1 = 0u, c1 = 0u;
      const uint32_t c0 = code16_bad(__ldg(reinterpret_cast<const uint4*>(b0)), &m0);
      if (h + rem > 16) c1 = code16_bad(__ldg(reinterpret_cast<const uint4*>(b0 + 16)), &m1);
      word = __funnelshift_l(c1, c0, 2 * h);
      if (rem < 16) word &= ~0u << (32 - 2 * rem);
      const uint32_t in = (rem >= 16 ? 0xFFFFu : ((1u << rem) - 1u)) << h;
      if ((m0 | (m1 << 16)) & in) bad = true;
    }
    out[j] = word;
  }
  return Team<WPP>::reduce_or(bad ? 1 : 0, flags, round) == 0;
}

// A pair that did not fit: onto the overflow list, with no CIGAR until a
// retry aligns it (so that a compaction run before the retry reads nothing).
__device__ __forceinline__ void overflow_pair_to(const AlignArgs& a, int64_t pair, int32_t* count) {
  const int idx = atomicAdd(count, 1);
  a.overflow_list[idx] = (int32_t)pair;
  a.nruns[pair] = 0;
  a.run_src[pair] = 0;
}

// After the forward pass of a pair (single thread): its outcome, and for a
// score its CIGAR, backtraced into a reservation of the run pool.
template <class V>
__device__ void finish_cigar(const AlignArgs& a, const V& view, int64_t pair, int n, int m, ScaledPen pen, int res,
                             int s, int k_end, int h_end, int32_t* overflow_count) {
  if (res == kFwdOverflow) {
    overflow_pair_to(a, pair, overflow_count);
    return;
  }
  if (res == kFwdLimit) {
    write_result(a, pair, 1, -1, 0, 0);
    return;
  }
  long bound = runs_bound_scaled(s, pen.x, pen.oe);
  if (bound > (long)n + m + 1) bound = (long)n + m + 1;
  const unsigned long long pos = atomicAdd(&a.ctrl->pool_top, (unsigned long long)bound);
  if ((long long)(pos + bound) > a.pool_cap) {
    atomicExch(&a.ctrl->pool_short, 1);
    overflow_pair_to(a, pair, overflow_count);
    return;
  }
  const int64_t src = -(int64_t)pos - 1;  // negative: an index into the pool
  const int nr = wfa_backtrace(view, n, m, pen, s, k_end, h_end, a.pool + pos, (int)bound);
  if (nr < 0) {
    atomicExch(&a.ctrl->internal_error, 1);
    write_result(a, pair, 0, s * a.g, 0, src);
  } else {
    write_result(a, pair, 0, s * a.g, nr, src);
  }
}

// Shared memory of one team: both packed sequences when they fit (seq_words
// 64-bit words each), the rotating reduction words and a broadcast slot.
struct TeamShm {
  int flags[3];
  int bcast;
};

template <int WPP>
__device__ void arena_body(const AlignArgs& a, const int32_t* list, const int32_t* count, int32_t* next,
                           int32_t* overflow_count, unsigned char* arena, long slot_bytes, int nteams,
                           int seq_words, unsigned char* smem) {
  using T = Team<WPP>;
  const int team = WPP == 1 ? (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) : (int)blockIdx.x;
  if (team >= nteams) return;  // whole team: uniform
  if (*(volatile const int32_t*)&a.ctrl->bad_input) return;  // inputs rejected by the validation kernel
  const int team_in_block = WPP == 1 ? (int)(threadIdx.x >> 5) : 0;
  // seq_words 64-bit words per sequence = 2 * seq_words 32-bit words
  const size_t team_smem = sizeof(TeamShm) + 2 * (size_t)seq_words * sizeof(uint64_t);
  unsigned char* my = smem + team_in_block * team_smem;
  TeamShm* ts = reinterpret_cast<TeamShm*>(my);
  const int sw32 = 2 * seq_words;
  uint32_t* spw = reinterpret_cast<uint32_t*>(my + sizeof(TeamShm));
  uint32_t* stw = spw + sw32;
  const int r = T::rank();
  if (r == 0) ts->flags[0] = ts->flags[1] = ts->flags[2] = 0;
  T::sync();
  int round = 0;
  unsigned char* slot = arena + (size_t)team * (size_t)slot_bytes;
  const ScaledPen pen{a.xs, a.oes, a.es};
  for (;;) {
    const int idx = T::broadcast(r == 0 ? atomicAdd(next, 1) : 0, &ts->bcast);
    if (idx >= *(volatile const int32_t*)count) break;
    const int64_t pair = list[idx];
    const int n = a.plen[pair], m = a.tlen[pair];
    const long nwp = (n + 15) / 16 + 1, nwt = (m + 15) / 16 + 1;  // 32-bit words incl. the zero pad
    // sequences in shared memory if they fit, else at the slice's start
    const bool in_smem = nwp <= sw32 && nwt <= sw32;
    uint32_t* pw = in_smem ? spw : reinterpret_cast<uint32_t*>(slot);
    uint32_t* tw = in_smem ? stw : reinterpret_cast<uint32_t*>(slot) + nwp;
    const long seq_bytes = in_smem ? 0 : (4L * (nwp + nwt) + 15) & ~15L;
    const long room = slot_bytes - seq_bytes;
    if (room < 1024) {
      if (r == 0) overflow_pair_to(a, pair, overflow_count);
      T::sync();
      continue;
    }
    const bool okp = team_pack32<WPP>(a.pat + a.poff[pair], n, pw, ts->flags, round);
    const bool okt = team_pack32<WPP>(a.txt + a.toff[pair], m, tw, ts->flags, round);
    if (!(okp && okt)) {
      if (r == 0) write_result(a, pair, 2, -1, 0, 0);
      T::sync();
      continue;
    }
    unsigned char* wf = slot + seq_bytes;
    int s = 0, res, k_end = m - n, h_end = m;
    const bool small = n < 32000 && m < 32000;
    if (a.score_only) {
      const int R = max(pen.x, max(pen.oe, pen.e)) + 1;
      const int W = n + m + 3;
      const long need = 16L * R + 3L * R * W * (small ? 2 : 4);
      if (need > room) {
        res = kFwdOverflow;
      } else if (small) {
        RingView<int16_t> v{reinterpret_cast<int32_t*>(wf), reinterpret_cast<int16_t*>(wf + 16L * R), R, W};
        res = team_forward<WPP>(v, pw, tw, n, m, pen, a.s_cap, a, ts->flags, round, &s, &k_end, &h_end);
      } else {
        RingView<int32_t> v{reinterpret_cast<int32_t*>(wf), reinterpret_cast<int32_t*>(wf + 16L * R), R, W};
        res = team_forward<WPP>(v, pw, tw, n, m, pen, a.s_cap, a, ts->flags, round, &s, &k_end, &h_end);
      }
      if (r == 0) {
        if (res == kFwdOverflow) overflow_pair_to(a, pair, overflow_count);
        else if (res == kFwdLimit) write_result(a, pair, 1, -1, 0, 0);
        else write_result(a, pair, 0, s * a.g, 0, 0);
      }
    } else {
      const long cap = room & ~15L;
      if (small) {
        ArenaViewT<int16_t> v{reinterpret_cast<int32_t*>(wf), reinterpret_cast<int16_t*>(wf + cap), cap};
        res = team_forward<WPP>(v, pw, tw, n, m, pen, a.s_cap, a, ts->flags, round, &s, &k_end, &h_end);
        if (r == 0) finish_cigar(a, v, pair, n, m, pen, res, s, k_end, h_end, overflow_count);
      } else {
        ArenaViewT<int32_t> v{reinterpret_cast<int32_t*>(wf), reinterpret_cast<int32_t*>(wf + cap), cap};
        res = team_forward<WPP>(v, pw, tw, n, m, pen, a.s_cap, a, ts->flags, round, &s, &k_end, &h_end);
        if (r == 0) finish_cigar(a, v, pair, n, m, pen, res, s, k_end, h_end, overflow_count);
      }
    }
    T::sync();
  }
}

}  // namespace wfa
