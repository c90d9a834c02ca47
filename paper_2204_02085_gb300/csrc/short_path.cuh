// short_path.cuh -- body of the fused short-read kernel (pack + gap-affine
// WFA with uniform per-score geometry + backtrace), shared by the kernel in
// kernels.cu.  See the comment on short_body.
#pragma once

#include "launch.h"
#include "wfa_device.cuh"

namespace wfa {

constexpr int kShortBlock = 128;

// Hand a pair to the arena kernels: pairs with a sequence longer than
// kMediumMaxLen to the one-CTA kernel, the rest to the one-warp kernel.
__device__ __forceinline__ void defer_pair(const AlignArgs& a, int64_t pair) {
  if (max(a.plen[pair], a.tlen[pair]) > kMediumMaxLen) {
    const int idx = atomicAdd(&a.ctrl->defer_long_count, 1);
    a.defer_long_list[idx] = (int32_t)pair;
  } else {
    const int idx = atomicAdd(&a.ctrl->defer_count, 1);
    a.defer_list[idx] = (int32_t)pair;
  }
}

__device__ __forceinline__ void write_result(const AlignArgs& a, int64_t pair, int status, int score, int nr,
                                             int64_t src) {
  a.score[pair] = score;
  a.status[pair] = (int8_t)status;
  a.nruns[pair] = nr;
  a.run_src[pair] = src;
}

// Shared-memory layout of the short kernel: the geometry table, then one
// region per warp holding its P = 32/G pairs' packed sequences and M/I/D
// cells, interleaved by pair (element c of pair slot q at [c * P + q]).
template <int G, int LMAX, int CELLS, int SCAP, typename Off, bool LIN = false>
struct ShortCfg {
  static constexpr int P = 32 / G;
  // packed sequence: 32-bit words (16 bases), data + two zero pad words,
  // stored every PS elements (PS = P + 1 keeps the lanes of one pair on
  // different banks)
  static constexpr int NW = 2 * ((LMAX + 31) / 32 + 1);
  static constexpr int PS = P + 1;
  struct WarpShm {
    uint32_t pw[NW * PS];
    uint32_t tw[NW * PS];
    Off M[CELLS * P];
    Off I[LIN ? 4 : CELLS * P];  // gap-linear model: I and D follow from M
    Off D[LIN ? 4 : CELLS * P];
    // the pairs still running, ascending slot: slot | n << 8 | m << 20
    uint32_t act[P];
  };
  // the packer's span scratch (the raw bytes of up to P back-to-back
  // sequences, 16-byte chunks) borrows the cell arrays, unused while
  // packing; longer spans take the packer's per-slot path
  static constexpr int kSpanAll = (P * LMAX + 15) / 16 + 1;
  static constexpr int kCellBytes = (int)(sizeof(Off) * (LIN ? CELLS * P : 3 * CELLS * P));
  static constexpr int kSpanFit = kCellBytes / 16;
  static constexpr int SPAN = kSpanAll < kSpanFit ? kSpanAll : kSpanFit;
  static_assert(16 * SPAN <= kCellBytes, "packer scratch does not fit the cell arrays");
  static constexpr size_t kTabBytes = ((SCAP + 1) * sizeof(UGeo) + 15) / 16 * 16;
  static constexpr size_t kWarpBytes = (sizeof(WarpShm) + 15) / 16 * 16;
  static constexpr size_t smem_bytes(int warps) { return kTabBytes + (size_t)warps * kWarpBytes; }
};

// A source wavefront of one score step: cell (k, slot r) of its stored
// component lies at row0 + k * P + r, for diagonals lo <= k < lo + w.
struct SrcRow {
  int row0, lo;
  unsigned w;
};
template <int P>
__device__ __forceinline__ SrcRow src_row(const Geo& g) {
  return SrcRow{(g.base - g.lo) * P, g.lo, (unsigned)g.w};
}

// One wavefront cell of the shared-lane score loop: item f of na running
// pairs (pair index fastest) at the score whose geometry is g; load()
// gathers its sources and applies the recurrences (the mismatch, insertion
// and deletion candidates, each null past the sequence ends) giving the
// offset h to extend, store() writes M, I and D.
template <typename Off, int P, bool LIN = false>
struct Cell {
  int r, k, kp, n, m, h, iv, dv;
  __device__ __forceinline__ void load(const Off* M, const Off* I, const Off* D, const uint32_t* act, int glo,
                                       const SrcRow& sx, const SrcRow& so, const SrcRow& se, int f, int na,
                                       unsigned inv_na) {
    constexpr int NUL = NullOf<Off>::value;
    const int i = na > 1 ? (int)__umulhi((unsigned)f, inv_na) : f;
    const uint32_t info = act[f - i * na];
    r = (int)(info & 0xffu);
    n = (int)((info >> 8) & 0xfffu);
    m = (int)(info >> 20);
    k = glo + i;
    kp = k * P + r;
    auto at = [&](const Off* A, const SrcRow& sr, int dk) -> int {
      return (unsigned)(k + dk - sr.lo) < sr.w ? (int)A[sr.row0 + kp + dk * P] : NUL;
    };
    const int mx = at(M, sx, 0);
    const int mlo = at(M, so, -1);
    const int mro = at(M, so, 1);
    // gap-linear model (o = 0): I[s-e][k-1] <= M[s-e][k-1] and D[s-e][k+1] <=
    // M[s-e][k+1] (M is the maximum over them), so the M sources alone give
    // the same I and D
    const int il = LIN ? NUL : at(I, se, -1);
    const int dr = LIN ? NUL : at(D, se, 1);
    // a null source stays negative through the +1 steps of the stored
    // scores, so only the far end needs testing; negative = null
    iv = max(mlo, il) + 1;
    if (iv > m) iv = NUL;
    dv = max(mro, dr);
    if (dv - k > n) dv = NUL;
    int xv = mx + 1;
    if (xv > m || xv - k > n) xv = NUL;
    h = __vimax3_s32(xv, iv, dv);
  }
  __device__ __forceinline__ void store(Off* M, Off* I, Off* D, int row0) const {
    constexpr int NUL = NullOf<Off>::value;
    const int c = row0 + kp;
    M[c] = (Off)(h >= 0 ? h : NUL);
    if (!LIN) {
      I[c] = (Off)iv;
      D[c] = (Off)dv;
    }
  }
};

// The short kernel's store seen by the backtrace under the gap-linear model
// (o = 0): only M is kept, and I_s[k] = M_{s-e}[k-1] + 1, D_s[k] =
// M_{s-e}[k+1] (each null past the sequence ends), which is what the
// gap-affine recurrences give when o = 0.
template <typename Off, int P>
struct LinUView : UView<Off, P> {
  int n, m, e;
};
template <typename Off, int P>
__device__ __forceinline__ int bt_I(const LinUView<Off, P>& v, int s, int k) {
  constexpr int NUL = NullOf<Off>::value;
  const UView<Off, P>& u = v;
  const int ml = get_off<UView<Off, P>, 0>(u, geo_of(u, s - v.e, 1), k - 1, NUL);
  return ml >= 0 && ml + 1 <= v.m ? ml + 1 : NUL;
}
template <typename Off, int P>
__device__ __forceinline__ int bt_D(const LinUView<Off, P>& v, int s, int k) {
  constexpr int NUL = NullOf<Off>::value;
  const UView<Off, P>& u = v;
  const int mr = get_off<UView<Off, P>, 0>(u, geo_of(u, s - v.e, 1), k + 1, NUL);
  return mr >= 0 && mr - k <= v.n ? mr : NUL;
}

// Fused short-read kernel: 32/G pairs per warp advance through the scores
// together; per pair: pack both sequences (2 bits per base, G lanes) into
// shared memory, run the wavefront recurrences with cells in shared memory
// (at each score the cells of the pairs still running are spread over all
// 32 lanes), then walk the backtrace (the pair's first lane) and write the
// CIGAR runs (last first) into the pair's slot.  Pairs longer than LMAX, or
// whose score passes the last storable wavefront (but not the caller's
// max_score), are deferred to the arena kernel.  LIN: the gap-linear model
// (o = 0, the edit distance at x = e = 1), only M stored.  EF: ends-free
// calls (free pattern / text ends; the first wavefront spans the free
// starts, the end test scans the free diagonals).
template <int G, int LMAX, int CELLS, int SCAP, typename Off, bool LIN = false, bool EF = false>
__device__ __forceinline__ void short_body(const AlignArgs& a, unsigned char* smem, int* s_last_shared) {
  using C = ShortCfg<G, LMAX, CELLS, SCAP, Off, LIN>;
  constexpr int P = C::P;
  constexpr int NUL = NullOf<Off>::value;
  static_assert(NUL + SCAP + 1 < 0, "a null offset must stay negative over the stored scores");
  constexpr unsigned FULL = 0xffffffffu;
  if (*(volatile int32_t*)&a.ctrl->bad_input) return;  // inputs rejected by the validation kernel
  int& s_last = *s_last_shared;
  UGeo* tab = reinterpret_cast<UGeo*>(smem);
  const int warp = threadIdx.x >> 5, lane32 = threadIdx.x & 31;
  const int lane = lane32 & (G - 1), q = lane32 / G;
  auto* W = reinterpret_cast<typename C::WarpShm*>(smem + C::kTabBytes + warp * C::kWarpBytes);
  const ScaledPen pen{a.xs, a.oes, a.es};
  // the first wavefront spans the free starts (diagonal 0 alone for a
  // global alignment)
  const int lo0 = EF ? -min(a.pb, LMAX) : 0, hi0 = EF ? min(a.tb, LMAX) : 0;
  constexpr bool ends_free = EF;  // the variant for ends-free calls
  if (threadIdx.x == 0) s_last = build_ugeo(tab, SCAP, CELLS, pen, lo0, hi0);
  __syncthreads();
  // -1: the first wavefront does not fit; also when a global variant is
  // handed an ends-free call (then the arena kernels take every pair)
  const int s_store = (!EF && (a.pb | a.pe | a.tb | a.te) != 0) ? -1 : s_last;
  const int s_hi = min(s_store, a.s_cap);
  const unsigned gmask = group_mask(G);
  UView<Off, P> view{tab, W->M, W->I, W->D, q};
  constexpr int PS = C::PS;
  uint32_t* pw = W->pw + q;
  uint32_t* tw = W->tw + q;
  const int64_t wpb = blockDim.x >> 5;
  const int64_t stride = (int64_t)gridDim.x * wpb * P;
  for (int64_t first = ((int64_t)blockIdx.x * wpb + warp) * P; first < a.n; first += stride) {
    const int64_t pair = first + q;
    bool active = pair < a.n;
    int n = 0, m = 0;
    if (active) {
      n = a.plen[pair];
      m = a.tlen[pair];
      if (n > LMAX || m > LMAX || s_store < 0) {
        if (lane == 0) defer_pair(a, pair);
        active = false;
      }
    }
    {
      // all lanes take part: the warp reads its pairs' sequences together
      uint32_t* scratch = reinterpret_cast<uint32_t*>(W->M);
      const char* ps = active ? a.pat + a.poff[pair] : nullptr;
      const char* ts = active ? a.txt + a.toff[pair] : nullptr;
      bool okp, okt;
      if (!a.host_seqs) {
        pack_pair_warp32<G, C::kSpanFit>(ps, n, ts, m, active, pw, tw, PS, scratch, lane, gmask, &okp, &okt);
      } else {
        okp = pack_warp32<G, C::SPAN>(ps, n, active, pw, PS, scratch, lane, gmask, false);
        okt = pack_warp32<G, C::SPAN>(ts, m, active, tw, PS, scratch, lane, gmask, false);
      }
      if (active && !(okp && okt)) {
        if (lane == 0) write_result(a, pair, 2, -1, 0, 0);
        active = false;
      }
    }
    __syncwarp();
    const int kf = m - n;
    int s_fin = -1, k_end = kf, h_end = m;
    // End test of a score (every lane of the pair, the same answer): the
    // diagonal nearest kf whose offset reaches an end cell -- the text end
    // (M == m) on kf .. kf + pe, the pattern end (M == n + k) on kf - te ..
    // kf - 1 -- the larger k on a tie; kf alone for a global alignment.
    auto reaches_end = [&](const UGeo& g) -> bool {
      const int dmax = max(a.pe, a.te);
      for (int d = 0; d <= dmax; ++d) {
        if (d <= a.pe && kf + d >= g.lo && kf + d < g.lo + g.w &&
            view.getM(Geo{g.lo, g.w, g.base}, kf + d - g.lo) == m) {
          k_end = kf + d;
          h_end = m;
          return true;
        }
        if (d > 0 && d <= a.te && kf - d >= g.lo && kf - d < g.lo + g.w &&
            view.getM(Geo{g.lo, g.w, g.base}, kf - d - g.lo) == m - d) {
          k_end = kf - d;
          h_end = m - d;
          return true;
        }
      }
      return false;
    };
    // The running pairs share the warp's lanes: at each score the cells of
    // all of them are spread over the 32 lanes, pair index fastest (cell
    // (i, j) of the j-th running pair is item i * na + j), so a pair that has
    // finished costs nothing while the others go on.
    unsigned amask = __ballot_sync(FULL, active && lane == 0);
    int na = __popc(amask);
    unsigned inv_na = 0;  // ceil(2^32 / na): item / na by one __umulhi
    auto relist = [&]() {
      if (active && lane == 0)
        W->act[__popc(amask & ((1u << lane32) - 1u))] = (uint32_t)q | (uint32_t)n << 8 | (uint32_t)m << 20;
      inv_na = na > 1 ? 0xffffffffu / (unsigned)na + 1u : 0u;
      __syncwarp();
    };
    if constexpr (!ends_free) {
      // global alignment: score 0 is diagonal 0 alone, one lane per pair
      if (active && lane == 0) {
        const int h0 = extend_diag32(pw, tw, n, m, 0, 0, PS);
        if constexpr (LIN) W->M[q] = (Off)h0;
        else view.put(0, 0, h0, NUL, NUL);
      }
      __syncwarp();
      if (active && kf == 0 && view.getM(Geo{0, 1, 0}, 0) == m) {
        s_fin = 0;
        active = false;
      }
      amask = __ballot_sync(FULL, active && lane == 0);
      na = __popc(amask);
      relist();
    } else {
      relist();
      // score 0: M_0[k] = extend(max(k, 0)) on the first wavefront's
      // diagonals that start inside both sequences
      const UGeo g0 = tab[0];
      const int items = na * g0.w;
      for (int f = lane32; f < items; f += 32) {
        const int i = na > 1 ? (int)__umulhi((unsigned)f, inv_na) : f;
        const uint32_t info = W->act[f - i * na];
        const int r = (int)(info & 0xffu), rn = (int)((info >> 8) & 0xfffu), rm = (int)(info >> 20);
        const int k = g0.lo + i;
        int h = NUL;
        if (k <= rm && -k <= rn) h = extend_diag32(W->pw + r, W->tw + r, rn, rm, k, k > 0 ? k : 0, PS);
        const int c = (g0.base + i) * P + r;
        W->M[c] = (Off)h;
        if constexpr (!LIN) {
          W->I[c] = (Off)NUL;
          W->D[c] = (Off)NUL;
        }
      }
      __syncwarp();
      if (active && reaches_end(g0)) {
        s_fin = 0;
        active = false;
      }
      const unsigned now = __ballot_sync(FULL, active && lane == 0);
      if (now != amask) {
        amask = now;
        na = __popc(amask);
        relist();
      }
    }
    for (int s = 1; s <= s_hi && na > 0; ++s) {
      const UGeo g = tab[s];
      if (!g.ex) continue;
      const SrcRow sx = src_row<P>(geo_of(view, s - pen.x, 1));
      const SrcRow so = src_row<P>(geo_of(view, s - pen.oe, 1));
      const SrcRow se = src_row<P>(geo_of(view, s - pen.e, 2));
      const int row0 = (g.base - g.lo) * P;
      const int items = na * g.w;
      for (int f = lane32; f < items; f += 32) {
        Cell<Off, P, LIN> c;
        c.load(W->M, W->I, W->D, W->act, g.lo, sx, so, se, f, na, inv_na);
        if (c.h >= 0) c.h = extend_diag32(W->pw + c.r, W->tw + c.r, c.n, c.m, c.k, c.h, PS);
        c.store(W->M, W->I, W->D, row0);
      }
      __syncwarp();
      bool done;
      if constexpr (ends_free) done = active && reaches_end(g);
      else done = active && kf >= g.lo && kf < g.lo + g.w && view.getM(Geo{g.lo, g.w, g.base}, kf - g.lo) == m;
      if (done) {
        s_fin = s;
        active = false;
      }
      const unsigned now = __ballot_sync(FULL, active && lane == 0);
      if (now != amask) {
        amask = now;
        na = __popc(amask);
        relist();
      }
    }
    if (lane == 0) {
      if (active) {
        // every stored score was tried: beyond the caller's bound, or beyond
        // what this kernel stores (then the arena kernel takes the pair)
        if (a.s_cap <= s_store) write_result(a, pair, 1, -1, 0, 0);
        else defer_pair(a, pair);
      } else if (s_fin >= 0) {
        if (a.score_only) {
          write_result(a, pair, 0, s_fin * a.g, 0, 0);
        } else {
          const int64_t src = pair * kSlot;
          int nr;
          if constexpr (LIN) {
            LinUView<Off, P> lv{view, n, m, pen.e};
            nr = wfa_backtrace<true>(lv, n, m, pen, s_fin, k_end, h_end, a.runs + src, kSlot);
          } else {
            nr = wfa_backtrace<true>(view, n, m, pen, s_fin, k_end, h_end, a.runs + src, kSlot);
          }
          if (nr == -1) {
            defer_pair(a, pair);  // more runs than a slot holds
          } else if (nr < 0) {
            atomicExch(&a.ctrl->internal_error, 1);
            write_result(a, pair, 0, s_fin * a.g, 0, src);
          } else {
            write_result(a, pair, 0, s_fin * a.g, nr, src);
          }
        }
      }
    }
    __syncwarp();
  }
}

}  // namespace wfa
