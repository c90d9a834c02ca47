// lane_path.cuh -- body of the lane-per-pair short-read kernel: every lane
// of a warp owns one pair, and the warp's 32 pairs advance through the
// scores together over the uniform wavefront geometry.
//
// The recurrences are the gap-affine WFA of the paper's method (Sec. I),
// with penalties scaled by g = gcd(x, o, e):
//
//   I_s[k] = max(M_{s-o-e}[k-1], I_{s-e}[k-1]) + 1
//   D_s[k] = max(M_{s-o-e}[k+1], D_{s-e}[k+1])
//   M_s[k] = extend(max(M_{s-x}[k] + 1, I_s[k], D_s[k]))
//
// Storage, all of it [row][32 lanes] so that a lane only ever touches its
// own bank whatever row it reads:
//
//   * M of every stored score, one byte per cell: u = B_k - h, the distance
//     of the offset h to the end of diagonal k (B_k = min(m, n + k)).  In
//     these terms the sequence-end tests vanish: a mismatch step is u - 1,
//     an insertion min(u_M, u_I) - [k > m - n], a deletion
//     min(u_M, u_D) - [k < m - n] (B_k - B_{k-1} = [k <= m - n]); an offset
//     past the end wraps to a large unsigned value, which every later
//     minimum ignores; extension lowers u by the matches, at most to 0; the
//     end cell is u = 0 on diagonal m - n.
//   * I and D only for the scores the recurrences still read, in place:
//     I_s[k] lives at position k - s/e (row s mod e), where I_{s-e}[k-1]
//     was, and D_s[k] at k + s/e, where D_{s-e}[k+1] was; a cell reads its
//     source and overwrites it with its own value.  Positions never written
//     hold the null offset (lane_layout checks, per penalty set, that every
//     read finds the previous score's value or an unwritten position).
//
//   * two bit streams in cell order (32 cells to a word): whether I_s[k]
//     extended I_{s-e}[k-1] (I_{s-e}[k-1] >= M_{s-o-e}[k-1]; ties extend),
//     and the same for D.  A row's bits collect in two registers and join
//     the streams once the row is done.
//
// The backtrace needs I_s[k] and D_s[k] only on the cells it visits: it
// follows the extension bits from (s, k) along (s - j e, k - j) to the
// opening level J, and I_s[k] = M_{s-Je-o-e}[k-J-1] + 1 + J (null past the
// text end, or when the walk leaves the stored rows); D_s[k] the same
// towards k + j with D_s[k] = M_{s-Je-o-e}[k+J+1].  With M, this is all
// the walk of the method's tie-break needs.
//
// Two forward passes share the packing, the batch loop, the cell loop and
// the backtrace: LaneRunForward reads the geometry of any penalties from a
// table; LaneCtForward<x, o+e, e> has the geometry of one scaled penalty
// set at compile time, so every source row, range and store address of the
// cell loop is a constant.
//
// Extension compares 16 bases a round (XOR of two 2-bit packed windows,
// count leading zeros).  The first round of every cell runs in the cell
// loop; cells whose first 16 bases all matched finish in a second pass in
// which every lane works through its own pending cells one round at a time,
// so a long match on one pair does not hold up the other 31.
#pragma once

#include <type_traits>

#include "launch.h"
#include "short_path.cuh"
#include "wfa_device.cuh"

namespace wfa {

// Layout of the in-place I and D rows for the geometry tab of scores
// 0..last (see LaneGeo): the largest prefix of scores whose wavefronts are
// at most 32 diagonals wide (a lane's pending extensions are a 32-bit mask),
// whose rows fit rw positions, and whose row reads each find the value the
// score e before wrote there (source diagonal inside that score's range) or
// a position no score wrote (null), checked by replaying the writes.
struct LaneLayout {
  int s_store, off_i, off_d, span_i, span_d;
};
__host__ __device__ constexpr LaneLayout lane_layout(const UGeo* tab, int last, int E, int rw) {
  LaneLayout out{-1, 0, 0, 0, 0};
  for (int s = 1; s <= last; ++s)
    if ((tab[s].ex & 1) && tab[s].w > 32) {
      last = s - 1;
      break;
    }
  for (; last >= 0; --last) {
    int mi = 1 << 30, xi = -(1 << 30), md = 1 << 30, xd = -(1 << 30);
    for (int s = 0; s <= last; ++s) {
      if (!(tab[s].ex & 1)) continue;
      const int q = s / E, lo = tab[s].lo, hi = tab[s].lo + tab[s].w - 1;
      mi = lo - q < mi ? lo - q : mi;
      xi = hi - q > xi ? hi - q : xi;
      md = lo + q < md ? lo + q : md;
      xd = hi + q > xd ? hi + q : xd;
    }
    const int span_i = xi - mi + 1, span_d = xd - md + 1, off_i = -mi, off_d = -md;
    if (E * span_i > rw || E * span_d > rw || E * span_i > 64 || E * span_d > 64) continue;
    int wi[64] = {}, wd[64] = {};
    for (int i = 0; i < 64; ++i) wi[i] = wd[i] = -1;
    bool ok = true;
    for (int s = 0; s <= last && ok; ++s) {
      if (!(tab[s].ex & 1)) continue;
      const int q = s / E, r = s % E, lo = tab[s].lo, hi = tab[s].lo + tab[s].w - 1;
      const int prev = s - E;
      const bool has_prev = prev >= 0 && (tab[prev].ex & 1);
      const int plo = has_prev ? tab[prev].lo : 0, phi = has_prev ? tab[prev].lo + tab[prev].w - 1 : -1;
      for (int k = lo; k <= hi && ok; ++k) {
        const int pi = r * span_i + k - q + off_i, pd = r * span_d + k + q + off_d;
        if (s > 0) {
          const int want_i = has_prev && k - 1 >= plo && k - 1 <= phi ? prev : -1;
          const int want_d = has_prev && k + 1 >= plo && k + 1 <= phi ? prev : -1;
          ok = wi[pi] == want_i && wd[pd] == want_d;
        }
      }
      for (int k = lo; k <= hi; ++k) {
        wi[r * span_i + k - q + off_i] = s;
        wd[r * span_d + k + q + off_d] = s;
      }
    }
    if (ok) {
      out = LaneLayout{last, off_i, off_d, span_i, span_d};
      break;
    }
  }
  return out;
}

// The compile-time geometry of the lane-per-pair kernel for scaled
// penalties (X, OE = o + e, E) and a store of CELLS cells, RW row positions.
template <int X, int OE, int E, int CELLS, int RW>
struct LaneCtGeo {
  UGeo tab[32];
  LaneLayout L;
  constexpr LaneCtGeo() : tab{}, L{} {
    const int last = build_ugeo(tab, 31, CELLS, ScaledPen{X, OE, E}, 0, 0);
    L = lane_layout(tab, last, E, RW);
  }
};

// Shared memory of one warp of the lane-per-pair kernel: packed sequences,
// then a region that holds the raw sequence bytes while packing and the
// wavefront store afterwards (M offsets, extension bits, the I and D rows).
template <int LMAX, int CELLS, int RW, int SPAN_BYTES>
struct LaneCfg {
  static_assert(LMAX <= 127, "one-byte offsets");
  static constexpr int NW = LMAX / 16 + 2;  // packed 16-base words a window may touch
  static constexpr int kHBytes = CELLS * 32;
  static constexpr int kXWords = (CELLS + 31) / 32;  // words of each bit stream
  static constexpr int kXBytes = 2 * kXWords * 4 * 32;
  static constexpr int kRowBytes = 2 * RW * 32;
  static constexpr int kStore = kHBytes + kXBytes + kRowBytes;
  static constexpr int kUnion = ((kStore > SPAN_BYTES ? kStore : SPAN_BYTES) + 15) / 16 * 16;
  static constexpr int kSpanFit = kUnion / 16;
  struct WarpShm {
    uint32_t pw[NW * 32];
    uint32_t tw[NW * 32];
    alignas(16) unsigned char u[kUnion];
  };
  static constexpr size_t kTabBytes = (sizeof(UGeo) * 32 + 15) / 16 * 16;
  static constexpr size_t kRowsBytes = sizeof(LaneRow) * 32;  // forward passes that read row records
  static constexpr size_t smem_bytes(int warps, bool rows) {
    return kTabBytes + (rows ? kRowsBytes : 0) + (size_t)warps * sizeof(WarpShm);
  }
};

// One lane's view of its pair and store during the forward pass.
struct LaneSt {
  const uint32_t* pw;  // packed pattern words, word j at pw[j * 32]
  const uint32_t* tw;  // packed text words
  uint8_t* H;          // store cell c at H[c * 32]: u of M_s[k]
  uint32_t* XI;        // I extension bits of cells 32 w .. 32 w + 31 at XI[w * 32]
  uint32_t* XD;        // D extension bits, likewise
  uint32_t ai, ad;     // the bits of the words being filled
  int cnext;           // the next cell to be written (cells run in order)
  uint8_t* IR;         // I row position p at IR[p * 32]
  uint8_t* DR;         // D row position p at DR[p * 32]
  int n, m, kf;
  int s_hi;            // last score to try (store and caller's bound)
  bool active;         // not finished (and a real pair)
  int s_fin;           // scaled score once finished
};

// Matches from pattern position v and text position h, up to 32 (kLaneNW
// packed words at pw[j * 32], tw[j * 32]): the XOR of the two 32-base
// windows in two 32-bit halves, leading zeros halved.  A window's third word
// past the last one (j + 2 = kLaneNW) would hold only positions beyond any
// sequence's end, which no caller counts: the last word stands in for it.
__device__ __forceinline__ int lane_match32(const uint32_t* pw, int v, const uint32_t* tw, int h) {
  const int jp = v >> 4, sp = (v & 15) << 1, jt = h >> 4, st = (h & 15) << 1;
  const uint32_t p1 = pw[(jp + 1) * 32];
  const uint32_t t1 = tw[(jt + 1) * 32];
  const uint32_t p2 = pw[min(jp + 2, kLaneNW - 1) * 32];
  const uint32_t t2 = tw[min(jt + 2, kLaneNW - 1) * 32];
  const uint32_t dh = __funnelshift_l(p1, pw[jp * 32], sp) ^ __funnelshift_l(t1, tw[jt * 32], st);
  const uint32_t dl = __funnelshift_l(p2, p1, sp) ^ __funnelshift_l(t2, t1, st);
  return dh ? (int)(__clz(dh) >> 1) : 16 + (int)(__clz(dl) >> 1);
}

// A lane's remaining extension rounds for the cells of one score whose first
// 16 bases matched (bit i: item i); each pass of the loop runs one round of
// 32 bases on every lane that has a cell left.
__device__ __forceinline__ void lane_pending(LaneSt& st, uint32_t pend, int lo, int base) {
  constexpr unsigned FULL = 0xffffffffu;
  int ci = -1, ck = 0, cb = 0, ch = 0;
  while (__any_sync(FULL, pend != 0 || ci >= 0)) {
    if (ci < 0 && pend) {
      ci = __ffs(pend) - 1;
      pend &= pend - 1;
      ck = lo + ci;
      cb = min(st.m, st.n + ck);
      ch = cb - (int)st.H[(base + ci) * 32];
    }
    if (ci >= 0) {
      const int eq = lane_match32(st.pw, ch - ck, st.tw, ch);
      ch += eq;
      if (eq < 32 || ch >= cb) {
        st.H[(base + ci) * 32] = (uint8_t)(cb - min(ch, cb));
        ci = -1;
      }
    }
  }
}

// The items of a row whose M sources all lie inside their rows: a .. b - 1
// (the mismatch source ax <= i < ax + wx, the k + 1 source
// ao - 1 <= i < ao + wo - 1).
__host__ __device__ constexpr int lane_mid_a(int ax, int ao, int w) {
  const int a = ax > ao - 1 ? ax : ao - 1;
  return a < 0 ? 0 : a > w ? w : a;
}
__host__ __device__ constexpr int lane_mid_b(int ax, int wx, int ao, int wo, int w, int a) {
  const int b = ax + wx < ao + wo - 1 ? ax + wx : ao + wo - 1;
  return (b < w ? b : w) > a ? (b < w ? b : w) : a;
}

// One score's row: the cells of items i = 0 .. w-1 (diagonal lo + i), stored
// at cells base + i.  Sources: row s - x has item i at cell cx + i while
// 0 <= i - ax < wx, row s - o - e likewise (ao, wo, co) for diagonals k - 1
// and k + 1; the I and D rows at positions pi0 + i and pd0 + i.  The items
// a .. b - 1, whose M sources all lie inside their rows (the middle of the
// row), run without range tests.  Then the pending extensions and the end
// test.
__device__ __forceinline__ void lane_row(LaneSt& st, int s, int lo, int w, int base, int ax, int wx, int cx, int ao,
                                         int wo, int co, int pi0, int pd0, int a, int b) {
  const int m = st.m;
  const int t0 = lo - st.kf;  // k - (m - n) at item 0
  const int nk0 = st.n + lo;  // n + k at item 0
  const uint8_t* H = st.H;
  // u of M_{s-o-e} on diagonals k - 1, k (carried) and k + 1 (loaded)
  auto ldo = [&](int item) -> uint32_t {
    return (unsigned)(item - ao) < (unsigned)wo ? (uint32_t)H[(co + item) * 32] : 0xFFu;
  };
  uint32_t oa = ldo(-1), ob = ldo(0);
  uint32_t pend = 0, bitv = 1, im = 0, dm = 0;  // pending extensions, this row's extension bits
  auto cell = [&](int i, auto tested) {
    constexpr bool T = decltype(tested)::value;
    const uint32_t oc = T ? ldo(i + 1) : (uint32_t)H[(co + i + 1) * 32];
    const uint32_t mx = !T ? (uint32_t)H[(cx + i) * 32]
                           : (unsigned)(i - ax) < (unsigned)wx ? (uint32_t)H[(cx + i) * 32] : 0xFFu;
    const uint32_t il = st.IR[(pi0 + i) * 32];  // I_{s-e}[k-1]
    const uint32_t dr = st.DR[(pd0 + i) * 32];  // D_{s-e}[k+1]
    const int t = t0 + i;
    const bool ei = il <= oa, ed = dr <= oc;  // extension (ties extend)
    const uint32_t uI = (ei ? il : oa) - (t > 0 ? 1u : 0u);
    const uint32_t uD = (ed ? dr : oc) - (t < 0 ? 1u : 0u);
    if (ei) im |= bitv;
    if (ed) dm |= bitv;
    bitv <<= 1;
    uint32_t uM = min(mx - 1u, min(uI, uD));
    if (uM < 128u) {
      const int h = min(m, nk0 + i) - (int)uM;
      const uint32_t d = window32s(st.pw, h - (lo + i), 32) ^ window32s(st.tw, h, 32);
      const uint32_t eq = __clz(d) >> 1;
      if (eq == 16u && uM > 16u) pend |= 1u << i;
      uM -= min(eq, uM);
    }
    st.H[(base + i) * 32] = (uint8_t)uM;
    st.IR[(pi0 + i) * 32] = (uint8_t)uI;
    st.DR[(pd0 + i) * 32] = (uint8_t)uD;
    oa = ob;
    ob = oc;
  };
  using Tested = std::integral_constant<bool, true>;
  using Untested = std::integral_constant<bool, false>;
#pragma unroll 1
  for (int i = 0; i < a; ++i) cell(i, Tested{});
#pragma unroll 4
  for (int i = a; i < b; ++i) cell(i, Untested{});
#pragma unroll 1
  for (int i = b; i < w; ++i) cell(i, Tested{});
  // the row's bits join the streams at bit base (cells run in order: the
  // words before hold the earlier rows)
  {
    const int r = base & 31, wi = base >> 5;
    st.ai |= im << r;
    st.ad |= dm << r;
    if (r + w >= 32) {
      st.XI[wi * 32] = st.ai;
      st.XD[wi * 32] = st.ad;
      st.ai = r ? im >> (32 - r) : 0u;
      st.ad = r ? dm >> (32 - r) : 0u;
    }
  }
  st.cnext = base + w;
  lane_pending(st, pend, lo, base);
  if (st.active && (unsigned)(st.kf - lo) < (unsigned)w && H[(base + st.kf - lo) * 32] == 0) {
    st.s_fin = s;
    st.active = false;
  }
}

// Score 0: diagonal 0 alone, u = B_0 - extend(0).
__device__ __forceinline__ void lane_score0(LaneSt& st) {
  const int u0 = st.active ? min(st.m, st.n) - extend_diag32(st.pw, st.tw, st.n, st.m, 0, 0, 32) : 0xFF;
  st.H[0] = (uint8_t)u0;
  st.ai = st.ad = 0;  // cell 0 has no gap
  st.cnext = 1;
  if (st.active && st.kf == 0 && u0 == 0) {
    st.s_fin = 0;
    st.active = false;
  }
}

// Forward pass over the call's row records (any penalties): four 16-byte
// loads a score.
struct LaneRunForward {
  static constexpr bool kRows = true;
  static __device__ __forceinline__ void run(LaneSt& st, const LaneRow* rows) {
    constexpr unsigned FULL = 0xffffffffu;
    lane_score0(st);
    for (int s = 1; s <= st.s_hi && __any_sync(FULL, st.active); ++s) {
      const int4* r = reinterpret_cast<const int4*>(rows + s);
      const int4 r0 = r[0], r1 = r[1], r2 = r[2], r3 = r[3];
      if (!r3.y) continue;  // no M wavefront at this score
      lane_row(st, s, r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w, r2.x, r2.y, r2.z, r2.w, r3.x);
    }
  }
};

// Forward pass with the geometry of scaled penalties (X, OE, E) known at
// compile time.
template <int X, int OE, int E, int CELLS, int RW>
struct LaneCtForward {
  static constexpr LaneCtGeo<X, OE, E, CELLS, RW> G{};
  static_assert(G.L.s_store >= 0, "no score fits the store");

  template <int S>
  static __device__ __forceinline__ void score(LaneSt& st) {
    constexpr UGeo g = G.tab[S];
    constexpr bool HXS = S >= X && (G.tab[S >= X ? S - X : 0].ex & 1);
    constexpr UGeo gx = G.tab[S >= X ? S - X : 0];
    constexpr int AX = HXS ? gx.lo - g.lo : 0, WX = HXS ? gx.w : 0, CX = HXS ? gx.base - AX : 0;
    constexpr bool HOS = S >= OE && (G.tab[S >= OE ? S - OE : 0].ex & 1);
    constexpr UGeo go = G.tab[S >= OE ? S - OE : 0];
    constexpr int AO = HOS ? go.lo - g.lo : 0, WO = HOS ? go.w : 0, CO = HOS ? go.base - AO : 0;
    constexpr int Q = S / E, R = S % E;
    constexpr int PI0 = R * G.L.span_i + g.lo - Q + G.L.off_i;
    constexpr int PD0 = R * G.L.span_d + g.lo + Q + G.L.off_d;
    constexpr int A = lane_mid_a(AX, AO, g.w), B = lane_mid_b(AX, WX, AO, WO, g.w, A);
    lane_row(st, S, g.lo, g.w, g.base, AX, WX, CX, AO, WO, CO, PI0, PD0, A, B);
  }

  template <int S>
  static __device__ __forceinline__ void scores(LaneSt& st) {
    if constexpr (S <= G.L.s_store) {
      if (S > st.s_hi || !__any_sync(0xffffffffu, st.active)) return;
      if constexpr ((G.tab[S].ex & 1) != 0) score<S>(st);
      scores<S + 1>(st);
    }
  }

  static constexpr bool kRows = false;
  static __device__ __forceinline__ void run(LaneSt& st, const LaneRow*) {
    lane_score0(st);
    scores<1>(st);
  }
};

// Walk back from (M, s, m - n, m) over the lane's store (cell c: u of M at
// H[c*32], extension bits at bit c mod 32 of XI / XD[(c/32)*32]) and write
// the run-length CIGAR words, last run first.  Returns the number of runs,
// -1 when more than cap are needed, -2 when the store is inconsistent
// (never, for a store the forward pass wrote).
__device__ __forceinline__ int lane_backtrace(const UGeo* tab, const uint8_t* H, const uint32_t* XI,
                                              const uint32_t* XD, int n, int m,
                                              int X, int OE, int E, int s, int k, int h, uint32_t* runs, int cap) {
  uint32_t cur_op = 0xF, cur_len = 0;
  int nr = 0;
  bool over = false, bad = false;
  auto emit = [&](uint32_t op, int len) {
    if (len < 0) bad = true;
    if (len <= 0) return;
    if (op == cur_op) {
      cur_len += (uint32_t)len;
      return;
    }
    if (cur_len) {
      if (nr < cap) runs[nr] = (cur_len << 4) | cur_op;
      else over = true;
      ++nr;
    }
    cur_op = op;
    cur_len = (uint32_t)len;
  };
  const int s_top = s;
  // store cell of (ss, kk), or -1 outside the stored rows
  auto cell = [&](int ss, int kk) -> int {
    if ((unsigned)ss > (unsigned)s_top) return -1;
    const UGeo t = tab[ss];
    const unsigned i = (unsigned)(kk - t.lo);
    return ((t.ex & 1) && i < (unsigned)t.w) ? t.base + (int)i : -1;
  };
  // the offset h of M_ss[kk], or -1 (outside, or null)
  auto mh = [&](int ss, int kk) -> int {
    const int c = cell(ss, kk);
    if (c < 0) return -1;
    const int u = H[c * 32];
    return u < 128 ? min(m, n + kk) - u : -1;
  };
  for (int guard = 2 * s_top + 8; guard > 0 && !bad; --guard) {
    if (s == 0) {
      if (k != 0) bad = true;
      emit(kOpM, h);
      break;
    }
    // the three candidates of M_s[k]: M_{s-x}[k] + 1, and I_s[k], D_s[k]
    // found by following their extension bits (both chains in one loop)
    const int xm = mh(s - X, k);
    int ji = 0, jd = 0;
    bool open_i = false, open_d = false, null_i = false, null_d = false;
    while (!((open_i || null_i) && (open_d || null_d))) {
      if (!(open_i || null_i)) {
        const int c = cell(s - ji * E, k - ji);
        if (c < 0) null_i = true;
        else if ((XI[(c >> 5) * 32] >> (c & 31)) & 1u) ++ji;
        else open_i = true;
      }
      if (!(open_d || null_d)) {
        const int c = cell(s - jd * E, k + jd);
        if (c < 0) null_d = true;
        else if ((XD[(c >> 5) * 32] >> (c & 31)) & 1u) ++jd;
        else open_d = true;
      }
    }
    const int im = null_i ? -1 : mh(s - ji * E - OE, k - ji - 1);
    const int dm = null_d ? -1 : mh(s - jd * E - OE, k + jd + 1);
    const int bk = min(m, n + k);
    const int xv = xm >= 0 && xm + 1 <= bk ? xm + 1 : -1;
    const int iv = im >= 0 && im + 1 + ji <= m ? im + 1 + ji : -1;
    const int dv = dm >= 0 && dm - k <= n ? dm : -1;
    // the largest; ties: mismatch, then insertion, then deletion
    const bool px = xv >= 0 && xv >= iv && xv >= dv;
    const bool pi = !px && iv >= 0 && iv >= dv;
    if (!px && !pi && dv < 0) return -2;
    const int c = px ? xv : pi ? iv : dv;
    const int j = pi ? ji : jd;
    emit(kOpM, h - c);
    emit(px ? kOpX : pi ? kOpI : kOpD, px ? 1 : j + 1);
    s -= px ? X : j * E + OE;
    k += px ? 0 : pi ? -(j + 1) : j + 1;
    h = px ? c - 1 : pi ? c - j - 1 : c;
    if (s < 0) return -2;
  }
  if (bad || s != 0) return -2;
  if (cur_len) {
    if (nr < cap) runs[nr] = (cur_len << 4) | cur_op;
    else over = true;
    ++nr;
  }
  return over ? -1 : nr;
}

// ------------------------------------------------------------ ordering
//
// The warp's 32 pairs run in lockstep until the last of them ends, so a
// warp's cost is set by its highest score.  The ordering pass puts pairs of
// similar score into the same warp: every group of kLaneGroup consecutive
// pairs is packed, each pair gets a cheap upper bound on its scaled score,
// and the group is sorted by it (stable counting sort, in the block).  The
// packed words go out in the sorted order, so the lane kernel reads them
// with coalesced loads and packs nothing itself.

// Largest estimate kept apart; empty slots take it too.
constexpr int kLaneEstMax = 63;

// The furthest offset of diagonal k from offset h (packed words at W[j * 32]):
// 32 bases a round.
__device__ __forceinline__ int lane_extend32(const uint32_t* pw, const uint32_t* tw, int n, int m, int k, int h) {
  for (;;) {
    const int rem = min(n - (h - k), m - h);
    if (rem <= 0) return h;
    const int eq = lane_match32(pw, h - k, tw, h);
    if (eq >= rem) return h + rem;
    h += eq;
    if (eq < 32) return h;
  }
}

// Cost of a greedy alignment, an upper bound on the optimal scaled score,
// followed only up to cap (a higher bound changes nothing: such a pair
// passes the store): from the furthest point of diagonal 0, repeatedly take
// one edit and extend.  A mismatch followed by at least four matches is
// taken at once; otherwise the mismatch, one inserted and one deleted base
// (each priced as a fresh event) are all tried, and the one whose extension
// ends furthest along v + h, less its cost, is taken.  The rest of the
// longer sequence at an end is one gap.  Packed words at pw[j * 32].
__device__ __forceinline__ int lane_estimate(const uint32_t* pw, const uint32_t* tw, int n, int m, int X, int OE,
                                             int E, int cap) {
  int k = 0, h = lane_extend32(pw, tw, n, m, 0, 0), cost = 0;
#pragma unroll 1
  while (cost < cap) {  // every edit costs at least 1
    const int v = h - k;
    if (v >= n || h >= m) {
      const int rem = (n - v) + (m - h);
      return min(cost + (rem > 0 ? OE + E * (rem - 1) : 0), cap);
    }
    const int hx = lane_extend32(pw, tw, n, m, k, h + 1);  // mismatch: v + 1, h + 1
    if (hx - h >= 5 || hx - k >= n || hx >= m) {
      h = hx;
      cost += X;
      continue;
    }
    const int hi = lane_extend32(pw, tw, n, m, k + 1, h + 1);  // insertion: h + 1
    const int hd = lane_extend32(pw, tw, n, m, k - 1, h);      // deletion: v + 1
    // v + h after the extension, less the edit's cost (v = h - k)
    const int gx = 2 * hx - k - X, gi = 2 * hi - (k + 1) - OE, gd = 2 * hd - (k - 1) - OE;
    if (gx >= gi && gx >= gd) {
      h = hx;
      cost += X;
    } else if (gi >= gd) {
      ++k;
      h = hi;
      cost += OE;
    } else {
      --k;
      h = hd;
      cost += OE;
    }
  }
  return cap;
}

// 16 ASCII bytes -> 16 two-bit codes, first byte in the top bits (A C G T
// = 0 1 2 3 in either case: bits 1 and 2 of the byte, XORed), and whether a
// byte is not A/C/G/T: the upper-case letter of each byte's code is picked
// from "ACGT" by a byte permute with the codes as selectors and compared
// with the byte folded to upper case.  Only when some byte differs is the
// per-byte mask (bit i: byte i) worked out.
__device__ __forceinline__ uint32_t lane_code16(uint4 v, uint32_t* bad16) {
  const uint32_t q[4] = {v.x, v.y, v.z, v.w};
  uint32_t code = 0u, xs[4], any = 0u;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t w = q[i];
    const uint32_t c = ((w >> 1) ^ (w >> 2)) & 0x03030303u;  // byte j's code in bits 8j, 8j + 1
    const uint32_t sel = __byte_perm(c | (c >> 4), 0u, 0x4420u);  // nibble j = byte j's code
    xs[i] = (w & 0xDFDFDFDFu) ^ __byte_perm(0x54474341u, 0u, sel);  // zero byte <=> valid
    any |= xs[i];
    code = (code << 8) | ((c * 0x40100401u) >> 24);
  }
  uint32_t bad = 0u;
  if (any) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t x = xs[i];
      const uint32_t hb = ((((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x) >> 7) & 0x01010101u;  // 1 per nonzero byte
      bad |= ((hb * 0x01020408u) >> 24 & 0xFu) << (4 * i);
    }
  }
  *bad16 = bad;
  return code;
}

// One lane packs one sequence of at most 16 * NCH - 15 bases from device
// memory into words 0 .. NCH - 1 (16 bases each, first base in the top bits,
// zero past the end) at out[j * 32]: every aligned 16-byte chunk holding a
// base is loaded at once, then the words are cut from the chunks' 2-bit
// codes.  Returns whether a byte of the sequence is not A/C/G/T.
template <int NCH>
__device__ __forceinline__ bool lane_pack_direct(const char* seq, int len, uint32_t* out) {
  const unsigned long long a0 = reinterpret_cast<uintptr_t>(seq), b0 = a0 & ~15ull;
  const int h = (int)(a0 - b0);
  const int nch = (h + len + 15) >> 4;
  uint4 raw[NCH];
#pragma unroll
  for (int c = 0; c < NCH; ++c)  // all loads first: their latencies overlap
    raw[c] = c < nch ? __ldg(reinterpret_cast<const uint4*>(b0 + 16ull * c)) : make_uint4(0u, 0u, 0u, 0u);
  uint32_t code[NCH + 1], bad[NCH + 1];
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    code[c] = 0u;
    bad[c] = 0u;
    if (c < nch) code[c] = lane_code16(raw[c], &bad[c]);
  }
  code[NCH] = 0u;
  bad[NCH] = 0u;
  const int nw = (len + 15) >> 4;
  bool any_bad = false;
#pragma unroll
  for (int j = 0; j < NCH; ++j) {
    uint32_t word = 0u;
    if (j < nw) {
      const int rem = min(16, len - 16 * j);
      word = __funnelshift_l(code[j + 1], code[j], 2 * h);
      if (rem < 16) word &= ~0u << (32 - 2 * rem);
      const uint32_t in = (rem >= 16 ? 0xFFFFu : ((1u << rem) - 1u)) << h;  // the word's bytes in chunks j, j + 1
      if ((bad[j] | (bad[j + 1] << 16)) & in) any_bad = true;
    }
    out[j * 32] = word;
  }
  return any_bad;
}

// Shared memory of the ordering pass: per warp the packed words of its 32
// pairs; the per-warp counts of each estimate and each estimate's first slot.
template <int LMAX>
struct LaneOrderShm {
  static constexpr int NW = LMAX / 16 + 2;
  static constexpr int kWarps = kLaneGroup / 32;
  struct Warp {
    uint32_t pw[NW * 32];
    uint32_t tw[NW * 32];
  } w[kWarps];
  int cnt[2][kWarps][kLaneEstMax + 1];  // alternate groups use alternate halves
  int start[kLaneEstMax + 1];
};

// The ordering pass (block of kLaneGroup threads, one per pair of a group;
// sequences in device memory, each lane reading its own pair's aligned
// 16-byte chunks).  est_cap = 0: pack only, every slot keeps its pair's
// place in the group (for stores so small that every warp ends within a few
// scores anyway, where the estimate would cost more than it saves).  Pairs longer than LMAX are deferred and pairs with a
// byte other than A/C/G/T get their status here; both, and the slots past
// the last pair, become empty slots (pair -1) at the end of their group.
template <int LMAX>
__device__ void lane_order_body(const AlignArgs& a, int est_cap, unsigned char* smem) {
  using S_t = LaneOrderShm<LMAX>;
  constexpr int NW = S_t::NW, WG = S_t::kWarps, NK = kLaneEstMax + 1;
  static_assert(NW == kLaneNW, "packed words per sequence");
  static_assert(NK <= 64, "two estimates per lane in the scan");
  constexpr unsigned FULL = 0xffffffffu;
  if (*(volatile int32_t*)&a.ctrl->bad_input) return;  // inputs rejected by the validation kernel
  auto& S = *reinterpret_cast<S_t*>(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto& W = S.w[warp];
  const int64_t groups = (a.n + kLaneGroup - 1) / kLaneGroup;
  for (int i = threadIdx.x; i < 2 * WG * NK; i += kLaneGroup) (&S.cnt[0][0][0])[i] = 0;
  __syncthreads();
  int half = 0;
  for (int64_t gi = blockIdx.x; gi < groups; gi += gridDim.x, half ^= 1) {
    const int64_t pair = gi * kLaneGroup + threadIdx.x;
    bool active = pair < a.n;
    int n = 0, m = 0;
    int64_t po = 0, to = 0;
    if (active) {
      n = a.plen[pair];
      m = a.tlen[pair];
      po = a.poff[pair];  // with the lengths: one round trip for all four
      to = a.toff[pair];
      if (n > LMAX || m > LMAX) {
        defer_pair(a, pair);
        active = false;
      }
    }
    if (active) {
      static_assert(16 * NW - 15 >= LMAX, "chunks of the longest sequence");
      const bool bad = lane_pack_direct<NW>(a.pat + po, n, W.pw + lane) |
                       lane_pack_direct<NW>(a.txt + to, m, W.tw + lane);
      if (bad) {
        write_result(a, pair, 2, -1, 0, 0);
        active = false;
      }
    }
    if (est_cap <= 0) {  // call order (uniform over the launch)
      uint32_t* out = a.lane_words + gi * (2 * NW * kLaneGroup) + threadIdx.x;
#pragma unroll
      for (int j = 0; j < NW; ++j) {
        out[j * kLaneGroup] = active ? W.pw[j * 32 + lane] : 0u;
        out[(NW + j) * kLaneGroup] = active ? W.tw[j * 32 + lane] : 0u;
      }
      a.lane_slots[pair] = make_int2(active ? (int)pair : -1, active ? n | (m << 8) : 0);
      continue;
    }
    const int key = active ? lane_estimate(W.pw + lane, W.tw + lane, n, m, a.xs, a.oes, a.es, est_cap) : kLaneEstMax;
    // stable: a pair's slot follows every pair of a lower estimate and every
    // earlier pair of its own.  This group's counts are in half `half` (zero:
    // cleared while the group before used the other half)
    auto& cnt = S.cnt[half];
    const unsigned same = __match_any_sync(FULL, key);
    const int before = __popc(same & ((1u << lane) - 1u));
    if (before == 0) cnt[warp][key] = __popc(same);
    __syncthreads();
    // every warp is past its reads of the other half (the group before)
    for (int i = threadIdx.x; i < WG * NK; i += kLaneGroup) (&S.cnt[half ^ 1][0][0])[i] = 0;
    if (warp == 0) {
      // lane l: estimates 2l and 2l + 1; each warp's count becomes the count
      // of the warps before it, then each estimate's first slot
      int tot[2] = {0, 0};
      for (int q = 0; q < 2; ++q) {
        const int e = 2 * lane + q;
        if (e >= NK) continue;
        int run = 0;
        for (int w = 0; w < WG; ++w) {
          const int c = cnt[w][e];
          cnt[w][e] = run;
          run += c;
        }
        tot[q] = run;
      }
      const int both = tot[0] + tot[1];
      int incl = both;
      for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += o;
      }
      if (2 * lane < NK) S.start[2 * lane] = incl - both;
      if (2 * lane + 1 < NK) S.start[2 * lane + 1] = incl - both + tot[0];
    }
    __syncthreads();
    const int slot = S.start[key] + cnt[warp][key] + before;
    uint32_t* out = a.lane_words + gi * (2 * NW * kLaneGroup) + slot;
#pragma unroll
    for (int j = 0; j < NW; ++j) {
      out[j * kLaneGroup] = active ? W.pw[j * 32 + lane] : 0u;
      out[(NW + j) * kLaneGroup] = active ? W.tw[j * 32 + lane] : 0u;
    }
    a.lane_slots[gi * kLaneGroup + slot] = make_int2(active ? (int)pair : -1, active ? n | (m << 8) : 0);
    // no barrier here: the next group's first barrier comes after every
    // warp's reads of this group's counts and first slots
  }
}

// The lane-per-pair kernel body (global gap-affine alignment, both sequences
// <= LMAX).  Pairs longer than LMAX, or whose score passes the last stored
// wavefront (but not the caller's max_score), are deferred to the arena
// kernels, as are pairs whose CIGAR needs more than kSlot runs.
template <int LMAX, int CELLS, int RW, int SPAN_BYTES, class Fwd>
__device__ __forceinline__ void lane_body(const AlignArgs& a, const LaneGeo& lg, unsigned char* smem) {
  using C = LaneCfg<LMAX, CELLS, RW, SPAN_BYTES>;
  if (*(volatile int32_t*)&a.ctrl->bad_input) return;  // inputs rejected by the validation kernel
  UGeo* tab = reinterpret_cast<UGeo*>(smem);
  LaneRow* rows = reinterpret_cast<LaneRow*>(smem + C::kTabBytes);  // when Fwd reads them
  for (int i = threadIdx.x; i < 32; i += blockDim.x) tab[i] = lg.tab[i];
  if constexpr (Fwd::kRows)
    for (int i = threadIdx.x; i < 32; i += blockDim.x) rows[i] = lg.rows[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr size_t kHead = C::kTabBytes + (Fwd::kRows ? C::kRowsBytes : 0);
  auto* W = reinterpret_cast<typename C::WarpShm*>(smem + kHead + warp * sizeof(typename C::WarpShm));
  const int s_store = lg.s_store;
  const int X = a.xs, OE = a.oes, E = a.es;
  LaneSt st;
  st.pw = W->pw + lane;
  st.tw = W->tw + lane;
  st.H = W->u + lane;
  st.XI = reinterpret_cast<uint32_t*>(W->u + C::kHBytes) + lane;
  st.XD = st.XI + C::kXWords * 32;
  st.IR = W->u + C::kHBytes + C::kXBytes + lane;
  st.DR = st.IR + RW * 32;
  st.s_hi = min(s_store, a.s_cap);
  const int64_t wpb = blockDim.x >> 5;
  const int64_t stride = (int64_t)gridDim.x * wpb * 32;
  // ordered input: slots of the ordering pass, whole groups, taken by the
  // warps in batches of 32 from a queue (within a group the batches' costs
  // rise with the estimates, so a fixed share would give some warps only
  // the dearest batches); call order: a fixed stride
  const bool ordered = a.lane_slots != nullptr;
  static_assert(C::NW == kLaneNW, "packed words per sequence");
  const int64_t total = ordered ? (a.n + kLaneGroup - 1) / kLaneGroup * kLaneGroup : a.n;
  // ordered input: the next batch's slot and packed words are loaded into
  // registers while the current batch computes
  int64_t next = total;
  int2 nsl = make_int2(-1, 0);
  uint32_t nwd[2 * kLaneNW];
  auto grab = [&]() -> int64_t {
    int b = 0;
    if (lane == 0) b = atomicAdd(&a.ctrl->lane_next, 1);
    return (int64_t)__shfl_sync(0xffffffffu, b, 0) * 32;
  };
  auto fetch = [&](int64_t f) {
    if (f >= total) return;
    nsl = a.lane_slots[f + lane];
    const uint32_t* src = a.lane_words + (f / kLaneGroup) * (2 * kLaneNW * kLaneGroup) + f % kLaneGroup + lane;
#pragma unroll
    for (int j = 0; j < 2 * kLaneNW; ++j) nwd[j] = src[j * kLaneGroup];
  };
  if (ordered) {
    next = grab();
    fetch(next);
  }
  for (int64_t first = ((int64_t)blockIdx.x * wpb + warp) * 32;; first += stride) {
    if (ordered) first = next;
    if (first >= total) break;
    int64_t pair;
    bool active;
    int n = 0, m = 0;
    if (ordered) {
      const int2 sl = nsl;
#pragma unroll
      for (int j = 0; j < kLaneNW; ++j) {
        W->pw[j * 32 + lane] = nwd[j];
        W->tw[j * 32 + lane] = nwd[kLaneNW + j];
      }
      next = grab();
      fetch(next);
      pair = sl.x;
      active = pair >= 0;
      n = sl.y & 255;
      m = sl.y >> 8;
      if (active && s_store < 0) {
        defer_pair(a, pair);
        active = false;
      }
    } else {
      pair = first + lane;
      active = pair < a.n;
      if (active) {
        n = a.plen[pair];
        m = a.tlen[pair];
        if (n > LMAX || m > LMAX || s_store < 0) {
          defer_pair(a, pair);
          active = false;
        }
      }
      // all lanes take part: the warp reads its pairs' sequences together
      uint32_t* scratch = reinterpret_cast<uint32_t*>(W->u);
      const char* ps = active ? a.pat + a.poff[pair] : nullptr;
      const char* ts = active ? a.txt + a.toff[pair] : nullptr;
      const unsigned gm = 1u << lane;
      bool okp, okt;
      if (!a.host_seqs) {
        pack_pair_warp32<1, C::kSpanFit>(ps, n, ts, m, active, W->pw + lane, W->tw + lane, 32, scratch, 0, gm,
                                         &okp, &okt);
      } else {
        okp = pack_warp32<1, C::kSpanFit>(ps, n, active, W->pw + lane, 32, scratch, 0, gm, false);
        okt = pack_warp32<1, C::kSpanFit>(ts, m, active, W->tw + lane, 32, scratch, 0, gm, false);
      }
      if (active && !(okp && okt)) {
        write_result(a, pair, 2, -1, 0, 0);
        active = false;
      }
    }
    const bool real = ordered ? pair >= 0 : pair < a.n;
    __syncwarp();  // the packer's scratch becomes the store
    {
      // the I and D rows start null
      const uint32_t nul = 0xFFFFFFFFu;
      uint4* z = reinterpret_cast<uint4*>(W->u + C::kHBytes + C::kXBytes);
      for (int i = lane; i < C::kRowBytes / 16; i += 32) z[i] = make_uint4(nul, nul, nul, nul);
      __syncwarp();
    }
    if (!active) n = m = 0;  // idle lanes run with empty sequences: every offset stays null
    st.n = n;
    st.m = m;
    st.kf = m - n;
    st.active = active;
    st.s_fin = -1;
    Fwd::run(st, rows);
    if (st.cnext & 31) {  // the last, partly filled words
      st.XI[(st.cnext >> 5) * 32] = st.ai;
      st.XD[(st.cnext >> 5) * 32] = st.ad;
    }
    if (real) {
      if (st.active) {
        // every stored score was tried: beyond the caller's bound, or beyond
        // what this kernel stores (then the arena kernel takes the pair)
        if (a.s_cap <= s_store) write_result(a, pair, 1, -1, 0, 0);
        else defer_pair(a, pair);
      } else if (st.s_fin >= 0) {
        if (a.score_only) {
          write_result(a, pair, 0, st.s_fin * a.g, 0, 0);
        } else {
          const int64_t src = pair * kSlot;
          const int nr = lane_backtrace(tab, st.H, st.XI, st.XD, n, m, X, OE, E, st.s_fin, st.kf, m, a.runs + src, kSlot);
          if (nr == -1) {
            defer_pair(a, pair);  // more runs than a slot holds
          } else if (nr < 0) {
            atomicExch(&a.ctrl->internal_error, 1);
            write_result(a, pair, 0, st.s_fin * a.g, 0, src);
          } else {
            write_result(a, pair, 0, st.s_fin * a.g, nr, src);
          }
        }
      }
    }
    __syncwarp();  // the store is the next batch's packing scratch
  }
}

}  // namespace wfa
