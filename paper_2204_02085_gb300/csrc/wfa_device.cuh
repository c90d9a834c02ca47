// wfa_device.cuh -- device building blocks of the batched gap-affine WFA.
//
// The method is the wavefront algorithm (WFA) the paper runs unmodified on
// every read pair (Sec. I).  With offsets h (text position) on diagonals
// k = h - v (v = pattern position), and penalties scaled by
// g = gcd(x, o, e) so that only integer scores s = 0, 1, 2, ... occur:
//
//   I_s[k] = max(M_{s-o-e}[k-1], I_{s-e}[k-1]) + 1        (consumes text)
//   D_s[k] = max(M_{s-o-e}[k+1], D_{s-e}[k+1])            (consumes pattern)
//   M_s[k] = extend(max(M_{s-x}[k] + 1, I_s[k], D_s[k]))
//   M_0[0] = extend(0);   score = g * (first s with M_s[m-n] == m)
//
// A candidate past either sequence end is dropped before the maximum.
// extend() advances h while pattern[h-k] == text[h]; here it compares 32
// bases at a time: XOR of two 2-bit packed 64-bit windows, count leading
// zeros, halve.
//
// A "group" of G lanes (G divides 32) owns one pair; lanes stride over the
// diagonals of a wavefront.  The wavefronts live behind a View: shared
// memory (int16 offsets) for short reads, a slice of a global scratch arena
// (int32 offsets) otherwise.  The backtrace walks the stored wavefronts
// back from the end with the library's tie-break and emits run-length
// CIGAR words, last run first.
#pragma once

#include <cstdint>
#include <climits>

namespace wfa {

// ------------------------------------------------------------------ common

constexpr int kOpM = 0, kOpX = 1, kOpI = 2, kOpD = 3;

// forward-pass outcomes
constexpr int kFwdOk = 0, kFwdLimit = 1, kFwdOverflow = 3;

// missing offset: negative, and stays negative after +1 (offsets are
// bounded by the sequence length, far from these values)
constexpr int kNull16 = -16384;
constexpr int kNull32 = -(1 << 30);

constexpr int kNull8 = -128;

template <typename Off> struct NullOf;
template <> struct NullOf<int8_t> { static constexpr int value = kNull8; };
template <> struct NullOf<int16_t> { static constexpr int value = kNull16; };
template <> struct NullOf<int32_t> { static constexpr int value = kNull32; };

struct ScaledPen {
  int x, oe, e;  // penalties divided by g; oe = o + e
};

__device__ __forceinline__ unsigned group_mask(int G) {
  const unsigned lane = threadIdx.x & 31u;
  return G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(unsigned)(G - 1)));
}

// ------------------------------------------------------------------ packing

// 16 ASCII bytes -> 16 two-bit codes (A0 C1 G2 T3, either case), first byte
// in the top bits.  Bytes with chunk-local index in [lo_b, hi_b) are
// validated; *bad is set if one of them is not A/C/G/T.
__device__ __forceinline__ uint32_t code16(uint4 v, int lo_b, int hi_b, bool* bad) {
  const uint32_t q[4] = {v.x, v.y, v.z, v.w};
  uint32_t code = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t w = q[i];
    // ((b >> 1) ^ (b >> 2)) & 3 maps A,C,G,T and a,c,g,t to 0,1,2,3
    const uint32_t c = ((w >> 1) ^ (w >> 2)) & 0x03030303u;
    const uint32_t u = w & 0xDFDFDFDFu;  // fold case
    const uint32_t ok = __vcmpeq4(u, 0x41414141u) | __vcmpeq4(u, 0x43434343u) |
                        __vcmpeq4(u, 0x47474747u) | __vcmpeq4(u, 0x54545454u);
    // bytes of this quad inside [lo_b, hi_b)
    const int b0 = 4 * i;
    const int lo = max(lo_b - b0, 0), hi = min(hi_b - b0, 4);
    uint32_t in = 0;
    if (hi > lo) in = (hi >= 4 ? 0xffffffffu : ((1u << (8 * hi)) - 1u)) & ~((1u << (8 * lo)) - 1u);
    if (~ok & in) *bad = true;
    const uint32_t p8 = ((c & 3u) << 6) | ((c >> 4) & 0x30u) | ((c >> 14) & 0x0Cu) | ((c >> 24) & 3u);
    code = (code << 8) | p8;
  }
  return code;
}

// Packed word w of the sequence at `seq` (len bases): bases 32w .. 32w+31
// (fewer at the end, zero-filled).  Loads only the 16-byte aligned chunks
// that hold at least one of those bases, so it never touches a chunk
// without a byte of the sequence (a 16-byte aligned chunk never straddles a
// page).
__device__ __forceinline__ uint64_t pack_word(const char* __restrict__ seq, int len, int w, bool* bad) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(seq) + 32u * (uintptr_t)w;
  const int nb = min(32, len - 32 * w);  // bases in this word, >= 1
  const uintptr_t a0 = a & ~(uintptr_t)15;
  const int head = (int)(a - a0);
  const int nch = (head + nb + 15) >> 4;  // 2 or 3 chunks (1 if nb small)
  uint32_t c[3] = {0u, 0u, 0u};
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    if (j < nch) {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(a0 + 16u * j));
      const int lo_b = head - 16 * j, hi_b = head + nb - 16 * j;
      c[j] = code16(v, lo_b, hi_b, bad);
    }
  }
  const int r = 2 * head;  // bits to drop from the front
  const uint32_t hi = __funnelshift_l(c[1], c[0], r);
  const uint32_t lo = __funnelshift_l(c[2], c[1], r);
  uint64_t word = ((uint64_t)hi << 32) | lo;
  if (nb < 32) word &= ~0ull << (64 - 2 * nb);
  return word;
}

// The group packs one sequence into out[0 .. ceil(len/32)] (last word = pad
// 0).  Returns, uniformly across the group, whether every byte is valid.
template <int G>
__device__ __forceinline__ bool pack_seq(const char* __restrict__ seq, int len, uint64_t* out, int lane,
                                         unsigned gmask) {
  const int nwords = (len + 31) >> 5;
  bool bad = false;
  for (int w = lane; w <= nwords; w += G) out[w] = (w < nwords) ? pack_word(seq, len, w, &bad) : 0ull;
  return __any_sync(gmask, bad) == 0;
}

// As pack_seq, but word w goes to out[w * stride] (words of several pairs
// interleaved in shared memory).
template <int G>
__device__ __forceinline__ bool pack_seq_strided(const char* __restrict__ seq, int len, uint64_t* out, int stride,
                                                 int lane, unsigned gmask) {
  const int nwords = (len + 31) >> 5;
  bool bad = false;
  for (int w = lane; w <= nwords; w += G) out[w * stride] = (w < nwords) ? pack_word(seq, len, w, &bad) : 0ull;
  return __any_sync(gmask, bad) == 0;
}

// As pack_seq_strided, into 32-bit words (16 bases each, first base in the
// top bits): 64-bit word w becomes 32-bit words 2w (high half) and 2w + 1.
// Writes ceil(len/32)*2 + 2 words, the last two zero.
template <int G>
__device__ __forceinline__ bool pack_seq_strided32(const char* __restrict__ seq, int len, uint32_t* out, int stride,
                                                   int lane, unsigned gmask) {
  const int nwords = (len + 31) >> 5;
  bool bad = false;
  for (int w = lane; w <= nwords; w += G) {
    const uint64_t v = (w < nwords) ? pack_word(seq, len, w, &bad) : 0ull;
    out[(2 * w) * stride] = (uint32_t)(v >> 32);
    out[(2 * w + 1) * stride] = (uint32_t)v;
  }
  return __any_sync(gmask, bad) == 0;
}

// 16 ASCII bytes -> 16 two-bit codes (first byte in the top bits) and, in
// *bad16, bit i set when byte i is not A/C/G/T in either case.  The check
// rebuilds the upper-case letter of each byte's code (A C G T = 0x41 0x43
// 0x47 0x54 = 0x41 + 2 b0 + 6 b1 + 11 b0 b1 for code bits b1 b0) and
// compares it with the byte folded to upper case.
__device__ __forceinline__ uint32_t code16_bad(uint4 v, uint32_t* bad16) {
  const uint32_t q[4] = {v.x, v.y, v.z, v.w};
  uint32_t code = 0, xs[4], any = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t w = q[i];
    const uint32_t c = ((w >> 1) ^ (w >> 2)) & 0x03030303u;
    const uint32_t b0 = c & 0x01010101u, b1 = (c >> 1) & 0x01010101u;
    const uint32_t f = 0x41414141u + 2u * b0 + 6u * b1 + 11u * (b0 & b1);
    xs[i] = (w & 0xDFDFDFDFu) ^ f;  // zero byte <=> valid
    any |= xs[i];
    code = (code << 8) | ((c * 0x40100401u) >> 24);  // 4 codes, first in the top bits
  }
  uint32_t bad = 0;
  if (any) {  // rare: which bytes are not A/C/G/T
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t x = xs[i];
      const uint32_t hb = ((((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x) >> 7) & 0x01010101u;  // 1 per bad byte
      bad |= ((hb * 0x01020408u) >> 24 & 0xFu) << (4 * i);
    }
  }
  *bad16 = bad;
  return code;
}

// 16-byte asynchronous global -> shared copy (both addresses 16-byte
// aligned) and the wait for all of this thread's copies.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// The span (16-byte aligned chunks) holding the active slots' sequences of
// a warp; `fits`: non-empty and at most span_chunks chunks.  All 32 lanes.
struct WarpSpan {
  unsigned long long base;
  int nch;
  bool fits;
};
__device__ __forceinline__ WarpSpan warp_span(const char* seq, int len, bool active, int span_chunks) {
  constexpr unsigned FULL = 0xffffffffu;
  const unsigned long long a = reinterpret_cast<uintptr_t>(seq);
  unsigned long long lo = active && len > 0 ? a : ~0ull;
  unsigned long long hi = active && len > 0 ? a + (unsigned)len : 0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long l2 = __shfl_xor_sync(FULL, lo, o), h2 = __shfl_xor_sync(FULL, hi, o);
    lo = l2 < lo ? l2 : lo;
    hi = h2 > hi ? h2 : hi;
  }
  WarpSpan w{lo & ~15ull, 0, false};
  if (hi > lo && hi - w.base <= 16ull * span_chunks) {
    w.nch = (int)((hi - w.base + 15) >> 4);
    w.fits = true;
  }
  return w;
}

// Raw span bytes staged at scratch -> (2-bit codes, bad-byte mask) per
// chunk, in place, 32 chunks a round: a round writes its 8-byte entries
// below the raw bytes of the rounds still to come; then the zero sentinel
// entry at nch.  All 32 lanes.
__device__ __forceinline__ void convert_span(uint32_t* scratch, int nch, int lane32) {
  const uint4* raw = reinterpret_cast<const uint4*>(scratch);
  uint2* ent = reinterpret_cast<uint2*>(scratch);
  for (int c0 = 0; c0 < nch; c0 += 32) {
    const int c = c0 + lane32;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (c < nch) v = raw[c];
    __syncwarp();
    if (c < nch) {
      uint32_t b16;
      const uint32_t code = code16_bad(v, &b16);
      ent[c] = make_uint2(code, b16);
    }
  }
  __syncwarp();
  if (lane32 == 0) ent[nch] = make_uint2(0u, 0u);
  __syncwarp();
}

// A slot cuts its words 0 .. ceil(len/16) (the last one zero) from the
// converted span entries; returns whether one of its bytes is bad.
template <int G>
__device__ __forceinline__ bool cut_words(const uint2* ent, unsigned long long base, const char* seq, int len,
                                          uint32_t* out, int stride, int lane) {
  const int nw = (len + 15) >> 4;
  const int off = (int)(reinterpret_cast<uintptr_t>(seq) - base);  // bytes from the span start
  const int c0 = off >> 4, r = (off & 15) << 1;
  bool bad = false;
  for (int j = lane; j <= nw; j += G) {
    uint32_t word = 0u;
    if (j < nw) {
      const uint2 e0 = ent[c0 + j], e1 = ent[c0 + j + 1];
      word = __funnelshift_l(e1.x, e0.x, r);
      const int rem = len - 16 * j;
      if (rem < 16) word &= ~0u << (32 - 2 * rem);
      // bad bytes among this word's 16 (at most 2 chunks)
      const uint32_t m2 = e0.y | (e1.y << 16);
      if (m2) {
        const int nb = min(16, rem);
        const uint32_t in = (nb >= 16 ? 0xFFFFu : ((1u << nb) - 1u)) << (off & 15);
        if (m2 & in) bad = true;
      }
    }
    out[j * stride] = word;
  }
  return bad;
}

// A slot reads its own chunks (the span is too wide or not staged).
template <int G>
__device__ __forceinline__ bool pack_slot_direct(const char* seq, int len, uint32_t* out, int stride, int lane) {
  const unsigned long long a = reinterpret_cast<uintptr_t>(seq);
  const int nw = (len + 15) >> 4;
  bool bad = false;
  for (int j = lane; j <= nw; j += G) {
    uint32_t word = 0u;
    if (j < nw) {
      // the 16 bytes of word j span at most two aligned chunks
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
    out[j * stride] = word;
  }
  return bad;
}

// Warp-cooperative packing of one sequence per pair slot of a warp (P pair
// slots of G lanes).  When the active slots' sequences lie in one span of at
// most 16 * SPAN_CHUNKS bytes (aligned 16-byte chunks), the warp copies the
// span once into shared scratch and converts it there to (2-bit codes,
// bad-byte mask) per chunk, and every slot cuts its 32-bit words (16 bases,
// first base in the top bits) from that; otherwise every slot reads its own
// chunks.  Slot q writes words 0 .. ceil(len/16) (the last one zero) to
// out[j * stride].  scratch: 16 * SPAN_CHUNKS bytes, 16-byte aligned.
// async_copy: stage the span with asynchronous copies (device memory) rather
// than plain loads (host memory read over the link).
// Returns, per slot, whether every byte of its sequence is A/C/G/T.  All 32
// lanes call it.
template <int G>
__device__ __forceinline__ bool pack_span_warp32(const WarpSpan& sp, const char* seq, int len, bool active,
                                                 uint32_t* out, int stride, uint32_t* scratch, int lane,
                                                 unsigned gmask, bool async_copy) {
  const int lane32 = threadIdx.x & 31;
  bool bad = false;
  if (sp.fits) {
    if (async_copy) {
      // device memory: every chunk copied to shared memory asynchronously
      // (all loads in flight at once), then converted in place
      for (int c = lane32; c < sp.nch; c += 32)
        cp_async16(scratch + 4 * c, reinterpret_cast<const void*>(sp.base + 16ull * c));
      cp_async_wait_all();
      __syncwarp();
      convert_span(scratch, sp.nch, lane32);
    } else {
      // page-locked host memory read in place: plain coalesced loads (the
      // asynchronous copies measured slower over the host link)
      uint2* ent = reinterpret_cast<uint2*>(scratch);
      for (int c = lane32; c < sp.nch; c += 32) {
        uint32_t b16;
        const uint32_t code = code16_bad(__ldg(reinterpret_cast<const uint4*>(sp.base + 16ull * c)), &b16);
        ent[c] = make_uint2(code, b16);
      }
      __syncwarp();
      if (lane32 == 0) ent[sp.nch] = make_uint2(0u, 0u);
      __syncwarp();
    }
    if (active) bad = cut_words<G>(reinterpret_cast<const uint2*>(scratch), sp.base, seq, len, out, stride, lane);
    __syncwarp();
  } else if (active) {
    bad = pack_slot_direct<G>(seq, len, out, stride, lane);
  }
  return __any_sync(gmask, bad) == 0;
}

template <int G, int SPAN_CHUNKS>
__device__ __forceinline__ bool pack_warp32(const char* seq, int len, bool active, uint32_t* out, int stride,
                                            uint32_t* scratch, int lane, unsigned gmask, bool async_copy) {
  return pack_span_warp32<G>(warp_span(seq, len, active, SPAN_CHUNKS), seq, len, active, out, stride, scratch,
                             lane, gmask, async_copy);
}

// Both sequences of the warp's pairs (device memory): when the pattern span
// and the text span fit the scratch together, one round of asynchronous
// copies stages both (one wait instead of two), else one sequence after the
// other.  Sets *okp / *okt per slot as pack_warp32 returns.
template <int G, int SCRATCH_CHUNKS>
__device__ __forceinline__ void pack_pair_warp32(const char* pseq, int n, const char* tseq, int m, bool active,
                                                 uint32_t* pout, uint32_t* tout, int stride, uint32_t* scratch,
                                                 int lane, unsigned gmask, bool* okp, bool* okt) {
  const int lane32 = threadIdx.x & 31;
  const WarpSpan sp = warp_span(pseq, n, active, SCRATCH_CHUNKS);
  const WarpSpan st = warp_span(tseq, m, active, SCRATCH_CHUNKS);
  if (sp.fits && st.fits && sp.nch + st.nch <= SCRATCH_CHUNKS) {
    uint32_t* tscr = scratch + 4 * sp.nch;  // the text span's raw bytes after the pattern's
    for (int c = lane32; c < sp.nch; c += 32)
      cp_async16(scratch + 4 * c, reinterpret_cast<const void*>(sp.base + 16ull * c));
    for (int c = lane32; c < st.nch; c += 32)
      cp_async16(tscr + 4 * c, reinterpret_cast<const void*>(st.base + 16ull * c));
    cp_async_wait_all();
    __syncwarp();
    // the pattern's entries stay below its own raw bytes, so below the text's
    convert_span(scratch, sp.nch, lane32);
    convert_span(tscr, st.nch, lane32);
    bool badp = false, badt = false;
    if (active) {
      badp = cut_words<G>(reinterpret_cast<const uint2*>(scratch), sp.base, pseq, n, pout, stride, lane);
      badt = cut_words<G>(reinterpret_cast<const uint2*>(tscr), st.base, tseq, m, tout, stride, lane);
    }
    __syncwarp();
    *okp = __any_sync(gmask, badp) == 0;
    *okt = __any_sync(gmask, badt) == 0;
  } else {
    *okp = pack_span_warp32<G>(sp, pseq, n, active, pout, stride, scratch, lane, gmask, true);
    *okt = pack_span_warp32<G>(st, tseq, m, active, tout, stride, scratch, lane, gmask, true);
  }
}

// ----------------------------------------------------------------- extend

// 16 bases starting at base position pos of a sequence packed into 32-bit
// words stored every `stride` elements (reads words pos/16 and pos/16 + 1).
__device__ __forceinline__ uint32_t window32s(const uint32_t* W, int pos, int stride) {
  const int j = pos >> 4;
  return __funnelshift_l(W[(j + 1) * stride], W[j * stride], (pos & 15) << 1);
}

// extend_diag over 32-bit packed words: 16 bases per compare.
__device__ __forceinline__ int extend_diag32(const uint32_t* pw, const uint32_t* tw, int n, int m, int k, int h,
                                             int stride) {
  for (;;) {
    const int v = h - k;
    const int rem = min(n - v, m - h);
    if (rem <= 0) break;
    const uint32_t d = window32s(pw, v, stride) ^ window32s(tw, h, stride);
    const int eq = __clz(d) >> 1;  // 16 when the windows are equal
    if (eq >= rem) {
      h += rem;
      break;
    }
    h += eq;
    if (eq < 16) break;
  }
  return h;
}

// 32 bases starting at base position pos of a packed sequence (reads words
// pos/32 and pos/32 + 1; the pad word makes the second one exist).
__device__ __forceinline__ uint64_t window64(const uint64_t* W, int pos) {
  const int w = pos >> 5;
  const int sh = (pos & 31) << 1;
  const uint64_t a = W[w], b = W[w + 1];
  return (a << sh) | ((b >> 1) >> (63 - sh));
}

// window64 over words stored every `stride` elements
__device__ __forceinline__ uint64_t window64s(const uint64_t* W, int pos, int stride) {
  const int w = pos >> 5;
  const int sh = (pos & 31) << 1;
  const uint64_t a = W[w * stride], b = W[(w + 1) * stride];
  return (a << sh) | ((b >> 1) >> (63 - sh));
}

// Advance offset h on diagonal k while pattern[h-k] == text[h]; h is a
// valid offset (0 <= h <= m, 0 <= h-k <= n).  Packed words are read every
// `stride` elements.
__device__ __forceinline__ int extend_diag(const uint64_t* pw, const uint64_t* tw, int n, int m, int k, int h,
                                           int stride = 1) {
  for (;;) {
    const int v = h - k;
    const int rem = min(n - v, m - h);
    if (rem <= 0) break;
    const uint64_t d = window64s(pw, v, stride) ^ window64s(tw, h, stride);
    const int eq = d ? (__clzll(d) >> 1) : 32;
    if (eq >= rem) {
      h += rem;
      break;
    }
    h += eq;
    if (eq < 32) break;
  }
  return h;
}

// ------------------------------------------------------------------ views

// Geometry of one stored wavefront: diagonals [lo, lo + w), cells at `base`
// (w == 0: component absent).
struct Geo {
  int lo, w, base;
};

// Shared-memory wavefronts: int16 offsets, per-score metadata arrays.
struct SmemView {
  using Off = int16_t;
  int16_t *M, *I, *D;            // cells [cell_cap]
  int16_t *lo, *hi, *base;       // per score [score_cap + 1]
  uint8_t* ex;                   // per score: bit0 M, bit1 I, bit2 D exist
  int cell_cap, score_cap;

  __device__ __forceinline__ int lo_of(int s) const { return lo[s]; }
  __device__ __forceinline__ int hi_of(int s) const { return hi[s]; }
  __device__ __forceinline__ int base_of(int s) const { return base[s]; }
  __device__ __forceinline__ int ex_of(int s) const { return ex[s]; }
  __device__ __forceinline__ void set_meta(int s, int l, int h, int b, int e) {
    lo[s] = (int16_t)l; hi[s] = (int16_t)h; base[s] = (int16_t)b; ex[s] = (uint8_t)e;
  }
  __device__ __forceinline__ void set_absent(int s) { ex[s] = 0; }
  // room for the metadata of score s
  __device__ __forceinline__ bool score_ok(int s, int top) const { (void)top; return s <= score_cap; }
  // reserve `w` cells for score s; `top` counts cells in use
  __device__ __forceinline__ bool alloc(int s, int w, int& top, int& b) const {
    if (s > score_cap || top + w > cell_cap) return false;
    b = top;
    top += w;
    return true;
  }
  __device__ __forceinline__ void release(int b, int& top) const { top = b; }
  __device__ __forceinline__ int getM(const Geo& g, int i) const { return M[g.base + i]; }
  __device__ __forceinline__ int getI(const Geo& g, int i) const { return I[g.base + i]; }
  __device__ __forceinline__ int getD(const Geo& g, int i) const { return D[g.base + i]; }
  __device__ __forceinline__ void put(int b, int w, int i, int mv, int iv, int dv) {
    (void)w;
    M[b + i] = (int16_t)mv; I[b + i] = (int16_t)iv; D[b + i] = (int16_t)dv;
  }
};

// Arena wavefronts: int32 offsets.  Per-score metadata (4 ints: lo, hi,
// base, exist bits) grows up from `meta`; each wavefront's block
// [M w][I w][D w] grows down from `end`; `base` counts ints from `end` to
// the block start.  The two meet at `cap_ints`.
struct ArenaView {
  using Off = int32_t;
  int32_t* meta;
  int32_t* end;
  long cap_ints;

  __device__ __forceinline__ int lo_of(int s) const { return meta[4 * s]; }
  __device__ __forceinline__ int hi_of(int s) const { return meta[4 * s + 1]; }
  __device__ __forceinline__ int base_of(int s) const { return meta[4 * s + 2]; }
  __device__ __forceinline__ int ex_of(int s) const { return meta[4 * s + 3]; }
  __device__ __forceinline__ void set_meta(int s, int l, int h, int b, int e) {
    meta[4 * s] = l; meta[4 * s + 1] = h; meta[4 * s + 2] = b; meta[4 * s + 3] = e;
  }
  __device__ __forceinline__ void set_absent(int s) { meta[4 * s + 3] = 0; }
  __device__ __forceinline__ bool score_ok(int s, int top) const { return 4L * (s + 1) + (long)top <= cap_ints; }
  __device__ __forceinline__ bool alloc(int s, int w, int& top, int& b) const {
    const long need = 4L * (s + 1) + (long)top + 3L * w;
    if (need > cap_ints || (long)top + 3L * w > INT_MAX) return false;
    top += 3 * w;
    b = top;
    return true;
  }
  __device__ __forceinline__ void release(int b, int& top) const { (void)b; (void)top; }
  __device__ __forceinline__ const int32_t* blk(const Geo& g) const { return end - g.base; }
  __device__ __forceinline__ int getM(const Geo& g, int i) const { return blk(g)[i]; }
  __device__ __forceinline__ int getI(const Geo& g, int i) const { return blk(g)[g.w + i]; }
  __device__ __forceinline__ int getD(const Geo& g, int i) const { return blk(g)[2 * g.w + i]; }
  __device__ __forceinline__ void put(int b, int w, int i, int mv, int iv, int dv) {
    int32_t* p = end - b;
    p[i] = mv; p[w + i] = iv; p[2 * w + i] = dv;
  }
};

// Uniform geometry: without trimming to the sequence ends, the diagonal
// range of every wavefront depends only on the (scaled) penalties, so one
// table serves every pair of a launch.  ex: bit0 M exists, bit1 I and D
// exist (they always exist together); base: first cell of the wavefront in a
// pair's store.
struct __align__(8) UGeo {
  int16_t lo, w, base;
  uint8_t ex, pad;
};

// Fill tab[0..scap] for penalties p and a first wavefront on diagonals
// lo0 .. hi0; wavefronts whose cells would pass cellcap are marked absent
// and the last storable score is returned (-1: not even the first).
// constexpr: the lane-per-pair kernel also builds its table at compile time.
__host__ __device__ constexpr int build_ugeo(UGeo* tab, int scap, int cellcap, ScaledPen p, int lo0 = 0,
                                            int hi0 = 0) {
  int top = 0, last = scap;
  for (int s = 0; s <= scap; ++s) {
    UGeo g{0, 0, 0, 0, 0};
    int lo = 1 << 14, hi = -(1 << 14);
    bool exM = false, exG = false;
    if (s == 0) {
      exM = true;  // diagonals lo0 .. hi0: the free starts (0 .. 0: global)
      lo = lo0;
      hi = hi0;
    } else {
      const bool eX = s - p.x >= 0 && (tab[s - p.x].ex & 1);
      const bool eO = s - p.oe >= 0 && (tab[s - p.oe].ex & 1);
      const bool eE = s - p.e >= 0 && (tab[s - p.e].ex & 2);
      exG = eO || eE;
      exM = eX || exG;
      if (eX) {
        const int l = tab[s - p.x].lo, h = tab[s - p.x].lo + tab[s - p.x].w - 1;
        lo = l < lo ? l : lo;
        hi = h > hi ? h : hi;
      }
      if (eO) {
        const int l = tab[s - p.oe].lo - 1, h = tab[s - p.oe].lo + tab[s - p.oe].w;
        lo = l < lo ? l : lo;
        hi = h > hi ? h : hi;
      }
      if (eE) {
        const int l = tab[s - p.e].lo - 1, h = tab[s - p.e].lo + tab[s - p.e].w;
        lo = l < lo ? l : lo;
        hi = h > hi ? h : hi;
      }
    }
    if (exM) {
      const int w = hi - lo + 1;
      if (top + w > cellcap) {
        last = s - 1;
        for (int r = s; r <= scap; ++r) tab[r] = UGeo{0, 0, 0, 0, 0};
        break;
      }
      g.lo = (int16_t)lo;
      g.w = (int16_t)w;
      g.base = (int16_t)top;
      g.ex = (uint8_t)(1 | (exG ? 2 : 0));
      top += w;
    }
    tab[s] = g;
  }
  return last;
}

// View over a warp's interleaved shared-memory store: cell c of the warp's
// pair slot p at [c * P + p]; geometry from the shared table.
template <typename OffT, int P>
struct UView {
  using Off = OffT;
  const UGeo* tab;
  OffT *M, *I, *D;
  int p;
  __device__ __forceinline__ int lo_of(int s) const { return tab[s].lo; }
  __device__ __forceinline__ int hi_of(int s) const { return tab[s].lo + tab[s].w - 1; }
  __device__ __forceinline__ int base_of(int s) const { return tab[s].base; }
  __device__ __forceinline__ int ex_of(int s) const { return tab[s].ex & 2 ? 7 : tab[s].ex; }
  __device__ __forceinline__ int getM(const Geo& g, int i) const { return M[(g.base + i) * P + p]; }
  __device__ __forceinline__ int getI(const Geo& g, int i) const { return I[(g.base + i) * P + p]; }
  __device__ __forceinline__ int getD(const Geo& g, int i) const { return D[(g.base + i) * P + p]; }
  __device__ __forceinline__ void put(int b, int i, int mv, int iv, int dv) {
    M[(b + i) * P + p] = (OffT)mv; I[(b + i) * P + p] = (OffT)iv; D[(b + i) * P + p] = (OffT)dv;
  }
};

// geometry of component `bit` of stored score s (w = 0 if absent)
template <class V>
__device__ __forceinline__ Geo geo_of(const V& view, int s, int bit) {
  Geo g{0, 0, 0};
  if (s >= 0) {
    const int e = view.ex_of(s);
    if (e & bit) {
      g.lo = view.lo_of(s);
      g.w = view.hi_of(s) - g.lo + 1;
      g.base = view.base_of(s);
    }
  }
  return g;
}

// The same for the short kernel's store: one 8-byte load of the table entry.
template <typename OffT, int P>
__device__ __forceinline__ Geo geo_of(const UView<OffT, P>& view, int s, int bit) {
  Geo g{0, 0, 0};
  if (s >= 0) {
    const UGeo t = view.tab[s];
    const int e = t.ex & 2 ? 7 : t.ex;
    if (e & bit) {
      g.lo = t.lo;
      g.w = t.w;
      g.base = t.base;
    }
  }
  return g;
}

template <class V, int WHICH>
__device__ __forceinline__ int get_off(const V& view, const Geo& g, int k, int null_v) {
  const unsigned i = (unsigned)(k - g.lo);
  if (i >= (unsigned)g.w) return null_v;
  return WHICH == 0 ? view.getM(g, (int)i) : WHICH == 1 ? view.getI(g, (int)i) : view.getD(g, (int)i);
}

// ------------------------------------------------------------ forward pass

// Runs the score loop for one pair on a group of G lanes.  Returns kFwdOk
// with *s_out = scaled score, kFwdLimit when the scaled score would exceed
// s_cap (the caller's max_score bound), or kFwdOverflow when the view runs
// out of room.  Every lane returns the same value.
template <int G, class V>
__device__ int wfa_forward(V& view, const uint64_t* pw, const uint64_t* tw, int n, int m, ScaledPen p, int s_cap,
                           int lane, unsigned gmask, int* s_out) {
  using Off = typename V::Off;
  constexpr int NUL = NullOf<Off>::value;
  const int kf = m - n;
  int top = 0, b0 = 0;
  if (!view.alloc(0, 1, top, b0)) return kFwdOverflow;
  if (lane == 0) {
    const int h = extend_diag(pw, tw, n, m, 0, 0);
    view.put(b0, 1, 0, h, NUL, NUL);
    view.set_meta(0, 0, 0, b0, 1);
  }
  __syncwarp(gmask);
  if (kf == 0 && view.getM(Geo{0, 1, b0}, 0) == m) {
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
    lo = max(lo, -n);  // diagonals outside [-n, m] hold no valid offset
    hi = min(hi, m);
    if (lo > hi) {
      if (lane == 0) view.set_absent(s);
      __syncwarp(gmask);
      continue;
    }
    const int w = hi - lo + 1;
    int b = 0;
    if (!view.alloc(s, w, top, b)) return kFwdOverflow;
    bool anyM = false, anyI = false, anyD = false;
    for (int k = lo + lane; k <= hi; k += G) {
      const int mx = get_off<V, 0>(view, gx, k, NUL);
      const int ml = get_off<V, 0>(view, go, k - 1, NUL);
      const int mr = get_off<V, 0>(view, go, k + 1, NUL);
      const int il = get_off<V, 1>(view, gi, k - 1, NUL);
      const int dr = get_off<V, 2>(view, gd, k + 1, NUL);
      int iv = max(ml, il) + 1;
      if (iv < 0 || iv > m) iv = NUL;
      int dv = max(mr, dr);
      if (dv < 0 || dv - k > n) dv = NUL;
      int xv = mx + 1;
      if (mx < 0 || xv > m || xv - k > n) xv = NUL;
      int mv = max(xv, max(iv, dv));
      if (mv >= 0) {
        mv = extend_diag(pw, tw, n, m, k, mv);
        anyM = true;
      } else {
        mv = NUL;
      }
      anyI |= iv >= 0;
      anyD |= dv >= 0;
      view.put(b, w, k - lo, mv, iv, dv);
    }
    const int exbits = (__any_sync(gmask, anyM) ? 1 : 0) | (__any_sync(gmask, anyI) ? 2 : 0) |
                       (__any_sync(gmask, anyD) ? 4 : 0);
    if (exbits == 0) view.release(b, top);
    if (lane == 0) view.set_meta(s, lo, hi, b, exbits);
    __syncwarp(gmask);
    if ((exbits & 1) && kf >= lo && kf <= hi && view.getM(Geo{lo, w, b}, kf - lo) == m) {
      *s_out = s;
      return kFwdOk;
    }
  }
}

// -------------------------------------------------------------- backtrace

// I_s[k] and D_s[k] as the backtrace reads them (null past the stored
// range); views that do not store I and D overload these.
template <class V>
__device__ __forceinline__ int bt_I(const V& view, int s, int k) {
  return get_off<V, 1>(view, geo_of(view, s, 2), k, NullOf<typename V::Off>::value);
}
template <class V>
__device__ __forceinline__ int bt_D(const V& view, int s, int k) {
  return get_off<V, 2>(view, geo_of(view, s, 4), k, NullOf<typename V::Off>::value);
}

// Walk back from the end cell (M, s_final, k_end, h_end) -- (m-n, m) for a
// global alignment -- and write run-length CIGAR words into runs[0 ..), LAST
// run first.  Under ends-free alignment the characters past the end cell
// come out first (D run if k_end > m-n, I run if k_end < m-n), and the walk
// stops at score 0 on any diagonal k of the first wavefront: matches back to
// the free start (0, k) or (-k, 0), then its skipped prefix (I or D run).
// Returns the number of runs, -1 if more than cap runs are needed, -2 if the
// stored wavefronts are inconsistent (which the forward pass never
// produces).  Single lane.
template <bool CONVERGENT = false, class V>
__device__ int wfa_backtrace(const V& view, int n, int m, ScaledPen p, int s_final, int k_end, int h_end,
                             uint32_t* runs, int cap) {
  using Off = typename V::Off;
  constexpr int NUL = NullOf<Off>::value;
  int s = s_final, k = k_end, h = h_end, state = kOpM;
  uint32_t cur_op = 0xF, cur_len = 0;
  int nr = 0;
  long guard = 2L * ((long)n + (long)m) + 4;
  bool over = false;
  auto emit = [&](uint32_t op, uint32_t len) {
    if (len == 0) return;
    if (op == cur_op) {
      cur_len += len;
      return;
    }
    if (cur_len) {
      if (nr < cap) runs[nr] = (cur_len << 4) | cur_op; else over = true;
      ++nr;
    }
    cur_op = op;
    cur_len = len;
  };
  // free end: the characters past the end cell
  if (k_end > m - n) emit(kOpD, (uint32_t)(k_end - (m - n)));
  if (k_end < m - n) emit(kOpI, (uint32_t)((m - n) - k_end));
  while (guard-- > 0) {
    if (s < 0) return -2;
    const bool in_m = state == kOpM;
    if (in_m && s == 0) {
      // a start on diagonal k: (0, k) or (-k, 0), then matches to h
      const int h0 = k > 0 ? k : 0;
      if (h < h0 || k > m || -k > n) return -2;
      emit(kOpM, (uint32_t)(h - h0));
      if (k > 0) emit(kOpI, (uint32_t)k);
      if (k < 0) emit(kOpD, (uint32_t)(-k));
      break;
    }
    // CONVERGENT (lanes of a warp walking different pairs): every state
    // reads the same three cells, so the lanes stay together -- state M its
    // mismatch, insertion and deletion candidates M_{s-x}[k], I_s[k],
    // D_s[k]; state I the extension test's I_{s-e}[k-1]; state D its
    // D_{s-e}[k+1].  Otherwise (one thread) each state reads only its own.
    int xv = NUL, iv = NUL, dv = NUL;
    if (CONVERGENT || in_m) xv = get_off<V, 0>(view, geo_of(view, in_m ? s - p.x : -1, 1), k, NUL);
    if (CONVERGENT || state != kOpD) iv = bt_I(view, in_m ? s : s - p.e, in_m ? k : k - 1);
    if (CONVERGENT || state != kOpI) dv = bt_D(view, in_m ? s : s - p.e, in_m ? k : k + 1);
    if (in_m) {
      if (xv >= 0) {
        xv += 1;
        if (xv > m || xv - k > n) xv = NUL;
      } else {
        xv = NUL;
      }
      int pick, c;
      if (xv >= 0 && xv >= iv && xv >= dv) {
        pick = kOpX; c = xv;
      } else if (iv >= 0 && iv >= dv) {
        pick = kOpI; c = iv;
      } else if (dv >= 0) {
        pick = kOpD; c = dv;
      } else {
        return -2;
      }
      if (c > h) return -2;
      emit(kOpM, (uint32_t)(h - c));
      if (pick == kOpX) {
        emit(kOpX, 1);
        s -= p.x;
        h = c - 1;
      } else {
        state = pick;
        h = c;
      }
    } else if (state == kOpI) {
      emit(kOpI, 1);
      if (iv == h - 1) {  // extend before open
        s -= p.e;
      } else {
        s -= p.oe;
        state = kOpM;
      }
      k -= 1;
      h -= 1;
    } else {
      emit(kOpD, 1);
      if (dv == h) {
        s -= p.e;
      } else {
        s -= p.oe;
        state = kOpM;
      }
      k += 1;
    }
  }
  if (guard < 0) return -2;
  if (cur_len) {
    if (nr < cap) runs[nr] = (cur_len << 4) | cur_op; else over = true;
    ++nr;
  }
  return over ? -1 : nr;
}

// largest number of CIGAR runs of an alignment of scaled score s
__host__ __device__ __forceinline__ long runs_bound_scaled(long s, int x, int oe) {
  const int mn = x < oe ? x : oe;
  return 2L * (s / mn) + 1 + 2;  // + the free end runs of an ends-free alignment
}

}  // namespace wfa
