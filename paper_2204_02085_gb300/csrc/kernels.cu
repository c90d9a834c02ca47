// kernels.cu -- the CUDA kernels of libwfa_gpu.so (sm_103a) and their
// launchers.
//
//   short_kernel    fused pack + gap-affine WFA + backtrace for pairs whose
//                   sequences are at most kShortLmax long and whose
//                   wavefronts fit the group's shared memory (the paper's
//                   100 bp workload, Sec. II); everything else is deferred
//   general_kernel  one warp per deferred pair, wavefronts in a slice of the
//                   global scratch arena, pairs taken from a device work
//                   queue (atomic counter)
//   validate/scan/compact/pack  bookkeeping around them
#include <algorithm>
#include <type_traits>
#include <climits>

#include <cstring>

#include "arena_path.cuh"
#include "lane_path.cuh"
#include "launch.h"
#include "short_path.cuh"
#include "wfa_device.cuh"

namespace wfa {

namespace {

// ------------------------------------------------------------ short kernel

template <int G, int LMAX, int CELLS, int SCAP, typename Off, bool LIN, bool EF>
__global__ void __launch_bounds__(kShortBlock, 8) short_kernel(const AlignArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_last;
  short_body<G, LMAX, CELLS, SCAP, Off, LIN, EF>(a, smem, &s_last);
}

// One lane per pair, the warp's pairs in lockstep (lane_path.cuh); Fwd is
// the forward pass: geometry from the table (any penalties) or fixed at
// compile time (one scaled penalty set).
template <int LMAX, int CELLS, int RW, int SPAN, int WPB, class Fwd>
__global__ void __launch_bounds__(32 * WPB) lane_kernel(const AlignArgs a, const LaneGeo g) {
  extern __shared__ __align__(16) unsigned char smem[];
  lane_body<LMAX, CELLS, RW, SPAN, Fwd>(a, g, smem);
}
// One large block per SM: its warps fill the shared memory that blocks of a
// few warps leave unused (the 197-cell store: 17 warps in one block where
// 2-warp blocks fit 16), and the explicit minimum of one block keeps the
// compiler from capping its registers for more blocks.
template <int LMAX, int CELLS, int RW, int SPAN, int WPB, class Fwd>
__global__ void __launch_bounds__(32 * WPB, 1) lane_kernel_wide(const AlignArgs a, const LaneGeo g) {
  extern __shared__ __align__(16) unsigned char smem[];
  lane_body<LMAX, CELLS, RW, SPAN, Fwd>(a, g, smem);
}

// The lane kernel's ordering pass: a block per group of kLaneGroup pairs
// (lane_path.cuh).
template <int LMAX>
__global__ void __launch_bounds__(kLaneGroup) lane_order_kernel(const AlignArgs a, int est_cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  lane_order_body<LMAX>(a, est_cap, smem);
}

// ----------------------------------------------------------- arena kernels

template <int WPP>
__global__ void __launch_bounds__(WPP == 1 ? 128 : 32 * WPP)
    arena_kernel(const AlignArgs a, const int32_t* list, const int32_t* count, int32_t* next, int32_t* overflow_count,
                 unsigned char* arena, long slot_bytes, int nteams, int seq_words, int32_t count_lo,
                 int32_t count_hi) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int32_t c = *(volatile const int32_t*)count;
  // nothing deferred (a graph replays the launch anyway), or the other team
  // width takes this list
  if (c <= count_lo || c > count_hi) return;
  arena_body<WPP>(a, list, count, next, overflow_count, arena, slot_bytes, nteams, seq_words, smem);
}

// Every pair onto the arena work lists (the plain path), by length.
__global__ void route_all_kernel(const AlignArgs a) {
  if (*(volatile const int32_t*)&a.ctrl->bad_input) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) defer_pair(a, i);
}

// ----------------------------------------------------------------- helpers

constexpr int kAuxBlock = 256;

__device__ __forceinline__ long long warp_max64(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  return v;
}

__global__ void validate_kernel(int64_t n, const int64_t* poff, const int32_t* plen, const int64_t* toff,
                                const int32_t* tlen, Ctrl* ctrl) {
  long long pe = 0, te = 0;
  int ml = 0;
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int pl = plen[i], tl = tlen[i];
    const long long po = poff[i], to = toff[i];
    if (pl < 0 || tl < 0 || pl > ((1 << 28) - 1) || tl > ((1 << 28) - 1) || po < 0 || to < 0) {
      bad = true;
      continue;
    }
    pe = max(pe, po + pl);
    te = max(te, to + tl);
    ml = max(ml, max(pl, tl));
  }
  pe = warp_max64(pe);
  te = warp_max64(te);
  ml = __reduce_max_sync(0xffffffffu, ml);
  if ((threadIdx.x & 31) == 0) {
    if (pe) atomicMax(&ctrl->pat_extent, pe);
    if (te) atomicMax(&ctrl->txt_extent, te);
    if (ml) atomicMax(&ctrl->max_len, ml);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(&ctrl->bad_input, 1);
}

// -------------------------------------------------------------------- scan
//
// Prefix sums in three kernels: the tile sums (scan_reduce*), the tiles'
// offsets (scan_tiles, one block), and each tile scanned again with its
// offset (scan_apply*).  A tile of kScanTile elements is kScanItems items per
// thread, an item being four consecutive elements moved with one 16-byte
// load (and two 16-byte stores of the int64 results) when the array is
// 16-byte aligned; item r of thread t holds elements
// r * 4 * kScanBlock + 4 t .. + 3, so each warp access covers 512 consecutive
// bytes of input.

constexpr int kScanBlock = 256;
constexpr int kScanWarps = kScanBlock / 32;
constexpr int kScanItems = kScanTile / (4 * kScanBlock);
static_assert(kScanItems * 4 * kScanBlock == kScanTile, "whole items per tile");

__device__ __forceinline__ bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Elements i .. i + 3 (zero from n on); kind 1: packed words per sequence,
// ceil(len / 32) + 1, for the elements below n.
__device__ __forceinline__ int4 scan_load4(const int32_t* in, int64_t i, int64_t n, int kind, bool vec) {
  int4 v;
  if (vec && i + 3 < n) {
    v = __ldg(reinterpret_cast<const int4*>(in + i));
  } else {
    v.x = i < n ? in[i] : 0;
    v.y = i + 1 < n ? in[i + 1] : 0;
    v.z = i + 2 < n ? in[i + 2] : 0;
    v.w = i + 3 < n ? in[i + 3] : 0;
  }
  if (kind == 1) {
    v.x = i < n ? (v.x + 31) / 32 + 1 : 0;
    v.y = i + 1 < n ? (v.y + 31) / 32 + 1 : 0;
    v.z = i + 2 < n ? (v.z + 31) / 32 + 1 : 0;
    v.w = i + 3 < n ? (v.w + 31) / 32 + 1 : 0;
  }
  return v;
}

// out[i .. i + 3] = c, c + v.x, c + v.x + v.y, c + v.x + v.y + v.z (the
// exclusive sums of the item from c), only the positions up to n.
__device__ __forceinline__ void scan_store4(int64_t* out, int64_t i, int64_t n, bool vec, int64_t c, int4 v) {
  const int64_t a = c, b = a + v.x, d = b + v.y, e = d + v.z;
  if (vec && i + 3 <= n) {
    longlong2* o = reinterpret_cast<longlong2*>(out + i);
    o[0] = make_longlong2(a, b);
    o[1] = make_longlong2(d, e);
  } else {
    if (i <= n) out[i] = a;
    if (i + 1 <= n) out[i + 1] = b;
    if (i + 2 <= n) out[i + 2] = d;
    if (i + 3 <= n) out[i + 3] = e;
  }
}

__device__ __forceinline__ int64_t item_sum(int4 v) { return (int64_t)v.x + v.y + v.z + v.w; }

// Exclusive scan of R values per thread in element order (value r of thread
// t comes after every value of rows < r and of threads < t in row r): each
// warp scans its 32 values of every row with shuffles, the warps' row sums
// go to shared memory (sh: R * kScanWarps + 1 entries) and warp 0 scans them
// in order.  Two block barriers; ex[r] = the sum before value r; *total =
// the sum of all.  A caller that scans again with the same sh synchronises
// the block first.
template <int R>
__device__ __forceinline__ void tile_exclusive(const int64_t (&v)[R], int64_t (&ex)[R], int64_t* total, int64_t* sh) {
  constexpr int NE = R * kScanWarps, P = (NE + 31) / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    int64_t x = v[r];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    ex[r] = x;  // inclusive within the warp's row for now
    if (lane == 31) sh[r * kScanWarps + warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
    int64_t q[P], run = 0;
#pragma unroll
    for (int j = 0; j < P; ++j) {
      q[j] = lane * P + j < NE ? sh[lane * P + j] : 0;
      run += q[j];
    }
    int64_t inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    int64_t pre = inc - run;
#pragma unroll
    for (int j = 0; j < P; ++j) {
      if (lane * P + j < NE) sh[lane * P + j] = pre;
      pre += q[j];
    }
    if (lane == 31) sh[NE] = inc;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < R; ++r) ex[r] += sh[r * kScanWarps + warp] - v[r];
  *total = sh[NE];
}

// The block's sums of a and b, valid in thread 0.
__device__ __forceinline__ void block_sum2(int64_t& a, int64_t& b) {
  __shared__ int64_t sa[kScanWarps], sb[kScanWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (lane == 0) {
    sa[warp] = a;
    sb[warp] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = b = 0;
#pragma unroll
    for (int w = 0; w < kScanWarps; ++w) {
      a += sa[w];
      b += sb[w];
    }
  }
}

__global__ void __launch_bounds__(kScanBlock) scan_reduce(const int32_t* in, int64_t n, int kind, int64_t* tile_sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + 4 * threadIdx.x;
  const bool vec = aligned16(in);
  int64_t acc = 0, none = 0;
#pragma unroll
  for (int r = 0; r < kScanItems; ++r) acc += item_sum(scan_load4(in, base + r * 4 * kScanBlock, n, kind, vec));
  block_sum2(acc, none);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = acc;
}

// pattern and text lengths in one pass: the two tile-sum arrays side by side
__global__ void __launch_bounds__(kScanBlock) scan_reduce2(const int32_t* in1, const int32_t* in2, int64_t n,
                                                           int64_t* tile_sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + 4 * threadIdx.x;
  const bool vec1 = aligned16(in1), vec2 = aligned16(in2);
  int64_t a1 = 0, a2 = 0;
#pragma unroll
  for (int r = 0; r < kScanItems; ++r) {
    a1 += item_sum(scan_load4(in1, base + r * 4 * kScanBlock, n, 0, vec1));
    a2 += item_sum(scan_load4(in2, base + r * 4 * kScanBlock, n, 0, vec2));
  }
  block_sum2(a1, a2);
  if (threadIdx.x == 0) {
    tile_sums[blockIdx.x] = a1;
    tile_sums[gridDim.x + blockIdx.x] = a2;
  }
}

// tile offsets of array blockIdx.x (tile_sums + blockIdx.x * ntiles):
// 8 * kScanBlock tile sums a pass
__global__ void __launch_bounds__(kScanBlock) scan_tiles(int64_t* tile_sums, int64_t ntiles) {
  constexpr int R = 8;
  __shared__ int64_t sh[R * kScanWarps + 1];
  tile_sums += (int64_t)blockIdx.x * ntiles;
  int64_t carry = 0;
  for (int64_t b = 0; b < ntiles; b += R * kScanBlock) {
    int64_t v[R], ex[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t i = b + r * kScanBlock + threadIdx.x;
      v[r] = i < ntiles ? tile_sums[i] : 0;
    }
    int64_t total;
    tile_exclusive(v, ex, &total, sh);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t i = b + r * kScanBlock + threadIdx.x;
      if (i < ntiles) tile_sums[i] = carry + ex[r];
    }
    carry += total;
    __syncthreads();  // sh is scanned again
  }
}

// offsets of both sequences (out[n] = the totals) and the input checks of
// validate_kernel on the way (lengths in range; offsets come from the scan).
// Both arrays' items are loaded at once, then scanned in registers.
__global__ void __launch_bounds__(kScanBlock, 4) scan_apply2_validate(const int32_t* in1, const int32_t* in2, int64_t n,
                                                                   const int64_t* tile_off, int64_t* out1,
                                                                   int64_t* out2, Ctrl* ctrl) {
  __shared__ int64_t sh[2][kScanItems * kScanWarps + 1];
  __shared__ long long s_pe[kScanWarps], s_te[kScanWarps];
  __shared__ int s_ml[kScanWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + 4 * threadIdx.x;
  const bool vin1 = aligned16(in1), vin2 = aligned16(in2), vout = aligned16(out1) && aligned16(out2);
  int4 v1[kScanItems], v2[kScanItems];
  int64_t s1[kScanItems], s2[kScanItems], e1[kScanItems], e2[kScanItems];
#pragma unroll
  for (int r = 0; r < kScanItems; ++r) {
    v1[r] = scan_load4(in1, base + r * 4 * kScanBlock, n, 0, vin1);
    v2[r] = scan_load4(in2, base + r * 4 * kScanBlock, n, 0, vin2);
    s1[r] = item_sum(v1[r]);
    s2[r] = item_sum(v2[r]);
  }
  int64_t t1, t2;
  tile_exclusive(s1, e1, &t1, sh[0]);
  tile_exclusive(s2, e2, &t2, sh[1]);
  const int64_t c1 = tile_off[blockIdx.x], c2 = tile_off[gridDim.x + blockIdx.x];
  long long pe = 0, te = 0;
  int ml = 0;
  bool bad = false;
#pragma unroll
  for (int r = 0; r < kScanItems; ++r) {
    const int64_t i = base + r * 4 * kScanBlock;
    scan_store4(out1, i, n, vout, c1 + e1[r], v1[r]);
    scan_store4(out2, i, n, vout, c2 + e2[r], v2[r]);
    const int x1[4] = {v1[r].x, v1[r].y, v1[r].z, v1[r].w}, x2[4] = {v2[r].x, v2[r].y, v2[r].z, v2[r].w};
    int64_t o1 = c1 + e1[r], o2 = c2 + e2[r];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      o1 += x1[j];  // the end of element i + j
      o2 += x2[j];
      if (i + j < n) {
        if (x1[j] < 0 || x2[j] < 0 || x1[j] > ((1 << 28) - 1) || x2[j] > ((1 << 28) - 1)) {
          bad = true;
        } else {
          pe = max(pe, (long long)o1);
          te = max(te, (long long)o2);
          ml = max(ml, max(x1[j], x2[j]));
        }
      }
    }
  }
  // the block's extents in one atomic each
  pe = warp_max64(pe);
  te = warp_max64(te);
  ml = __reduce_max_sync(0xffffffffu, ml);
  if (lane == 0) {
    s_pe[warp] = pe;
    s_te[warp] = te;
    s_ml[warp] = ml;
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicExch(&ctrl->bad_input, 1);
  __syncthreads();
  if (warp == 0) {
    pe = warp_max64(lane < kScanWarps ? s_pe[lane] : 0);
    te = warp_max64(lane < kScanWarps ? s_te[lane] : 0);
    ml = __reduce_max_sync(0xffffffffu, lane < kScanWarps ? s_ml[lane] : 0);
    if (lane == 0) {
      if (pe) atomicMax(&ctrl->pat_extent, pe);
      if (te) atomicMax(&ctrl->txt_extent, te);
      if (ml) atomicMax(&ctrl->max_len, ml);
    }
  }
}

__global__ void __launch_bounds__(kScanBlock) scan_apply(const int32_t* in, int64_t n, int kind,
                                                         const int64_t* tile_off, int64_t* out) {
  __shared__ int64_t sh[kScanItems * kScanWarps + 1];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + 4 * threadIdx.x;
  const bool vin = aligned16(in), vout = aligned16(out);
  int4 v[kScanItems];
  int64_t sum[kScanItems], ex[kScanItems];
#pragma unroll
  for (int r = 0; r < kScanItems; ++r) {
    v[r] = scan_load4(in, base + r * 4 * kScanBlock, n, kind, vin);
    sum[r] = item_sum(v[r]);
  }
  int64_t total;
  tile_exclusive(sum, ex, &total, sh);
  const int64_t carry = tile_off[blockIdx.x];
#pragma unroll
  for (int r = 0; r < kScanItems; ++r) scan_store4(out, base + r * 4 * kScanBlock, n, vout, carry + ex[r], v[r]);  // out[n] = total
}

// ---------------------------------------------------------------- compact

// One warp per 32 consecutive pairs: the lanes write the pairs' words to
// consecutive output positions (coalesced); lane w's word belongs to the
// last of the 32 pairs whose offset is <= its position (binary search over
// the offsets in shared memory; a pair without runs shares the next pair's
// offset, so the search lands on a pair that has the word).
__global__ void __launch_bounds__(kAuxBlock) compact_kernel(int64_t n, const int32_t* nruns, const int64_t* run_src,
                                                             const uint32_t* runs, const uint32_t* pool,
                                                             const int64_t* off, uint32_t* out, int64_t cap,
                                                             const Ctrl* ctrl) {
  if (off[n] > cap || (ctrl && *(volatile const int32_t*)&ctrl->bad_input)) return;
  __shared__ int64_t s_off[kAuxBlock / 32][32];
  __shared__ int64_t s_src[kAuxBlock / 32][32];
  __shared__ int32_t s_cnt[kAuxBlock / 32][32];
  __shared__ uint32_t s_words[kAuxBlock / 32][32 * kSlot];  // a batch's runs in output order
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5 << 5; i0 < n; i0 += nwarps * 32) {
    const int cnt = n - i0 < 32 ? (int)(n - i0) : 32;
    const int64_t i = i0 + lane;
    int64_t my_off = 0, my_src = 0;
    int my_cnt = 0;
    if (lane < cnt) {
      my_off = off[i];
      my_src = run_src[i];
      my_cnt = nruns[i];
      s_off[wib][lane] = my_off;
      s_src[wib][lane] = my_src;
      s_cnt[wib][lane] = my_cnt;
    }
    const int64_t begin = off[i0], end = off[i0 + cnt];
    // every pair of the batch with its runs in its own slot (the short-read
    // kernels'): each lane puts its pair's runs in output order in shared
    // memory, then the warp writes the batch's words with coalesced stores
    if (__all_sync(0xffffffffu, lane >= cnt || (my_src >= 0 && my_cnt <= kSlot))) {
      if (lane < cnt) {
        const uint32_t* r = runs + my_src;
        uint32_t* d = s_words[wib] + (my_off - begin);
        for (int j = 0; j < my_cnt; ++j) d[j] = r[my_cnt - 1 - j];  // runs are stored last first
      }
      __syncwarp();
      for (int t = lane; t < (int)(end - begin); t += 32) out[begin + t] = s_words[wib][t];
      __syncwarp();
      continue;
    }
    __syncwarp();
    for (int64_t w = begin + lane; w < end; w += 32) {
      int l = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1)
        if (l + step < cnt && s_off[wib][l + step] <= w) l += step;
      const int64_t src = s_src[wib][l];
      const uint32_t* r = src >= 0 ? runs + src : pool + (-src - 1);
      out[w] = r[s_cnt[wib][l] - 1 - (int)(w - s_off[wib][l])];  // runs are stored last first
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------- pack

constexpr int kPackG = 8;

__global__ void __launch_bounds__(kAuxBlock) pack_kernel(int64_t n, const char* seqs, const int64_t* off,
                                                         const int32_t* len, const int64_t* woff, uint64_t* words,
                                                         int8_t* invalid) {
  const int lane = threadIdx.x & (kPackG - 1);
  const unsigned gmask = group_mask(kPackG);
  const int64_t gpb = blockDim.x / kPackG;
  const int64_t total = (int64_t)gridDim.x * gpb;
  for (int64_t i = (int64_t)blockIdx.x * gpb + threadIdx.x / kPackG; __any_sync(0xffffffffu, i < n); i += total) {
    if (i < n) {
      const bool ok = pack_seq<kPackG>(seqs + off[i], len[i], words + woff[i], lane, gmask);
      if (lane == 0) invalid[i] = ok ? 0 : 1;
    }
    __syncwarp();
  }
}

// ------------------------------------------------ longest-first work order

__device__ __forceinline__ int len_bucket(const AlignArgs& a, int32_t pair, int max_len) {
  const int L = max(a.plen[pair], a.tlen[pair]);
  const int b = (int)(((long long)L * kSortBuckets) / ((long long)max_len + 1));
  return b < kSortBuckets ? b : kSortBuckets - 1;
}

__global__ void sort_hist_kernel(const AlignArgs a, const int32_t* list, const int32_t* count, int32_t* hist) {
  __shared__ int h[kSortBuckets];
  for (int i = threadIdx.x; i < kSortBuckets; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const int n = *count, ml = a.ctrl->max_len;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    atomicAdd(&h[len_bucket(a, list[i], ml)], 1);
  __syncthreads();
  for (int i = threadIdx.x; i < kSortBuckets; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

// bucket starts, longest bucket first (one thread: 64 buckets)
__global__ void sort_scan_kernel(const int32_t* hist, int32_t* cursor) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int at = 0;
  for (int b = kSortBuckets - 1; b >= 0; --b) {
    cursor[b] = at;
    at += hist[b];
  }
}

__global__ void sort_scatter_kernel(const AlignArgs a, const int32_t* list, const int32_t* count, int32_t* cursor,
                                    int32_t* out) {
  const int n = *count, ml = a.ctrl->max_len;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int32_t p = list[i];
    out[atomicAdd(&cursor[len_bucket(a, p, ml)], 1)] = p;
  }
}

__global__ void add_kernel(int64_t* p, int64_t count, int64_t v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    p[i] += v;
}

// Small transfers as kernels (see launch_put_ctrl).
__global__ void put_ctrl_kernel(Ctrl* dst, const Ctrl v) { *dst = v; }

__global__ void copy_small_kernel(uint32_t* dst, const uint32_t* src, int words) {
  if ((int)threadIdx.x < words) dst[threadIdx.x] = src[threadIdx.x];
  __threadfence_system();  // page-locked host destination: visible once the stream is done
}

int sm_count(int device) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
  return v > 0 ? v : 1;
}

int aux_grid(int64_t n, int device) {
  const int64_t want = (n + kAuxBlock - 1) / kAuxBlock;
  const int64_t cap = (int64_t)sm_count(device) * 8;
  return (int)(want < 1 ? 1 : want > cap ? cap : want);
}

int current_device() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}

}  // namespace

// ---------------------------------------------------------------- launchers

namespace {

template <int G, int LMAX, int CELLS, int SCAP, typename Off, bool LIN = false, bool EF = false>
cudaError_t plan_one(int device, ShortVariant* v, const char* name) {
  using C = ShortCfg<G, LMAX, CELLS, SCAP, Off, LIN>;
  auto k = short_kernel<G, LMAX, CELLS, SCAP, Off, LIN, EF>;
  const int warps = kShortBlock / 32;
  const size_t smem = C::smem_bytes(warps);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kShortBlock, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  v->grid = sm_count(device) * per_sm;
  v->block = kShortBlock;
  v->smem = smem;
  v->max_len = LMAX;
  v->pairs_per_block = warps * C::P;
  v->kernel = reinterpret_cast<const void*>(k);
  v->name = name;
  v->cells = CELLS;
  v->scap = SCAP;
  v->linear = LIN ? 1 : 0;
  v->ends_free = EF ? 1 : 0;
  v->kind = 0;
  v->rw = 0;
  v->ct_x = v->ct_oe = v->ct_e = 0;
  return cudaSuccess;
}

// Raw sequence bytes a lane-per-pair warp stages at once: both spans of 32
// back-to-back pairs of up to 127 bases (kLaneSpan), or one (kLaneSpan1:
// small stores, where the scratch would otherwise set the shared memory).
constexpr int kLaneSpan = 8192;
constexpr int kLaneSpan1 = 4096;
// warps of the 197-cell store's one block per SM (18 x 12.3 KB of shared
// memory, with 30 row positions: the 4/6/2 geometry's rows need 30, penalty
// sets whose rows are wider keep a shorter store)
constexpr int kWide197 = 18;

// The ordering pass's shared memory and its resident grid (the same for
// every lane variant).
using OrderShm = LaneOrderShm<127>;

cudaError_t plan_order(int device, int* grid) {
  auto k = lane_order_kernel<127>;
  const size_t smem = sizeof(OrderShm);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kLaneGroup, smem);
  if (e != cudaSuccess) return e;
  *grid = sm_count(device) * (per_sm < 1 ? 1 : per_sm);
  return cudaSuccess;
}

// A lane-per-pair variant; CT_X, CT_OE, CT_E: the scaled penalties whose
// geometry is compiled in (0: any penalties, geometry from the table).
template <int LMAX, int CELLS, int RW, int WPB, int CT_X = 0, int CT_OE = 0, int CT_E = 0, int SPAN = kLaneSpan>
cudaError_t plan_lane(int device, ShortVariant* v, const char* name) {
  using C = LaneCfg<LMAX, CELLS, RW, SPAN>;
  using Fwd = typename std::conditional<CT_X == 0, LaneRunForward,
                                        LaneCtForward<(CT_X ? CT_X : 1), (CT_OE ? CT_OE : 1), (CT_E ? CT_E : 1), CELLS,
                                                      RW>>::type;
  const void* k;
  if constexpr (WPB >= 8) k = reinterpret_cast<const void*>(lane_kernel_wide<LMAX, CELLS, RW, SPAN, WPB, Fwd>);
  else k = reinterpret_cast<const void*>(lane_kernel<LMAX, CELLS, RW, SPAN, WPB, Fwd>);
  const size_t smem = C::smem_bytes(WPB, Fwd::kRows);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * WPB, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  v->grid = sm_count(device) * per_sm;
  v->block = 32 * WPB;
  v->smem = smem;
  v->max_len = LMAX;
  v->pairs_per_block = 32 * WPB;
  v->kernel = reinterpret_cast<const void*>(k);
  v->name = name;
  v->cells = CELLS;
  v->scap = 31;
  v->linear = 0;
  v->ends_free = 0;
  v->kind = 1;
  v->rw = RW;
  v->ct_x = CT_X;
  v->ct_oe = CT_OE;
  v->ct_e = CT_E;
  return plan_order(device, &v->order_grid);
}

}  // namespace

void lane_geometry(const AlignArgs& a, int cells, int rw, LaneGeo* g) {
  std::memset(g, 0, sizeof *g);
  const int last = build_ugeo(g->tab, 31, cells, ScaledPen{a.xs, a.oes, a.es}, 0, 0);
  const LaneLayout L = lane_layout(g->tab, last, a.es, rw);
  g->s_store = (a.pb | a.pe | a.tb | a.te) != 0 ? -1 : L.s_store;  // global alignment only
  g->off_i = L.off_i;
  g->off_d = L.off_d;
  g->span_i = L.span_i;
  g->span_d = L.span_d;
  // each score's row record (LaneRunForward): sources, I/D positions and
  // the untested middle of the row
  const int X = a.xs, OE = a.oes, E = a.es;
  for (int s = 1; s < 32; ++s) {
    const UGeo& t = g->tab[s];
    LaneRow& r = g->rows[s];
    if (!(t.ex & 1)) continue;  // ex = 0: the score has no M wavefront
    r.ex = 1;
    r.lo = t.lo;
    r.w = t.w;
    r.base = t.base;
    if (s - X >= 0 && (g->tab[s - X].ex & 1)) {
      const UGeo& x = g->tab[s - X];
      r.ax = x.lo - t.lo;  // item of the source's first diagonal
      r.wx = x.w;
      r.cx = x.base - r.ax;
    }
    if (s - OE >= 0 && (g->tab[s - OE].ex & 1)) {
      const UGeo& o = g->tab[s - OE];
      r.ao = o.lo - t.lo;
      r.wo = o.w;
      r.co = o.base - r.ao;
    }
    const int q = s / E, rm = s % E;
    r.pi0 = rm * L.span_i + t.lo - q + L.off_i;
    r.pd0 = rm * L.span_d + t.lo + q + L.off_d;
    r.a = lane_mid_a(r.ax, r.ao, r.w);
    r.b = lane_mid_b(r.ax, r.wx, r.ao, r.wo, r.w, r.a);
  }
}

// The short-kernel variants: (lanes per pair, longest sequence, cells per
// pair, largest score index, offset type, gap-linear model).
cudaError_t short_plan(int device, ShortPlan* plan) {
  cudaError_t e;
  int i = 0;
  // 197 cells: every wavefront up to scaled score 16 under 4/6/2, and a
  // block of four G = 2 warps small enough for five blocks per SM
  if ((e = plan_one<1, 127, 197, 31, int8_t>(device, &plan->v[i++], "g1_l127_c197_i8"))) return e;
  if ((e = plan_one<2, 127, 197, 31, int8_t>(device, &plan->v[i++], "g2_l127_c197_i8"))) return e;
  if ((e = plan_one<4, 127, 197, 31, int8_t>(device, &plan->v[i++], "g4_l127_c197_i8"))) return e;
  if ((e = plan_one<8, 127, 197, 31, int8_t>(device, &plan->v[i++], "g8_l127_c197_i8"))) return e;
  if ((e = plan_one<1, 127, 64, 15, int8_t>(device, &plan->v[i++], "g1_l127_c64_i8"))) return e;
  if ((e = plan_one<2, 255, 197, 31, int16_t>(device, &plan->v[i++], "g2_l255_c197_i16"))) return e;
  if ((e = plan_one<4, 255, 197, 31, int16_t>(device, &plan->v[i++], "g4_l255_c197_i16"))) return e;
  if ((e = plan_one<1, 127, 40, 15, int8_t>(device, &plan->v[i++], "g1_l127_c40_i8"))) return e;
  // gap-linear model (o = 0): M only, so a third of the store per cell
  if ((e = plan_one<1, 127, 64, 15, int8_t, true>(device, &plan->v[i++], "g1_l127_c64_lin"))) return e;
  if ((e = plan_one<2, 127, 256, 31, int8_t, true>(device, &plan->v[i++], "g2_l127_c256_lin"))) return e;
  if ((e = plan_one<2, 255, 256, 31, int16_t, true>(device, &plan->v[i++], "g2_l255_c256_lin_i16"))) return e;
  // ends-free calls (first wavefront over the free starts, end test over the
  // free diagonals)
  if ((e = plan_one<2, 127, 197, 31, int8_t, false, true>(device, &plan->v[i++], "g2_l127_c197_i8_ef"))) return e;
  if ((e = plan_one<4, 255, 197, 31, int16_t, false, true>(device, &plan->v[i++], "g4_l255_c197_i16_ef")))
    return e;
  if ((e = plan_one<2, 127, 256, 31, int8_t, true, true>(device, &plan->v[i++], "g2_l127_c256_lin_ef"))) return e;
  if ((e = plan_one<2, 255, 256, 31, int16_t, true, true>(device, &plan->v[i++], "g2_l255_c256_lin_i16_ef")))
    return e;
  // one lane per pair (gap-affine, global): stores of scores 0-8, 0-9, 0-12
  // and 0-16 under 4/6/2; any penalties (15-18), and with the geometry of
  // scaled penalties x = 2, o + e = 4, e = 1 (4/6/2 and its multiples)
  // compiled in (19-22)
  if ((e = plan_lane<127, 40, 16, 4, 0, 0, 0, kLaneSpan1>(device, &plan->v[i++], "lane_l127_c40"))) return e;
  if ((e = plan_lane<127, 64, 16, 4, 0, 0, 0, kLaneSpan1>(device, &plan->v[i++], "lane_l127_c64"))) return e;
  if ((e = plan_lane<127, 104, 32, 2>(device, &plan->v[i++], "lane_l127_c104"))) return e;
  if ((e = plan_lane<127, 197, 30, kWide197>(device, &plan->v[i++], "lane_l127_c197"))) return e;
  if ((e = plan_lane<127, 40, 16, 4, 2, 4, 1, kLaneSpan1>(device, &plan->v[i++], "lane_ct241_l127_c40"))) return e;
  if ((e = plan_lane<127, 64, 16, 4, 2, 4, 1, kLaneSpan1>(device, &plan->v[i++], "lane_ct241_l127_c64"))) return e;
  if ((e = plan_lane<127, 104, 32, 2, 2, 4, 1>(device, &plan->v[i++], "lane_ct241_l127_c104"))) return e;
  if ((e = plan_lane<127, 197, 32, 2, 2, 4, 1>(device, &plan->v[i++], "lane_ct241_l127_c197"))) return e;
  plan->count = i;
  // the one-CTA arena kernels keep two sequences of up to 32,768 bases in
  // shared memory
  const size_t arena_smem = sizeof(TeamShm) + 2 * (size_t)(32768 / 32 + 2) * sizeof(uint64_t);
  if ((e = cudaFuncSetAttribute(arena_kernel<kLongTeamWide>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)arena_smem)))
    return e;
  return cudaFuncSetAttribute(arena_kernel<kLongTeamNarrow>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)arena_smem);
}

// Ordered input only for sequences in device memory (the ordering pass
// reads each pair's bytes with its own loads, which page-locked host memory
// read in place over the link would turn into many small transfers).
static bool lane_ordered(const AlignArgs& a, const ShortVariant& v) {
  return a.n > 0 && v.kind == 1 && a.lane_slots && a.lane_words && !a.host_seqs;
}

int short_launches(const AlignArgs& a, const ShortVariant& v) { return lane_ordered(a, v) ? 2 : 1; }

cudaError_t launch_short(const AlignArgs& a, const ShortVariant& v, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  int grid = v.grid;
  AlignArgs copy = a;
  const bool ordered = lane_ordered(a, v);
  if (!ordered) copy.lane_words = nullptr, copy.lane_slots = nullptr;
  const int64_t groups = (a.n + kLaneGroup - 1) / kLaneGroup;
  const int64_t units = ordered ? groups * kLaneGroup : a.n;  // pairs, or slots of whole groups
  const int64_t need = (units + v.pairs_per_block - 1) / v.pairs_per_block;
  if (need < grid) grid = (int)need;
  if (v.kind == 1) {
    LaneGeo g;
    lane_geometry(a, v.cells, v.rw, &g);
    if (ordered) {
      // estimates above the store's last score all mean "deferred": the
      // greedy walk stops there; a small store is ordered by packing alone
      const int cap = g.s_store < a.lane_sort_min ? 0 : std::min(g.s_store + 1, kLaneEstMax);
      const int og = groups < v.order_grid ? (int)groups : v.order_grid;
      lane_order_kernel<127><<<og, kLaneGroup, sizeof(OrderShm), st>>>(copy, cap);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    void* args[] = {&copy, &g};
    return cudaLaunchKernel(v.kernel, dim3(grid), dim3(v.block), args, v.smem, st);
  }
  void* args[] = {&copy};
  return cudaLaunchKernel(v.kernel, dim3(grid), dim3(v.block), args, v.smem, st);
}

cudaError_t launch_route_all(const AlignArgs& a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  route_all_kernel<<<aux_grid(a.n, current_device()), kAuxBlock, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t arena_occupancy(int team_warps, int* teams_per_sm) {
  int per_sm = 0;
  cudaError_t e;
  if (team_warps == 1) {
    const int seq_words = kMediumMaxLen / 32 + 2;
    const size_t smem = 4 * (sizeof(TeamShm) + 2 * (size_t)seq_words * sizeof(uint64_t));
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, arena_kernel<1>, 128, smem);
    *teams_per_sm = 4 * per_sm;
  } else {
    const size_t smem = sizeof(TeamShm) + 2 * (size_t)(32768 / 32 + 2) * sizeof(uint64_t);
    e = team_warps == kLongTeamNarrow
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, arena_kernel<kLongTeamNarrow>,
                                                            32 * kLongTeamNarrow, smem)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, arena_kernel<kLongTeamWide>, 32 * kLongTeamWide,
                                                            smem);
    *teams_per_sm = per_sm;
  }
  if (*teams_per_sm < 1) *teams_per_sm = 1;
  return e;
}

cudaError_t launch_arena(int team_warps, const AlignArgs& a, const int32_t* list, const int32_t* count,
                         int32_t* next, int32_t* overflow_count, unsigned char* arena, long slot_bytes, int nteams,
                         cudaStream_t st, int32_t count_lo, int32_t count_hi) {
  if (nteams < 1) return cudaSuccess;
  if (team_warps == 1) {
    // four one-warp teams per block; sequences of medium pairs in shared memory
    const int seq_words = kMediumMaxLen / 32 + 2;
    const size_t smem = 4 * (sizeof(TeamShm) + 2 * (size_t)seq_words * sizeof(uint64_t));
    const int grid = (nteams + 3) / 4;
    arena_kernel<1><<<grid, 128, smem, st>>>(a, list, count, next, overflow_count, arena, slot_bytes, nteams,
                                            seq_words, count_lo, count_hi);
  } else {
    // one CTA per team; sequences up to 32,768 bases in shared memory
    const int seq_words = 32768 / 32 + 2;
    const size_t smem = sizeof(TeamShm) + 2 * (size_t)seq_words * sizeof(uint64_t);
    if (team_warps == kLongTeamNarrow)
      arena_kernel<kLongTeamNarrow><<<nteams, 32 * kLongTeamNarrow, smem, st>>>(
          a, list, count, next, overflow_count, arena, slot_bytes, nteams, seq_words, count_lo, count_hi);
    else
      arena_kernel<kLongTeamWide><<<nteams, 32 * kLongTeamWide, smem, st>>>(
          a, list, count, next, overflow_count, arena, slot_bytes, nteams, seq_words, count_lo, count_hi);
  }
  return cudaGetLastError();
}

cudaError_t launch_sort_longest_first(const AlignArgs& a, const int32_t* list, const int32_t* count, int64_t n_cap,
                                      int32_t* aux, int32_t* out, cudaStream_t st) {
  if (n_cap <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(aux, 0, kSortBuckets * sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  const int grid = std::min(aux_grid(n_cap, current_device()), 2 * sm_count(current_device()));
  sort_hist_kernel<<<grid, kAuxBlock, 0, st>>>(a, list, count, aux);
  sort_scan_kernel<<<1, 32, 0, st>>>(aux, aux + kSortBuckets);
  sort_scatter_kernel<<<grid, kAuxBlock, 0, st>>>(a, list, count, aux + kSortBuckets, out);
  return cudaGetLastError();
}

cudaError_t launch_put_ctrl(Ctrl* dst, const Ctrl& v, cudaStream_t st) {
  put_ctrl_kernel<<<1, 1, 0, st>>>(dst, v);
  return cudaGetLastError();
}

cudaError_t launch_copy_small(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  if (bytes % 4 != 0 || bytes > 4096 || reinterpret_cast<uintptr_t>(dst) % 4 != 0 ||
      reinterpret_cast<uintptr_t>(src) % 4 != 0)
    return cudaErrorInvalidValue;
  const int words = (int)(bytes / 4);
  copy_small_kernel<<<1, (unsigned)((words + 31) / 32 * 32), 0, st>>>(static_cast<uint32_t*>(dst),
                                                                      static_cast<const uint32_t*>(src), words);
  return cudaGetLastError();
}

cudaError_t launch_add(int64_t* p, int64_t count, int64_t v, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  add_kernel<<<aux_grid(count, current_device()), kAuxBlock, 0, st>>>(p, count, v);
  return cudaGetLastError();
}

cudaError_t launch_validate(int64_t n, const int64_t* poff, const int32_t* plen, const int64_t* toff,
                            const int32_t* tlen, Ctrl* ctrl, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  validate_kernel<<<aux_grid(n, current_device()), kAuxBlock, 0, st>>>(n, poff, plen, toff, tlen, ctrl);
  return cudaGetLastError();
}

// room for two tile-sum arrays (launch_offsets_validate)
int64_t scan_tmp_elems(int64_t n) { return 2 * ((n + 1 + kScanTile - 1) / kScanTile) + 2; }

cudaError_t launch_offsets_validate(const int32_t* plen, const int32_t* tlen, int64_t n, int64_t* poff,
                                    int64_t* toff, int64_t* tmp, Ctrl* ctrl, cudaStream_t st) {
  const int64_t ntiles = (n + 1 + kScanTile - 1) / kScanTile;
  scan_reduce2<<<(unsigned)ntiles, kScanBlock, 0, st>>>(plen, tlen, n, tmp);
  scan_tiles<<<2, kScanBlock, 0, st>>>(tmp, ntiles);
  scan_apply2_validate<<<(unsigned)ntiles, kScanBlock, 0, st>>>(plen, tlen, n, tmp, poff, toff, ctrl);
  return cudaGetLastError();
}

cudaError_t launch_scan(const int32_t* in, int64_t n, int kind, int64_t* out, int64_t* tmp, cudaStream_t st) {
  // tiles cover indices 0..n (out[n] is the total)
  const int64_t ntiles = (n + 1 + kScanTile - 1) / kScanTile;
  scan_reduce<<<(unsigned)ntiles, kScanBlock, 0, st>>>(in, n, kind, tmp);
  scan_tiles<<<1, kScanBlock, 0, st>>>(tmp, ntiles);
  scan_apply<<<(unsigned)ntiles, kScanBlock, 0, st>>>(in, n, kind, tmp, out);
  return cudaGetLastError();
}

cudaError_t launch_compact(int64_t n, const int32_t* nruns, const int64_t* run_src, const uint32_t* runs,
                           const uint32_t* pool, const int64_t* off, uint32_t* out, int64_t cap, const Ctrl* ctrl,
                           cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  compact_kernel<<<aux_grid(n, current_device()), kAuxBlock, 0, st>>>(n, nruns, run_src, runs, pool, off, out, cap,
                                                                       ctrl);
  return cudaGetLastError();
}

cudaError_t launch_pack(int64_t n, const char* seqs, const int64_t* off, const int32_t* len, const int64_t* woff,
                        uint64_t* words, int8_t* invalid, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t groups_per_block = kAuxBlock / kPackG;
  int64_t grid = (n + groups_per_block - 1) / groups_per_block;
  const int64_t cap = (int64_t)sm_count(current_device()) * 16;
  if (grid > cap) grid = cap;
  pack_kernel<<<(unsigned)grid, kAuxBlock, 0, st>>>(n, seqs, off, len, woff, words, invalid);
  return cudaGetLastError();
}

}  // namespace wfa
