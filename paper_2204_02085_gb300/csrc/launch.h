// launch.h -- host-side launchers of the library's kernels (C++ linkage,
// internal to libwfa_gpu.so; the public interface is include/wfa_gpu.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "wfa_device.cuh"

namespace wfa {

// Per-call device control block, zeroed before each batch.
struct Ctrl {
  int32_t bad_input;        // a length or offset out of range
  int32_t internal_error;   // stored wavefronts inconsistent in a backtrace
  int32_t defer_count;      // pairs handed to the one-warp arena kernel
  int32_t defer_long_count; // pairs handed to the one-CTA arena kernel
  int32_t next_medium;      // work-queue heads of the arena kernels
  int32_t next_long;
  int32_t retry_count;      // pairs of the current retry list
  int32_t next_retry;
  int32_t overflow_count;   // pairs an arena kernel could not fit
  int32_t pool_short;       // the CIGAR pool ran out
  unsigned long long pool_top;  // words used in the CIGAR pool
  long long pat_extent;     // max(offset + length) over patterns
  long long txt_extent;     // max(offset + length) over texts
  int32_t max_len;          // longest pattern or text
  int32_t lane_next;        // work-queue head of the lane kernel on ordered input
};

struct AlignArgs {
  int64_t n;
  const char* pat;
  const int64_t* poff;
  const int32_t* plen;
  const char* txt;
  const int64_t* toff;
  const int32_t* tlen;
  int xs, oes, es;  // penalties divided by g
  int g;            // gcd(x, o, e)
  int s_cap;        // largest scaled score reported (INT_MAX: none)
  int score_only;
  int host_seqs;  // sequences read in place from page-locked host memory
  // ends-free alignment: free leading / trailing pattern (pb, pe) and text
  // (tb, te) characters; all 0 for a global alignment
  int pb, pe, tb, te;
  int32_t* score;
  int8_t* status;
  int32_t* nruns;
  int64_t* run_src;   // where a pair's runs (last run first) are: >= 0 an
                      // index into `runs`, < 0 the index -src-1 into `pool`
  uint32_t* runs;     // [n * kSlot] per-pair slots of the short kernel
  uint32_t* pool;     // runs of arena-kernel pairs, reserved by atomics
  int64_t pool_cap;   // words in the pool
  int32_t* defer_list;       // [n] pairs for the one-warp arena kernel
  int32_t* defer_long_list;  // [n] pairs for the one-CTA arena kernel
  int32_t* overflow_list;    // [n]
  Ctrl* ctrl;
  // lane-per-pair kernel input order (both null: pairs in call order).  Each
  // group of kLaneGroup consecutive pairs is packed and sorted by an
  // estimate of its score; slot q of group j holds its pair's packed words
  // at lane_words[(j * 2 * kLaneNW + w) * kLaneGroup + q] (w < kLaneNW the
  // pattern's word w, then the text's) and (pair or -1, n | m << 8) at
  // lane_slots[j * kLaneGroup + q].
  uint32_t* lane_words;
  int2* lane_slots;
  int lane_sort_min;  // smallest store (last stored score) whose ordering sorts
};

// Pairs the lane ordering sorts together, and packed 16-base words per
// sequence of at most 127 bases the lane kernel reads.
constexpr int kLaneGroup = 1024;
constexpr int kLaneNW = 127 / 16 + 2;

// longest sequence handled by a one-warp arena team; longer pairs go to a
// one-CTA team
constexpr int kMediumMaxLen = 2048;
// A one-CTA arena team (pairs longer than kMediumMaxLen) has 8 warps when
// few long pairs are deferred (each pair's latency sets the call's) and 4
// when they outnumber the 8-warp teams that fit (more teams in flight).
constexpr int kLongTeamWide = 8;
constexpr int kLongTeamNarrow = 4;

constexpr int kSlot = 16;  // CIGAR runs a short-kernel pair may keep

// Fused short-read kernel (pack + wavefronts in shared memory + backtrace),
// one instantiation per variant.  kind 0: the running pairs of a warp share
// its lanes cell by cell (short_path.cuh); kind 1: one lane per pair, the
// warp's 32 pairs in lockstep over a host-built geometry (lane_path.cuh).
struct ShortVariant {
  const void* kernel;
  const char* name;
  int grid, block, pairs_per_block;
  size_t smem;
  int max_len;  // longest sequence the variant takes
  int cells;    // wavefront cells stored per pair
  int scap;     // largest score index of the geometry table
  int linear;   // 1: gap-linear model only (o = 0; M stored, I and D derived)
  int ends_free;  // 1: for ends-free calls only
  int kind;     // 0 shared-lane, 1 lane-per-pair
  int rw;       // kind 1: positions of each in-place I and D row
  int ct_x, ct_oe, ct_e;  // kind 1: scaled penalties compiled in (0: any)
  int order_grid;         // kind 1: blocks of the ordering pass that fit the GPU at once
};
struct ShortPlan {
  ShortVariant v[24];
  int count;
};
cudaError_t short_plan(int device, ShortPlan* plan);
cudaError_t launch_short(const AlignArgs& a, const ShortVariant& v, cudaStream_t st);
// Kernels launch_short enqueues: the ordering pass and the lane kernel for a
// lane variant with lane_slots set (sequences in device memory), else one.
int short_launches(const AlignArgs& a, const ShortVariant& v);

// Geometry of the lane-per-pair kernel for one call (a kernel parameter):
// the uniform table of scores 0..31, the last score the kernel stores (-1:
// it takes no pair, e.g. ends-free calls), and where the in-place I and D
// rows keep each score: I_s[k] at position (s mod e) * span_i + k - s/e +
// off_i, D_s[k] at (s mod e) * span_d + k + s/e + off_d.
// rows[s]: score s's row as the forward pass with the table read at run
// time takes it (every lane of every warp the same, so it is worked out
// once on the host): its diagonals and store cells, where its sources lie,
// and the items whose sources all lie inside their rows.
struct alignas(16) LaneRow {
  int32_t lo, w, base;  // first diagonal, width, store cell of item 0
  int32_t ax, wx, cx;   // row s - x: its first item, its width, the cell of item 0
  int32_t ao, wo, co;   // row s - o - e, likewise
  int32_t pi0, pd0;     // I and D row positions of item 0
  int32_t a, b;         // items a .. b - 1 need no range test
  int32_t ex;           // 1: the score has an M wavefront
  int32_t pad[2];
};
struct LaneGeo {
  UGeo tab[32];
  LaneRow rows[32];
  int32_t s_store, off_i, off_d, span_i, span_d, pad[3];
};
// Fills g for the call's penalties and a variant of `cells` cells and
// in-place rows of `rw` positions (lane_layout in lane_path.cuh: the last
// stored score is the largest whose wavefronts fit the cells, are at most 32
// diagonals wide, fit the rows, and whose row reads each find the previous
// score's value or a position not yet written).
void lane_geometry(const AlignArgs& a, int cells, int rw, LaneGeo* g);

// Arena kernels for pairs deferred by the short kernel: pairs list[0 ..
// *count), taken through the work-queue head *next; `nteams` teams (one
// warp each when long_team is false, one CTA of 8 warps otherwise), each
// with slot_bytes of the arena; pairs that do not fit go to a.overflow_list.
// The plain path: every pair onto the arena work lists.
cudaError_t launch_route_all(const AlignArgs& a, cudaStream_t st);

// Resident teams per SM of an arena kernel with teams of team_warps warps
// (1: one-warp teams of medium pairs; kLongTeamWide or kLongTeamNarrow:
// one-CTA teams of long pairs).
cudaError_t arena_occupancy(int team_warps, int* teams_per_sm);
// The launch works through the list only while count_lo < *count <=
// count_hi: a graph holds both one-CTA widths and the count, known on the
// device only, picks the one that runs.
cudaError_t launch_arena(int team_warps, const AlignArgs& a, const int32_t* list, const int32_t* count,
                         int32_t* next, int32_t* overflow_count, unsigned char* arena, long slot_bytes, int nteams,
                         cudaStream_t st, int32_t count_lo = 0, int32_t count_hi = 0x7fffffff);

// Longest-first order of a work list (batched path): list[0 .. *count) ->
// out, by the longer sequence of each pair in kSortBuckets equal-width
// buckets over [0, ctrl->max_len], longest bucket first (order inside a
// bucket unspecified).  aux: 2 * kSortBuckets ints of scratch.  n_cap bounds
// *count (sizes the grid).  Reads the count on the device, so it can be
// captured into a graph.
constexpr int kSortBuckets = 64;
cudaError_t launch_sort_longest_first(const AlignArgs& a, const int32_t* list, const int32_t* count, int64_t n_cap,
                                      int32_t* aux, int32_t* out, cudaStream_t st);

// Offsets of back-to-back patterns and texts (both exclusive scans of the
// lengths, [n] = totals) and the checks and extents of launch_validate, in
// one pass of three kernels; ctrl must be zeroed first.
cudaError_t launch_offsets_validate(const int32_t* plen, const int32_t* tlen, int64_t n, int64_t* poff,
                                    int64_t* toff, int64_t* tmp, Ctrl* ctrl, cudaStream_t st);

// Validate lengths / offsets, record max(offset + length) extents.
cudaError_t launch_validate(int64_t n, const int64_t* poff, const int32_t* plen, const int64_t* toff,
                            const int32_t* tlen, Ctrl* ctrl, cudaStream_t st);

// Elements per tile of the prefix-sum kernels (one tile sum each in tmp).
constexpr int kScanTile = 2048;

// Exclusive prefix sums into out[0..n] (out[n] = total).  `kind`:
//   0: values in[i];  1: ceil(in[i]/32) + 1 (packed words per sequence).
// tmp must hold scan_tmp_elems(n) int64.
int64_t scan_tmp_elems(int64_t n);
cudaError_t launch_scan(const int32_t* in, int64_t n, int kind, int64_t* out, int64_t* tmp, cudaStream_t st);

// CIGAR compaction: pair i's runs (stored last first, see run_src) to
// out[off[i] .. off[i+1]) in order; writes nothing if off[n] > cap or the
// inputs were rejected (ctrl may be NULL).
cudaError_t launch_compact(int64_t n, const int32_t* nruns, const int64_t* run_src, const uint32_t* runs,
                           const uint32_t* pool, const int64_t* off, uint32_t* out, int64_t cap, const Ctrl* ctrl,
                           cudaStream_t st);

// p[0 .. count) += v (int64).
cudaError_t launch_add(int64_t* p, int64_t count, int64_t v, cudaStream_t st);

// Small transfers as one-block kernels.  A copy engine serves the copies of
// every stream in order, so a small copy queued behind another stream's
// bulk copy (a chunk of input bases, a chunk of outputs) waits for all of
// it; a kernel's loads and stores do not.  launch_put_ctrl writes v (a
// kernel argument) to dst; launch_copy_small copies bytes (a multiple of 4,
// at most 4 KiB, both addresses 4-byte aligned; dst may be the device
// address of page-locked host memory).
cudaError_t launch_put_ctrl(Ctrl* dst, const Ctrl& v, cudaStream_t st);
cudaError_t launch_copy_small(void* dst, const void* src, size_t bytes, cudaStream_t st);

// Standalone packer: sequence i -> words[woff[i] ..], invalid[i].
cudaError_t launch_pack(int64_t n, const char* seqs, const int64_t* off, const int32_t* len, const int64_t* woff,
                        uint64_t* words, int8_t* invalid, cudaStream_t st);

}  // namespace wfa
