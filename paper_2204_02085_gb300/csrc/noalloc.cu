// noalloc.cu -- wfa_gpu_align_short_noalloc: the short-read alignment path
// for callers that cannot allocate device memory.  Its scratch lives in one
// file-scope device array instead of buffers from cudaMalloc; see the
// declaration in include/wfa_gpu.h for the contract.
#include <cstdint>
#include <mutex>

#include "launch.h"
#include "wfa_gpu.h"

namespace {

// The scratch: every GPU that loads this library holds it until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[WFA_GPU_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
constexpr int64_t kN = WFA_GPU_NOALLOC_MAX_PAIRS;

struct DeviceState {
  bool ready = false;
  unsigned char* scratch = nullptr;  // device address of g_noalloc_scratch
  wfa::ShortPlan plan{};
};

std::mutex g_mutex;
DeviceState g_state[kMaxDevices];

// Carve-up of the scratch array (offsets in bytes, 256-aligned).
constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kOffCtrl = 0;
constexpr size_t kOffScanTmp = align256(kOffCtrl + 2 * sizeof(wfa::Ctrl));
constexpr size_t kScanTmpBytes = ((kN + 1 + wfa::kScanTile - 1) / wfa::kScanTile + 2) * sizeof(int64_t);
constexpr size_t kOffPoff = align256(kOffScanTmp + kScanTmpBytes);
constexpr size_t kOffToff = align256(kOffPoff + (kN + 1) * sizeof(int64_t));
constexpr size_t kOffNruns = align256(kOffToff + (kN + 1) * sizeof(int64_t));
constexpr size_t kOffRunSrc = align256(kOffNruns + kN * sizeof(int32_t));
constexpr size_t kOffDefer = align256(kOffRunSrc + kN * sizeof(int64_t));
constexpr size_t kOffRuns = align256(kOffDefer + kN * sizeof(int32_t));
constexpr size_t kEnd = kOffRuns + (size_t)kN * wfa::kSlot * sizeof(uint32_t);
static_assert(kEnd <= WFA_GPU_NOALLOC_SCRATCH_BYTES, "scratch array too small for its carve-up");

// Index of the short-kernel variant with the large store and int8 offsets
// (sequences <= 127 bases) in the plan built by wfa::short_plan.
constexpr int kVariant = 1;

// Once per device, with that device current: the scratch array's device
// address (the name g_noalloc_scratch is only a host-side stand-in) and the
// kernel configuration.
int setup(int device, DeviceState** out) {
  if (device < 0 || device >= kMaxDevices) return WFA_GPU_ECUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceState& st = g_state[device];
  if (!st.ready) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return WFA_GPU_ECUDA;
    if (wfa::short_plan(device, &st.plan) != cudaSuccess) return WFA_GPU_ECUDA;
    if (st.plan.count <= kVariant || st.plan.v[kVariant].max_len < WFA_GPU_NOALLOC_MAX_LEN) return WFA_GPU_ECUDA;
    st.scratch = static_cast<unsigned char*>(ptr);
    st.ready = true;
  }
  *out = &st;
  return WFA_GPU_OK;
}

int gcd(int a, int b) {
  while (b) {
    const int t = a % b;
    a = b;
    b = t;
  }
  return a;
}

}  // namespace

extern "C" int wfa_gpu_align_short_noalloc(void* stream, int64_t n, const char* patterns,
                                           const int64_t* pattern_offsets, const int32_t* pattern_lengths,
                                           const char* texts, const int64_t* text_offsets,
                                           const int32_t* text_lengths, wfa_gpu_penalties pen, int32_t max_score,
                                           int32_t* out_scores, int8_t* out_status, uint32_t* out_cigars,
                                           int64_t cap, int64_t* out_cigar_offsets) {
  if (n < 0 || n > kN || cap < 0 || !out_cigar_offsets) return WFA_GPU_EINVAL;
  if (pen.x < 1 || pen.o < 0 || pen.e < 1 || pen.x > WFA_GPU_MAX_PENALTY || pen.o > WFA_GPU_MAX_PENALTY ||
      pen.e > WFA_GPU_MAX_PENALTY)
    return WFA_GPU_EINVAL;
  if (n > 0 && (!patterns || !pattern_lengths || !texts || !text_lengths || !out_scores || !out_status))
    return WFA_GPU_EINVAL;
  if (cap > 0 && !out_cigars) return WFA_GPU_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return WFA_GPU_ECUDA;
  DeviceState* ds = nullptr;
  int rc = setup(device, &ds);
  if (rc) return rc;
  if (n == 0) {
    if (cudaMemsetAsync(out_cigar_offsets, 0, sizeof(int64_t), st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return WFA_GPU_ECUDA;
    return WFA_GPU_OK;
  }
  unsigned char* base = ds->scratch;
  wfa::Ctrl* ctrl = reinterpret_cast<wfa::Ctrl*>(base + kOffCtrl);
  int64_t* scan_tmp = reinterpret_cast<int64_t*>(base + kOffScanTmp);
  const int64_t* poff = pattern_offsets;
  const int64_t* toff = text_offsets;
  // the previous call's contents are still there: clear what must start at 0
  if (cudaMemsetAsync(ctrl, 0, 2 * sizeof(wfa::Ctrl), st) != cudaSuccess) return WFA_GPU_ECUDA;
  if (!poff) {
    int64_t* p = reinterpret_cast<int64_t*>(base + kOffPoff);
    if (wfa::launch_scan(pattern_lengths, n, 0, p, scan_tmp, st) != cudaSuccess) return WFA_GPU_ECUDA;
    poff = p;
  }
  if (!toff) {
    int64_t* p = reinterpret_cast<int64_t*>(base + kOffToff);
    if (wfa::launch_scan(text_lengths, n, 0, p, scan_tmp, st) != cudaSuccess) return WFA_GPU_ECUDA;
    toff = p;
  }
  if (wfa::launch_validate(n, poff, pattern_lengths, toff, text_lengths, ctrl, st) != cudaSuccess)
    return WFA_GPU_ECUDA;
  wfa::Ctrl h{};
  if (cudaMemcpyAsync(&h, ctrl, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return WFA_GPU_ECUDA;
  if (h.bad_input || h.max_len > WFA_GPU_NOALLOC_MAX_LEN) return WFA_GPU_EINVAL;

  const int g = gcd(pen.x, gcd(pen.o, pen.e));
  wfa::AlignArgs a{};
  a.n = n;
  a.pat = patterns; a.poff = poff; a.plen = pattern_lengths;
  a.txt = texts; a.toff = toff; a.tlen = text_lengths;
  a.g = g;
  a.xs = pen.x / g;
  a.es = pen.e / g;
  a.oes = (pen.o + pen.e) / g;
  a.s_cap = max_score > 0 ? max_score / g : INT32_MAX;
  a.score_only = 0;
  a.score = out_scores;
  a.status = out_status;
  a.nruns = reinterpret_cast<int32_t*>(base + kOffNruns);
  a.run_src = reinterpret_cast<int64_t*>(base + kOffRunSrc);
  a.runs = reinterpret_cast<uint32_t*>(base + kOffRuns);
  a.pool = nullptr;
  a.pool_cap = 0;
  // deferred pairs of either kind land in the one list; any makes the call fail
  a.defer_list = reinterpret_cast<int32_t*>(base + kOffDefer);
  a.defer_long_list = a.defer_list;
  a.overflow_list = nullptr;
  a.ctrl = ctrl;
  if (wfa::launch_short(a, ds->plan.v[kVariant], st) != cudaSuccess) return WFA_GPU_ECUDA;
  if (wfa::launch_scan(a.nruns, n, 0, out_cigar_offsets, scan_tmp, st) != cudaSuccess) return WFA_GPU_ECUDA;
  int64_t total = 0;
  if (cudaMemcpyAsync(&h, ctrl, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&total, out_cigar_offsets + n, sizeof total, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return WFA_GPU_ECUDA;
  if (h.internal_error) return WFA_GPU_ECUDA;
  if (h.defer_count > 0 || h.defer_long_count > 0) return WFA_GPU_ENOMEM;  // a pair outgrew the short kernel
  if (total > cap) return WFA_GPU_ECIGAR_CAPACITY;
  if (total > 0) {
    if (wfa::launch_compact(n, a.nruns, a.run_src, a.runs, nullptr, out_cigar_offsets, out_cigars, cap, ctrl, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return WFA_GPU_ECUDA;
  }
  return WFA_GPU_OK;
}
