// internal.h -- hooks shared by the library's translation units; not part
// of the C ABI (hidden symbols).
#pragma once
#include <cstdint>

struct wfa_gpu_ctx;

namespace wfa {

// Asked once by a host-pointer wfa_gpu_align_batch call, when the call's
// CIGAR word count is known (and fits its capacity): returns a buffer of at
// least `words` uint32 words that receives the CIGAR words in place of the
// caller's out_cigars, or NULL (the call then fails with WFA_GPU_ENOMEM).
using CigarSink = uint32_t* (*)(void* user, int64_t words);

// Install (or, with sink NULL, remove) the hook on a context.  Not
// thread-safe against calls on the same context.
__attribute__((visibility("hidden"))) void set_cigar_sink(wfa_gpu_ctx* ctx, CigarSink sink, void* user);

// Run the context's later calls with the scratch arena [arena, arena +
// bytes) of device memory the caller owns (arena teams and slices sized
// for it), or, with arena NULL, with the context's own arena again.  Not
// thread-safe against calls on the same context.
__attribute__((visibility("hidden"))) void set_arena(wfa_gpu_ctx* ctx, void* arena, size_t bytes);

}  // namespace wfa
