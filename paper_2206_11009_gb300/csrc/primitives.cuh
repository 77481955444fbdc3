// Device-wide primitives: exclusive scan and a stable LSD radix sort of (uint64 key, uint32
// value) pairs.  Host launchers; temporaries come from the stream-ordered allocator.
#pragma once

#include "common.cuh"

namespace ot {

// out[i] = sum_{k<i} in[k]; if total != nullptr, *total (device) = sum of all.  In-place OK.
Error scan_exclusive_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total,
                         cudaStream_t st);

// Stable sort of n pairs by the bits [0, key_bits) of keys (values follow).  Sorted output is
// written back into keys/vals.  key_bits is rounded up to a multiple of 8.
Error radix_sort_pairs(uint64_t *keys, uint32_t *vals, int64_t n, int key_bits, cudaStream_t st);

// Caller-provided device workspace handed out as a stack (LIFO release).  While one is active on
// the calling thread (ArenaScope), DevTemp draws from it instead of the stream-ordered allocator.
struct Arena {
    char *base = nullptr;
    size_t size = 0;
    size_t top = 0;
    size_t high = 0;  // high-water mark
};
Arena *&active_arena();

struct ArenaScope {
    Arena *prev;
    explicit ArenaScope(Arena *a) : prev(active_arena()) { active_arena() = a; }
    ~ArenaScope() { active_arena() = prev; }
};

// Temporary device buffer: stream-ordered (cudaMallocAsync / cudaFreeAsync), or carved from the
// active Arena when there is one.
template <typename T>
struct DevTemp {
    T *p = nullptr;
    cudaStream_t st = nullptr;
    Arena *arena = nullptr;
    size_t mark = 0;
    DevTemp() = default;
    DevTemp(const DevTemp &) = delete;
    DevTemp &operator=(const DevTemp &) = delete;
    Error alloc(int64_t count, cudaStream_t s) {
        st = s;
        if (count <= 0) count = 1;
        const size_t bytes = sizeof(T) * (size_t)count;
        if (Arena *a = active_arena()) {
            const size_t off = (a->top + 255) & ~(size_t)255;
            if (off + bytes > a->size)
                return fail(OT_ERR_BUF_TOO_SMALL, "device workspace exhausted");
            arena = a;
            mark = a->top;
            p = (T *)(a->base + off);
            a->top = off + bytes;
            if (a->top > a->high) a->high = a->top;
            return ok();
        }
        OT_CUDA(cudaMallocAsync((void **)&p, bytes, s));
        return ok();
    }
    ~DevTemp() {
        if (arena) {
            if (p) arena->top = mark;
        } else if (p) {
            cudaFreeAsync(p, st);
        }
    }
};

}  // namespace ot
