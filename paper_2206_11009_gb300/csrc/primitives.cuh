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

// Stream-ordered temporary buffer (cudaMallocAsync / cudaFreeAsync).
template <typename T>
struct DevTemp {
    T *p = nullptr;
    cudaStream_t st = nullptr;
    DevTemp() = default;
    DevTemp(const DevTemp &) = delete;
    DevTemp &operator=(const DevTemp &) = delete;
    Error alloc(int64_t count, cudaStream_t s) {
        st = s;
        if (count <= 0) count = 1;
        OT_CUDA(cudaMallocAsync((void **)&p, sizeof(T) * (size_t)count, s));
        return ok();
    }
    ~DevTemp() {
        if (p) cudaFreeAsync(p, st);
    }
};

}  // namespace ot
