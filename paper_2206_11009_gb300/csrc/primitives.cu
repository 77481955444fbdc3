// Exclusive scan and stable LSD radix sort (8-bit digits), written for small-to-medium
// arrays (pricing candidates, support entries: 1e3 .. 1e7 items).
#include "primitives.cuh"

#include <mutex>

namespace ot {

Arena *&active_arena() {
    static thread_local Arena *a = nullptr;
    return a;
}

// ----------------------------------------------------------------------------- scan
namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void __launch_bounds__(kScanThreads)
scan_tile_kernel(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, int64_t n,
                 uint32_t *__restrict__ block_sums) {
    __shared__ uint32_t warp_tot[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t local = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0u;
        uint32_t t = v[k];
        v[k] = local;
        local += t;
    }
    // inclusive warp scan of `local`
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = lane < kScanThreads / 32 ? warp_tot[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = w;
    }
    __syncthreads();
    uint32_t prefix = (x - local) + (wid > 0 ? warp_tot[wid - 1] : 0u);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) out[base + k] = prefix + v[k];
    if (threadIdx.x == kScanThreads - 1 && block_sums) block_sums[blockIdx.x] = prefix + local;
}

__global__ void scan_add_kernel(uint32_t *__restrict__ out, int64_t n,
                                const uint32_t *__restrict__ block_off) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += block_off[i / kScanTile];
}

__global__ void scan_total_kernel(const uint32_t *in, const uint32_t *out, int64_t n,
                                  uint32_t *total) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *total = n > 0 ? out[n - 1] + in[n - 1] : 0u;
}

}  // namespace

Error scan_exclusive_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total,
                         cudaStream_t st) {
    if (n <= 0) {
        if (total) OT_CUDA(cudaMemsetAsync(total, 0, sizeof(uint32_t), st));
        return ok();
    }
    // keep the last input element for the total when scanning in place
    DevTemp<uint32_t> last;
    if (total) {
        OT_TRY(last.alloc(1, st));
        OT_CUDA(cudaMemcpyAsync(last.p, in + n - 1, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    }
    const int64_t nb = ceil_div(n, kScanTile);
    if (nb == 1) {
        scan_tile_kernel<<<1, kScanThreads, 0, st>>>(in, out, n, nullptr);
        OT_LAUNCHED();
    } else {
        DevTemp<uint32_t> sums;
        OT_TRY(sums.alloc(nb, st));
        scan_tile_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, sums.p);
        OT_LAUNCHED();
        OT_TRY(scan_exclusive_u32(sums.p, sums.p, nb, nullptr, st));
        scan_add_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(out, n, sums.p);
        OT_LAUNCHED();
    }
    if (total) {
        scan_total_kernel<<<1, 32, 0, st>>>(last.p, out + n - 1, 1, total);
        OT_LAUNCHED();
    }
    return ok();
}

// ----------------------------------------------------------------------------- radix sort
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortChunks = 16;                       // items per thread per tile
constexpr int kSortTile = kSortThreads * kSortChunks;  // 4096 items per block

__global__ void __launch_bounds__(kSortThreads)
radix_hist_kernel(const uint64_t *__restrict__ keys, int64_t n, int shift, int nblocks,
                  uint32_t *__restrict__ hist /* [256][nblocks] */) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int c = 0; c < kSortChunks; ++c) {
        int64_t i = base + (int64_t)c * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads)
radix_scatter_kernel(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                     uint64_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n,
                     int shift, int nblocks, const uint32_t *__restrict__ offs) {
    __shared__ uint32_t running[256];
    __shared__ uint32_t wcount[kSortWarps][256];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    running[threadIdx.x] = offs[(int64_t)threadIdx.x * nblocks + blockIdx.x];
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int c = 0; c < kSortChunks; ++c) {
        for (int w = 0; w < kSortWarps; ++w) wcount[w][threadIdx.x] = 0;
        __syncthreads();
        const int64_t i = base + (int64_t)c * kSortThreads + threadIdx.x;
        const bool valid = i < n;
        uint64_t k = valid ? kin[i] : ~0ull;
        uint32_t val = valid ? vin[i] : 0u;
        unsigned d = valid ? (unsigned)(k >> shift) & 255u : 256u;   // 256 = padding bucket
        unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned rank = __popc(peers & lt_mask);
        if (valid && rank == 0) wcount[wid][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pos = running[d] + rank;
            for (int w = 0; w < wid; ++w) pos += wcount[w][d];
            kout[pos] = k;
            vout[pos] = val;
        }
        __syncthreads();
        uint32_t add = 0;
        for (int w = 0; w < kSortWarps; ++w) add += wcount[w][threadIdx.x];
        running[threadIdx.x] += add;
        __syncthreads();
    }
}

// Up to kSmallN items: the whole sort in one CTA, both buffers and the per-warp digit counters in
// shared memory, one launch for all passes.  Warp w owns items [w * 256, w * 256 + 256), taken 32
// at a time in index order; per pass a counting sweep (warp-private digit counts: the lane that
// leads each group of equal digits adds the group's size), the exclusive offsets of (digit, warp)
// in digit-major order, and a scatter sweep in the same order (stable).
constexpr int kSmallN = 8192;
constexpr int kSmallThreads = 1024;
constexpr int kSmallWarps = kSmallThreads / 32;
constexpr int kSmallSteps = kSmallN / kSmallThreads;   // 32-item steps per warp
constexpr int kSmallSmem = kSmallN * (8 + 8 + 4 + 4) + kSmallWarps * 256 * 4 + 256 * 4;

__global__ void __launch_bounds__(kSmallThreads, 1)
radix_small_kernel(uint64_t *__restrict__ keys, uint32_t *__restrict__ vals, int n, int passes) {
    extern __shared__ __align__(16) unsigned char sm[];
    uint64_t *K0 = (uint64_t *)sm, *K1 = K0 + kSmallN;
    uint32_t *V0 = (uint32_t *)(K1 + kSmallN), *V1 = V0 + kSmallN;
    uint32_t (*cnt)[256] = (uint32_t (*)[256])(V1 + kSmallN);
    uint32_t *dtot = (uint32_t *)(cnt + kSmallWarps);
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int i = threadIdx.x; i < n; i += kSmallThreads) {
        K0[i] = keys[i];
        V0[i] = vals[i];
    }
    __syncthreads();
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        for (int d = lane; d < 256; d += 32) cnt[w][d] = 0u;
        __syncwarp();
        for (int k = 0; k < kSmallSteps; ++k) {
            const int idx = w * (kSmallSteps * 32) + k * 32 + lane;
            const bool valid = idx < n;
            const unsigned d = valid ? (unsigned)(K0[idx] >> shift) & 255u : 256u;
            const unsigned peers = __match_any_sync(full, d);
            if (valid && (peers & lt) == 0u) cnt[w][d] += (uint32_t)__popc(peers);
            __syncwarp();
        }
        __syncthreads();
        if (threadIdx.x < 256) {
            const int d = threadIdx.x;
            uint32_t run = 0;
            for (int ww = 0; ww < kSmallWarps; ++ww) {
                const uint32_t c = cnt[ww][d];
                cnt[ww][d] = run;
                run += c;
            }
            dtot[d] = run;
        }
        __syncthreads();
        if (threadIdx.x < 32) {   // exclusive scan of the 256 digit totals, 8 per lane
            uint32_t v[8], t = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                v[q] = dtot[lane * 8 + q];
                t += v[q];
            }
            uint32_t x = t;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(full, x, o);
                if (lane >= o) x += y;
            }
            uint32_t pre = x - t;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                dtot[lane * 8 + q] = pre;
                pre += v[q];
            }
        }
        __syncthreads();
        if (threadIdx.x < 256) {
            const uint32_t b = dtot[threadIdx.x];
            for (int ww = 0; ww < kSmallWarps; ++ww) cnt[ww][threadIdx.x] += b;
        }
        __syncthreads();
        for (int k = 0; k < kSmallSteps; ++k) {
            const int idx = w * (kSmallSteps * 32) + k * 32 + lane;
            const bool valid = idx < n;
            const uint64_t key = valid ? K0[idx] : 0ull;
            const uint32_t val = valid ? V0[idx] : 0u;
            const unsigned d = valid ? (unsigned)(key >> shift) & 255u : 256u;
            const unsigned peers = __match_any_sync(full, d);
            const uint32_t rank = (uint32_t)__popc(peers & lt);
            const uint32_t base = valid ? cnt[w][d] : 0u;
            __syncwarp();
            if (valid) {
                K1[base + rank] = key;
                V1[base + rank] = val;
                if (rank == 0u) cnt[w][d] = base + (uint32_t)__popc(peers);
            }
            __syncwarp();
        }
        __syncthreads();
        uint64_t *tk = K0; K0 = K1; K1 = tk;
        uint32_t *tv = V0; V0 = V1; V1 = tv;
    }
    for (int i = threadIdx.x; i < n; i += kSmallThreads) {
        keys[i] = K0[i];
        vals[i] = V0[i];
    }
}

}  // namespace

Error radix_sort_pairs(uint64_t *keys, uint32_t *vals, int64_t n, int key_bits, cudaStream_t st) {
    if (n <= 1 || key_bits <= 0) return ok();
    if (n > 0x7fffffffLL) return fail(OT_ERR_ARG, "radix_sort_pairs: too many items");
    if (n <= kSmallN) {
        static std::once_flag once;
        static cudaError_t attr = cudaSuccess;
        std::call_once(once, [] {
            attr = cudaFuncSetAttribute(radix_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmallSmem);
        });
        if (attr != cudaSuccess) return fail(OT_ERR_CUDA, cudaGetErrorString(attr));
        radix_small_kernel<<<1, kSmallThreads, kSmallSmem, st>>>(keys, vals, (int)n, (key_bits + 7) / 8);
        OT_LAUNCHED();
        return ok();
    }
    const int passes = (key_bits + 7) / 8;
    const int nb = (int)ceil_div(n, kSortTile);
    DevTemp<uint64_t> k2;
    DevTemp<uint32_t> v2, hist;
    OT_TRY(k2.alloc(n, st));
    OT_TRY(v2.alloc(n, st));
    OT_TRY(hist.alloc((int64_t)256 * nb, st));
    uint64_t *ka = keys, *kb = k2.p;
    uint32_t *va = vals, *vb = v2.p;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        radix_hist_kernel<<<nb, kSortThreads, 0, st>>>(ka, n, shift, nb, hist.p);
        OT_LAUNCHED();
        OT_TRY(scan_exclusive_u32(hist.p, hist.p, (int64_t)256 * nb, nullptr, st));
        radix_scatter_kernel<<<nb, kSortThreads, 0, st>>>(ka, va, kb, vb, n, shift, nb, hist.p);
        OT_LAUNCHED();
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    if (ka != keys) {
        OT_CUDA(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st));
        OT_CUDA(cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st));
    }
    return ok();
}

}  // namespace ot
