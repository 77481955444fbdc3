// Tensor-core form of the FP32 dense factor's bulk rank-64 update C -= A_op B_op^T (not yet used by
// the library): tcgen05 MMAs in split TF32 (hi*hi + hi*lo + lo*hi with hi = TF32 rounding, FP32
// accumulation in TMEM), one CTA per 128 x 128 tile.  Standalone and self-checking against an FP64
// CPU product; exits 0 and prints OK when every case is within 1e-5 relative.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o tc_update_check tc_update_check.cu
// Layouts: A_op(r, l) = PA[l * lda + r], B_op(c, l) = PB[l * ldb + c], C(r, c) = C[c * ldc + r].
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>

namespace {

constexpr int TM = 128, TN = 128, TK = 64;   // tile rows, tile columns, depth (the panel width)
constexpr int kThreads = 256;
constexpr int kOpBytes = TM * TK * 4;        // one operand piece (hi or lo): 32 KB
constexpr int kSmem = 4 * kOpBytes + 16;     // A hi, A lo, B hi, B lo, mbarrier, TMEM address
constexpr long long kWaitLimit = 1LL << 22;  // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major canonical layout without swizzle: 8-row x 16-byte core matrices; the core matrix
// (row / 8, k / 4) sits at ((k / 4) * (TM / 8) + row / 8) * 128 bytes, its row (row % 8) at 16-byte
// steps.  So the stride between core matrices along K (LBO) is (TM / 8) * 128 = 2048 bytes and
// along M / N (SBO) 128 bytes.
__device__ __forceinline__ uint32_t kmajor_off(int row, int kq) {
    return (uint32_t)((kq * (TM / 8) + (row >> 3)) * 128 + (row & 7) * 16);
}
constexpr uint32_t kLBO = (TM / 8) * 128;
constexpr uint32_t kSBO = 128;

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((kLBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((kSBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of the tcgen05 family; base offset 0, no swizzle
    return d;
}

// instruction descriptor, kind::tf32: D = F32 (bits 4-5), A = B = TF32 (bits 7-9, 10-12), both
// K-major (bits 15, 16 clear), N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
        :: "r"(tmem), "l"(a), "l"(b), "r"(kIdesc), "r"(acc) : "memory");
}

__device__ __forceinline__ bool wait_parity(uint32_t mbar, uint32_t parity) {
    for (long long i = 0; i < kWaitLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// one CTA per 128 x 128 tile (ti, tj) of a tiles_n x tiles_n grid from (r0base, c0base)
__global__ void __launch_bounds__(kThreads, 1)
tc_update_kernel(int n, int climit, int tri, const float *__restrict__ PA, int lda, const float *__restrict__ PB,
                 int ldb, float *__restrict__ C, int ldc, int r0base, int c0base, int tiles_n, int *err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *mbar = (uint64_t *)(smem + 4 * kOpBytes);
    uint32_t *tslot = (uint32_t *)(smem + 4 * kOpBytes + 8);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = r0base + (int)(blockIdx.x / tiles_n) * TM, c0 = c0base + (int)(blockIdx.x % tiles_n) * TN;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tslot)), "r"(TN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // operands: thread (row, h) stages the k-quads h, h + 2, ... of row `row` of A_op and B_op
    // (four coalesced global loads per quad, one 16-byte shared store per piece)
    {
        const int row = threadIdx.x & (TM - 1), h = threadIdx.x >> 7;
        const int r = r0 + row, c = c0 + row;
        for (int kq = h; kq < TK / 4; kq += 2) {
            float a[4], b[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int l = kq * 4 + j;
                a[j] = r < n ? PA[(size_t)l * lda + r] : 0.f;
                b[j] = c < climit ? PB[(size_t)l * ldb + c] : 0.f;
            }
            float ah[4], al[4], bh[4], bl[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                ah[j] = tf32_round(a[j]);
                al[j] = a[j] - ah[j];
                bh[j] = tf32_round(b[j]);
                bl[j] = b[j] - bh[j];
            }
            const uint32_t off = kmajor_off(row, kq);
            *(float4 *)(smem + off) = make_float4(ah[0], ah[1], ah[2], ah[3]);
            *(float4 *)(smem + kOpBytes + off) = make_float4(al[0], al[1], al[2], al[3]);
            *(float4 *)(smem + 2 * kOpBytes + off) = make_float4(bh[0], bh[1], bh[2], bh[3]);
            *(float4 *)(smem + 3 * kOpBytes + off) = make_float4(bl[0], bl[1], bl[2], bl[3]);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    if (threadIdx.x == 0) {
        const uint32_t base = smem_u32(smem);
        for (int ks = 0; ks < TK / 8; ++ks) {
            const uint32_t koff = (uint32_t)ks * 2 * kLBO;   // 8 tf32 of K = two core matrices
            const uint64_t ah = smem_desc(base + koff), al = smem_desc(base + kOpBytes + koff);
            const uint64_t bh = smem_desc(base + 2 * kOpBytes + koff), bl = smem_desc(base + 3 * kOpBytes + koff);
            mma_tf32(tmem, ah, bh, ks > 0 ? 1u : 0u);
            mma_tf32(tmem, ah, bl, 1u);
            mma_tf32(tmem, al, bh, 1u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(smem_u32(mbar)) : "memory");
    }
    const bool ok = __syncthreads_and(wait_parity(smem_u32(mbar), 0) ? 1 : 0) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
        if (threadIdx.x == 0) atomicExch(err, 1);
    } else {
        // warp w reads TMEM lanes 32 (w % 4) .. (its quarter) and the columns 64 (w / 4) ..
        const int q = warp & 3, ch = warp >> 2;
        const int r = r0 + q * 32 + lane;
#pragma unroll
        for (int part = 0; part < 2; ++part) {
            const int col0 = ch * 64 + part * 32;
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)col0, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int c = c0 + col0 + j;
                if (r < n && c < climit && (!tri || r > c)) C[(size_t)c * ldc + r] -= __uint_as_float(v[j]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TN) : "memory");
}

double run(int n, int tri, bool timing) {
    const int ld = (n + 31) / 32 * 32, tiles = (n + TM - 1) / TM;
    std::vector<float> hA((size_t)TK * ld), hB((size_t)TK * ld), hC((size_t)ld * n);
    srand(12345 + n);
    auto rnd = [] { return (float)rand() / (float)RAND_MAX; };
    for (auto &x : hA) x = -rnd();
    for (auto &x : hB) x = -rnd();
    for (auto &x : hC) x = -rnd();
    float *dA, *dB, *dC;
    int *derr;
    cudaMalloc(&dA, hA.size() * 4);
    cudaMalloc(&dB, hB.size() * 4);
    cudaMalloc(&dC, hC.size() * 4);
    cudaMalloc(&derr, 4);
    cudaMemcpy(dA, hA.data(), hA.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(dB, hB.data(), hB.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(dC, hC.data(), hC.size() * 4, cudaMemcpyHostToDevice);
    cudaMemset(derr, 0, 4);
    cudaFuncSetAttribute(tc_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    tc_update_kernel<<<tiles * tiles, kThreads, kSmem>>>(n, n, tri, dA, ld, dB, ld, dC, ld, 0, 0, tiles, derr);
    cudaError_t e = cudaDeviceSynchronize();
    int herr = 0;
    cudaMemcpy(&herr, derr, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess || herr) {
        printf("n=%d: %s, wait timeout flag %d\n", n, cudaGetErrorString(e), herr);
        return -1;
    }
    std::vector<float> gC(hC.size());
    cudaMemcpy(gC.data(), dC, gC.size() * 4, cudaMemcpyDeviceToHost);
    double worst = 0.0;
    for (int c = 0; c < n; ++c)
        for (int r = 0; r < n; ++r) {
            double want = hC[(size_t)c * ld + r];
            if (!tri || r > c) {
                double s = 0.0;
                for (int l = 0; l < TK; ++l) s += (double)hA[(size_t)l * ld + r] * (double)hB[(size_t)l * ld + c];
                want -= s;
            }
            worst = fmax(worst, fabs((double)gC[(size_t)c * ld + r] - want) / (1.0 + fabs(want)));
        }
    if (timing) {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a);
        for (int it = 0; it < 10; ++it)
            tc_update_kernel<<<tiles * tiles, kThreads, kSmem>>>(n, n, 0, dA, ld, dB, ld, dC, ld, 0, 0, tiles, derr);
        cudaEventRecord(b);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        const double flops = 2.0 * TK * (double)n * n;   // useful work of one launch
        printf("n=%d: %.1f us per launch, %.1f TFLOP/s useful (x3 tensor work)\n", n, 1e3 * ms / 10,
               flops / (1e-3 * ms / 10) / 1e12);
    }
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dC);
    cudaFree(derr);
    return worst;
}

}  // namespace

int main() {
    int bad = 0;
    for (int n : {128, 300, 1000}) {
        for (int tri = 0; tri < 2; ++tri) {
            const double w = run(n, tri, false);
            printf("n=%d tri=%d: max |gpu - fp64| / (1 + |ref|) = %.3e\n", n, tri, w);
            if (!(w >= 0 && w < 1e-5)) bad = 1;
        }
    }
    if (!bad) run(4096, 0, true);
    printf(bad ? "FAILED\n" : "OK\n");
    return bad;
}
