// Dense LDL^T of the assembled Schur complement S_M (Section 4.2's direct solve) for moderate n.
//
// When the support is still large, the exact factor of S_M is a sizeable fraction of dense
// (a quarter of n^2 on 64x64 images), and a sparse factorisation then only adds dependency-chain
// latency.  This path factors the dense matrix (column-major, FP64) with a blocked right-looking
// LDL^T: per panel of kB columns
//   (1) the kB x kB diagonal block in shared memory, one CTA (pivots keeping less than eps of
//       their original diagonal become +infinity: the column is zeroed, Section 4.2);
//   (2) the panel below, L21 = A21 L11^-T D1^-1, one thread per row, and LD = L21 D1;
//   (3) the trailing update A22 -= LD L21^T on 64 x 64 tiles of the lower triangle.
// Solves run in one cooperative launch: forward and backward substitution panel by panel with a
// bounded grid barrier between the diagonal-block step and the update of the rest.
#include "chol.cuh"
#include "primitives.cuh"

#include <cmath>

namespace ot {
namespace {

constexpr int kB = 64;      // panel width
constexpr int kT = 256;

#define GSD(var, count) \
    for (int64_t var = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; var < (count); var += (int64_t)gridDim.x * blockDim.x)

inline unsigned gridd(int64_t work) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(4096, ceil_div(work, kT)));
}

__global__ void dense_scatter_kernel(int n, const int32_t *__restrict__ Ap, const int32_t *__restrict__ Aj,
                                     const double *__restrict__ Ax, const double *__restrict__ Adiag,
                                     double *__restrict__ A, double *__restrict__ d0) {
    GSD(r, n) {
        for (int e = Ap[r]; e < Ap[r + 1]; ++e) A[(int64_t)Aj[e] * n + r] = Ax[e];
        A[(int64_t)r * n + r] = Adiag[r];
        d0[r] = Adiag[r];
    }
}

// (1) diagonal block [k, k+bs) in shared memory
__global__ void __launch_bounds__(kT)
dense_diag_kernel(int n, int k, int bs, double *__restrict__ A, double *__restrict__ D,
                  const double *__restrict__ d0, double eps, double *__restrict__ Linv) {
    __shared__ double S[kB][kB + 1];
    __shared__ double s_d;
    __shared__ int s_inf;
    for (int t = threadIdx.x; t < bs * bs; t += blockDim.x) {
        const int i = t % bs, j = t / bs;
        S[i][j] = (i >= j) ? A[(int64_t)(k + j) * n + (k + i)] : 0.0;
    }
    __syncthreads();
    for (int j = 0; j < bs; ++j) {
        if (threadIdx.x == 0) {
            const double d = S[j][j];
            s_inf = !(d > eps * d0[k + j]);
            s_d = d;
            D[k + j] = s_inf ? INFINITY : d;
        }
        __syncthreads();
        const double d = s_d;
        const int inf = s_inf;
        for (int i = j + 1 + threadIdx.x; i < bs; i += blockDim.x) S[i][j] = inf ? 0.0 : S[i][j] / d;
        __syncthreads();
        if (!inf) {
            // S[i][l] -= l_ij d l_lj  for j < l <= i < bs
            const int m2 = bs - j - 1;
            for (int t = threadIdx.x; t < m2 * m2; t += blockDim.x) {
                const int i = j + 1 + t / m2, l = j + 1 + t % m2;
                if (l <= i) S[i][l] -= S[i][j] * d * S[l][j];
            }
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < bs * bs; t += blockDim.x) {
        const int i = t % bs, j = t / bs;
        if (i > j) A[(int64_t)(k + j) * n + (k + i)] = S[i][j];
    }
    // inverse of the unit lower block, column by column: X[:,c] solves L X[:,c] = e_c, written
    // to Linv (row k+i, column c) so that the solves need no serial substitution
    __syncthreads();
    for (int c = threadIdx.x; c < bs; c += blockDim.x) {
        double x[kB];
        for (int i = 0; i < bs; ++i) {
            double t = (i == c) ? 1.0 : 0.0;
            for (int l = c; l < i; ++l) t -= S[i][l] * x[l];
            x[i] = (i < c) ? 0.0 : t;
        }
        for (int i = 0; i < bs; ++i) Linv[(int64_t)c * n + (k + i)] = x[i];
    }
}

// (2) panel rows r in [k+bs, n): x D1 L11^T = A(r, k:k+bs)  ->  L21(r,:) = x, LD(r,:) = x D1
__global__ void __launch_bounds__(kT)
dense_panel_kernel(int n, int k, int bs, double *__restrict__ A, const double *__restrict__ D,
                   double *__restrict__ LD /* n x kB, column-major with ld n */) {
    __shared__ double L11[kB][kB + 1];
    __shared__ double Ds[kB];
    for (int t = threadIdx.x; t < bs * bs; t += blockDim.x) {
        const int i = t % bs, j = t / bs;
        L11[i][j] = (i > j) ? A[(int64_t)(k + j) * n + (k + i)] : 0.0;
    }
    for (int t = threadIdx.x; t < bs; t += blockDim.x) Ds[t] = D[k + t];
    __syncthreads();
    const int r = k + bs + blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double x[kB];
#pragma unroll 8
    for (int j = 0; j < kB; ++j) {
        if (j >= bs) break;
        double t = A[(int64_t)(k + j) * n + r];
        for (int l = 0; l < j; ++l) t -= x[l] * Ds[l] * L11[j][l];
        const double dj = Ds[j];
        x[j] = isinf(dj) ? 0.0 : t / dj;
    }
    for (int j = 0; j < bs; ++j) {
        A[(int64_t)(k + j) * n + r] = x[j];
        const double dj = Ds[j];
        LD[(int64_t)j * n + r] = isinf(dj) ? 0.0 : x[j] * dj;
    }
}

// (3) A22(r, c) -= sum_l LD(r, l) L21(c, l) on the lower triangle, 64x64 tiles, 4x4 per thread
__global__ void __launch_bounds__(kT)
dense_update_kernel(int n, int k, int bs, double *__restrict__ A, const double *__restrict__ LD) {
    const int base = k + bs;
    const int t = (n - base + 63) / 64;
    // tile index -> (ti, tj) with ti >= tj
    const int idx = blockIdx.x;
    int ti = (int)((sqrt(8.0 * idx + 1.0) - 1.0) * 0.5);
    while ((ti + 1) * (ti + 2) / 2 <= idx) ++ti;
    while (ti * (ti + 1) / 2 > idx) --ti;
    const int tj = idx - ti * (ti + 1) / 2;
    if (ti >= t) return;
    __shared__ double Ls[32][64 + 1];   // LD rows of tile ti   [l][r]
    __shared__ double Rs[32][64 + 1];   // L21 rows of tile tj  [l][c]
    const int r0 = base + ti * 64, c0 = base + tj * 64;
    const int tr = (threadIdx.x % 16) * 4, tc = (threadIdx.x / 16) * 4;
    double acc[4][4] = {};
    for (int l0 = 0; l0 < bs; l0 += 32) {
        const int lb = min(32, bs - l0);
        __syncthreads();
        for (int q = threadIdx.x; q < lb * 64; q += blockDim.x) {
            const int l = q / 64, rr = q % 64;
            const int r = r0 + rr, c = c0 + rr;
            Ls[l][rr] = r < n ? LD[(int64_t)(l0 + l) * n + r] : 0.0;
            Rs[l][rr] = c < n ? A[(int64_t)(k + l0 + l) * n + c] : 0.0;
        }
        __syncthreads();
        for (int l = 0; l < lb; ++l) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) { a[u] = Ls[l][tr + u]; b[u] = Rs[l][tc + u]; }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[u][w] += a[u] * b[w];
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int r = r0 + tr + u, c = c0 + tc + w;
            if (r < n && c < n && r >= c) A[(int64_t)c * n + r] -= acc[u][w];
        }
}

// forward L z = b, y = D^-1 z, backward L^T x = y; one cooperative launch.  The diagonal blocks
// are applied through their stored inverses (small GEMVs by block 0), the off-diagonal panels by
// all blocks; one grid barrier after each step.
__global__ void __launch_bounds__(kT)
dense_solve_kernel(int n, const double *__restrict__ A, const double *__restrict__ Linv,
                   const double *__restrict__ D, const double *__restrict__ b, double *z, double *x,
                   double *part /* gridDim x kB */, unsigned *bar, int *err) {
    __shared__ double vb[kB];
    __shared__ double red[kT / 32][32];
    __shared__ double Ls[kB][kB + 1];      // inverse diagonal block (block 0 only)
    const int lane = threadIdx.x & 31;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = tid; r < n; r += stride) z[r] = b[r];
    if (!grid_barrier(bar, gridDim.x, err)) return;
    // ---- forward
    for (int k = 0; k < n; k += kB) {
        const int bs = min(kB, n - k);
        if (blockIdx.x == 0) {
            // z_blk = L11^-1 z_blk, the inverse block staged in shared memory
            for (int q = threadIdx.x; q < kB * kB; q += blockDim.x) {
                const int i = q % kB, c = q / kB;
                Ls[c][i] = (i < bs && c < bs) ? Linv[(int64_t)c * n + (k + i)] : 0.0;
            }
            if (threadIdx.x < kB) vb[threadIdx.x] = threadIdx.x < bs ? z[k + threadIdx.x] : 0.0;
            __syncthreads();
            if (threadIdx.x < bs) {
                const int i = threadIdx.x;
                double t = 0;
#pragma unroll 16
                for (int c = 0; c < kB; ++c) t += Ls[c][i] * vb[c];
                z[k + i] = t;
            }
            __syncthreads();
        }
        if (!grid_barrier(bar, gridDim.x, err)) return;
        if (k + bs < n) {
            if (threadIdx.x < kB) vb[threadIdx.x] = threadIdx.x < bs ? z[k + threadIdx.x] : 0.0;
            __syncthreads();
            for (int64_t r = k + bs + tid; r < n; r += stride) {
                double acc = 0;
                if (bs == kB) {
#pragma unroll 16
                    for (int l = 0; l < kB; ++l) acc += A[(int64_t)(k + l) * n + r] * vb[l];
                } else {
                    for (int l = 0; l < bs; ++l) acc += A[(int64_t)(k + l) * n + r] * vb[l];
                }
                z[r] -= acc;
            }
            __syncthreads();
            if (!grid_barrier(bar, gridDim.x, err)) return;
        }
    }
    // ---- diagonal
    for (int64_t r = tid; r < n; r += stride) x[r] = isinf(D[r]) ? 0.0 : z[r] / D[r];
    if (!grid_barrier(bar, gridDim.x, err)) return;
    // ---- backward: t = y_blk - L21^T x_rest, then x_blk = L11^-T t
    for (int k = ((n - 1) / kB) * kB; k >= 0; k -= kB) {
        const int bs = min(kB, n - k);
        if (k + bs < n) {
            for (int h = 0; h < bs; h += 32) {
                const int hb = min(32, bs - h);
                double acc[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[j] = 0.0;
                for (int64_t r = k + bs + tid; r < n; r += stride) {
                    const double xr = x[r];
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (j < hb) acc[j] += A[(int64_t)(k + h + j) * n + r] * xr;
                }
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const double v = warp_sum(acc[j]);
                    if (lane == 0) red[threadIdx.x >> 5][j] = v;
                }
                __syncthreads();
                if (threadIdx.x < hb) {
                    double sum = 0;
                    for (int w = 0; w < kT / 32; ++w) sum += red[w][threadIdx.x];
                    part[(int64_t)blockIdx.x * kB + h + threadIdx.x] = sum;
                }
                __syncthreads();
            }
            if (!grid_barrier(bar, gridDim.x, err)) return;
        }
        if (blockIdx.x == 0) {
            for (int q = threadIdx.x; q < kB * kB; q += blockDim.x) {
                const int i = q % kB, c = q / kB;
                Ls[c][i] = (i < bs && c < bs) ? Linv[(int64_t)c * n + (k + i)] : 0.0;
            }
            if (threadIdx.x < kB) {
                double t = 0.0;
                if (threadIdx.x < bs) {
                    t = x[k + threadIdx.x];
                    if (k + bs < n)
                        for (unsigned g = 0; g < gridDim.x; ++g) t -= part[(int64_t)g * kB + threadIdx.x];
                }
                vb[threadIdx.x] = t;
            }
            __syncthreads();
            if (threadIdx.x < bs) {
                const int c = threadIdx.x;  // x_c = sum_i Linv(i, c) t_i   (L11^-T t)
                double v = 0;
#pragma unroll 16
                for (int i = 0; i < kB; ++i) v += Ls[c][i] * vb[i];
                x[k + c] = v;
            }
            __syncthreads();
        }
        if (!grid_barrier(bar, gridDim.x, err)) return;
    }
}

}  // namespace

Error dense_alloc(DenseLDL &M, int32_t n) {
    M.n = n;
    OT_CUDA(cudaMalloc((void **)&M.A, sizeof(double) * (size_t)n * n));
    OT_CUDA(cudaMalloc((void **)&M.LD, sizeof(double) * (size_t)n * kB));
    OT_CUDA(cudaMalloc((void **)&M.Linv, sizeof(double) * (size_t)n * kB));
    OT_CUDA(cudaMalloc((void **)&M.D, sizeof(double) * n));
    OT_CUDA(cudaMalloc((void **)&M.d0, sizeof(double) * n));
    OT_CUDA(cudaMalloc((void **)&M.z, sizeof(double) * n));
    OT_CUDA(cudaMalloc((void **)&M.part, sizeof(double) * 4096 * kB));
    OT_CUDA(cudaMalloc((void **)&M.bar, sizeof(unsigned) * 2));
    OT_CUDA(cudaMalloc((void **)&M.err, sizeof(int)));
    return ok();
}

void dense_free(DenseLDL &M) {
    for (void *p : {(void *)M.A, (void *)M.LD, (void *)M.Linv, (void *)M.D, (void *)M.d0, (void *)M.z, (void *)M.part,
                    (void *)M.bar, (void *)M.err})
        if (p) cudaFree(p);
    M = DenseLDL();
}

Error dense_factor(DenseLDL &M, const Chol &C, double eps, cudaStream_t st) {
    const int n = M.n;
    OT_CUDA(cudaMemsetAsync(M.A, 0, sizeof(double) * (size_t)n * n, st));
    dense_scatter_kernel<<<gridd(n), kT, 0, st>>>(n, C.Ap, C.Aj, C.Ax, C.Adiag, M.A, M.d0);
    OT_LAUNCHED();
    ktimer_begin(KT_LDL_NUMERIC, st);
    for (int k = 0; k < n; k += kB) {
        const int bs = std::min(kB, n - k);
        dense_diag_kernel<<<1, kT, 0, st>>>(n, k, bs, M.A, M.D, M.d0, eps, M.Linv);
        OT_LAUNCHED();
        if (k + bs < n) {
            dense_panel_kernel<<<(unsigned)ceil_div(n - k - bs, kT), kT, 0, st>>>(n, k, bs, M.A, M.D, M.LD);
            OT_LAUNCHED();
            const int t = (int)ceil_div(n - k - bs, 64);
            dense_update_kernel<<<(unsigned)(t * (t + 1) / 2), kT, 0, st>>>(n, k, bs, M.A, M.LD);
            OT_LAUNCHED();
        }
    }
    ktimer_end(KT_LDL_NUMERIC, st);
    ktimer_add_work(KT_LDL_NUMERIC, (double)n * n * n / 3.0);  // L D L^T: n^3/3 flops
    return ok();
}

Error dense_solve(DenseLDL &M, const double *b, double *x, cudaStream_t st) {
    int dev = 0, sms = 0, per_sm = 0;
    OT_CUDA(cudaGetDevice(&dev));
    OT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    OT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dense_solve_kernel, kT, 0));
    int grid = std::max(1, std::min<int>(std::min(per_sm, 2) * sms, (int)ceil_div(M.n, kT)));
    grid = std::min(grid, 4096);
    OT_CUDA(cudaMemsetAsync(M.bar, 0, 2 * sizeof(unsigned), st));
    int n = M.n;
    const double *A = M.A, *Li = M.Linv, *D = M.D;
    double *z = M.z, *part = M.part;
    unsigned *bar = M.bar;
    int *err = M.err;
    void *args[] = {&n, &A, &Li, &D, &b, &z, &x, &part, &bar, &err};
    ktimer_begin(KT_LDL_SOLVE, st);
    OT_CUDA(cudaLaunchCooperativeKernel((void *)dense_solve_kernel, dim3(grid), dim3(kT), args, 0, st));
    OT_LAUNCHED();
    ktimer_end(KT_LDL_SOLVE, st);
    ktimer_add_work(KT_LDL_SOLVE, 8.0 * (double)n * n);  // reads L twice
    return ok();
}

}  // namespace ot
