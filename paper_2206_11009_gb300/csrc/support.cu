// Support bookkeeping kernels: initial support, views, removal selection, merge.
#include "support.cuh"
#include "pricing.cuh"
#include "primitives.cuh"

#include <algorithm>
#include <vector>

namespace ot {
namespace {

int host_bits_for(uint64_t maxkey) {
    int b = 1;
    while (b < 64 && (maxkey >> b)) ++b;
    return b;
}

constexpr int kIT = 64;  // init tile: 64 x 64 pairs, 256 threads

// PHASE 0: per-row and per-column minimum cost key.  PHASE 1: smallest index attaining it,
// plus the pairs with c <= thr (appended).
template <int PHASE>
__global__ void __launch_bounds__(256)
init_scan_kernel(CostDev c, double thr, unsigned long long *__restrict__ rowmin,
                 unsigned long long *__restrict__ colmin, unsigned *__restrict__ rowarg,
                 unsigned *__restrict__ colarg, uint64_t *__restrict__ keys, unsigned long long cap,
                 unsigned long long *__restrict__ cnt) {
    __shared__ unsigned long long s_row[kIT], s_col[kIT];
    const int m = c.m, n = c.n;
    const int nbj = (n + kIT - 1) / kIT;
    const int64_t ntiles = (int64_t)((m + kIT - 1) / kIT) * nbj;
    const int tx = threadIdx.x & (kIT - 1), ty = threadIdx.x / kIT;  // ty in [0, 4)
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int i0 = (int)(t / nbj) * kIT, j0 = (int)(t % nbj) * kIT;
        __syncthreads();
        if (threadIdx.x < kIT) { s_row[threadIdx.x] = ~0ull; s_col[threadIdx.x] = ~0ull; }
        __syncthreads();
        const int j = j0 + tx;
        unsigned long long cbest = ~0ull;
        for (int r = ty; r < kIT; r += 4) {
            const int i = i0 + r;
            if (i >= m || j >= n) continue;
            const double cc = cost_at(c, i, j);
            const unsigned long long k = f64_key(cc);
            if (PHASE == 0) {
                atomicMin(&s_row[r], k);
                cbest = min(cbest, k);
            } else {
                if (k == rowmin[i]) atomicMin(&s_row[r], (unsigned long long)j);
                if (k == colmin[j]) cbest = min(cbest, (unsigned long long)i);
                if (cc <= thr) {
                    unsigned long long pos = atomicAdd(cnt, 1ull);
                    if (pos < cap) keys[pos] = (uint64_t)i * (uint64_t)n + (uint64_t)j;
                }
            }
        }
        if (j < n && cbest != ~0ull) atomicMin(&s_col[tx], cbest);
        __syncthreads();
        if (threadIdx.x < kIT) {
            const int i = i0 + threadIdx.x, jj = j0 + threadIdx.x;
            if (PHASE == 0) {
                if (i < m && s_row[threadIdx.x] != ~0ull) atomicMin(&rowmin[i], s_row[threadIdx.x]);
                if (jj < n && s_col[threadIdx.x] != ~0ull) atomicMin(&colmin[jj], s_col[threadIdx.x]);
            } else {
                if (i < m && s_row[threadIdx.x] != ~0ull) atomicMin(&rowarg[i], (unsigned)s_row[threadIdx.x]);
                if (jj < n && s_col[threadIdx.x] != ~0ull) atomicMin(&colarg[jj], (unsigned)s_col[threadIdx.x]);
            }
        }
    }
}

__global__ void init_extra_keys(int m, int n, const unsigned *__restrict__ rowarg,
                                const unsigned *__restrict__ colarg, uint64_t *__restrict__ keys) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)m + n;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t < m) keys[t] = (uint64_t)t * n + rowarg[t];
        else keys[t] = (uint64_t)colarg[t - m] * n + (uint64_t)(t - m);
    }
}

__global__ void unique_flags(int64_t cnt, const uint64_t *__restrict__ keys, uint32_t *__restrict__ f) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x)
        f[t] = (t == 0 || keys[t] != keys[t - 1]) ? 1u : 0u;
}

__global__ void unique_scatter(int64_t cnt, int n, const uint64_t *__restrict__ keys, const uint32_t *__restrict__ f,
                               const uint32_t *__restrict__ pos, int32_t *__restrict__ oi, int32_t *__restrict__ oj) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x)
        if (f[t]) {
            oi[pos[t]] = (int32_t)(keys[t] / (uint64_t)n);
            oj[pos[t]] = (int32_t)(keys[t] % (uint64_t)n);
        }
}

// ------------------------------------------------------------------------- views
__global__ void col_keys_kernel(int64_t psi, const int32_t *__restrict__ j, uint64_t *__restrict__ key,
                                uint32_t *__restrict__ val) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < psi; e += (int64_t)gridDim.x * blockDim.x) {
        key[e] = (uint64_t)j[e];
        val[e] = (uint32_t)e;
    }
}

__global__ void col_view_kernel(int64_t psi, const uint32_t *__restrict__ val, const int32_t *__restrict__ si,
                                int32_t *__restrict__ perm, int32_t *__restrict__ crow) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < psi; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = (int32_t)val[k];
        perm[k] = e;
        crow[k] = si[e];
    }
}

__global__ void col_ptr_kernel(int64_t psi, int n, const uint64_t *__restrict__ sorted_j, int32_t *__restrict__ cp) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q <= n; q += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = psi;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (sorted_j[mid] < (uint64_t)q) lo = mid + 1; else hi = mid;
        }
        cp[q] = (int32_t)lo;
    }
}

// ------------------------------------------------------------------------- removal
__global__ void removal_cand_kernel(int64_t psi, const int32_t *__restrict__ si, const int32_t *__restrict__ sj,
                                    const double *__restrict__ p, const double *__restrict__ s,
                                    const double *__restrict__ a, const double *__restrict__ b, double frac,
                                    uint8_t *__restrict__ flag) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < psi; e += (int64_t)gridDim.x * blockDim.x) {
        const double thr = frac * fmin(a[si[e]], b[sj[e]]);
        flag[e] = (p[e] < thr && p[e] / s[e] < 1.0) ? 1 : 0;
    }
}

__global__ void count_flags_kernel(int64_t psi, const uint8_t *__restrict__ flag, uint32_t *__restrict__ f32) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < psi; e += (int64_t)gridDim.x * blockDim.x)
        f32[e] = flag[e];
}

__global__ void removal_keys_kernel(int64_t psi, int m, const uint32_t *__restrict__ f32, const uint32_t *__restrict__ pos,
                                    const int32_t *__restrict__ si, const int32_t *__restrict__ sj,
                                    uint64_t *__restrict__ key, uint32_t *__restrict__ val) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < psi; e += (int64_t)gridDim.x * blockDim.x)
        if (f32[e]) {
            key[pos[e]] = (uint64_t)si[e] + (uint64_t)sj[e] * (uint64_t)m;
            val[pos[e]] = (uint32_t)e;
        }
}

__global__ void removal_rekey_kernel(int64_t cnt, const uint32_t *__restrict__ val, const double *__restrict__ p,
                                     uint64_t *__restrict__ key) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += (int64_t)gridDim.x * blockDim.x)
        key[k] = f64_key(p[val[k]]);
}

__global__ void removal_trim_kernel(int64_t cnt, int64_t kmax, const uint32_t *__restrict__ val, uint8_t *__restrict__ flag) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += (int64_t)gridDim.x * blockDim.x)
        if (k >= kmax) flag[val[k]] = 0;
}

// ------------------------------------------------------------------------- merge
// ---- maximum-weight spanning forest of the support graph by Boruvka rounds.  Edge order: larger
// p first, then smaller jlin = i + j*m (all keys distinct, so the forest is unique and equals the
// one Kruskal's rule builds).  Vertices: sources 0..m-1, targets m..m+n-1.
__global__ void bv_reset_kernel(int V, unsigned long long *__restrict__ bestp, unsigned long long *__restrict__ bestk) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
        bestp[v] = 0ull;
        bestk[v] = ~0ull;
    }
}

// heaviest p leaving each component (positive doubles order like their bit patterns)
__global__ void bv_max_kernel(int64_t psi, int m, const int32_t *__restrict__ si, const int32_t *__restrict__ sj,
                              const double *__restrict__ p, const int32_t *__restrict__ comp,
                              unsigned long long *__restrict__ bestp) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < psi; e += (int64_t)gridDim.x * blockDim.x) {
        const int cu = comp[si[e]], cv = comp[m + sj[e]];
        if (cu == cv) continue;
        const unsigned long long b = (unsigned long long)__double_as_longlong(p[e]);
        atomicMax(&bestp[cu], b);
        atomicMax(&bestp[cv], b);
    }
}

// among the edges of that p, the smallest jlin
__global__ void bv_tie_kernel(int64_t psi, int m, const int32_t *__restrict__ si, const int32_t *__restrict__ sj,
                              const double *__restrict__ p, const int32_t *__restrict__ comp,
                              const unsigned long long *__restrict__ bestp, unsigned long long *__restrict__ bestk) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < psi; e += (int64_t)gridDim.x * blockDim.x) {
        const int cu = comp[si[e]], cv = comp[m + sj[e]];
        if (cu == cv) continue;
        const unsigned long long b = (unsigned long long)__double_as_longlong(p[e]);
        const unsigned long long jl = (unsigned long long)si[e] + (unsigned long long)sj[e] * (unsigned long long)m;
        if (bestp[cu] == b) atomicMin(&bestk[cu], jl);
        if (bestp[cv] == b) atomicMin(&bestk[cv], jl);
    }
}

// every component root takes its chosen edge into the forest and hooks onto the component at its
// other end; of two components that chose the same edge, the smaller id hooks onto the larger
__global__ void bv_hook_kernel(int V, int m, const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ sj,
                               const int32_t *__restrict__ comp, const unsigned long long *__restrict__ bestp,
                               const unsigned long long *__restrict__ bestk, int32_t *__restrict__ parent,
                               uint8_t *__restrict__ flag, int *__restrict__ changed) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < V; c += gridDim.x * blockDim.x) {
        if (comp[c] != c || bestp[c] == 0ull) continue;
        const unsigned long long jl = bestk[c];
        const int i = (int)(jl % (unsigned long long)m), j = (int)(jl / (unsigned long long)m);
        int lo = row_ptr[i], hi = row_ptr[i + 1];  // the support is sorted by (i, j)
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (sj[mid] < j) lo = mid + 1; else hi = mid;
        }
        flag[lo] = 0;
        const int ci = comp[i], cj = comp[m + j];
        const int other = ci == c ? cj : ci;
        const bool mutual = bestk[other] == jl && bestp[other] == bestp[c];
        if (!mutual || c < other) parent[c] = other;
        *changed = 1;
    }
}

// comp[v] <- root of its hook chain (at most 64 steps per launch; *more when a chain is longer)
__global__ void bv_jump_kernel(int V, const int32_t *__restrict__ parent, int32_t *__restrict__ comp, int *__restrict__ more) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
        int r = comp[v];
        for (int s = 0; s < 64 && parent[r] != r; ++s) r = parent[r];
        comp[v] = r;
        if (parent[r] != r) *more = 1;
    }
}

// All Boruvka rounds in one cooperative launch: the same five stages per round as the kernels
// above, separated by grid barriers instead of launches, and the round / jump-pass decisions taken
// by every block from flags that a barrier has published (one fresh flag word per round and per
// jump pass, zeroed before the launch, so no block can see a flag reset under it).
struct BvArgs {
    int64_t psi;
    int m, V, max_passes;             // jump passes per round at most (chains of 64 steps each)
    const int32_t *si, *sj, *row_ptr;
    const double *p;
    int32_t *comp, *parent;
    unsigned long long *bestp, *bestk;
    uint8_t *flag;
    int *changed;                     // [64]: a component hooked in round r
    int *more;                        // [64 * max_passes]: a chain outlived jump pass k of round r
    unsigned *bar;
    int *err;                         // barrier timeout; 2 = a round needed more jump passes
};

__global__ void __launch_bounds__(256) bv_coop_kernel(BvArgs A) {
    const unsigned G = gridDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)G * blockDim.x;
    for (int64_t v = tid; v < A.V; v += stride) {
        A.comp[v] = (int32_t)v;
        A.parent[v] = (int32_t)v;
    }
    if (!grid_barrier(A.bar, G, A.err)) return;
    for (int round = 0; round < 64; ++round) {
        for (int64_t v = tid; v < A.V; v += stride) {
            A.bestp[v] = 0ull;
            A.bestk[v] = ~0ull;
        }
        if (!grid_barrier(A.bar, G, A.err)) return;
        for (int64_t e = tid; e < A.psi; e += stride) {
            const int cu = A.comp[A.si[e]], cv = A.comp[A.m + A.sj[e]];
            if (cu == cv) continue;
            const unsigned long long b = (unsigned long long)__double_as_longlong(A.p[e]);
            atomicMax(&A.bestp[cu], b);
            atomicMax(&A.bestp[cv], b);
        }
        if (!grid_barrier(A.bar, G, A.err)) return;
        for (int64_t e = tid; e < A.psi; e += stride) {
            const int cu = A.comp[A.si[e]], cv = A.comp[A.m + A.sj[e]];
            if (cu == cv) continue;
            const unsigned long long b = (unsigned long long)__double_as_longlong(A.p[e]);
            const unsigned long long jl = (unsigned long long)A.si[e] + (unsigned long long)A.sj[e] * (unsigned long long)A.m;
            if (A.bestp[cu] == b) atomicMin(&A.bestk[cu], jl);
            if (A.bestp[cv] == b) atomicMin(&A.bestk[cv], jl);
        }
        if (!grid_barrier(A.bar, G, A.err)) return;
        for (int64_t c = tid; c < A.V; c += stride) {
            if (A.comp[c] != c || A.bestp[c] == 0ull) continue;
            const unsigned long long jl = A.bestk[c];
            const int i = (int)(jl % (unsigned long long)A.m), j = (int)(jl / (unsigned long long)A.m);
            int lo = A.row_ptr[i], hi = A.row_ptr[i + 1];
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (A.sj[mid] < j) lo = mid + 1; else hi = mid;
            }
            A.flag[lo] = 0;
            const int ci = A.comp[i], cj = A.comp[A.m + j];
            const int other = ci == (int)c ? cj : ci;
            const bool mutual = A.bestk[other] == jl && A.bestp[other] == A.bestp[c];
            if (!mutual || (int)c < other) A.parent[c] = other;
            A.changed[round] = 1;
        }
        if (!grid_barrier(A.bar, G, A.err)) return;
        for (int pass = 0;; ++pass) {
            int *more = A.more + (int64_t)round * A.max_passes + pass;
            for (int64_t v = tid; v < A.V; v += stride) {
                int r = A.comp[v];
                for (int s = 0; s < 64 && A.parent[r] != r; ++s) r = A.parent[r];
                A.comp[v] = r;
                if (A.parent[r] != r) *more = 1;
            }
            if (!grid_barrier(A.bar, G, A.err)) return;
            if (!*(volatile int *)more) break;
            if (pass + 1 >= A.max_passes) {
                if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(A.err, 0, 2);
                return;
            }
        }
        if (!*(volatile int *)(A.changed + round)) break;
    }
}

__global__ void bv_init_kernel(int V, int32_t *__restrict__ comp, int32_t *__restrict__ parent) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
        comp[v] = v;
        parent[v] = v;
    }
}

__global__ void keep_flags_kernel(int64_t psi, const uint8_t *__restrict__ flag, uint32_t *__restrict__ keep) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < psi; e += (int64_t)gridDim.x * blockDim.x)
        keep[e] = flag ? (flag[e] ? 0u : 1u) : 1u;
}

__global__ void new_keys_kernel(int64_t k, int n, const int32_t *__restrict__ ni, const int32_t *__restrict__ nj,
                                uint64_t *__restrict__ key, uint32_t *__restrict__ val) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < k; t += (int64_t)gridDim.x * blockDim.x) {
        key[t] = (uint64_t)ni[t] * (uint64_t)n + (uint64_t)nj[t];
        val[t] = (uint32_t)t;
    }
}

__device__ __forceinline__ int64_t count_less_kept(uint64_t K, const int32_t *ki, const int32_t *kj, int64_t nk, int n) {
    int64_t lo = 0, hi = nk;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        uint64_t km = (uint64_t)ki[mid] * (uint64_t)n + (uint64_t)kj[mid];
        if (km < K) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int64_t count_less_new(uint64_t K, const uint64_t *nk, int64_t k) {
    int64_t lo = 0, hi = k;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (nk[mid] < K) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// kept entries: S entries with keep == 1, compacted position pos[e]
__global__ void merge_kept_kernel(int64_t psi, int n, const uint32_t *__restrict__ keep, const uint32_t *__restrict__ pos,
                                  const int32_t *__restrict__ si, const int32_t *__restrict__ sj,
                                  const double *__restrict__ sp, const double *__restrict__ ss,
                                  const uint64_t *__restrict__ nkey, int64_t k,
                                  int32_t *__restrict__ ti, int32_t *__restrict__ tj, double *__restrict__ tp,
                                  double *__restrict__ ts) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < psi; e += (int64_t)gridDim.x * blockDim.x) {
        if (!keep[e]) continue;
        const uint64_t K = (uint64_t)si[e] * (uint64_t)n + (uint64_t)sj[e];
        const int64_t q = (int64_t)pos[e] + count_less_new(K, nkey, k);
        ti[q] = si[e]; tj[q] = sj[e]; tp[q] = sp[e]; ts[q] = ss[e];
    }
}

// new entries: binary search in the compacted kept list (read back from T's positions is not
// possible yet, so search the kept entries through S with the keep prefix)
__global__ void merge_new_kernel(int64_t k, int n, const uint64_t *__restrict__ nkey, const uint32_t *__restrict__ nval,
                                 const int32_t *__restrict__ ni, const int32_t *__restrict__ nj,
                                 const int32_t *__restrict__ ki, const int32_t *__restrict__ kj, int64_t nkept,
                                 double p_new, const double *__restrict__ a_cap, const double *__restrict__ b_cap,
                                 int32_t *__restrict__ ti, int32_t *__restrict__ tj,
                                 double *__restrict__ tp, double *__restrict__ ts) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < k; t += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t K = nkey[t];
        const int64_t q = t + count_less_kept(K, ki, kj, nkept, n);
        const uint32_t src = nval[t];
        const int i = ni[src], j = nj[src];
        ti[q] = i; tj[q] = j;
        if (a_cap) {
            // p s = mu with p no larger than the pair's smaller mass
            const double p = fmin(p_new, fmin(a_cap[i], b_cap[j]));
            tp[q] = p;
            ts[q] = p_new * p_new / p;
        } else {
            tp[q] = p_new;
            ts[q] = p_new;
        }
    }
}

__global__ void compact_ij_kernel(int64_t psi, const uint32_t *__restrict__ keep, const uint32_t *__restrict__ pos,
                                  const int32_t *__restrict__ si, const int32_t *__restrict__ sj,
                                  int32_t *__restrict__ ki, int32_t *__restrict__ kj) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < psi; e += (int64_t)gridDim.x * blockDim.x)
        if (keep[e]) { ki[pos[e]] = si[e]; kj[pos[e]] = sj[e]; }
}

inline unsigned grid_for(int64_t work, int cap = 1184) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cap, ceil_div(work, 256)));
}

}  // namespace

Error initial_support(const CostDev &c, double thr, int32_t **out_i, int32_t **out_j, int64_t *psi,
                      cudaStream_t st) {
    const int m = c.m, n = c.n;
    DevTemp<unsigned long long> rowmin, colmin, cnt;
    DevTemp<unsigned> rowarg, colarg;
    OT_TRY(rowmin.alloc(m, st)); OT_TRY(colmin.alloc(n, st)); OT_TRY(cnt.alloc(1, st));
    OT_TRY(rowarg.alloc(m, st)); OT_TRY(colarg.alloc(n, st));
    OT_CUDA(cudaMemsetAsync(rowmin.p, 0xff, sizeof(unsigned long long) * m, st));
    OT_CUDA(cudaMemsetAsync(colmin.p, 0xff, sizeof(unsigned long long) * n, st));
    OT_CUDA(cudaMemsetAsync(rowarg.p, 0xff, sizeof(unsigned) * m, st));
    OT_CUDA(cudaMemsetAsync(colarg.p, 0xff, sizeof(unsigned) * n, st));
    const int64_t ntiles = ceil_div(m, kIT) * ceil_div(n, kIT);
    const unsigned g = (unsigned)std::min<int64_t>(ntiles, 2048);
    init_scan_kernel<0><<<g, 256, 0, st>>>(c, thr, rowmin.p, colmin.p, rowarg.p, colarg.p, nullptr, 0, nullptr);
    OT_LAUNCHED();
    unsigned long long cap = 16ull * (m + n) + 1024, got = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        DevTemp<uint64_t> keys;
        OT_TRY(keys.alloc((int64_t)cap + m + n, st));
        OT_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long), st));
        if (attempt == 1) {
            OT_CUDA(cudaMemsetAsync(rowarg.p, 0xff, sizeof(unsigned) * m, st));
            OT_CUDA(cudaMemsetAsync(colarg.p, 0xff, sizeof(unsigned) * n, st));
        }
        init_scan_kernel<1><<<g, 256, 0, st>>>(c, thr, rowmin.p, colmin.p, rowarg.p, colarg.p, keys.p, cap, cnt.p);
        OT_LAUNCHED();
        OT_CUDA(cudaMemcpyAsync(&got, cnt.p, sizeof(got), cudaMemcpyDeviceToHost, st));
        OT_CUDA(cudaStreamSynchronize(st));
        if (got > cap) { cap = got; continue; }
        const int64_t total = (int64_t)got + m + n;
        init_extra_keys<<<grid_for(m + n), 256, 0, st>>>(m, n, rowarg.p, colarg.p, keys.p + got);
        OT_LAUNCHED();
        DevTemp<uint32_t> vals, flags, pos;
        OT_TRY(vals.alloc(total, st)); OT_TRY(flags.alloc(total, st)); OT_TRY(pos.alloc(total, st));
        OT_TRY(radix_sort_pairs(keys.p, vals.p, total, host_bits_for((uint64_t)m * n - 1), st));
        unique_flags<<<grid_for(total), 256, 0, st>>>(total, keys.p, flags.p);
        OT_LAUNCHED();
        DevTemp<uint32_t> nuniq;
        OT_TRY(nuniq.alloc(1, st));
        OT_TRY(scan_exclusive_u32(flags.p, pos.p, total, nuniq.p, st));
        uint32_t nu = 0;
        OT_CUDA(cudaMemcpyAsync(&nu, nuniq.p, sizeof(nu), cudaMemcpyDeviceToHost, st));
        OT_CUDA(cudaStreamSynchronize(st));
        int32_t *oi = nullptr, *oj = nullptr;
        OT_CUDA(cudaMalloc((void **)&oi, sizeof(int32_t) * std::max<uint32_t>(nu, 1)));
        cudaError_t e = cudaMalloc((void **)&oj, sizeof(int32_t) * std::max<uint32_t>(nu, 1));
        if (e != cudaSuccess) { cudaFree(oi); return fail(OT_ERR_OOM, "initial_support: allocation"); }
        unique_scatter<<<grid_for(total), 256, 0, st>>>(total, n, keys.p, flags.p, pos.p, oi, oj);
        OT_LAUNCHED();
        *out_i = oi; *out_j = oj; *psi = nu;
        return ok();
    }
    return fail(OT_ERR_ARG, "initial_support: threshold set keeps growing");
}

Error rebuild_views(Support &S, int32_t m, int32_t n, cudaStream_t st) {
    OT_TRY(build_row_ptr(S.i, S.psi, m, S.row_ptr, st));
    DevTemp<uint64_t> key;
    DevTemp<uint32_t> val;
    OT_TRY(key.alloc(S.psi, st));
    OT_TRY(val.alloc(S.psi, st));
    if (S.psi > 0) {
        col_keys_kernel<<<grid_for(S.psi), 256, 0, st>>>(S.psi, S.j, key.p, val.p);
        OT_LAUNCHED();
        OT_TRY(radix_sort_pairs(key.p, val.p, S.psi, host_bits_for((uint64_t)std::max(n - 1, 1)), st));
        col_view_kernel<<<grid_for(S.psi), 256, 0, st>>>(S.psi, val.p, S.i, S.col_perm, S.col_row);
        OT_LAUNCHED();
    }
    col_ptr_kernel<<<grid_for((int64_t)n + 1), 256, 0, st>>>(S.psi, n, key.p, S.col_ptr);
    OT_LAUNCHED();
    return ok();
}

Error removal_flags(const Support &S, int32_t m, int32_t n, const double *a_s, const double *b_s,
                    double rm_p_frac, int32_t kmax, uint8_t *flag, int64_t *count, cudaStream_t st) {
    const int64_t psi = S.psi;
    *count = 0;
    if (psi == 0) return ok();
    removal_cand_kernel<<<grid_for(psi), 256, 0, st>>>(psi, S.i, S.j, S.p, S.s, a_s, b_s, rm_p_frac, flag);
    OT_LAUNCHED();
    // Keep a maximum-weight spanning forest of the support graph (weights p, ties: smaller jlin
    // first): the support stays connected, so the restricted problem cannot split into components
    // whose masses do not balance (and no row or column empties).  Boruvka rounds on the device.
    DevTemp<uint32_t> f32, pos, tot;
    OT_TRY(f32.alloc(psi, st)); OT_TRY(pos.alloc(psi, st)); OT_TRY(tot.alloc(1, st));
    count_flags_kernel<<<grid_for(psi), 256, 0, st>>>(psi, flag, f32.p);
    OT_LAUNCHED();
    OT_TRY(scan_exclusive_u32(f32.p, pos.p, psi, tot.p, st));
    uint32_t ncand = 0;
    OT_CUDA(cudaMemcpyAsync(&ncand, tot.p, sizeof(ncand), cudaMemcpyDeviceToHost, st));
    OT_CUDA(cudaStreamSynchronize(st));
    if (ncand == 0) return ok();
    {
        const int V = m + n;
        DevTemp<int32_t> comp, parent;
        DevTemp<unsigned long long> bestp, bestk;
        DevTemp<int> flags;  // [0] a component hooked, [1] a hook chain is longer than one jump pass
        OT_TRY(comp.alloc(V, st)); OT_TRY(parent.alloc(V, st));
        OT_TRY(bestp.alloc(V, st)); OT_TRY(bestk.alloc(V, st));
        OT_TRY(flags.alloc(2, st));
        // one cooperative launch when the device can hold its grid; else the launch-per-stage rounds
        bool done = false;
        {
            const int max_passes = V / 64 + 2;
            DevTemp<int> chg, more, err;
            DevTemp<unsigned> bar;
            OT_TRY(chg.alloc(64, st)); OT_TRY(more.alloc((int64_t)64 * max_passes, st));
            OT_TRY(err.alloc(1, st)); OT_TRY(bar.alloc(2, st));
            OT_CUDA(cudaMemsetAsync(chg.p, 0, sizeof(int) * 64, st));
            OT_CUDA(cudaMemsetAsync(more.p, 0, sizeof(int) * 64 * (size_t)max_passes, st));
            OT_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
            OT_CUDA(cudaMemsetAsync(bar.p, 0, 2 * sizeof(unsigned), st));
            int dev = 0, sms = 0, per_sm = 0;
            OT_CUDA(cudaGetDevice(&dev));
            OT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            OT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bv_coop_kernel, 256, 0));
            const int64_t want = ceil_div(std::max<int64_t>(psi, V), 256);
            const int G = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)std::max(per_sm, 0) * sms));
            if (per_sm > 0) {
                BvArgs A{psi, m, V, max_passes, S.i, S.j, S.row_ptr, S.p, comp.p, parent.p, bestp.p, bestk.p, flag,
                         chg.p, more.p, bar.p, err.p};
                void *args[] = {&A};
                const cudaError_t le =
                    cudaLaunchCooperativeKernel((const void *)bv_coop_kernel, dim3(G), dim3(256), args, 0, st);
                if (le == cudaErrorCooperativeLaunchTooLarge) {
                    cudaGetLastError();
                    OT_CUDA(cudaMemsetAsync(err.p, 0xff, sizeof(int), st));   // -1: not launched
                } else {
                    OT_CUDA(le);
                    OT_LAUNCHED();
                }
                int ev = 0;
                OT_CUDA(cudaMemcpyAsync(&ev, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
                OT_CUDA(cudaStreamSynchronize(st));
                if (ev == (int)OT_ERR_TIMEOUT) return fail(OT_ERR_TIMEOUT, "removal guard: grid barrier wait limit reached");
                done = ev == 0;
            }
        }
        if (!done) {
        // the flags of the forest edges are reset again by the rounds below
        removal_cand_kernel<<<grid_for(psi), 256, 0, st>>>(psi, S.i, S.j, S.p, S.s, a_s, b_s, rm_p_frac, flag);
        OT_LAUNCHED();
        bv_init_kernel<<<grid_for(V), 256, 0, st>>>(V, comp.p, parent.p);
        OT_LAUNCHED();
        int hf[2] = {1, 0};
        for (int round = 0; round < 64 && hf[0]; ++round) {
            OT_CUDA(cudaMemsetAsync(flags.p, 0, 2 * sizeof(int), st));
            bv_reset_kernel<<<grid_for(V), 256, 0, st>>>(V, bestp.p, bestk.p);
            OT_LAUNCHED();
            bv_max_kernel<<<grid_for(psi), 256, 0, st>>>(psi, m, S.i, S.j, S.p, comp.p, bestp.p);
            OT_LAUNCHED();
            bv_tie_kernel<<<grid_for(psi), 256, 0, st>>>(psi, m, S.i, S.j, S.p, comp.p, bestp.p, bestk.p);
            OT_LAUNCHED();
            bv_hook_kernel<<<grid_for(V), 256, 0, st>>>(V, m, S.row_ptr, S.j, comp.p, bestp.p, bestk.p, parent.p, flag,
                                                        flags.p);
            OT_LAUNCHED();
            do {
                OT_CUDA(cudaMemsetAsync(flags.p + 1, 0, sizeof(int), st));
                bv_jump_kernel<<<grid_for(V), 256, 0, st>>>(V, parent.p, comp.p, flags.p + 1);
                OT_LAUNCHED();
                OT_CUDA(cudaMemcpyAsync(hf, flags.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
                OT_CUDA(cudaStreamSynchronize(st));
            } while (hf[1]);
        }
        }
    }
    count_flags_kernel<<<grid_for(psi), 256, 0, st>>>(psi, flag, f32.p);
    OT_LAUNCHED();
    OT_TRY(scan_exclusive_u32(f32.p, pos.p, psi, tot.p, st));
    uint32_t nf = 0;
    OT_CUDA(cudaMemcpyAsync(&nf, tot.p, sizeof(nf), cudaMemcpyDeviceToHost, st));
    OT_CUDA(cudaStreamSynchronize(st));
    if ((int64_t)nf > kmax) {
        DevTemp<uint64_t> key;
        DevTemp<uint32_t> val;
        OT_TRY(key.alloc(nf, st)); OT_TRY(val.alloc(nf, st));
        removal_keys_kernel<<<grid_for(psi), 256, 0, st>>>(psi, m, f32.p, pos.p, S.i, S.j, key.p, val.p);
        OT_LAUNCHED();
        OT_TRY(radix_sort_pairs(key.p, val.p, nf, host_bits_for((uint64_t)m * n - 1), st));
        removal_rekey_kernel<<<grid_for(nf), 256, 0, st>>>(nf, val.p, S.p, key.p);
        OT_LAUNCHED();
        OT_TRY(radix_sort_pairs(key.p, val.p, nf, 64, st));
        removal_trim_kernel<<<grid_for(nf), 256, 0, st>>>(nf, kmax, val.p, flag);
        OT_LAUNCHED();
        nf = (uint32_t)kmax;
    }
    *count = nf;
    return ok();
}

Error merge_support(const Support &S, const uint8_t *flag, const int32_t *ni, const int32_t *nj,
                    int64_t k, double p_new, int32_t m, int32_t n, Support &T, cudaStream_t st,
                    const double *a_cap, const double *b_cap) {
    const int64_t psi = S.psi;
    DevTemp<uint32_t> keep, pos, tot;
    OT_TRY(keep.alloc(psi, st)); OT_TRY(pos.alloc(psi, st)); OT_TRY(tot.alloc(1, st));
    if (psi > 0) {
        keep_flags_kernel<<<grid_for(psi), 256, 0, st>>>(psi, flag, keep.p);
        OT_LAUNCHED();
    }
    OT_TRY(scan_exclusive_u32(keep.p, pos.p, psi, tot.p, st));
    uint32_t nkept = 0;
    OT_CUDA(cudaMemcpyAsync(&nkept, tot.p, sizeof(nkept), cudaMemcpyDeviceToHost, st));
    OT_CUDA(cudaStreamSynchronize(st));
    const int64_t total = (int64_t)nkept + k;
    if (total > T.cap) return fail(OT_ERR_ARG, "merge_support: target capacity too small");
    DevTemp<uint64_t> nkey;
    DevTemp<uint32_t> nval;
    DevTemp<int32_t> ki, kj;
    OT_TRY(nkey.alloc(k, st)); OT_TRY(nval.alloc(k, st));
    OT_TRY(ki.alloc(nkept, st)); OT_TRY(kj.alloc(nkept, st));
    if (k > 0) {
        new_keys_kernel<<<grid_for(k), 256, 0, st>>>(k, n, ni, nj, nkey.p, nval.p);
        OT_LAUNCHED();
        OT_TRY(radix_sort_pairs(nkey.p, nval.p, k, host_bits_for((uint64_t)m * n - 1), st));
    }
    if (psi > 0) {
        compact_ij_kernel<<<grid_for(psi), 256, 0, st>>>(psi, keep.p, pos.p, S.i, S.j, ki.p, kj.p);
        OT_LAUNCHED();
        merge_kept_kernel<<<grid_for(psi), 256, 0, st>>>(psi, n, keep.p, pos.p, S.i, S.j, S.p, S.s, nkey.p, k,
                                                         T.i, T.j, T.p, T.s);
        OT_LAUNCHED();
    }
    if (k > 0) {
        merge_new_kernel<<<grid_for(k), 256, 0, st>>>(k, n, nkey.p, nval.p, ni, nj, ki.p, kj.p, nkept, p_new, a_cap,
                                                      b_cap, T.i, T.j, T.p, T.s);
        OT_LAUNCHED();
    }
    T.psi = total;
    OT_TRY(rebuild_views(T, m, n, st));
    return ok();
}

}  // namespace ot
