// ot_price_topk_noalloc: the pricing selection of ot_price_topk with every temporary buffer
// taken from one statically sized device array instead of the stream-ordered allocator.
//
// Who needs it: host programs that must not allocate device memory once they are running --
// a serving process that reserved its whole memory budget at start-up (any further cudaMalloc
// fails or evicts its caches), or a latency-critical loop that cannot afford the implicit
// device-wide synchronisation an allocation or release may cause.  Such a caller still owns the
// inputs and outputs; only the scratch moves into this file-scope array.
#include "pricing.cuh"
#include "primitives.cuh"

namespace {

// 24 MiB of scratch on every device where the library's module is loaded (held until the process
// exits).  With lazy module loading that happens at the first call on the device.  Enough for
// m, n <= 16384 and a pricing candidate set of about 400k pairs.
constexpr size_t kScratchBytes = (size_t)24 << 20;
constexpr int32_t kMaxSide = 16384;

static __device__ __align__(256) unsigned char g_price_scratch[kScratchBytes];

// Device address of the scratch array on the current device.  Host code must not use
// g_price_scratch directly: on the host that name is only a stand-in for the device symbol.  The
// address is looked up on every call (the lookup allocates nothing), so it always belongs to the
// current context, also after a device reset made a new one.
ot::Error scratch_for_current_device(void **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_price_scratch);
    if (e != cudaSuccess || !p)
        return ot::fail(OT_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    *out = p;
    return ot::ok();
}

}  // namespace

extern "C" int ot_price_topk_noalloc(int32_t m, int32_t n, const int32_t *sx, const int32_t *sy, const int32_t *tx,
                                     const int32_t *ty, const double *u, const double *v, const int32_t *sup_i,
                                     const int32_t *sup_j, int64_t psi, int32_t kmax, int32_t precision,
                                     int32_t *out_i, int32_t *out_j, double *out_d, int32_t *out_count,
                                     void *stream) {
    using namespace ot;
    if (m <= 0 || n <= 0 || kmax < 0 || psi < 0 || !sx || !sy || !tx || !ty || !u || !v || !out_i || !out_j ||
        !out_count || (psi > 0 && (!sup_i || !sup_j)) || (precision != 0 && precision != 1)) {
        set_thread_error("ot_price_topk_noalloc: invalid argument");
        return OT_ERR_ARG;
    }
    if (m > kMaxSide || n > kMaxSide) {
        set_thread_error("ot_price_topk_noalloc: m and n must not exceed 16384 (scratch is a fixed 24 MiB array)");
        return OT_ERR_ARG;
    }
    void *base = nullptr;
    Error e = scratch_for_current_device(&base);
    if (e.code != OT_OK) {
        set_thread_error(e.msg.c_str());
        return e.code;
    }
    Arena arena;
    arena.base = (char *)base;
    arena.size = kScratchBytes;
    cudaStream_t st = (cudaStream_t)stream;
    {
        ArenaScope scope(&arena);
        PriceInput in;
        in.m = m; in.n = n;
        in.sx = sx; in.sy = sy; in.tx = tx; in.ty = ty;
        in.u = u; in.v = v;
        in.sup_i = sup_i; in.sup_j = sup_j; in.psi = psi;
        in.kmax = kmax;
        in.precision = precision;
        e = coord_origin(m, n, sx, sy, tx, ty, &in.origin_x, &in.origin_y, st);
        if (e.code == OT_OK) e = price_topk(in, out_i, out_j, out_d, out_count, nullptr, st);
    }
    if (e.code == OT_ERR_BUF_TOO_SMALL)
        e.msg = "ot_price_topk_noalloc: the candidate set of this call does not fit the fixed 24 MiB scratch; "
                "use ot_price_topk";
    if (e.code != OT_OK) set_thread_error(e.msg.c_str());
    return e.code;
}
