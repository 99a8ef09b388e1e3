// Context, errors, device memory pool, kernel timing and point layouts.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <cub/device/device_radix_sort.cuh>

#include "internal.h"

namespace ssd {

int set_error(ssd_ctx *ctx, int status, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return status;
}

int cuda_check(ssd_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return SSD_OK;
    const int st = (e == cudaErrorMemoryAllocation) ? SSD_ENOMEM : SSD_ECUDA;
    return set_error(ctx, st, std::string(what) + ": " + cudaGetErrorString(e));
}

int launch_check(ssd_ctx *ctx, const char *what) { return cuda_check(ctx, cudaGetLastError(), what); }

int dev_alloc(ssd_ctx *ctx, size_t bytes, void **p) {
    bytes = (bytes + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    int best = -1;
    for (size_t k = 0; k < ctx->pool.size(); ++k) {
        const auto &b = ctx->pool[k];
        if (!b.used && b.bytes >= bytes && (best < 0 || b.bytes < ctx->pool[best].bytes)) best = (int)k;
    }
    if (best >= 0) {
        ctx->pool[best].used = true;
        *p = ctx->pool[best].p;
        return SSD_OK;
    }
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        // release unused cached blocks and retry once
        cudaGetLastError();
        for (auto &b : ctx->pool)
            if (!b.used) { cudaFree(b.p); b.p = nullptr; }
        ctx->pool.erase(std::remove_if(ctx->pool.begin(), ctx->pool.end(),
                                       [](const ssd_ctx::Block &b) { return b.p == nullptr; }),
                        ctx->pool.end());
        e = cudaMalloc(&q, bytes);
        if (e != cudaSuccess) return cuda_check(ctx, e, "device allocation");
    }
    ctx->pool.push_back({q, bytes, true});
    *p = q;
    return SSD_OK;
}

void dev_free(ssd_ctx *ctx, void *p) {
    if (!p) return;
    for (auto &b : ctx->pool)
        if (b.p == p) { b.used = false; return; }
}

int timed_begin(ssd_ctx *ctx, cudaStream_t s, cudaEvent_t *beg) {
    *beg = nullptr;
    if (!ctx->timing) return SSD_OK;
    cudaEvent_t e;
    if (!ctx->event_pool.empty()) {
        e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
    } else {
        SSD_TRY(cuda_check(ctx, cudaEventCreate(&e), "event create"));
    }
    *beg = e;
    return cuda_check(ctx, cudaEventRecord(e, s), "event record");
}

void timed_end(ssd_ctx *ctx, cudaStream_t s, cudaEvent_t beg, int cls, int prec, double pairs) {
    if (!ctx->timing || !beg) return;
    cudaEvent_t e;
    if (!ctx->event_pool.empty()) {
        e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        return;
    }
    cudaEventRecord(e, s);
    ctx->pending.push_back({beg, e, cls, prec == SSD_FP32C ? 1 : 0, pairs});
}

int frame_acquire(ssd_ctx *ctx, double **slots, cudaEvent_t ev[2]) {
    if (ctx->hsp >= kHostFrames) return set_error(ctx, SSD_EINVAL, "GMRES nesting too deep");
    const int f = ctx->hsp;
    while ((int)ctx->sync_ev.size() < 2 * (f + 1)) {
        cudaEvent_t e;
        SSD_TRY(cuda_check(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event create"));
        ctx->sync_ev.push_back(e);
    }
    *slots = ctx->hbuf + 512 + 4 * f;
    ev[0] = ctx->sync_ev[2 * f];
    ev[1] = ctx->sync_ev[2 * f + 1];
    ctx->hsp++;
    return SSD_OK;
}

void frame_release(ssd_ctx *ctx) {
    if (ctx->hsp > 0) ctx->hsp--;
}

static int drain_timing(ssd_ctx *ctx) {
    for (auto &t : ctx->pending) {
        float ms = 0.f;
        SSD_TRY(cuda_check(ctx, cudaEventSynchronize(t.end), "event sync"));
        SSD_TRY(cuda_check(ctx, cudaEventElapsedTime(&ms, t.beg, t.end), "event time"));
        ctx->stat_ms[t.cls][t.prec] += ms;
        ctx->stat_pairs[t.cls][t.prec] += t.pairs;
        ctx->stat_launches[t.cls][t.prec] += 1;
        ctx->event_pool.push_back(t.beg);
        ctx->event_pool.push_back(t.end);
    }
    ctx->pending.clear();
    return SSD_OK;
}

// ------------------------------------------------------------------ layouts
namespace {

__global__ void bbox_kernel(const double *xyz, int64_t n, double *out /* 6 */) {
    __shared__ double lo[3][256], hi[3][256];
    double l[3] = {1e300, 1e300, 1e300}, h[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
        for (int k = 0; k < 3; ++k) {
            const double v = xyz[k * n + i];
            l[k] = fmin(l[k], v);
            h[k] = fmax(h[k], v);
        }
    for (int k = 0; k < 3; ++k) { lo[k][threadIdx.x] = l[k]; hi[k][threadIdx.x] = h[k]; }
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st)
            for (int k = 0; k < 3; ++k) {
                lo[k][threadIdx.x] = fmin(lo[k][threadIdx.x], lo[k][threadIdx.x + st]);
                hi[k][threadIdx.x] = fmax(hi[k][threadIdx.x], hi[k][threadIdx.x + st]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) { out[k] = lo[k][0]; out[3 + k] = hi[k][0]; }
}

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// 30-bit Morton key of each point inside the bounding box
__global__ void morton_kernel(const double *xyz, int64_t n, const double *bb, uint32_t *key, int32_t *idx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t q[3];
    for (int k = 0; k < 3; ++k) {
        const double ext = bb[3 + k] - bb[k];
        double f = ext > 0 ? (xyz[k * n + i] - bb[k]) / ext : 0.0;
        f = fmin(fmax(f, 0.0), 1.0);
        q[k] = (uint32_t)(f * 1023.0);
    }
    key[i] = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
    idx[i] = (int32_t)i;
}

__global__ void fill_layout_kernel(const double *xyz, const double *nrm, const double *w, int64_t n, int64_t n_pad,
                                   const int32_t *sorted_idx, Layout L) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pad) return;
    if (i < n) {
        const int32_t o = sorted_idx ? sorted_idx[i] : (int32_t)i;
        const double x = xyz[o], y = xyz[n + o], z = xyz[2 * n + o];
        const double ww = w[o];
        const double wx = ww * nrm[o], wy = ww * nrm[n + o], wz = ww * nrm[2 * n + o];
        L.perm[i] = o;
        L.pos64[i] = d4{x, y, z, ww};
        L.wn64[i] = d4{wx, wy, wz, 0.0};
        L.pos32[i] = make_float4((float)x, (float)y, (float)z, (float)ww);
        L.wn32[i] = make_float4((float)wx, (float)wy, (float)wz, 0.f);
    } else {
        // padding: zero weight far from every point
        const double far = 1.0e4;
        L.perm[i] = -1;
        L.pos64[i] = d4{far, far, far, 0.0};
        L.wn64[i] = d4{0.0, 0.0, 0.0, 0.0};
        L.pos32[i] = make_float4((float)far, (float)far, (float)far, 0.f);
        L.wn32[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Bounding box of each 32-point chunk of the sorted layout (real points only;
// a chunk of padding gets the padding position as a degenerate box).
__global__ void chunk_box_kernel(Layout L) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= L.n_pad / kChunk) return;
    float lo[3] = {1e30f, 1e30f, 1e30f}, hi[3] = {-1e30f, -1e30f, -1e30f};
    bool any = false;
    for (int k = 0; k < kChunk; ++k) {
        const int64_t i = c * kChunk + k;
        if (i >= L.n) break;
        const float4 p = L.pos32[i];
        lo[0] = fminf(lo[0], p.x); lo[1] = fminf(lo[1], p.y); lo[2] = fminf(lo[2], p.z);
        hi[0] = fmaxf(hi[0], p.x); hi[1] = fmaxf(hi[1], p.y); hi[2] = fmaxf(hi[2], p.z);
        any = true;
    }
    if (!any) {
        const float4 p = L.pos32[c * kChunk];
        lo[0] = hi[0] = p.x; lo[1] = hi[1] = p.y; lo[2] = hi[2] = p.z;
    }
    L.cbox[2 * c] = make_float4(lo[0], lo[1], lo[2], 0.f);
    L.cbox[2 * c + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
}

// fixed-order FP64 sum of the weights (one block)
__global__ void wsum_kernel(const double *w, int64_t n, double *out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += w[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// ------------------------------------------------------------- batched layouts
// key = surface index above a 30-bit Morton code of the position in the
// batch's bounding box: sorting groups each surface's points in Morton order
__global__ void batch_key_kernel(const double *xyz, int64_t n, const double *bb, const int32_t *esurf,
                                 uint64_t *key, int32_t *idx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t q[3];
    for (int k = 0; k < 3; ++k) {
        const double ext = bb[3 + k] - bb[k];
        double f = ext > 0 ? (xyz[k * n + i] - bb[k]) / ext : 0.0;
        f = fmin(fmax(f, 0.0), 1.0);
        q[k] = (uint32_t)(f * 1023.0);
    }
    const uint32_t m = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
    key[i] = ((uint64_t)esurf[i] << 30) | m;
    idx[i] = (int32_t)i;
}

struct BatchFillArgs {
    int32_t nsurf;
    const int64_t *off, *cnt, *poff;   // device copies
    const double *xyz, *nrm, *w;
    int64_t n_total, n_pad_total;
    const int32_t *sorted;             // sorted position -> caller index
};

__global__ void batch_fill_kernel(const BatchFillArgs a, Layout L) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_pad_total) return;
    // surface owning padded index i (binary search over padded offsets)
    int lo = 0, hi = a.nsurf - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.poff[mid] <= i) lo = mid; else hi = mid - 1;
    }
    const int64_t local = i - a.poff[lo];
    const int64_t n = a.n_total;
    if (local < a.cnt[lo]) {
        const int32_t o = a.sorted[a.off[lo] + local];
        const double x = a.xyz[o], y = a.xyz[n + o], z = a.xyz[2 * n + o];
        const double ww = a.w[o];
        const double wx = ww * a.nrm[o], wy = ww * a.nrm[n + o], wz = ww * a.nrm[2 * n + o];
        L.perm[i] = o;
        L.pos64[i] = d4{x, y, z, ww};
        L.wn64[i] = d4{wx, wy, wz, 0.0};
        L.pos32[i] = make_float4((float)x, (float)y, (float)z, (float)ww);
        L.wn32[i] = make_float4((float)wx, (float)wy, (float)wz, 0.f);
    } else {
        const double far = 1.0e4;
        L.perm[i] = -1;
        L.pos64[i] = d4{far, far, far, 0.0};
        L.wn64[i] = d4{0.0, 0.0, 0.0, 0.0};
        L.pos32[i] = make_float4((float)far, (float)far, (float)far, 0.f);
        L.wn32[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// chunk boxes of the batched layout; chunks never straddle surfaces because
// every surface is padded to a multiple of kRowAlign
__global__ void batch_chunk_box_kernel(Layout L) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= L.n_pad / kChunk) return;
    float lo[3] = {1e30f, 1e30f, 1e30f}, hi[3] = {-1e30f, -1e30f, -1e30f};
    bool any = false;
    for (int k = 0; k < kChunk; ++k) {
        const int64_t i = c * kChunk + k;
        if (L.perm[i] < 0) continue;
        const float4 p = L.pos32[i];
        lo[0] = fminf(lo[0], p.x); lo[1] = fminf(lo[1], p.y); lo[2] = fminf(lo[2], p.z);
        hi[0] = fmaxf(hi[0], p.x); hi[1] = fmaxf(hi[1], p.y); hi[2] = fmaxf(hi[2], p.z);
        any = true;
    }
    if (!any) {
        const float4 p = L.pos32[c * kChunk];
        lo[0] = hi[0] = p.x; lo[1] = hi[1] = p.y; lo[2] = hi[2] = p.z;
    }
    L.cbox[2 * c] = make_float4(lo[0], lo[1], lo[2], 0.f);
    L.cbox[2 * c + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
}

// weight sum per surface, fixed order (one block per surface)
__global__ void batch_wsum_kernel(const double *w, const int64_t *off, double *out) {
    __shared__ double red[256];
    const int s = blockIdx.x;
    double acc = 0.0;
    for (int64_t i = off[s] + threadIdx.x; i < off[s + 1]; i += blockDim.x) acc += w[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[s] = red[0];
}

__global__ void batch_esurf_kernel(const int64_t *off, int32_t nsurf, int64_t n, int32_t *esurf) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = nsurf - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    esurf[i] = lo;
}

}  // namespace

void batch_layout_release(ssd_ctx *ctx, BatchLayout *B) {
    if (B->block) dev_free(ctx, B->block);
    for (int k = 0; k < 2; ++k) {
        if (B->items[k]) dev_free(ctx, B->items[k]);
    }
    *B = BatchLayout();
}

int batch_layout_build(ssd_ctx *ctx, const ssd_batch *b, BatchLayout *B, cudaStream_t s) {
    if (!b || b->nsurf < 1 || b->nsurf > (1 << 20) || !b->offsets || !b->delta)
        return set_error(ctx, SSD_EINVAL, "bad batch description");
    if (!b->xyz || !b->nrm || !b->w) return set_error(ctx, SSD_EINVAL, "NULL batch point array");
    BatchLayout out;
    out.nsurf = b->nsurf;
    if (b->offsets[0] != 0) return set_error(ctx, SSD_EINVAL, "offsets[0] must be 0");
    int64_t pacc = 0;
    for (int k = 0; k < b->nsurf; ++k) {
        const int64_t nk = b->offsets[k + 1] - b->offsets[k];
        if (nk <= 0) return set_error(ctx, SSD_EINVAL, "every surface needs at least one point");
        if (!(b->delta[k] > 0.0) || !isfinite(b->delta[k]))
            return set_error(ctx, SSD_EINVAL, "delta must be positive per surface");
        out.off.push_back(b->offsets[k]);
        out.n.push_back(nk);
        out.poff.push_back(pacc);
        const int64_t np = ((nk + kRowAlign - 1) / kRowAlign) * kRowAlign;
        out.n_pad.push_back(np);
        out.delta.push_back(b->delta[k]);
        pacc += np;
    }
    out.n_total = b->offsets[b->nsurf];
    out.n_pad_total = pacc;
    if (out.n_pad_total > (int64_t)0x7fffffff - 1024) return set_error(ctx, SSD_EINVAL, "batch too large");
    const int64_t n = out.n_total, np = out.n_pad_total;
    const int ns = out.nsurf;

    size_t off = 0;
    auto carve = [&](size_t bb) { size_t o = off; off += (bb + 255) & ~size_t(255); return o; };
    const size_t o_perm = carve(sizeof(int32_t) * np), o_p32 = carve(sizeof(float4) * np),
                 o_w32 = carve(sizeof(float4) * np), o_p64 = carve(sizeof(d4) * np),
                 o_w64 = carve(sizeof(d4) * np), o_cb = carve(sizeof(float4) * 2 * (np / kChunk)),
                 o_es = carve(sizeof(int32_t) * n), o_ws = carve(sizeof(double) * ns),
                 o_sc = carve(sizeof(double) * ns), o_meta = carve(sizeof(int64_t) * (4 * ns + 1));
    void *blk = nullptr;
    SSD_TRY(dev_alloc(ctx, off, &blk));
    char *bp = static_cast<char *>(blk);
    out.block = blk;
    out.L.n = np;   // the concatenated arrays as one padded set
    out.L.n_pad = np;
    out.L.perm = reinterpret_cast<int32_t *>(bp + o_perm);
    out.L.pos32 = reinterpret_cast<float4 *>(bp + o_p32);
    out.L.wn32 = reinterpret_cast<float4 *>(bp + o_w32);
    out.L.pos64 = reinterpret_cast<d4 *>(bp + o_p64);
    out.L.wn64 = reinterpret_cast<d4 *>(bp + o_w64);
    out.L.cbox = reinterpret_cast<float4 *>(bp + o_cb);
    out.elem_surf = reinterpret_cast<int32_t *>(bp + o_es);
    out.d_wsum = reinterpret_cast<double *>(bp + o_ws);
    out.d_selfc = reinterpret_cast<double *>(bp + o_sc);
    int64_t *dmeta = reinterpret_cast<int64_t *>(bp + o_meta);   // off[ns+1], cnt[ns], poff[ns]
    std::vector<int64_t> hmeta(4 * ns + 1, 0);
    for (int k = 0; k <= ns; ++k) hmeta[k] = b->offsets[k];
    for (int k = 0; k < ns; ++k) { hmeta[ns + 1 + k] = out.n[k]; hmeta[2 * ns + 1 + k] = out.poff[k]; }
    std::vector<double> selfc(ns);
    for (int k = 0; k < ns; ++k) selfc[k] = 16.0 / (3.0 * sqrt(M_PI) * out.delta[k]);
    int st = cuda_check(ctx, cudaMemcpyAsync(dmeta, hmeta.data(), sizeof(int64_t) * hmeta.size(),
                                             cudaMemcpyHostToDevice, s), "batch meta copy");
    if (st == SSD_OK)
        st = cuda_check(ctx, cudaMemcpyAsync(out.d_selfc, selfc.data(), sizeof(double) * ns,
                                             cudaMemcpyHostToDevice, s), "batch self copy");
    // sort by (surface, Morton)
    void *tmp = nullptr;
    if (st == SSD_OK) {
        size_t cub_bytes = 0;
        int nbits = 30;
        while ((1 << (nbits - 30)) < ns) ++nbits;
        cub::DeviceRadixSort::SortPairs(nullptr, cub_bytes, (const uint64_t *)nullptr, (uint64_t *)nullptr,
                                        (const int32_t *)nullptr, (int32_t *)nullptr, (int)n, 0, nbits, s);
        size_t t_off = 0;
        auto tcarve = [&](size_t bb) { size_t o = t_off; t_off += (bb + 255) & ~size_t(255); return o; };
        const size_t o_k0 = tcarve(sizeof(uint64_t) * n), o_k1 = tcarve(sizeof(uint64_t) * n);
        const size_t o_i0 = tcarve(sizeof(int32_t) * n), o_i1 = tcarve(sizeof(int32_t) * n);
        const size_t o_bb = tcarve(sizeof(double) * 6), o_cub = tcarve(cub_bytes);
        st = dev_alloc(ctx, t_off, &tmp);
        if (st == SSD_OK) {
            char *tb = static_cast<char *>(tmp);
            uint64_t *k0 = reinterpret_cast<uint64_t *>(tb + o_k0), *k1 = reinterpret_cast<uint64_t *>(tb + o_k1);
            int32_t *i0 = reinterpret_cast<int32_t *>(tb + o_i0), *i1 = reinterpret_cast<int32_t *>(tb + o_i1);
            double *bb = reinterpret_cast<double *>(tb + o_bb);
            const unsigned gn = (unsigned)((n + 255) / 256);
            batch_esurf_kernel<<<gn, 256, 0, s>>>(dmeta, ns, n, out.elem_surf);
            bbox_kernel<<<1, 256, 0, s>>>(b->xyz, n, bb);
            batch_key_kernel<<<gn, 256, 0, s>>>(b->xyz, n, bb, out.elem_surf, k0, i0);
            ctx->launches += 3;
            st = launch_check(ctx, "batch keys");
            if (st == SSD_OK) {
                cudaError_t e = cub::DeviceRadixSort::SortPairs(tb + o_cub, cub_bytes, k0, k1, i0, i1, (int)n, 0,
                                                                nbits, s);
                ctx->launches += 4;
                st = cuda_check(ctx, e, "batch radix sort");
            }
            if (st == SSD_OK) {
                BatchFillArgs fa;
                fa.nsurf = ns; fa.off = dmeta; fa.cnt = dmeta + ns + 1; fa.poff = dmeta + 2 * ns + 1;
                fa.xyz = b->xyz; fa.nrm = b->nrm; fa.w = b->w; fa.n_total = n; fa.n_pad_total = np;
                fa.sorted = i1;
                batch_fill_kernel<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(fa, out.L);
                batch_chunk_box_kernel<<<(unsigned)((np / kChunk + 127) / 128), 128, 0, s>>>(out.L);
                batch_wsum_kernel<<<ns, 256, 0, s>>>(b->w, dmeta, out.d_wsum);
                ctx->launches += 3;
                st = launch_check(ctx, "batch fill");
            }
        }
    }
    out.wsum.resize(ns);
    if (st == SSD_OK)
        st = cuda_check(ctx, cudaMemcpyAsync(out.wsum.data(), out.d_wsum, sizeof(double) * ns,
                                             cudaMemcpyDeviceToHost, s), "wsum copy");
    if (st == SSD_OK) st = cuda_check(ctx, cudaStreamSynchronize(s), "batch layout sync");
    if (tmp) dev_free(ctx, tmp);
    if (st == SSD_OK) {
        for (int k = 0; k < ns; ++k)
            if (!(out.wsum[k] > 0.0)) { st = set_error(ctx, SSD_EINVAL, "surface weights must sum to > 0"); break; }
    }
    if (st == SSD_OK) st = pair_batch_items(ctx, &out, s);
    if (st != SSD_OK) {
        batch_layout_release(ctx, &out);
        return st;
    }
    *B = out;
    return SSD_OK;
}

int check_points(ssd_ctx *ctx, const ssd_points *pts) {
    if (!pts) return set_error(ctx, SSD_EINVAL, "points is NULL");
    if (pts->n <= 0 || pts->n > (int64_t)0x7fffffff - 1024)
        return set_error(ctx, SSD_EINVAL, "point count out of range");
    if (!pts->xyz || !pts->nrm || !pts->w) return set_error(ctx, SSD_EINVAL, "NULL point array");
    if (pts->layout && pts->layout->L.n != pts->n)
        return set_error(ctx, SSD_EINVAL, "layout was built for a different point count");
    return SSD_OK;
}

void release_layout(ssd_ctx *ctx, Layout *L) {
    if (L->block) dev_free(ctx, L->block);
    for (int k = 0; k < 2; ++k)
        if (L->order32[k]) dev_free(ctx, L->order32[k]);
    for (auto &pl : L->sym)
        if (pl.block) dev_free(ctx, pl.block);
    *L = Layout();
}

int build_layout(ssd_ctx *ctx, const ssd_points *pts, bool sort, Layout *L, cudaStream_t s) {
    const int64_t n = pts->n;
    const int64_t n_pad = ((n + kRowAlign - 1) / kRowAlign) * kRowAlign;
    size_t off = 0;
    auto carve = [&](size_t b) { size_t o = off; off += (b + 255) & ~size_t(255); return o; };
    const size_t o_perm = carve(sizeof(int32_t) * n_pad);
    const size_t o_p32 = carve(sizeof(float4) * n_pad);
    const size_t o_w32 = carve(sizeof(float4) * n_pad);
    const size_t o_p64 = carve(sizeof(d4) * n_pad);
    const size_t o_w64 = carve(sizeof(d4) * n_pad);
    const size_t o_cb = carve(sizeof(float4) * 2 * (n_pad / kChunk));
    const size_t o_ws = carve(sizeof(double) * 8);
    void *blk = nullptr;
    SSD_TRY(dev_alloc(ctx, off, &blk));
    char *b = static_cast<char *>(blk);
    Layout out;
    out.n = n;
    out.n_pad = n_pad;
    out.block = blk;
    out.perm = reinterpret_cast<int32_t *>(b + o_perm);
    out.pos32 = reinterpret_cast<float4 *>(b + o_p32);
    out.wn32 = reinterpret_cast<float4 *>(b + o_w32);
    out.pos64 = reinterpret_cast<d4 *>(b + o_p64);
    out.wn64 = reinterpret_cast<d4 *>(b + o_w64);
    out.cbox = reinterpret_cast<float4 *>(b + o_cb);
    double *dsum = reinterpret_cast<double *>(b + o_ws);

    int32_t *sorted = nullptr;
    void *tmp = nullptr;
    int st = SSD_OK;
    if (sort) {
        // keys/values and CUB temporary storage
        size_t cub_bytes = 0;
        cub::DeviceRadixSort::SortPairs(nullptr, cub_bytes, (const uint32_t *)nullptr, (uint32_t *)nullptr,
                                        (const int32_t *)nullptr, (int32_t *)nullptr, (int)n, 0, 30, s);
        size_t t_off = 0;
        auto tcarve = [&](size_t bb) { size_t o = t_off; t_off += (bb + 255) & ~size_t(255); return o; };
        const size_t o_k0 = tcarve(sizeof(uint32_t) * n), o_k1 = tcarve(sizeof(uint32_t) * n);
        const size_t o_i0 = tcarve(sizeof(int32_t) * n), o_i1 = tcarve(sizeof(int32_t) * n);
        const size_t o_bb = tcarve(sizeof(double) * 6), o_cub = tcarve(cub_bytes);
        st = dev_alloc(ctx, t_off, &tmp);
        if (st != SSD_OK) { release_layout(ctx, &out); return st; }
        char *tb = static_cast<char *>(tmp);
        uint32_t *k0 = reinterpret_cast<uint32_t *>(tb + o_k0), *k1 = reinterpret_cast<uint32_t *>(tb + o_k1);
        int32_t *i0 = reinterpret_cast<int32_t *>(tb + o_i0), *i1 = reinterpret_cast<int32_t *>(tb + o_i1);
        double *bb = reinterpret_cast<double *>(tb + o_bb);
        bbox_kernel<<<1, 256, 0, s>>>(pts->xyz, n, bb);
        morton_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pts->xyz, n, bb, k0, i0);
        ctx->launches += 2;
        st = launch_check(ctx, "morton keys");
        if (st == SSD_OK) {
            cudaError_t e = cub::DeviceRadixSort::SortPairs(tb + o_cub, cub_bytes, k0, k1, i0, i1, (int)n, 0, 30, s);
            ctx->launches += 4;
            st = cuda_check(ctx, e, "radix sort");
        }
        sorted = i1;
    }
    if (st == SSD_OK) {
        fill_layout_kernel<<<(unsigned)((n_pad + 255) / 256), 256, 0, s>>>(pts->xyz, pts->nrm, pts->w, n, n_pad,
                                                                          sorted, out);
        wsum_kernel<<<1, 256, 0, s>>>(pts->w, n, dsum);
        chunk_box_kernel<<<(unsigned)((n_pad / kChunk + 127) / 128), 128, 0, s>>>(out);
        ctx->launches += 3;
        st = launch_check(ctx, "layout fill");
    }
    if (st == SSD_OK) st = cuda_check(ctx, cudaMemcpyAsync(ctx->hbuf, dsum, sizeof(double),
                                                           cudaMemcpyDeviceToHost, s), "wsum copy");
    if (st == SSD_OK) st = cuda_check(ctx, cudaStreamSynchronize(s), "layout sync");
    if (tmp) dev_free(ctx, tmp);
    if (st != SSD_OK) { release_layout(ctx, &out); return st; }
    out.wsum = ctx->hbuf[0];
    if (!(out.wsum > 0.0)) {
        release_layout(ctx, &out);
        return set_error(ctx, SSD_EINVAL, "quadrature weights must have a positive sum");
    }
    *L = out;
    return SSD_OK;
}

int get_layout(ssd_ctx *ctx, const ssd_points *pts, LayoutRef *ref, cudaStream_t s) {
    SSD_TRY(check_points(ctx, pts));
    if (pts->layout) {
        ref->L = &pts->layout->L;
        return SSD_OK;
    }
    SSD_TRY(build_layout(ctx, pts, false, &ref->tmp, s));
    ref->ctx = ctx;
    ref->L = &ref->tmp;
    return SSD_OK;
}

}  // namespace ssd

using namespace ssd;

extern "C" {

const char *ssd_status_string(int st) {
    switch (st) {
        case SSD_OK: return "ok";
        case SSD_EINVAL: return "invalid argument";
        case SSD_ENOMEM: return "out of memory";
        case SSD_ECUDA: return "CUDA error";
        case SSD_ENOTCONV: return "iteration limit reached";
        case SSD_ENUMERIC: return "non-finite value";
        default: return "unknown status";
    }
}

int ssd_ctx_create(ssd_ctx **out, int device) {
    if (!out) return SSD_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return SSD_EINVAL;
    }
    if (cudaSetDevice(device) != cudaSuccess) return SSD_ECUDA;
    ssd_ctx *ctx = new ssd_ctx();
    ctx->device = device;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) { delete ctx; return SSD_ECUDA; }
    ctx->num_sms = prop.multiProcessorCount;
    if (cudaMallocHost((void **)&ctx->hbuf, 8192) != cudaSuccess) { delete ctx; return SSD_ENOMEM; }
    if (pair_occupancy(ctx) != SSD_OK) { cudaFreeHost(ctx->hbuf); delete ctx; return SSD_ECUDA; }
    // tuning knob: waves of resident CTAs in an FP32C pair-kernel grid
    if (const char *w = getenv("SSD_PAIR_WAVES")) {
        const int v = atoi(w);
        if (v >= 1 && v <= 64) ctx->waves32 = v;
    }
    // tuning knob: 0 launches the FP32C grid in plain (tile, split) order
    if (const char *w = getenv("SSD_PAIR_LPT")) ctx->lpt = atoi(w) != 0;
    if (const char *w = getenv("SSD_PAIR_SYM")) ctx->sym = atoi(w) != 0;
    if (const char *w = getenv("SSD_PAIR_WAVES64")) {
        const int v = atoi(w);
        if (v >= 1 && v <= 64) ctx->waves64 = v;
    }
    *out = ctx;
    return SSD_OK;
}

int ssd_ctx_destroy(ssd_ctx *ctx) {
    if (!ctx) return SSD_OK;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto &b : ctx->pool) cudaFree(b.p);
    for (auto &t : ctx->pending) { cudaEventDestroy(t.beg); cudaEventDestroy(t.end); }
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    for (auto e : ctx->sync_ev) cudaEventDestroy(e);
    if (ctx->hbuf) cudaFreeHost(ctx->hbuf);
    delete ctx;
    return SSD_OK;
}

const char *ssd_ctx_last_error(const ssd_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

int ssd_ctx_set_timing(ssd_ctx *ctx, int enable) {
    if (!ctx) return SSD_EINVAL;
    ctx->timing = enable != 0;
    return SSD_OK;
}

int ssd_ctx_kernel_stats(ssd_ctx *ctx, int cls, int prec, ssd_kernel_stats *out) {
    if (!ctx || !out || cls < 0 || cls >= SSD_K_COUNT || (prec != SSD_FP64 && prec != SSD_FP32C))
        return set_error(ctx, SSD_EINVAL, "bad kernel class, precision or output");
    SSD_TRY(drain_timing(ctx));
    const int p = prec == SSD_FP32C ? 1 : 0;
    out->launches = ctx->stat_launches[cls][p];
    out->ms = ctx->stat_ms[cls][p];
    out->pairs = ctx->stat_pairs[cls][p];
    return SSD_OK;
}

int ssd_ctx_reset_stats(ssd_ctx *ctx) {
    if (!ctx) return SSD_EINVAL;
    SSD_TRY(drain_timing(ctx));
    for (int c = 0; c < SSD_K_COUNT; ++c)
        for (int p = 0; p < 2; ++p) {
            ctx->stat_ms[c][p] = 0;
            ctx->stat_pairs[c][p] = 0;
            ctx->stat_launches[c][p] = 0;
        }
    return SSD_OK;
}

int ssd_ctx_launch_count(const ssd_ctx *ctx, int64_t *out) {
    if (!ctx || !out) return SSD_EINVAL;
    *out = ctx->launches;
    return SSD_OK;
}

int ssd_sync(ssd_ctx *ctx, ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != ctx->device)
        return set_error(ctx, SSD_EINVAL, "the current device is not the context's device");
    const cudaError_t e = stream ? cudaStreamSynchronize((cudaStream_t)stream) : cudaDeviceSynchronize();
    return cuda_check(ctx, e, "synchronise");
}

int ssd_points_prepare(ssd_ctx *ctx, ssd_points *pts, ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    if (pts && pts->layout) return set_error(ctx, SSD_EINVAL, "points already have a layout");
    SSD_TRY(check_points(ctx, pts));
    ssd_layout *lay = new ssd_layout();
    int st = build_layout(ctx, pts, true, &lay->L, (cudaStream_t)stream);
    lay->L.order_ok = true;
    if (st != SSD_OK) { delete lay; return st; }
    pts->layout = lay;
    return SSD_OK;
}

int ssd_points_release(ssd_ctx *ctx, ssd_points *pts) {
    if (!ctx || !pts) return SSD_EINVAL;
    if (pts->layout) {
        release_layout(ctx, &pts->layout->L);
        delete pts->layout;
        pts->layout = nullptr;
    }
    return SSD_OK;
}

int ssd_batch_prepare(ssd_ctx *ctx, ssd_batch *b, ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    ctx->err.clear();
    if (!b) return set_error(ctx, SSD_EINVAL, "batch is NULL");
    if (b->layout) return set_error(ctx, SSD_EINVAL, "batch already has a layout");
    ssd_batch_layout *lay = new ssd_batch_layout();
    const int st = batch_layout_build(ctx, b, &lay->B, (cudaStream_t)stream);
    if (st != SSD_OK) { delete lay; return st; }
    b->layout = lay;
    return SSD_OK;
}

int ssd_batch_release(ssd_ctx *ctx, ssd_batch *b) {
    if (!ctx || !b) return SSD_EINVAL;
    if (b->layout) {
        batch_layout_release(ctx, &b->layout->B);
        delete b->layout;
        b->layout = nullptr;
    }
    return SSD_OK;
}

int ssd_quadrature_points(ssd_ctx *ctx, const ssd_surface *surf, double h, double angle_deg, int64_t capacity,
                          int64_t *n_out, double *xyz, double *nrm, double *w, int32_t *meta, ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    ctx->err.clear();
    return quadrature_points(ctx, surf, h, angle_deg, capacity, n_out, xyz, nrm, w, meta, (cudaStream_t)stream);
}

int ssd_quadrature_jacobian(ssd_ctx *ctx, const ssd_surface *surf, double h, double angle_deg, int64_t n,
                            double *dxyz, double *dnrm, double *dw, ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    ctx->err.clear();
    if (!surf) return set_error(ctx, SSD_EINVAL, "surface is NULL");
    return quadrature_jacobian(ctx, surf, h, angle_deg, n, dxyz, dnrm, dw, (cudaStream_t)stream);
}

}  // extern "C"

// ------------------------------------------------- FP32 FMA rate (measurement)
// Every thread keeps 16 independent FMA chains (8 packed f32x2 pairs, or 16
// scalars) for `iters` steps; the result is stored only when it equals a
// value it cannot reach, so nothing is optimised away.  Used to measure the
// FP32 rate the pair kernels can reach on this device.
namespace ssd {
namespace {
__global__ void __launch_bounds__(256) fma_rate_kernel(int packed, int iters, float m, float c, float *sink) {
    if (packed) {
        float2 a[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = make_float2(threadIdx.x * 1e-3f + k, blockIdx.x * 1e-3f - k);
        const float2 mm = make_float2(m, m), cc = make_float2(c, c);
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = __ffma2_rn(a[k], mm, cc);
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) s += a[k].x + a[k].y;
        if (s == -12345.678f) sink[0] = s;
    } else {
        float a[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) a[k] = threadIdx.x * 1e-3f + k;
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int k = 0; k < 16; ++k) a[k] = fmaf(a[k], m, c);
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < 16; ++k) s += a[k];
        if (s == -12345.678f) sink[0] = s;
    }
}
}  // namespace
}  // namespace ssd

extern "C" int ssd_fp32_fma_rate(ssd_ctx *ctx, int packed, double *tflops) {
    using namespace ssd;
    if (!ctx || !tflops) return SSD_EINVAL;
    ctx->err.clear();
    void *sink = nullptr;
    SSD_TRY(dev_alloc(ctx, 256, &sink));
    struct Release { ssd_ctx *c; void *p; ~Release() { dev_free(c, p); } } release{ctx, sink};
    const int blocks = ctx->num_sms * 8, threads = 256, iters = 1 << 14;
    cudaEvent_t e0, e1;
    SSD_TRY(cuda_check(ctx, cudaEventCreate(&e0), "event"));
    SSD_TRY(cuda_check(ctx, cudaEventCreate(&e1), "event"));
    float ms = 0.f;
    for (int rep = 0; rep < 3; ++rep) {   // the last of three launches is timed
        cudaEventRecord(e0, 0);
        fma_rate_kernel<<<blocks, threads, 0, 0>>>(packed, iters, 0.999999f, 1e-7f, static_cast<float *>(sink));
        cudaEventRecord(e1, 0);
        ctx->launches++;
    }
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    SSD_TRY(cuda_check(ctx, e, "fma rate kernel"));
    const double fmas = (double)blocks * threads * iters * 16.0;
    *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
    return SSD_OK;
}
