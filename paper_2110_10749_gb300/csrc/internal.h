// Internal declarations shared by the translation units of libssd.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ssd.h"

namespace ssd {

// ------------------------------------------------------------------ tiling
constexpr int kTile = 128;          // sources staged in shared memory per step
#ifndef SSD_TPB32
#define SSD_TPB32 128
#endif
#ifndef SSD_MINCTA32
#define SSD_MINCTA32 4
#endif
constexpr int kTPB32 = SSD_TPB32;         // threads per CTA, FP32C pair kernel
constexpr int kMinCTA32 = SSD_MINCTA32;   // resident CTAs per SM the FP32C kernel is compiled for
#ifndef SSD_TPT32
#define SSD_TPT32 4
#endif
constexpr int kTPT32 = SSD_TPT32;   // targets per thread, FP32C (pairs of packed f32x2 lanes)
#ifndef SSD_SYMTPT
#define SSD_SYMTPT 8
#endif
constexpr int kSymTPT = SSD_SYMTPT; // targets per thread of the FP32C symmetric kernel (4 or 8)
constexpr int kChunk = 32;          // sources per bounding-box chunk (near/far test per warp)
constexpr int kTPB64 = 128;         // threads per CTA, FP64 pair kernel
constexpr int kTPT64 = 1;           // targets per thread, FP64
constexpr int kRowAlign = 512;      // n_pad is a multiple of this (>= every CTA target span)

// Operators of the pair kernels.
// OP_LDLT, OP_SDLT: transposes of the subtracted double layers (adjoints)
enum Op { OP_LSL = 0, OP_LDL = 1, OP_SSL = 2, OP_SDL = 3, OP_SSLDL = 4, OP_LSLDL = 5, OP_LDLT = 6, OP_SDLT = 7 };
inline int op_components(int op) {
    return (op == OP_LSL || op == OP_LDL || op == OP_LSLDL || op == OP_LDLT) ? 1 : 3;
}

struct alignas(16) d4 { double x, y, z, w; };

// Plan that evaluates the far block pairs of a layout once for both
// directions, cached for the last rho_far delta it was built for: near items
// (generic or packed pair kernel in items mode) and far items (symmetric
// kernel) in one device block.
struct SymPlan {
    void *block = nullptr;
    int64_t near = 0, far = 0;
    double rfar2 = -1.0;
    bool use = false;
};

// Device layout of a point set: sorted copies used by the pair kernels.
struct Layout {
    int64_t n = 0, n_pad = 0;
    int32_t *perm = nullptr;   // sorted position -> caller index (n_pad entries, -1 for padding)
    float4 *pos32 = nullptr;   // (x, y, z, w)
    float4 *wn32 = nullptr;    // (w nx, w ny, w nz, 0)
    d4 *pos64 = nullptr;       // (x, y, z, w)
    d4 *wn64 = nullptr;        // (w nx, w ny, w nz, 0)
    float4 *cbox = nullptr;    // per 32-point chunk: [2 * c] = (lo x, y, z, 0), [2 * c + 1] = (hi ...)
    double wsum = 0.0;         // sum of weights (host copy)
    void *block = nullptr;     // single allocation backing the arrays
    // launch order of the FP32C pair grid (prepared layouts only), cached for
    // the last (grid, rho_far delta) it was built for
    // (slot 0: FP32C packed kernel, slot 1: FP64 generic kernel)
    bool order_ok = false;
    int2 *order32[2] = {nullptr, nullptr};
    int64_t order_nit[2] = {0, 0}, order_chunk[2] = {0, 0};
    float order_rfar2[2] = {-1.f, -1.f};
    // plans of the layer operators that evaluate far block pairs once for
    // both directions (prepared layouts only), one per precision:
    // [0] FP32C, [1] FP64
    SymPlan sym[2];
};

struct TimedLaunch {
    cudaEvent_t beg, end;
    int cls, prec;
    double pairs;
};

}  // namespace ssd

struct ssd_layout {
    ssd::Layout L;
};

struct ssd_ctx {
    int device = 0;
    int num_sms = 0;
    int occ32 = 1, occ64 = 1;  // resident CTAs per SM of the pair kernels
    int waves32 = 12;          // FP32C grid: about this many waves of resident CTAs (tuned)
    int lpt = 1;               // pair grids in near-first order on prepared layouts
    int sym = 1;               // layer operators (both precisions): far block pairs once for both directions
    int waves64 = 8;           // FP64 grid: about this many waves of resident CTAs (tuned)
    void *noalloc_scratch = nullptr;   // device address of the no-alloc scratch array (first no-alloc call)
    std::string err;
    // caching device allocator: blocks are reused in stream order
    struct Block { void *p; size_t bytes; bool used; };
    std::vector<Block> pool;
    // pinned host scratch for small device->host reads
    double *hbuf = nullptr;     // pinned: [0, 512) scalar reads, [512, 1024) GMRES frames
    int hsp = 0;                // GMRES frames in use (nested solves take one each)
    std::vector<cudaEvent_t> sync_ev;   // two per frame, created on first use
    // timing
    bool timing = false;
    std::vector<ssd::TimedLaunch> pending;
    std::vector<cudaEvent_t> event_pool;
    double stat_ms[SSD_K_COUNT][2] = {};
    double stat_pairs[SSD_K_COUNT][2] = {};
    int64_t stat_launches[SSD_K_COUNT][2] = {};
    int64_t launches = 0;
};

namespace ssd {

int set_error(ssd_ctx *ctx, int status, const std::string &msg);
int cuda_check(ssd_ctx *ctx, cudaError_t e, const char *what);
int launch_check(ssd_ctx *ctx, const char *what);

// Caching device allocator (ctx.cu).  Blocks return to the pool on free and
// are reused by later calls in stream order: a context's calls must be issued
// on one stream at a time.
int dev_alloc(ssd_ctx *ctx, size_t bytes, void **p);
void dev_free(ssd_ctx *ctx, void *p);

// Layout handling (ctx.cu).  A temporary (unsorted) layout is built into pool
// memory when pts->layout is NULL; release it with release_layout.
int build_layout(ssd_ctx *ctx, const ssd_points *pts, bool sort, Layout *L, cudaStream_t s);
void release_layout(ssd_ctx *ctx, Layout *L);
struct LayoutRef {
    const Layout *L = nullptr;
    Layout tmp;
    ssd_ctx *ctx = nullptr;
    ~LayoutRef() { if (ctx && tmp.block) release_layout(ctx, &tmp); }
};
int get_layout(ssd_ctx *ctx, const ssd_points *pts, LayoutRef *ref, cudaStream_t s);
int check_points(ssd_ctx *ctx, const ssd_points *pts);

// Pinned frame of 4 doubles and two events for one GMRES solve, so that
// its residual can be read back asynchronously while nested solves use their
// own frames (LIFO).  (ctx.cu)
constexpr int kHostFrames = 128;
int frame_acquire(ssd_ctx *ctx, double **slots, cudaEvent_t ev[2]);
void frame_release(ssd_ctx *ctx);

// Timing (ctx.cu)
int timed_begin(ssd_ctx *ctx, cudaStream_t s, cudaEvent_t *beg);
void timed_end(ssd_ctx *ctx, cudaStream_t s, cudaEvent_t beg, int cls, int prec, double pairs);

// Pair-sum pipeline (pair.cu).  Computes, for every point i (caller order),
//   out[c][i] = a_id * xin[c][i] + a_op * (S_c(i) + self_c(i)) + add_c + (add_dev ? *add_dev : 0)
// where S is the operator sum of `op` with its physical constants.  For the
// fused operators alpha and beta weight the two layers.  xin may be NULL when
// a_id == 0.  `dens0` is the operator's density (g, p, f, u; u for fused
// Stokes, p for fused Laplace), `dens1` the second density of fused ops (f or g).
struct PairCall {
    int op = OP_LSL;
    int prec = SSD_FP64;
    double delta = 1.0, mu = 1.0;
    double alpha = 1.0, beta = 1.0;       // fused ops only
    const double *dens0 = nullptr, *dens1 = nullptr;
    const double *xin = nullptr;
    double a_id = 0.0, a_op = 1.0;
    double add[3] = {0, 0, 0};
    const double *add_dev = nullptr;      // device scalar added to every entry
    bool rank1_weight_mean = false;       // add (w . dens0) / sum(w) to every entry (Darcy gauge)
    const double *rank1_nrm = nullptr;    // vector ops: add n (w . (dens0 . n)) / sum(w) (Stokes
                                          // normal-mode deflation); caller-order normals [3][n]
    bool transpose_sl = false;            // OP_LSL / OP_SSL: apply the transpose W S W^{-1}
    int64_t row_begin = 0, row_end = -1;  // layout rows [row_begin, row_end) only (row_end < 0: all rows)
    double *out = nullptr;
};
int pair_apply(ssd_ctx *ctx, const Layout &L, const PairCall &pc, cudaStream_t s);
int pair_occupancy(ssd_ctx *ctx);

// ------------------------------------------------------------ batched layout
// Many surfaces concatenated (caller order: surface s owns caller indices
// [off[s], off[s] + n[s])); each surface is Morton-sorted and padded to
// kRowAlign separately so no work item straddles two surfaces.
struct BatchLayout {
    int32_t nsurf = 0;
    int64_t n_total = 0, n_pad_total = 0;
    std::vector<int64_t> off, n, poff, n_pad;   // host copies
    std::vector<double> delta, wsum;
    Layout L;                 // concatenated padded arrays; L.perm maps to caller indices
    int32_t *elem_surf = nullptr;   // [n_total] surface of each caller index
    double *d_wsum = nullptr;       // [nsurf] weight sum per surface
    double *d_selfc = nullptr;      // [nsurf] lim s1(rho)/(rho delta) at rho = 0, i.e. 16/(3 sqrt(pi) delta)
    // work items and per-surface descriptors, FP32C (index 0) and FP64 (index 1)
    void *items[2] = {nullptr, nullptr};
    void *surfs[2] = {nullptr, nullptr};
    void *consts[2] = {nullptr, nullptr};
    int64_t nitems[2] = {0, 0};
    int64_t ptotal[2] = {0, 0};     // sum over surfaces of nsplit * n_pad
    void *block = nullptr;          // backing allocation of the device arrays above
};

}  // namespace ssd

struct ssd_batch_layout {
    ssd::BatchLayout B;
};

namespace ssd {

int batch_layout_build(ssd_ctx *ctx, const ssd_batch *b, BatchLayout *B, cudaStream_t s);
// work items and per-surface constants of both precisions (pair.cu)
int pair_batch_items(ssd_ctx *ctx, BatchLayout *B, cudaStream_t s);
void batch_layout_release(ssd_ctx *ctx, BatchLayout *B);
// Batched pair sums: out[r][c][i] for right-hand side r < nrhs of every surface;
// add[r][c] per right-hand side (nrhs <= kMaxRhs); other fields as in PairCall.
constexpr int kMaxRhs = 16;
struct BatchCall {
    PairCall pc;
    int nrhs = 1;
    double add[kMaxRhs][3] = {};
};
int pair_apply_batch(ssd_ctx *ctx, const BatchLayout &B, const BatchCall &bc, cudaStream_t s);

// Quadrature (quad.cu)
int quadrature_points(ssd_ctx *ctx, const ssd_surface *surf, double h, double angle_deg, int64_t capacity,
                      int64_t *n_out, double *xyz, double *nrm, double *w, int32_t *meta, cudaStream_t s);
int geometry_gradient(ssd_ctx *ctx, const ssd_points *pts, int op, double delta, double mu, double alpha,
                      const double *a, const double *b, double *gx, double *gn, double *gw, cudaStream_t s);
int quadrature_jacobian(ssd_ctx *ctx, const ssd_surface *surf, double h, double angle_deg, int64_t n, double *dxyz,
                        double *dnrm, double *dw, cudaStream_t s);

// Small vector kernels (solve.cu)
int dot(ssd_ctx *ctx, const double *a, const double *b, int64_t n, double *dev_out, cudaStream_t s);

}  // namespace ssd

#define SSD_TRY(expr)                 \
    do {                              \
        int _st = (expr);             \
        if (_st != SSD_OK) return _st; \
    } while (0)
