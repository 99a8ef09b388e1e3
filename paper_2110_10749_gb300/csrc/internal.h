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
constexpr int kTPB32 = 128;         // threads per CTA, FP32C pair kernel
constexpr int kTPT32 = 2;           // targets per thread, FP32C
constexpr int kTPB64 = 128;         // threads per CTA, FP64 pair kernel
constexpr int kTPT64 = 1;           // targets per thread, FP64
constexpr int kRowAlign = 256;      // n_pad is a multiple of this (>= every CTA target span)

// Operators of the pair kernels.
enum Op { OP_LSL = 0, OP_LDL = 1, OP_SSL = 2, OP_SDL = 3, OP_SSLDL = 4, OP_LSLDL = 5 };
inline int op_components(int op) { return (op == OP_LSL || op == OP_LDL || op == OP_LSLDL) ? 1 : 3; }

struct alignas(16) d4 { double x, y, z, w; };

// Device layout of a point set: sorted copies used by the pair kernels.
struct Layout {
    int64_t n = 0, n_pad = 0;
    int32_t *perm = nullptr;   // sorted position -> caller index (n_pad entries, -1 for padding)
    float4 *pos32 = nullptr;   // (x, y, z, w)
    float4 *wn32 = nullptr;    // (w nx, w ny, w nz, 0)
    d4 *pos64 = nullptr;       // (x, y, z, w)
    d4 *wn64 = nullptr;        // (w nx, w ny, w nz, 0)
    double wsum = 0.0;         // sum of weights (host copy)
    void *block = nullptr;     // single allocation backing the arrays
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
    std::string err;
    // caching device allocator: blocks are reused in stream order
    struct Block { void *p; size_t bytes; bool used; };
    std::vector<Block> pool;
    // pinned host scratch for small device->host reads
    double *hbuf = nullptr;
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
    double *out = nullptr;
};
int pair_apply(ssd_ctx *ctx, const Layout &L, const PairCall &pc, cudaStream_t s);
int pair_occupancy(ssd_ctx *ctx);

// Quadrature (quad.cu)
int quadrature_points(ssd_ctx *ctx, const ssd_surface *surf, double h, double angle_deg, int64_t capacity,
                      int64_t *n_out, double *xyz, double *nrm, double *w, int32_t *meta, cudaStream_t s);

// Small vector kernels (solve.cu)
int dot(ssd_ctx *ctx, const double *a, const double *b, int64_t n, double *dev_out, cudaStream_t s);

}  // namespace ssd

#define SSD_TRY(expr)                 \
    do {                              \
        int _st = (expr);             \
        if (_st != SSD_OK) return _st; \
    } while (0)
