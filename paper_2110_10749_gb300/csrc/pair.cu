// Pair-sum kernels of the four regularized layer operators (Sections 5.1-5.3)
// and their fused single+double layer forms.
//
// Work decomposition: a CTA owns a span of targets (one per thread and
// target slot, consecutive in the layout's spatially sorted order) and one
// contiguous source range ("split").  Source records are staged in shared
// memory kTile at a time; every warp walks the tile with all lanes reading the
// same record (broadcast).  For each source the warp votes whether any of its
// targets lies within rho_far*delta; if none does, the bare kernels 1/r^p are
// evaluated (s_i = 1 to the working precision), otherwise the smoothed ones.
// Each split writes its per-target partial sums; the epilogue kernel adds the
// splits in a fixed order in FP64, applies the physical constants, the FP64
// self term of the single layers and the identity/right-hand-side terms, and
// scatters to the caller's order.
//
// FP32C: pair terms in FP32; each thread adds a tile's terms in FP32 and folds
// the tile sum into a two-float (hi, lo) accumulator with an error-free
// transformation (Knuth's TwoSum), so the accumulated error does not grow
// with the number of tiles.
#include <math.h>
#include <string.h>


#include "internal.h"
#include "erfcx_coef.h"
#include "series_coef.h"

namespace ssd {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kRhoSeries = 0.5;   // series branch below this rho (both precisions)
constexpr double kRhoFar32 = 5.5;    // 1 - s_i(rho) < 2^-25 beyond this (FP32)
constexpr double kRhoFar64 = 8.0;    // 1 - s_i(rho) < 1e-21 beyond this (FP64)
// symmetric plans: blocks of 512 layout points (the FP32C CTA's target span,
// a divisor of n_pad), far items of at most kSymTiles source tiles
constexpr int kSymBlock = kTPB32 * kTPT32;
constexpr int kSymTiles = 8;
// FP32C symmetric kernel: threads per CTA and resident CTAs per SM for its
// targets per thread (4: 128 threads, as the direct kernel; 8: 64 threads).
// With 8 targets the Stokes layers keep every value in registers at 4
// resident CTAs (up to 255 registers); the Laplace layers fit 6 (measured at
// N = 138830: Stokes DL 11.5 ms at 4 against 12.1 ms at 6, where it spills;
// Laplace DL 7.55 ms at 6 against 7.72 ms at 4)
constexpr int kSymTPB32 = kSymBlock / kSymTPT;
constexpr int sym_min_cta(int op) {
#ifdef SSD_SYMMINCTA
    return op >= 0 ? SSD_SYMMINCTA : 0;
#else
    return kSymTPT == 4 ? kMinCTA32 : ((op == OP_SDL || op == OP_SSL) ? 4 : 6);
#endif
}
static_assert(kSymTPB32 % 32 == 0 && kSymTPT % 2 == 0, "whole warps and packed target pairs");

template <int OP> struct OpInfo;
template <> struct OpInfo<OP_LSL>   { enum { NC = 1, WN = 0, D1 = 0, SL = 1, DL = 0 }; };
template <> struct OpInfo<OP_LDL>   { enum { NC = 1, WN = 1, D1 = 0, SL = 0, DL = 1 }; };
template <> struct OpInfo<OP_SSL>   { enum { NC = 3, WN = 0, D1 = 0, SL = 1, DL = 0 }; };
template <> struct OpInfo<OP_SDL>   { enum { NC = 3, WN = 1, D1 = 0, SL = 0, DL = 1 }; };
template <> struct OpInfo<OP_SSLDL> { enum { NC = 3, WN = 1, D1 = 1, SL = 1, DL = 1 }; };
template <> struct OpInfo<OP_LSLDL> { enum { NC = 1, WN = 1, D1 = 0, SL = 1, DL = 1 }; };
template <> struct OpInfo<OP_LDLT>  { enum { NC = 1, WN = 1, D1 = 0, SL = 0, DL = 1 }; };
template <> struct OpInfo<OP_SDLT>  { enum { NC = 3, WN = 1, D1 = 0, SL = 0, DL = 1 }; };

// ---------------------------------------------------------------- precision
template <typename R> struct Prec;
template <> struct Prec<float> {
    typedef float4 V4;
    static __device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
    static __device__ __forceinline__ float erf_(float x) { return erff(x); }
    static __device__ __forceinline__ float exp_(float x) { return expf(x); }
    static __device__ __forceinline__ float ser(int i, float t) {
        float s = kSeries32[i][SSD_NSER32 - 1];
#pragma unroll
        for (int k = SSD_NSER32 - 2; k >= 0; --k) s = fmaf(s, t, kSeries32[i][k]);
        return s;
    }
};
template <> struct Prec<double> {
    typedef d4 V4;
    static __device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
    static __device__ __forceinline__ double erf_(double x) { return erf(x); }
    static __device__ __forceinline__ double exp_(double x) { return exp(x); }
    static __device__ __forceinline__ double ser(int i, double t) {
        double s = kSeries[i][SSD_NSER - 1];
#pragma unroll
        for (int k = SSD_NSER - 2; k >= 0; --k) s = fma(s, t, kSeries[i][k]);
        return s;
    }
};

// Work item of a batched launch: targets [tbase, tbase + span) against
// sources [s_beg, s_end) of surface `surf`, written to partial split `split`.
struct BItem {
    int32_t tbase, s_beg, s_end, surf, split, pad0, pad1, pad2;
};
// Surface of a batched layout: padded range [poff, poff + n_pad), n_real real
// points, pbase = sum over earlier surfaces of nsplit * n_pad (partial offset).
struct BSurf {
    int64_t poff, n_pad, n_real, pbase, nsplit, pad0, pad1, pad2;
};

template <typename R> struct Consts {
    R inv_d, inv_d2, inv_d3, inv_d5;
    R rfar2;      // (rho_far delta)^2
    R tser;       // rho_series^2
    R cg;         // 2/sqrt(pi)
};

template <typename R> struct KArgs {
    const typename Prec<R>::V4 *pos, *wn, *d0, *d1;
    int64_t n_pad;
    int64_t chunk;       // sources per split (multiple of kTile)
    Consts<R> c;
    R *part;             // [split][NC][2 or 1][n_pad]
    // batched mode (items != nullptr): blockIdx.x = work item, blockIdx.y = right-hand side
    const BItem *items;
    const BSurf *surfs;
    const Consts<R> *consts;   // per surface
    int64_t rec_stride;        // density records per right-hand side
    int64_t part_stride;       // partial values per right-hand side
    const int2 *order = nullptr;   // single-surface launch order: blockIdx.x -> (target tile, split)
    int64_t tile0 = 0;             // single-surface launch without order: first target tile
    double *acc = nullptr;         // items of one surface: add each sum to acc[c][i] atomically
                                   // instead of writing per-split partials
};

// Smoothed radial factors k1 = s1/r, k2 = s2/r^3, k3 = s3/r^3, k4 = s4/r^5
// (Section 5.3).  `ser` selects the Taylor branch (rho < rho_series); the
// closed forms are evaluated otherwise.
template <typename R, int OP>
__device__ __forceinline__ void smooth(R r2, const Consts<R> &c, bool anyser, R &k1, R &k2, R &k3, R &k4) {
    typedef Prec<R> P;
    const R rinv = P::rsq(r2);
    // clamp at the far threshold (FP32: t = 40, 1 - s_i < 2e-12; FP64: t = 64,
    // 1 - s_i < 1e-21): keeps the polynomials finite for distant pairs
    const R tmax = sizeof(R) == 4 ? R(40) : R(64);
    const R t = fmin(r2 * c.inv_d2, tmax);
    const R rho = fmin(r2 * rinv * c.inv_d, sizeof(R) == 4 ? R(6.324555320336759) : R(8));
    const R e = P::exp_(-t);
    const R er = P::erf_(rho);
    const R ce = c.cg * rho * e;
    const R rinv2 = rinv * rinv;
    const R rinv3 = rinv2 * rinv;
    const R third = R(1) / R(3);
    if (OpInfo<OP>::SL) {
        const R s1 = er + ce * ((R(5) - R(2) * t) * third);
        const R s3 = er + ce * ((t * (R(14) - R(4) * t) - R(3)) * third);
        k1 = s1 * rinv;
        k3 = s3 * rinv3;
    }
    if (OP == OP_LDL || OP == OP_LSLDL || OP == OP_LDLT) {
        const R s2 = er + ce * ((R(2) * t - R(3)) * third);
        k2 = s2 * rinv3;
    }
    if (OP == OP_SDL || OP == OP_SSLDL || OP == OP_SDLT) {
        const R s4 = er - ce * ((t * (t * (R(8) * t - R(36)) + R(6)) + R(9)) * (R(1) / R(9)));
        k4 = s4 * rinv3 * rinv2;
    }
    if (anyser && t < c.tser) {
        if (OpInfo<OP>::SL) {
            k1 = P::ser(0, t) * c.inv_d;
            k3 = P::ser(2, t) * c.inv_d3;
        }
        if (OP == OP_LDL || OP == OP_LSLDL || OP == OP_LDLT) k2 = P::ser(1, t) * c.inv_d3;
        if (OP == OP_SDL || OP == OP_SSLDL || OP == OP_SDLT) k4 = P::ser(3, t) * c.inv_d5;
    }
}

// Adds the pair (target with position y and density dt, source record s)
// into acc.  Near = smoothed kernels.  `self` removes the single-layer self
// term (added in FP64 by the epilogue).
template <typename R, int OP, bool NEAR>
__device__ __forceinline__ void pair_term(const R d[3], const R r2, const R dt[3], const typename Prec<R>::V4 &sw,
                                          const typename Prec<R>::V4 &s0, const typename Prec<R>::V4 &s1,
                                          const Consts<R> &c, bool anyser, bool self, R acc[3],
                                          const R *twn = nullptr) {
    const R dx = d[0], dy = d[1], dz = d[2];
    R k1, k2, k3, k4;
    if (NEAR) {
        smooth<R, OP>(r2, c, anyser, k1, k2, k3, k4);
        if (self) { k1 = R(0); k3 = R(0); }
    } else {
        const R rinv = Prec<R>::rsq(r2);
        const R rinv2 = rinv * rinv;
        k1 = rinv;
        k2 = rinv2 * rinv;
        k3 = k2;
        k4 = k2 * rinv2;
    }
    if (OP == OP_LSL) {
        acc[0] += s0.x * k1;
    } else if (OP == OP_LDL) {
        const R yn = dx * sw.x + dy * sw.y + dz * sw.z;
        acc[0] += (s0.x - dt[0]) * yn * k2;
    } else if (OP == OP_LSLDL) {
        const R yn = dx * sw.x + dy * sw.y + dz * sw.z;
        acc[0] += s0.y * k1 + (s0.x - dt[0]) * yn * k2;
    } else if (OP == OP_SSL) {
        const R yf = dx * s0.x + dy * s0.y + dz * s0.z;
        const R b = yf * k3;
        acc[0] += s0.x * k1 + dx * b;
        acc[1] += s0.y * k1 + dy * b;
        acc[2] += s0.z * k1 + dz * b;
    } else if (OP == OP_SDL) {
        const R uy = (s0.x - dt[0]) * dx + (s0.y - dt[1]) * dy + (s0.z - dt[2]) * dz;
        const R yn = dx * sw.x + dy * sw.y + dz * sw.z;
        const R b = uy * yn * k4;
        acc[0] += b * dx;
        acc[1] += b * dy;
        acc[2] += b * dz;
    } else if (OP == OP_LDLT) {
        // transpose of D^L: k2 [ (yhat . w_i n_i) v_j + (yhat . w_j n_j) v_i ]
        const R ynt = dx * twn[0] + dy * twn[1] + dz * twn[2];
        const R yns = dx * sw.x + dy * sw.y + dz * sw.z;
        acc[0] += k2 * (ynt * s0.x + yns * dt[0]);
    } else if (OP == OP_SDLT) {
        // transpose of D^S: k4 yhat [ (yhat . w_i n_i)(yhat . v_j) + (yhat . w_j n_j)(yhat . v_i) ]
        const R ynt = dx * twn[0] + dy * twn[1] + dz * twn[2];
        const R yns = dx * sw.x + dy * sw.y + dz * sw.z;
        const R yvs = dx * s0.x + dy * s0.y + dz * s0.z;
        const R yvt = dx * dt[0] + dy * dt[1] + dz * dt[2];
        const R b = k4 * (ynt * yvs + yns * yvt);
        acc[0] += b * dx;
        acc[1] += b * dy;
        acc[2] += b * dz;
    } else {  // OP_SSLDL: s0 = scaled u, s1 = scaled w f
        const R uy = (s0.x - dt[0]) * dx + (s0.y - dt[1]) * dy + (s0.z - dt[2]) * dz;
        const R yn = dx * sw.x + dy * sw.y + dz * sw.z;
        const R yf = dx * s1.x + dy * s1.y + dz * s1.z;
        const R b = yf * k3 + uy * yn * k4;
        acc[0] += s1.x * k1 + dx * b;
        acc[1] += s1.y * k1 + dy * b;
        acc[2] += s1.z * k1 + dz * b;
    }
}

template <typename R> struct Acc;
template <> struct Acc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float p) {
        const float s = hi + p;
        const float bp = s - hi;
        const float err = (hi - (s - bp)) + (p - bp);
        hi = s;
        lo += err;
    }
};
template <> struct Acc<double> {
    double hi = 0.0;
    __device__ __forceinline__ void add(double p) { hi += p; }
};

template <typename R, int OP, int TPB, int TPT>
__global__ void __launch_bounds__(TPB) pair_kernel(const KArgs<R> a) {
    typedef typename Prec<R>::V4 V4;
    constexpr int NC = OpInfo<OP>::NC;
    __shared__ V4 sm_pos[kTile];
    __shared__ V4 sm_wn[OpInfo<OP>::WN ? kTile : 1];
    __shared__ V4 sm_d0[kTile];
    __shared__ V4 sm_d1[OpInfo<OP>::D1 ? kTile : 1];

    int64_t tbase, s_beg, s_end, part_base, pstride;
    const V4 *d0 = a.d0, *d1 = a.d1;
    Consts<R> c;
    if (a.items) {
        const BItem it = a.items[blockIdx.x];
        const BSurf sf = a.surfs[it.surf];
        tbase = it.tbase; s_beg = it.s_beg; s_end = it.s_end;
        c = a.consts[it.surf];
        d0 += blockIdx.y * a.rec_stride;
        d1 += blockIdx.y * a.rec_stride;
        constexpr int NSL = sizeof(Acc<R>) / sizeof(R);
        part_base = blockIdx.y * a.part_stride + NC * NSL * sf.pbase + (int64_t)it.split * NC * NSL * sf.n_pad - sf.poff;
        pstride = sf.n_pad;
    } else {
        int64_t bt = blockIdx.x + a.tile0, bs = blockIdx.y;
        if (a.order) {
            const int2 o = a.order[blockIdx.x];
            bt = o.x;
            bs = o.y;
        }
        tbase = bt * (TPB * TPT);
        s_beg = bs * a.chunk;
        s_end = s_beg + a.chunk;
        if (s_end > a.n_pad) s_end = a.n_pad;
        c = a.c;
        constexpr int NSL = sizeof(Acc<R>) / sizeof(R);
        part_base = bs * NC * NSL * a.n_pad;
        pstride = a.n_pad;
    }
    constexpr bool TR = (OP == OP_LDLT || OP == OP_SDLT);
    R y[TPT][3], dt[TPT][3], twn[TPT][3];
    Acc<R> acc[TPT][NC];
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int64_t i = tbase + threadIdx.x + t * TPB;   // < n_pad by construction
        const V4 p = a.pos[i];
        y[t][0] = p.x; y[t][1] = p.y; y[t][2] = p.z;
        const V4 d = d0[i];
        dt[t][0] = d.x; dt[t][1] = d.y; dt[t][2] = d.z;
        if (TR) {
            const V4 q = a.wn[i];
            twn[t][0] = q.x; twn[t][1] = q.y; twn[t][2] = q.z;
        }
    }

    for (int64_t tile = s_beg; tile < s_end; tile += kTile) {
        __syncthreads();
        for (int k = threadIdx.x; k < kTile; k += TPB) {
            sm_pos[k] = a.pos[tile + k];
            if (OpInfo<OP>::WN) sm_wn[k] = a.wn[tile + k];
            sm_d0[k] = d0[tile + k];
            if (OpInfo<OP>::D1) sm_d1[k] = d1[tile + k];
        }
        __syncthreads();
        R part[TPT][3];
#pragma unroll
        for (int t = 0; t < TPT; ++t) part[t][0] = part[t][1] = part[t][2] = R(0);
#pragma unroll 2
        for (int j = 0; j < kTile; ++j) {
            const V4 sp = sm_pos[j];
            const V4 sw = OpInfo<OP>::WN ? sm_wn[j] : sp;
            const V4 s0 = sm_d0[j];
            const V4 s1 = OpInfo<OP>::D1 ? sm_d1[j] : s0;
            bool near = false, ser = false;
            R d[TPT][3], r2[TPT];
#pragma unroll
            for (int t = 0; t < TPT; ++t) {
                d[t][0] = y[t][0] - sp.x;
                d[t][1] = y[t][1] - sp.y;
                d[t][2] = y[t][2] - sp.z;
                r2[t] = d[t][0] * d[t][0] + d[t][1] * d[t][1] + d[t][2] * d[t][2];
                near |= r2[t] < c.rfar2;
                ser |= r2[t] * c.inv_d2 < c.tser;
            }
            if (__any_sync(0xffffffffu, near)) {
                const bool anyser = __any_sync(0xffffffffu, ser);
                const int64_t js = tile + j;
#pragma unroll
                for (int t = 0; t < TPT; ++t) {
                    const bool self = (js == tbase + threadIdx.x + t * TPB);
                    pair_term<R, OP, true>(d[t], r2[t], dt[t], sw, s0, s1, c, anyser, self, part[t], twn[t]);
                }
            } else {
#pragma unroll
                for (int t = 0; t < TPT; ++t)
                    pair_term<R, OP, false>(d[t], r2[t], dt[t], sw, s0, s1, c, false, false, part[t], twn[t]);
            }
        }
#pragma unroll
        for (int t = 0; t < TPT; ++t)
#pragma unroll
            for (int q = 0; q < NC; ++q) acc[t][q].add(part[t][q]);
    }
    // partial layout: [split][comp][slot][n_pad], slot = hi (and lo for FP32)
    constexpr int NS = sizeof(Acc<R>) / sizeof(R);
    if (a.acc) {
#pragma unroll
        for (int t = 0; t < TPT; ++t) {
            const int64_t i = tbase + threadIdx.x + t * TPB;
#pragma unroll
            for (int q = 0; q < NC; ++q) {
                const R *v = reinterpret_cast<const R *>(&acc[t][q]);
                atomicAdd(a.acc + q * a.n_pad + i, NS == 2 ? (double)v[0] + (double)v[1] : (double)v[0]);
            }
        }
        return;
    }
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int64_t i = tbase + threadIdx.x + t * TPB;
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            R *dst = a.part + part_base + (int64_t)(q * NS) * pstride + i;
            dst[0] = acc[t][q].hi;
            if (NS == 2) dst[pstride] = reinterpret_cast<const R *>(&acc[t][q])[1];
        }
    }
}

// --------------------------------------------------------- FP32C kernel (v2)
// Four targets per thread, held as two packed f32x2 pairs so that every
// target-dependent FP32 operation of the bare-kernel path issues as one
// FFMA2/FADD2/FMUL2 for two targets.  Each warp tests its targets' bounding
// box against the bounding box of every 32-source chunk: a chunk farther
// than rho_far*delta from all of them runs the bare kernels with no per-source
// test; otherwise each source is voted on as in the generic kernel, and the
// smoothed path runs (scalar, per target) only when a target of the warp is
// within rho_far*delta of it.
struct K32Args {
    const float4 *pos, *wn, *d0, *d1;
    const float4 *cbox;
    int64_t n, n_pad, chunk;
    Consts<float> c;
    float *part;
    // batched mode (items != nullptr): blockIdx.x = work item, blockIdx.y = right-hand side
    const BItem *items;
    const BSurf *surfs;
    const Consts<float> *consts;
    int64_t rec_stride, part_stride;
    // single-surface mode: optional launch order (blockIdx.x -> (target tile,
    // split)), and 1 partial slot per target when every CTA holds one tile
    const int2 *order = nullptr;
    int nslot = 2;
    int64_t tile0 = 0;          // single-surface launch without order: first target tile
    double *acc = nullptr;      // items of one surface: add (hi + lo) to acc[c][i] atomically
                                // instead of writing per-split partials
};

__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 rsq2(float2 a) { return make_float2(rsqrtf(a.x), rsqrtf(a.y)); }

// Packed pair terms for the target pair (dt = target densities) with the
// displacement (dx, dy, dz) = y - x and r2 = |y - x|^2 already formed.
// NEAR = false: bare kernels (s_i = 1).  NEAR = true: smoothed kernels written
// as s_i = 1 - E_i, E_i = e^{-t} (erfcx(rho) - (2/sqrt(pi)) rho Q_i(t)),
// t = rho^2, valid for rho >= 0.5 (the Taylor branch covers smaller rho);
// Q_1 = (5 - 2t)/3, Q_2 = (2t - 3)/3, Q_3 = (-4t^2 + 14t - 3)/3,
// Q_4 = -(8t^3 - 36t^2 + 6t + 9)/9 (Section 5.3).
template <int OP, bool NEAR>
__device__ __forceinline__ void pair2(const float2 dx, const float2 dy, const float2 dz, const float2 r2,
                                      const float2 dt[3], const float4 &sw, const float4 &s0, const float4 &s1,
                                      const Consts<float> &c, float2 acc[3]) {
    const float2 ri = rsq2(r2);
    const float2 ri2 = mul2(ri, ri);
    const float2 ri3 = mul2(ri2, ri);
    float2 k1 = ri, k2 = ri3, k3 = ri3, k4 = mul2(ri3, ri2);
    if (NEAR) {
        // t and rho clamped at t = 40 (e^{-t} < 5e-18): beyond it E_i is zero
        // to FP32 precision, and the clamp keeps the Q_i polynomials finite
        // for distant sources (zero-weight padding lies 1e4 away)
        const float2 tr = mul2(r2, bc2(c.inv_d2));
        const float2 t = make_float2(fminf(tr.x, 40.f), fminf(tr.y, 40.f));
        const float2 rr = mul2(mul2(r2, ri), bc2(c.inv_d));
        const float2 rho = make_float2(fminf(rr.x, 6.32455532f), fminf(rr.y, 6.32455532f));
        const float2 et = mul2(t, bc2(-1.4426950408889634f));
        const float2 e = make_float2(exp2f(et.x), exp2f(et.y));
        const float2 w = fma2(make_float2(__fdividef(1.f, 1.f + rho.x), __fdividef(1.f, 1.f + rho.y)),
                              bc2(kErfcxA), bc2(-kErfcxB));
        const float2 P = erfcx_fit2(w);
        const float2 cr = mul2(rho, bc2(c.cg));
        const float third = 1.f / 3.f;
        if (OpInfo<OP>::SL) {
            const float2 q1 = fma2(t, bc2(-2.f * third), bc2(5.f * third));
            const float2 q3 = fma2(fma2(t, bc2(-4.f * third), bc2(14.f * third)), t, bc2(-1.f));
            k1 = mul2(k1, fma2(e, fma2(cr, q1, make_float2(-P.x, -P.y)), bc2(1.f)));
            k3 = mul2(k3, fma2(e, fma2(cr, q3, make_float2(-P.x, -P.y)), bc2(1.f)));
        }
        if (OP == OP_LDL || OP == OP_LSLDL) {
            const float2 q2 = fma2(t, bc2(2.f * third), bc2(-1.f));
            k2 = mul2(k2, fma2(e, fma2(cr, q2, make_float2(-P.x, -P.y)), bc2(1.f)));
        }
        if (OP == OP_SDL || OP == OP_SSLDL) {
            const float ninth = 1.f / 9.f;
            const float2 q4 = fma2(fma2(fma2(t, bc2(-8.f * ninth), bc2(4.f)), t, bc2(-6.f * ninth)), t, bc2(-1.f));
            k4 = mul2(k4, fma2(e, fma2(cr, q4, make_float2(-P.x, -P.y)), bc2(1.f)));
        }
    }
    if (OP == OP_LSL) {
        acc[0] = fma2(bc2(s0.x), k1, acc[0]);
    } else if (OP == OP_LDL || OP == OP_LSLDL) {
        const float2 yn = fma2(dz, bc2(sw.z), fma2(dy, bc2(sw.y), mul2(dx, bc2(sw.x))));
        const float2 dp = sub2(bc2(s0.x), dt[0]);
        acc[0] = fma2(mul2(dp, yn), k2, acc[0]);
        if (OP == OP_LSLDL) acc[0] = fma2(bc2(s0.y), k1, acc[0]);
    } else if (OP == OP_SSL) {
        const float2 yf = fma2(dz, bc2(s0.z), fma2(dy, bc2(s0.y), mul2(dx, bc2(s0.x))));
        const float2 b = mul2(yf, k3);
        acc[0] = fma2(bc2(s0.x), k1, fma2(dx, b, acc[0]));
        acc[1] = fma2(bc2(s0.y), k1, fma2(dy, b, acc[1]));
        acc[2] = fma2(bc2(s0.z), k1, fma2(dz, b, acc[2]));
    } else {  // OP_SDL, OP_SSLDL
        const float2 ux = sub2(bc2(s0.x), dt[0]), uy = sub2(bc2(s0.y), dt[1]), uz = sub2(bc2(s0.z), dt[2]);
        const float2 du = fma2(uz, dz, fma2(uy, dy, mul2(ux, dx)));
        const float2 yn = fma2(dz, bc2(sw.z), fma2(dy, bc2(sw.y), mul2(dx, bc2(sw.x))));
        float2 b = mul2(mul2(du, yn), k4);
        if (OP == OP_SSLDL) {
            const float2 yf = fma2(dz, bc2(s1.z), fma2(dy, bc2(s1.y), mul2(dx, bc2(s1.x))));
            b = fma2(yf, k3, b);
            acc[0] = fma2(bc2(s1.x), k1, acc[0]);
            acc[1] = fma2(bc2(s1.y), k1, acc[1]);
            acc[2] = fma2(bc2(s1.z), k1, acc[2]);
        }
        acc[0] = fma2(b, dx, acc[0]);
        acc[1] = fma2(b, dy, acc[1]);
        acc[2] = fma2(b, dz, acc[2]);
    }
}

template <int OP>
__global__ void __launch_bounds__(kTPB32, kMinCTA32) pair32_kernel(const K32Args a) {
    constexpr int NC = OpInfo<OP>::NC;
    constexpr int NP = kTPT32 / 2;   // packed pairs per thread
    __shared__ float4 sm_pos[kTile];
    __shared__ float4 sm_wn[OpInfo<OP>::WN ? kTile : 1];
    __shared__ float4 sm_d0[kTile];
    __shared__ float4 sm_d1[OpInfo<OP>::D1 ? kTile : 1];

    int64_t tbase, s_beg, s_end, part_base, pstride, nreal_end;
    const float4 *d0 = a.d0, *d1 = a.d1;
    Consts<float> c;
    if (a.items) {
        const BItem it = a.items[blockIdx.x];
        const BSurf sf = a.surfs[it.surf];
        tbase = it.tbase; s_beg = it.s_beg; s_end = it.s_end;
        nreal_end = sf.poff + sf.n_real;
        c = a.consts[it.surf];
        d0 += blockIdx.y * a.rec_stride;
        d1 += blockIdx.y * a.rec_stride;
        part_base = blockIdx.y * a.part_stride + NC * 2 * sf.pbase + (int64_t)it.split * NC * 2 * sf.n_pad - sf.poff;
        pstride = sf.n_pad;
    } else {
        int64_t bt = blockIdx.x + a.tile0, bs = blockIdx.y;
        if (a.order) {
            const int2 o = a.order[blockIdx.x];
            bt = o.x;
            bs = o.y;
        }
        tbase = bt * (kTPB32 * kTPT32);
        s_beg = bs * a.chunk;
        s_end = s_beg + a.chunk;
        if (s_end > a.n_pad) s_end = a.n_pad;
        nreal_end = a.n;
        c = a.c;
        part_base = bs * NC * a.nslot * a.n_pad;
        pstride = a.n_pad;
    }
    // target t = 2k + j (pair k, lane j) is index tbase + threadIdx.x + t * kTPB32
    float2 y[NP][3], dt[NP][3];
    float blo[3] = {1e30f, 1e30f, 1e30f}, bhi[3] = {-1e30f, -1e30f, -1e30f};
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int64_t i0 = tbase + threadIdx.x + (2 * k) * kTPB32, i1 = i0 + kTPB32;
        const float4 p0 = a.pos[i0], p1 = a.pos[i1];
        const float4 e0 = d0[i0], e1 = d0[i1];
        y[k][0] = make_float2(p0.x, p1.x); y[k][1] = make_float2(p0.y, p1.y); y[k][2] = make_float2(p0.z, p1.z);
        dt[k][0] = make_float2(e0.x, e1.x); dt[k][1] = make_float2(e0.y, e1.y); dt[k][2] = make_float2(e0.z, e1.z);
        if (i0 < nreal_end) {
            blo[0] = fminf(blo[0], p0.x); blo[1] = fminf(blo[1], p0.y); blo[2] = fminf(blo[2], p0.z);
            bhi[0] = fmaxf(bhi[0], p0.x); bhi[1] = fmaxf(bhi[1], p0.y); bhi[2] = fmaxf(bhi[2], p0.z);
        }
        if (i1 < nreal_end) {
            blo[0] = fminf(blo[0], p1.x); blo[1] = fminf(blo[1], p1.y); blo[2] = fminf(blo[2], p1.z);
            bhi[0] = fmaxf(bhi[0], p1.x); bhi[1] = fmaxf(bhi[1], p1.y); bhi[2] = fmaxf(bhi[2], p1.z);
        }
    }
    // warp bounding box of its real targets
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            blo[q] = fminf(blo[q], __shfl_xor_sync(0xffffffffu, blo[q], off));
            bhi[q] = fmaxf(bhi[q], __shfl_xor_sync(0xffffffffu, bhi[q], off));
        }
    const bool warp_empty = blo[0] > bhi[0];
    float hi[kTPT32][NC], lo[kTPT32][NC];
#pragma unroll
    for (int t = 0; t < kTPT32; ++t)
#pragma unroll
        for (int q = 0; q < NC; ++q) hi[t][q] = lo[t][q] = 0.f;

    for (int64_t tile = s_beg; tile < s_end; tile += kTile) {
        __syncthreads();
        for (int k = threadIdx.x; k < kTile; k += kTPB32) {
            sm_pos[k] = a.pos[tile + k];
            if (OpInfo<OP>::WN) sm_wn[k] = a.wn[tile + k];
            sm_d0[k] = d0[tile + k];
            if (OpInfo<OP>::D1) sm_d1[k] = d1[tile + k];
        }
        __syncthreads();
        float2 part[NP][3];
#pragma unroll
        for (int k = 0; k < NP; ++k) part[k][0] = part[k][1] = part[k][2] = make_float2(0.f, 0.f);
        for (int ch = 0; ch < kTile / kChunk; ++ch) {
            const int64_t cidx = (tile + ch * kChunk) / kChunk;
            const float4 clo = a.cbox[2 * cidx], chi = a.cbox[2 * cidx + 1];
            const float gx = fmaxf(0.f, fmaxf(clo.x - bhi[0], blo[0] - chi.x));
            const float gy = fmaxf(0.f, fmaxf(clo.y - bhi[1], blo[1] - chi.y));
            const float gz = fmaxf(0.f, fmaxf(clo.z - bhi[2], blo[2] - chi.z));
            const bool far_chunk = warp_empty || (gx * gx + gy * gy + gz * gz >= c.rfar2);
            const int j0 = ch * kChunk;
            if (far_chunk) {
#pragma unroll 4
                for (int j = j0; j < j0 + kChunk; ++j) {
                    const float4 sp = sm_pos[j];
                    const float4 sw = OpInfo<OP>::WN ? sm_wn[j] : sp;
                    const float4 s0 = sm_d0[j];
                    const float4 s1 = OpInfo<OP>::D1 ? sm_d1[j] : s0;
#pragma unroll
                    for (int k = 0; k < NP; ++k) {
                        const float2 dx = sub2(y[k][0], bc2(sp.x)), dy = sub2(y[k][1], bc2(sp.y)),
                                     dz = sub2(y[k][2], bc2(sp.z));
                        const float2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
                        pair2<OP, false>(dx, dy, dz, r2, dt[k], sw, s0, s1, c, part[k]);
                    }
                }
            } else {
                for (int j = j0; j < j0 + kChunk; ++j) {
                    const float4 sp = sm_pos[j];
                    const float4 sw = OpInfo<OP>::WN ? sm_wn[j] : sp;
                    const float4 s0 = sm_d0[j];
                    const float4 s1 = OpInfo<OP>::D1 ? sm_d1[j] : s0;
                    bool nearv = false, serv = false;
                    float2 DX[NP], DY[NP], DZ[NP], R2[NP];
#pragma unroll
                    for (int k = 0; k < NP; ++k) {
                        DX[k] = sub2(y[k][0], bc2(sp.x));
                        DY[k] = sub2(y[k][1], bc2(sp.y));
                        DZ[k] = sub2(y[k][2], bc2(sp.z));
                        R2[k] = fma2(DZ[k], DZ[k], fma2(DY[k], DY[k], mul2(DX[k], DX[k])));
                        nearv |= (R2[k].x < c.rfar2) | (R2[k].y < c.rfar2);
                        serv |= (R2[k].x * c.inv_d2 < c.tser) | (R2[k].y * c.inv_d2 < c.tser);
                    }
                    if (__any_sync(0xffffffffu, serv)) {
                        // a target of the warp is within 0.5 delta of this source
                        // (the self pair or a close neighbour): scalar path with
                        // the Taylor branch
                        const int64_t js = tile + j;
#pragma unroll
                        for (int k = 0; k < NP; ++k) {
#pragma unroll
                            for (int l = 0; l < 2; ++l) {
                                const float dv[3] = {l ? DX[k].y : DX[k].x, l ? DY[k].y : DY[k].x,
                                                     l ? DZ[k].y : DZ[k].x};
                                const float rr = l ? R2[k].y : R2[k].x;
                                const float dd[3] = {l ? dt[k][0].y : dt[k][0].x, l ? dt[k][1].y : dt[k][1].x,
                                                     l ? dt[k][2].y : dt[k][2].x};
                                const bool self = (js == tbase + threadIdx.x + (2 * k + l) * kTPB32);
                                float accs[3] = {0.f, 0.f, 0.f};
                                if (rr < c.rfar2)
                                    pair_term<float, OP, true>(dv, rr, dd, sw, s0, s1, c, true, self, accs);
                                else
                                    pair_term<float, OP, false>(dv, rr, dd, sw, s0, s1, c, false, false, accs);
                                if (l) {
                                    part[k][0].y += accs[0]; part[k][1].y += accs[1]; part[k][2].y += accs[2];
                                } else {
                                    part[k][0].x += accs[0]; part[k][1].x += accs[1]; part[k][2].x += accs[2];
                                }
                            }
                        }
                    } else if (__any_sync(0xffffffffu, nearv)) {
#pragma unroll
                        for (int k = 0; k < NP; ++k)
                            pair2<OP, true>(DX[k], DY[k], DZ[k], R2[k], dt[k], sw, s0, s1, c, part[k]);
                    } else {
#pragma unroll
                        for (int k = 0; k < NP; ++k)
                            pair2<OP, false>(DX[k], DY[k], DZ[k], R2[k], dt[k], sw, s0, s1, c, part[k]);
                    }
                }
            }
        }
        // fold the tile's partial sums into the two-float accumulators (TwoSum)
#pragma unroll
        for (int k = 0; k < NP; ++k)
#pragma unroll
            for (int q = 0; q < NC; ++q)
#pragma unroll
                for (int l = 0; l < 2; ++l) {
                    const int t = 2 * k + l;
                    const float p = l ? part[k][q].y : part[k][q].x;
                    const float sum = hi[t][q] + p;
                    const float bp = sum - hi[t][q];
                    lo[t][q] += (hi[t][q] - (sum - bp)) + (p - bp);
                    hi[t][q] = sum;
                }
    }
#pragma unroll
    for (int t = 0; t < kTPT32; ++t) {
        const int64_t i = tbase + threadIdx.x + t * kTPB32;
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            if (a.acc) {
                atomicAdd(a.acc + q * a.n_pad + i, (double)hi[t][q] + (double)lo[t][q]);
                continue;
            }
            float *dst = a.part + part_base + (int64_t)(q * a.nslot) * pstride + i;
            dst[0] = hi[t][q];
            if (a.nslot == 2) dst[pstride] = lo[t][q];
        }
    }
}

// ------------------------------------------------- symmetric far block pairs
// The four layer operators evaluated once per unordered pair of points in
// two blocks of the layout that are farther apart than rho_far delta (bare
// kernels, s_i = 1).  For targets a and sources b with yh = y_a - x_b, and
// m = w n:
//   Stokes DL:  A = (yh . (u_b - u_a)) / r^5,
//               a <- A (yh . m_b) yh,   b <- A (yh . m_a) yh
//   Laplace DL: B = (p_b - p_a) / r^3,
//               a <- B (yh . m_b),      b <- B (yh . m_a)
//   single layers (kernels even in yh, densities packed with w):
//               a <- S(yh) (w f)_b,     b <- S(yh) (w f)_a
// (the reverse terms follow from yh -> -yh and swapping the roles), so r, its
// powers and the density difference are shared by both directions.
// A CTA holds the 512 targets of one block (kSymTPT per thread as packed
// f32x2 pairs: 8 per thread in 64 threads by default) and walks source tiles
// of 128 staged in shared memory.  At step s lane l takes source
// (l + s) mod 128, so the 32 lanes of a warp work on 32 different sources and
// add their reverse terms to the warp's own shared accumulator without
// conflict; after the tile the warps' accumulators are summed.  More targets
// per thread share each staged source and each reverse-sum update.  Forward
// sums fold per tile into (hi, lo) pairs; both directions end in an FP64
// atomic add to acc[c][point].
struct SymItem {
    int32_t tb, s0, s1, pad;   // targets [tb, tb + 512), sources [s0, s1) (whole tiles)
};

struct SymArgs {
    const float4 *pos, *wn, *d0;
    const SymItem *items;
    int64_t n_pad;
    double *acc;               // [NC][n_pad]
};

template <int OP>
__global__ void __launch_bounds__(kSymTPB32, sym_min_cta(OP)) sym32_kernel(const SymArgs a) {
    constexpr int NC = OpInfo<OP>::NC;
    constexpr int TPB = kSymTPB32;
    constexpr int NP = kSymTPT / 2;
    constexpr int NW = TPB / 32;
    static_assert(kTile % TPB == 0, "whole staged sources per thread");
    // source records packed for the step loop: (x, y, z, d0.x), (w n, d0.y), d0.z;
    // reverse sums one float per component, warp and source
    __shared__ float4 sm_a[kTile], sm_b[kTile];
    __shared__ float sm_c[NC == 3 ? kTile : 1];
    __shared__ float sm_rev[NC][NW][kTile];
    const SymItem it = a.items[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2 y[NP][3], dt[NP][3], tm[NP][3];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int64_t i0 = it.tb + threadIdx.x + (2 * k) * TPB, i1 = i0 + TPB;
        const float4 p0 = a.pos[i0], p1 = a.pos[i1];
        const float4 e0 = a.d0[i0], e1 = a.d0[i1];
        const float4 m0 = a.wn[i0], m1 = a.wn[i1];
        y[k][0] = make_float2(p0.x, p1.x); y[k][1] = make_float2(p0.y, p1.y); y[k][2] = make_float2(p0.z, p1.z);
        dt[k][0] = make_float2(e0.x, e1.x); dt[k][1] = make_float2(e0.y, e1.y); dt[k][2] = make_float2(e0.z, e1.z);
        tm[k][0] = make_float2(m0.x, m1.x); tm[k][1] = make_float2(m0.y, m1.y); tm[k][2] = make_float2(m0.z, m1.z);
    }
    float hi[kSymTPT][NC], lo[kSymTPT][NC];
#pragma unroll
    for (int t = 0; t < kSymTPT; ++t)
#pragma unroll
        for (int q = 0; q < NC; ++q) hi[t][q] = lo[t][q] = 0.f;

    for (int64_t tile = it.s0; tile < it.s1; tile += kTile) {
        __syncthreads();
#pragma unroll
        for (int js = threadIdx.x; js < kTile; js += TPB) {
            const float4 ps = a.pos[tile + js], ms = a.wn[tile + js], ds = a.d0[tile + js];
            sm_a[js] = make_float4(ps.x, ps.y, ps.z, ds.x);
            sm_b[js] = make_float4(ms.x, ms.y, ms.z, ds.y);
            if (NC == 3) sm_c[js] = ds.z;
#pragma unroll
            for (int q = 0; q < NC; ++q)
#pragma unroll
                for (int w = 0; w < NW; ++w) sm_rev[q][w][js] = 0.f;
        }
        __syncthreads();
        float2 part[NP][NC];
#pragma unroll
        for (int k = 0; k < NP; ++k)
#pragma unroll
            for (int q = 0; q < NC; ++q) part[k][q] = make_float2(0.f, 0.f);
#pragma unroll 2
        for (int st = 0; st < kTile; ++st) {
            const int j = (lane + st) & (kTile - 1);
            const float4 sp = sm_a[j], sw = sm_b[j];
            const float4 s0 = make_float4(sp.w, sw.w, NC == 3 ? sm_c[j] : 0.f, 0.f);
            float2 rv[NC];
#pragma unroll
            for (int q = 0; q < NC; ++q) rv[q] = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const float2 dx = sub2(y[k][0], bc2(sp.x)), dy = sub2(y[k][1], bc2(sp.y)), dz = sub2(y[k][2], bc2(sp.z));
                const float2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
                const float2 ri = rsq2(r2);
                const float2 ri2 = mul2(ri, ri);
                const float2 ynb = fma2(dz, bc2(sw.z), fma2(dy, bc2(sw.y), mul2(dx, bc2(sw.x))));
                const float2 yna = fma2(dz, tm[k][2], fma2(dy, tm[k][1], mul2(dx, tm[k][0])));
                if (OP == OP_LSL) {
                    // G is even in yh: a <- (w g)_b / r, b <- (w g)_a / r
                    part[k][0] = fma2(bc2(s0.x), ri, part[k][0]);
                    rv[0] = fma2(dt[k][0], ri, rv[0]);
                } else if (OP == OP_SSL) {
                    // S is even in yh: a <- f_b / r + yh (yh . f_b) / r^3 (f = w f), and so for b
                    const float2 ri3 = mul2(ri2, ri);
                    const float2 bb = mul2(fma2(dz, bc2(s0.z), fma2(dy, bc2(s0.y), mul2(dx, bc2(s0.x)))), ri3);
                    const float2 ba = mul2(fma2(dz, dt[k][2], fma2(dy, dt[k][1], mul2(dx, dt[k][0]))), ri3);
                    part[k][0] = fma2(bc2(s0.x), ri, fma2(bb, dx, part[k][0]));
                    part[k][1] = fma2(bc2(s0.y), ri, fma2(bb, dy, part[k][1]));
                    part[k][2] = fma2(bc2(s0.z), ri, fma2(bb, dz, part[k][2]));
                    rv[0] = fma2(dt[k][0], ri, fma2(ba, dx, rv[0]));
                    rv[1] = fma2(dt[k][1], ri, fma2(ba, dy, rv[1]));
                    rv[2] = fma2(dt[k][2], ri, fma2(ba, dz, rv[2]));
                } else if (OP == OP_SDL) {
                    const float2 ux = sub2(bc2(s0.x), dt[k][0]), uy = sub2(bc2(s0.y), dt[k][1]),
                                 uz = sub2(bc2(s0.z), dt[k][2]);
                    const float2 du = fma2(uz, dz, fma2(uy, dy, mul2(ux, dx)));
                    const float2 A = mul2(du, mul2(mul2(ri2, ri2), ri));
                    const float2 f = mul2(A, ynb), g = mul2(A, yna);
                    part[k][0] = fma2(f, dx, part[k][0]);
                    part[k][1] = fma2(f, dy, part[k][1]);
                    part[k][2] = fma2(f, dz, part[k][2]);
                    rv[0] = fma2(g, dx, rv[0]);
                    rv[1] = fma2(g, dy, rv[1]);
                    rv[2] = fma2(g, dz, rv[2]);
                } else {   // OP_LDL
                    const float2 B = mul2(sub2(bc2(s0.x), dt[k][0]), mul2(ri2, ri));
                    part[k][0] = fma2(B, ynb, part[k][0]);
                    rv[0] = fma2(B, yna, rv[0]);
                }
            }
#pragma unroll
            for (int q = 0; q < NC; ++q) sm_rev[q][warp][j] += rv[q].x + rv[q].y;
            __syncwarp();
        }
        // forward: fold the tile's sums into the (hi, lo) pairs (TwoSum)
#pragma unroll
        for (int k = 0; k < NP; ++k)
#pragma unroll
            for (int q = 0; q < NC; ++q)
#pragma unroll
                for (int l = 0; l < 2; ++l) {
                    const int t = 2 * k + l;
                    const float p = l ? part[k][q].y : part[k][q].x;
                    const float sum = hi[t][q] + p;
                    const float bp = sum - hi[t][q];
                    lo[t][q] += (hi[t][q] - (sum - bp)) + (p - bp);
                    hi[t][q] = sum;
                }
        // reverse: the warps' sums of each source of the tile
        __syncthreads();
#pragma unroll
        for (int js = threadIdx.x; js < kTile; js += TPB) {
#pragma unroll
            for (int q = 0; q < NC; ++q) {
                float r = sm_rev[q][0][js];
#pragma unroll
                for (int w = 1; w < NW; ++w) r += sm_rev[q][w][js];
                atomicAdd(a.acc + q * a.n_pad + tile + js, (double)r);
            }
        }
    }
#pragma unroll
    for (int t = 0; t < kSymTPT; ++t) {
        const int64_t i = it.tb + threadIdx.x + t * TPB;
#pragma unroll
        for (int q = 0; q < NC; ++q) atomicAdd(a.acc + q * a.n_pad + i, (double)hi[t][q] + (double)lo[t][q]);
    }
}

// FP64 counterpart of sym32_kernel on the same block plan: a CTA of 128
// threads holds the 512 targets of one block, 4 per thread (threadIdx.x +
// 128 t), and walks the source tiles of its item with the same lane-rotated
// source order and per-warp reverse sums.  Sources are staged as separate
// coordinate arrays (one double per bank pair per lane).  The per-pair work
// shared by both directions (the displacement, r, its powers, the density
// difference) is done once.
struct Sym64Args {
    const d4 *pos, *wn, *d0;
    const SymItem *items;
    int64_t n_pad;
    double *acc;               // [NC][n_pad]
};

template <int OP>
__global__ void __launch_bounds__(kTPB64) sym64_kernel(const Sym64Args a) {
    constexpr int NC = OpInfo<OP>::NC;
    constexpr int DL = OpInfo<OP>::DL;
    constexpr int TT = kSymBlock / kTPB64;
    constexpr int NW = kTPB64 / 32;
    static_assert(kTile == kTPB64, "one staged source per thread");
    __shared__ double sm_p[3][kTile];
    __shared__ double sm_m[DL ? 3 : 1][kTile];
    __shared__ double sm_d[NC][kTile];
    __shared__ double sm_rev[NC][NW][kTile];
    const SymItem it = a.items[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double y[TT][3], dt[TT][NC], tm[TT][DL ? 3 : 1], tacc[TT][NC];
#pragma unroll
    for (int t = 0; t < TT; ++t) {
        const int64_t i = it.tb + threadIdx.x + t * kTPB64;
        const d4 p = a.pos[i], d = a.d0[i];
        y[t][0] = p.x; y[t][1] = p.y; y[t][2] = p.z;
        dt[t][0] = d.x;
        if constexpr (NC == 3) { dt[t][1] = d.y; dt[t][2] = d.z; }
        if constexpr (DL) {
            const d4 m = a.wn[i];
            tm[t][0] = m.x; tm[t][1] = m.y; tm[t][2] = m.z;
        }
#pragma unroll
        for (int q = 0; q < NC; ++q) tacc[t][q] = 0.0;
    }
    for (int64_t tile = it.s0; tile < it.s1; tile += kTile) {
        __syncthreads();
        {
            const int64_t j = tile + threadIdx.x;
            const d4 p = a.pos[j], d = a.d0[j];
            sm_p[0][threadIdx.x] = p.x; sm_p[1][threadIdx.x] = p.y; sm_p[2][threadIdx.x] = p.z;
            sm_d[0][threadIdx.x] = d.x;
            if constexpr (NC == 3) { sm_d[1][threadIdx.x] = d.y; sm_d[2][threadIdx.x] = d.z; }
            if constexpr (DL) {
                const d4 m = a.wn[j];
                sm_m[0][threadIdx.x] = m.x; sm_m[1][threadIdx.x] = m.y; sm_m[2][threadIdx.x] = m.z;
            }
#pragma unroll
            for (int q = 0; q < NC; ++q)
#pragma unroll
                for (int w = 0; w < NW; ++w) sm_rev[q][w][threadIdx.x] = 0.0;
        }
        __syncthreads();
#pragma unroll 2
        for (int st = 0; st < kTile; ++st) {
            const int j = (lane + st) & (kTile - 1);
            const double sx = sm_p[0][j], sy = sm_p[1][j], sz = sm_p[2][j];
            double s0[NC], sm[3] = {0.0, 0.0, 0.0}, rv[NC];
#pragma unroll
            for (int q = 0; q < NC; ++q) { s0[q] = sm_d[q][j]; rv[q] = 0.0; }
            if constexpr (DL) { sm[0] = sm_m[0][j]; sm[1] = sm_m[1][j]; sm[2] = sm_m[2][j]; }
#pragma unroll
            for (int t = 0; t < TT; ++t) {
                const double dx = y[t][0] - sx, dy = y[t][1] - sy, dz = y[t][2] - sz;
                const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
                const double ri = rsqrt(r2);
                if constexpr (OP == OP_LSL) {
                    tacc[t][0] = fma(s0[0], ri, tacc[t][0]);
                    rv[0] = fma(dt[t][0], ri, rv[0]);
                } else if constexpr (OP == OP_SSL) {
                    const double ri3 = ri * ri * ri;
                    const double bb = fma(dz, s0[2], fma(dy, s0[1], dx * s0[0])) * ri3;
                    const double ba = fma(dz, dt[t][2], fma(dy, dt[t][1], dx * dt[t][0])) * ri3;
                    tacc[t][0] = fma(s0[0], ri, fma(bb, dx, tacc[t][0]));
                    tacc[t][1] = fma(s0[1], ri, fma(bb, dy, tacc[t][1]));
                    tacc[t][2] = fma(s0[2], ri, fma(bb, dz, tacc[t][2]));
                    rv[0] = fma(dt[t][0], ri, fma(ba, dx, rv[0]));
                    rv[1] = fma(dt[t][1], ri, fma(ba, dy, rv[1]));
                    rv[2] = fma(dt[t][2], ri, fma(ba, dz, rv[2]));
                } else {
                    const double ynb = fma(dz, sm[2], fma(dy, sm[1], dx * sm[0]));
                    const double yna = fma(dz, tm[t][2], fma(dy, tm[t][1], dx * tm[t][0]));
                    const double ri2 = ri * ri;
                    if constexpr (OP == OP_LDL) {
                        // B = (p_b - p_a) / r^3: a <- B (yh . m_b), b <- B (yh . m_a)
                        const double B = (s0[0] - dt[t][0]) * (ri2 * ri);
                        tacc[t][0] = fma(B, ynb, tacc[t][0]);
                        rv[0] = fma(B, yna, rv[0]);
                    } else {
                        // A = (yh . (u_b - u_a)) / r^5: a <- A (yh . m_b) yh, b <- A (yh . m_a) yh
                        const double du = fma(dz, s0[2] - dt[t][2], fma(dy, s0[1] - dt[t][1], dx * (s0[0] - dt[t][0])));
                        const double A = du * (ri2 * ri2 * ri);
                        const double ab = A * ynb, aa = A * yna;
                        tacc[t][0] = fma(ab, dx, tacc[t][0]);
                        tacc[t][1] = fma(ab, dy, tacc[t][1]);
                        tacc[t][2] = fma(ab, dz, tacc[t][2]);
                        rv[0] = fma(aa, dx, rv[0]);
                        rv[1] = fma(aa, dy, rv[1]);
                        rv[2] = fma(aa, dz, rv[2]);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < NC; ++q) sm_rev[q][warp][j] += rv[q];
        }
        // reverse: the four warps' sums of source tile + threadIdx.x
        __syncthreads();
        const int64_t jb = tile + threadIdx.x;
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            double r = sm_rev[q][0][threadIdx.x];
#pragma unroll
            for (int w = 1; w < NW; ++w) r += sm_rev[q][w][threadIdx.x];
            atomicAdd(a.acc + q * a.n_pad + jb, r);
        }
    }
#pragma unroll
    for (int t = 0; t < TT; ++t) {
        const int64_t i = it.tb + threadIdx.x + t * kTPB64;
#pragma unroll
        for (int q = 0; q < NC; ++q) atomicAdd(a.acc + q * a.n_pad + i, tacc[t][q]);
    }
}

// ------------------------------------------------------------------- packing
// Densities in the layout's order, scaled for the kernel; padding slots zero.
struct PackArgs {
    const int32_t *perm;
    int64_t n, n_pad;
    int op;
    const double *d0, *d1;    // caller order; [NC][n] for vectors
    const d4 *pos64;          // layout positions and weights (sorted order)
    const d4 *wn64;           // layout weighted normals (sorted order)
    double s0, s1;            // scale of d0, d1 records (fused ops)
    int no_weight;            // single layers: pack the density without w (transpose)
    void *out0, *out1;        // float4 or d4 [n_pad]
    double *wdot_part;        // optional: per-block partial of sum w * d0 (Darcy gauge)
};

template <typename V4, typename R>
__global__ void pack_kernel(const PackArgs a) {
    __shared__ double red[256];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double wd = 0.0;
    if (i < a.n_pad) {
        const int32_t o = a.perm[i];
        V4 r0 = {R(0), R(0), R(0), R(0)}, r1 = {R(0), R(0), R(0), R(0)};
        if (o >= 0) {
            const double w = a.no_weight ? 1.0 : a.pos64[i].w;
            switch (a.op) {
                case OP_LSL: r0.x = R(a.s0 * w * a.d0[o]); break;
                case OP_LDLT: r0.x = R(a.s0 * a.d0[o]); break;
                case OP_SDLT:
                    r0.x = R(a.s0 * a.d0[o]);
                    r0.y = R(a.s0 * a.d0[a.n + o]);
                    r0.z = R(a.s0 * a.d0[2 * a.n + o]);
                    break;
                case OP_LDL: r0.x = R(a.s0 * a.d0[o]); wd = w * a.d0[o]; break;
                case OP_SSL:
                    r0.x = R(a.s0 * w * a.d0[o]);
                    r0.y = R(a.s0 * w * a.d0[a.n + o]);
                    r0.z = R(a.s0 * w * a.d0[2 * a.n + o]);
                    break;
                case OP_SDL:
                    r0.x = R(a.s0 * a.d0[o]);
                    r0.y = R(a.s0 * a.d0[a.n + o]);
                    r0.z = R(a.s0 * a.d0[2 * a.n + o]);
                    wd = a.wn64[i].x * a.d0[o] + a.wn64[i].y * a.d0[a.n + o] + a.wn64[i].z * a.d0[2 * a.n + o];
                    break;
                case OP_SSLDL:
                    r0.x = R(a.s0 * a.d0[o]);
                    r0.y = R(a.s0 * a.d0[a.n + o]);
                    r0.z = R(a.s0 * a.d0[2 * a.n + o]);
                    wd = a.wn64[i].x * a.d0[o] + a.wn64[i].y * a.d0[a.n + o] + a.wn64[i].z * a.d0[2 * a.n + o];
                    r1.x = R(a.s1 * w * a.d1[o]);
                    r1.y = R(a.s1 * w * a.d1[a.n + o]);
                    r1.z = R(a.s1 * w * a.d1[2 * a.n + o]);
                    break;
                default:  // OP_LSLDL
                    r0.x = R(a.s0 * a.d0[o]);
                    r0.y = R(a.s1 * w * a.d1[o]);
                    wd = w * a.d0[o];
                    break;
            }
        }
        reinterpret_cast<V4 *>(a.out0)[i] = r0;
        if (a.out1) reinterpret_cast<V4 *>(a.out1)[i] = r1;
    }
    if (a.wdot_part) {
        red[threadIdx.x] = wd;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) a.wdot_part[blockIdx.x] = red[0];
    }
}

// ------------------------------------------------------------------ epilogue
struct EpiArgs {
    int weight_out;          // multiply the pair sum by the target weight (single-layer transpose)
    const int32_t *perm;
    int64_t n, n_pad;
    int nc, nsplit, nslot;   // nslot: 2 for FP32 (hi, lo), 1 for FP64
    int part_is_float;
    const void *part;
    double scale;            // physical constant of the operator sum
    double self_coef;        // single-layer self term: self_coef * w * self_src
    const double *self_src;  // caller order, [nc][n]
    const d4 *pos64;         // layout (sorted order): weight in .w
    const double *xin;       // identity term source, caller order
    double a_id, a_op;
    double add0, add1, add2;
    const double *add_dev;
    const double *wdot_part; // rank-one term: (sum of parts) * wdot_scale, times rank1_nrm if set
    int nwdot;
    double wdot_scale;
    const double *rank1_nrm; // caller order [3][n]
    double *out;
    int64_t row0 = 0, row1 = -1;   // only layout rows [row0, row1) are written (row1 < 0: all)
};

__global__ void epilogue_kernel(const EpiArgs a) {
    // one thread per (point, component): partial sums are summed over the
    // splits in a fixed order in FP64
    __shared__ double extra, rank1;
    if (threadIdx.x == 0) {
        double e = a.add_dev ? *a.add_dev : 0.0;
        double r1 = 0.0;
        if (a.wdot_part) {
            double s = 0.0;
            for (int k = 0; k < a.nwdot; ++k) s += a.wdot_part[k];
            if (a.rank1_nrm) r1 = s * a.wdot_scale;
            else e += s * a.wdot_scale;
        }
        extra = e;
        rank1 = r1;
    }
    __syncthreads();
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.n_pad * a.nc) return;
    const int q = (int)(g / a.n_pad);
    const int64_t i = g - (int64_t)q * a.n_pad;
    if (a.row1 >= 0 && (i < a.row0 || i >= a.row1)) return;
    const int32_t o = a.perm[i];
    if (o < 0) return;
    // four interleaved partial sums over the splits (loads stay in flight),
    // combined in a fixed order
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    const int64_t sstride = (int64_t)a.nc * a.nslot * a.n_pad;
    const int64_t base0 = ((int64_t)q * a.nslot) * a.n_pad + i;
    if (a.part_is_float) {
        // FP32 partials summed with an error-free transformation (TwoSum) into
        // a (hi, lo) pair: FP32 arithmetic, no rounding error beyond lo's
        // loads are issued eight splits ahead of the sums
        const float *pf = reinterpret_cast<const float *>(a.part);
        float hi = 0.f, lo = 0.f;
        auto two_sum = [&](float p) {
            const float t = hi + p;
            const float bp = t - hi;
            lo += (hi - (t - bp)) + (p - bp);
            hi = t;
        };
        int sp = 0;
        if (a.nslot == 1) {
            for (; sp + 7 < a.nsplit; sp += 8) {
                float p[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) p[u] = pf[base0 + (sp + u) * sstride];
#pragma unroll
                for (int u = 0; u < 8; ++u) two_sum(p[u]);
            }
        }
        for (; sp < a.nsplit; ++sp)
            for (int l = 0; l < a.nslot; ++l) two_sum(pf[base0 + sp * sstride + l * a.n_pad]);
        s0 = (double)hi + (double)lo;
    } else {
        const double *pd = reinterpret_cast<const double *>(a.part);
        int sp = 0;
        for (; sp + 3 < a.nsplit; sp += 4) {
            const int64_t b = base0 + sp * sstride;
            s0 += pd[b];
            s1 += pd[b + sstride];
            s2 += pd[b + 2 * sstride];
            s3 += pd[b + 3 * sstride];
        }
        for (; sp < a.nsplit; ++sp) s0 += pd[base0 + sp * sstride];
    }
    const double s = (s0 + s1) + (s2 + s3);
    double v = a.scale * s * (a.weight_out ? a.pos64[i].w : 1.0);
    if (a.self_src) v += a.self_coef * a.pos64[i].w * a.self_src[(int64_t)q * a.n + o];
    double r = a.a_op * v + extra + (q == 0 ? a.add0 : (q == 1 ? a.add1 : a.add2));
    if (a.rank1_nrm) r += rank1 * a.rank1_nrm[(int64_t)q * a.n + o];
    if (a.xin) r += a.a_id * a.xin[(int64_t)q * a.n + o];
    a.out[(int64_t)q * a.n + o] = r;
}

template <int OP>
cudaError_t launch64(dim3 grid, const KArgs<double> &ka, cudaStream_t s) {
    pair_kernel<double, OP, kTPB64, kTPT64><<<grid, kTPB64, 0, s>>>(ka);
    return cudaGetLastError();
}

cudaError_t launch_pair_op64(int op, dim3 grid, const KArgs<double> &ka, cudaStream_t s) {
    switch (op) {
        case OP_LSL: return launch64<OP_LSL>(grid, ka, s);
        case OP_LDL: return launch64<OP_LDL>(grid, ka, s);
        case OP_SSL: return launch64<OP_SSL>(grid, ka, s);
        case OP_SDL: return launch64<OP_SDL>(grid, ka, s);
        case OP_SSLDL: return launch64<OP_SSLDL>(grid, ka, s);
        default: return launch64<OP_LSLDL>(grid, ka, s);
    }
}

// transposed double layers run on the generic kernel in both precisions
template <typename R>
cudaError_t launch_transpose(int op, dim3 grid, const KArgs<R> &ka, cudaStream_t s) {
    if (op == OP_LDLT) pair_kernel<R, OP_LDLT, kTPB64, kTPT64><<<grid, kTPB64, 0, s>>>(ka);
    else pair_kernel<R, OP_SDLT, kTPB64, kTPT64><<<grid, kTPB64, 0, s>>>(ka);
    return cudaGetLastError();
}

template <int OP>
cudaError_t launch32(dim3 grid, const K32Args &ka, cudaStream_t s) {
    pair32_kernel<OP><<<grid, kTPB32, 0, s>>>(ka);
    return cudaGetLastError();
}

cudaError_t launch_pair_op32(int op, dim3 grid, const K32Args &ka, cudaStream_t s) {
    switch (op) {
        case OP_LSL: return launch32<OP_LSL>(grid, ka, s);
        case OP_LDL: return launch32<OP_LDL>(grid, ka, s);
        case OP_SSL: return launch32<OP_SSL>(grid, ka, s);
        case OP_SDL: return launch32<OP_SDL>(grid, ka, s);
        case OP_SSLDL: return launch32<OP_SSLDL>(grid, ka, s);
        default: return launch32<OP_LSLDL>(grid, ka, s);
    }
}

int kernel_class(int op) {
    switch (op) {
        case OP_LSL: return SSD_K_LAPLACE_SL;
        case OP_LDL: return SSD_K_LAPLACE_DL;
        case OP_SSL: return SSD_K_STOKES_SL;
        case OP_SDL: return SSD_K_STOKES_DL;
        case OP_SSLDL: return SSD_K_STOKES_SLDL;
        case OP_LDLT: return SSD_K_LAPLACE_DL_T;
        case OP_SDLT: return SSD_K_STOKES_DL_T;
        default: return SSD_K_LAPLACE_SLDL;
    }
}

template <typename R>
Consts<R> make_consts(double delta, double rho_far) {
    Consts<R> c;
    c.inv_d = R(1.0 / delta);
    c.inv_d2 = R(1.0 / (delta * delta));
    c.inv_d3 = R(1.0 / (delta * delta * delta));
    c.inv_d5 = R(1.0 / (delta * delta * delta * delta * delta));
    c.rfar2 = R(rho_far * rho_far * delta * delta);
    c.tser = R(kRhoSeries * kRhoSeries);
    c.cg = R(2.0 / sqrt(kPi));
    return c;
}

// ------------------------------------------------------------ batched pack/epilogue
struct BPackArgs {
    const int32_t *perm;
    int64_t n_total, n_pad;       // caller points, padded layout size
    int op;
    const double *d0, *d1;        // [nrhs][c][n_total]
    int nc0, nc1;                 // components of d0 and d1
    const d4 *pos64, *wn64;
    double s0, s1;
    void *out0, *out1;            // records [nrhs][n_pad]
    double *wdot_part;            // [nrhs][pack blocks]: w (d0 . n) (vector ops) or w d0 (scalar)
    int want_wdot;
};

template <typename V4, typename R>
__global__ void bpack_kernel(const BPackArgs a) {
    __shared__ double red[256];
    const int r = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double *d0 = a.d0 + (int64_t)r * a.nc0 * a.n_total;
    const double *d1 = a.d1 ? a.d1 + (int64_t)r * a.nc1 * a.n_total : nullptr;
    const int64_t n = a.n_total;
    double wd = 0.0;
    if (i < a.n_pad) {
        const int32_t o = a.perm[i];
        V4 r0 = {R(0), R(0), R(0), R(0)}, r1 = {R(0), R(0), R(0), R(0)};
        if (o >= 0) {
            const double w = a.pos64[i].w;
            switch (a.op) {
                case OP_LSL: r0.x = R(a.s0 * w * d0[o]); break;
                case OP_LDL: r0.x = R(a.s0 * d0[o]); wd = w * d0[o]; break;
                case OP_SSL:
                    r0.x = R(a.s0 * w * d0[o]); r0.y = R(a.s0 * w * d0[n + o]); r0.z = R(a.s0 * w * d0[2 * n + o]);
                    break;
                case OP_SDL:
                case OP_SSLDL:
                    r0.x = R(a.s0 * d0[o]); r0.y = R(a.s0 * d0[n + o]); r0.z = R(a.s0 * d0[2 * n + o]);
                    wd = a.wn64[i].x * d0[o] + a.wn64[i].y * d0[n + o] + a.wn64[i].z * d0[2 * n + o];
                    if (a.op == OP_SSLDL) {
                        r1.x = R(a.s1 * w * d1[o]); r1.y = R(a.s1 * w * d1[n + o]); r1.z = R(a.s1 * w * d1[2 * n + o]);
                    }
                    break;
                default:  // OP_LSLDL
                    r0.x = R(a.s0 * d0[o]);
                    r0.y = R(a.s1 * w * d1[o]);
                    wd = w * d0[o];
                    break;
            }
        }
        reinterpret_cast<V4 *>(a.out0)[(int64_t)r * a.n_pad + i] = r0;
        if (a.out1) reinterpret_cast<V4 *>(a.out1)[(int64_t)r * a.n_pad + i] = r1;
    }
    if (a.want_wdot) {
        red[threadIdx.x] = wd;
        __syncthreads();
        for (int st = blockDim.x / 2; st > 0; st >>= 1) {
            if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
            __syncthreads();
        }
        if (threadIdx.x == 0) a.wdot_part[(int64_t)r * gridDim.x + blockIdx.x] = red[0];
    }
}

// per (right-hand side, surface) sum of the pack blocks of that surface
__global__ void bwdot_kernel(const double *part, int nblocks, const BSurf *surfs, int nsurf, int nrhs,
                             const double *wsum, double *out) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nsurf * nrhs) return;
    const int r = g / nsurf, sidx = g % nsurf;
    const int64_t b0 = surfs[sidx].poff / 256, b1 = (surfs[sidx].poff + surfs[sidx].n_pad) / 256;
    double acc = 0.0;
    for (int64_t b = b0; b < b1; ++b) acc += part[(int64_t)r * nblocks + b];
    out[g] = acc / wsum[sidx];
}

struct BEpiArgs {
    const int32_t *perm;
    const int32_t *elem_surf;      // caller index -> surface
    const BSurf *surfs;
    int64_t n_total, n_pad;
    int nc, nslot, part_is_float, nrhs, nsurf;
    const void *part;
    int64_t part_stride;           // per right-hand side
    double scale;
    double self_coef;              // times selfc[surface]
    const double *selfc;
    const double *self_src;        // [nrhs][nc][n_total]
    const d4 *pos64;
    const double *xin;
    double a_id, a_op;
    double add[kMaxRhs][3];
    const double *rank1;           // [nrhs][nsurf] coefficient, or NULL
    const double *rank1_nrm;       // [3][n_total] (vector ops) or NULL (scalar: add to every entry)
    double *out;
};

__global__ void bepilogue_kernel(const BEpiArgs a) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per_rhs = a.n_pad * a.nc;
    if (g >= per_rhs * a.nrhs) return;
    const int r = (int)(g / per_rhs);
    const int64_t rem = g - (int64_t)r * per_rhs;
    const int q = (int)(rem / a.n_pad);
    const int64_t i = rem - (int64_t)q * a.n_pad;
    const int32_t o = a.perm[i];
    if (o < 0) return;
    const int sidx = a.elem_surf[o];
    const BSurf sf = a.surfs[sidx];
    const int64_t li = i - sf.poff;
    double s = 0.0;
    for (int64_t sp = 0; sp < sf.nsplit; ++sp) {
        const int64_t base = (int64_t)r * a.part_stride + (int64_t)a.nc * a.nslot * sf.pbase +
                             ((sp * a.nc + q) * a.nslot) * sf.n_pad + li;
        if (a.part_is_float) {
            const float *pf = reinterpret_cast<const float *>(a.part);
            s += (double)pf[base];
            if (a.nslot == 2) s += (double)pf[base + sf.n_pad];
        } else {
            s += reinterpret_cast<const double *>(a.part)[base];
        }
    }
    const int64_t oi = ((int64_t)r * a.nc + q) * a.n_total + o;
    double v = a.scale * s;
    if (a.self_src) v += a.self_coef * a.selfc[sidx] * a.pos64[i].w * a.self_src[oi];
    double res = a.a_op * v + a.add[r][q];
    if (a.rank1) {
        const double c1 = a.rank1[r * a.nsurf + sidx];
        res += a.rank1_nrm ? c1 * a.rank1_nrm[(int64_t)q * a.n_total + o] : c1;
    }
    if (a.xin) res += a.a_id * a.xin[oi];
    a.out[oi] = res;
}

}  // namespace

// Launch order of the single-surface FP32C grid: items (target tile, split)
// with more near (warp, 32-source chunk) pairs first, so that the cheap far
// items fill the last wave (longest-processing-time-first).  key = number of
// near (warp, chunk) pairs of the item.
__global__ void item_cost_kernel(const float4 *cbox, int64_t ntiles_t, int64_t nsplit, int64_t chunk, int64_t n_pad,
                                 float rfar2, int tpb, int tpt, int32_t *key) {
    const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= ntiles_t * nsplit) return;
    const int64_t t = it % ntiles_t, sp = it / ntiles_t;
    const int nwarps = tpb / 32;
    const int64_t c0 = t * ((int64_t)tpb * tpt / kChunk);
    int cnt = 0;
    for (int w = 0; w < nwarps; ++w) {
        float lo[3] = {1e30f, 1e30f, 1e30f}, hi[3] = {-1e30f, -1e30f, -1e30f};
        for (int k = 0; k < tpt; ++k) {
            const int64_t cc = c0 + w + k * nwarps;
            const float4 l = cbox[2 * cc], h = cbox[2 * cc + 1];
            lo[0] = fminf(lo[0], l.x); lo[1] = fminf(lo[1], l.y); lo[2] = fminf(lo[2], l.z);
            hi[0] = fmaxf(hi[0], h.x); hi[1] = fmaxf(hi[1], h.y); hi[2] = fmaxf(hi[2], h.z);
        }
        if (lo[0] > hi[0]) continue;
        int64_t send = (sp + 1) * chunk;
        if (send > n_pad) send = n_pad;
        for (int64_t sc = sp * chunk / kChunk; sc < send / kChunk; ++sc) {
            const float4 l = cbox[2 * sc], h = cbox[2 * sc + 1];
            const float gx = fmaxf(0.f, fmaxf(l.x - hi[0], lo[0] - h.x));
            const float gy = fmaxf(0.f, fmaxf(l.y - hi[1], lo[1] - h.y));
            const float gz = fmaxf(0.f, fmaxf(l.z - hi[2], lo[2] - h.z));
            cnt += (gx * gx + gy * gy + gz * gz < rfar2) ? 1 : 0;
        }
    }
    key[it] = cnt;
}

// Builds (once per layout, delta and grid) the launch order of the FP32C grid.
int item_order(ssd_ctx *ctx, const Layout &L, int slot, int tpb, int tpt, int64_t ntiles_t, int64_t nsplit,
               int64_t chunk, float rfar2, const int2 **order, cudaStream_t s) {
    Layout &M = const_cast<Layout &>(L);
    const int64_t nit = ntiles_t * nsplit;
    if (M.order32[slot] && M.order_nit[slot] == nit && M.order_chunk[slot] == chunk &&
        M.order_rfar2[slot] == rfar2) {
        *order = M.order32[slot];
        return SSD_OK;
    }
    if (M.order32[slot]) { dev_free(ctx, M.order32[slot]); M.order32[slot] = nullptr; }
    void *keys = nullptr;
    SSD_TRY(dev_alloc(ctx, sizeof(int32_t) * nit, &keys));
    struct Release { ssd_ctx *c; void *p; ~Release() { dev_free(c, p); } } release{ctx, keys};
    item_cost_kernel<<<(unsigned)((nit + 255) / 256), 256, 0, s>>>(L.cbox, ntiles_t, nsplit, chunk, L.n_pad, rfar2,
                                                                   tpb, tpt, static_cast<int32_t *>(keys));
    ctx->launches++;
    SSD_TRY(launch_check(ctx, "item cost kernel"));
    std::vector<int32_t> hk(nit);
    SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(hk.data(), keys, sizeof(int32_t) * nit, cudaMemcpyDeviceToHost, s),
                       "key copy"));
    SSD_TRY(cuda_check(ctx, cudaStreamSynchronize(s), "key sync"));
    // stable counting sort, largest key first
    int32_t kmax = 0;
    for (int64_t i = 0; i < nit; ++i) kmax = hk[i] > kmax ? hk[i] : kmax;
    std::vector<int64_t> start(kmax + 2, 0);
    for (int64_t i = 0; i < nit; ++i) start[kmax - hk[i] + 1]++;
    for (int k = 1; k <= kmax + 1; ++k) start[k] += start[k - 1];
    std::vector<int2> ho(nit);
    for (int64_t i = 0; i < nit; ++i) ho[start[kmax - hk[i]]++] = make_int2((int)(i % ntiles_t), (int)(i / ntiles_t));
    void *dev = nullptr;
    SSD_TRY(dev_alloc(ctx, sizeof(int2) * nit, &dev));
    M.order32[slot] = static_cast<int2 *>(dev);
    SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(M.order32[slot], ho.data(), sizeof(int2) * nit, cudaMemcpyHostToDevice,
                                            s), "order copy"));
    SSD_TRY(cuda_check(ctx, cudaStreamSynchronize(s), "order sync"));
    M.order_nit[slot] = nit;
    M.order_chunk[slot] = chunk;
    M.order_rfar2[slot] = rfar2;
    *order = M.order32[slot];
    return SSD_OK;
}

// Work lists of the symmetric plan of the layer operators (see sym32_kernel
// and sym64_kernel), built once per prepared layout, precision and
// rho_far delta from the chunk boxes.  Blocks of 512 points: a pair of blocks
// whose boxes (of their real points) are farther apart than rho_far delta
// goes to the symmetric kernel, in items of the target block against at most
// kSymTiles source tiles; the diagonal blocks and the near block pairs (both
// directions) are items of the pair kernel of the precision (slot 0:
// pair32_kernel, one item of 512 targets; slot 1: the generic FP64 kernel,
// four items of 128 targets).  The plan is used when far pairs are at least
// half of all pairs.  The device block holds the surface descriptor, the
// kernel constants (`cbytes` bytes at `consts`), the near and the far items.
int sym_plan(ssd_ctx *ctx, const Layout &L, int slot, double rfar2, const void *consts, size_t cbytes,
             cudaStream_t s) {
    Layout &M = const_cast<Layout &>(L);
    SymPlan &pl = M.sym[slot];
    if (pl.rfar2 == rfar2) return SSD_OK;
    if (pl.block) { dev_free(ctx, pl.block); pl.block = nullptr; }
    pl.use = false;
    pl.near = pl.far = 0;
    const int nsub = slot == 0 ? 1 : kSymBlock / (kTPB64 * kTPT64);   // near items per block pair
    const int sub = kSymBlock / nsub;
    const int64_t n = L.n, n_pad = L.n_pad, nb = n_pad / kSymBlock, nch = n_pad / kChunk;
    std::vector<float4> cb(2 * nch);
    SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(cb.data(), L.cbox, sizeof(float4) * 2 * nch, cudaMemcpyDeviceToHost, s),
                       "chunk box copy"));
    SSD_TRY(cuda_check(ctx, cudaStreamSynchronize(s), "chunk box sync"));
    // boxes of the real points of each block
    std::vector<float> blo(3 * nb, 1e30f), bhi(3 * nb, -1e30f);
    for (int64_t ch = 0; ch < nch && ch * kChunk < n; ++ch) {
        const int64_t b = ch * kChunk / kSymBlock;
        const float lo[3] = {cb[2 * ch].x, cb[2 * ch].y, cb[2 * ch].z};
        const float hi[3] = {cb[2 * ch + 1].x, cb[2 * ch + 1].y, cb[2 * ch + 1].z};
        for (int q = 0; q < 3; ++q) {
            blo[3 * b + q] = fminf(blo[3 * b + q], lo[q]);
            bhi[3 * b + q] = fmaxf(bhi[3 * b + q], hi[q]);
        }
    }
    auto far_pair = [&](int64_t i, int64_t k) {
        if (blo[3 * i] > bhi[3 * i] || blo[3 * k] > bhi[3 * k]) return true;   // a block of padding only
        double g2 = 0.0;
        for (int q = 0; q < 3; ++q) {
            const double g = fmax(0.0, fmax((double)blo[3 * k + q] - bhi[3 * i + q], (double)blo[3 * i + q] - bhi[3 * k + q]));
            g2 += g * g;
        }
        return g2 >= rfar2;
    };
    std::vector<BItem> near;
    std::vector<SymItem> far;
    int64_t far_blocks = 0;
    auto near_item = [&](int64_t ti, int64_t si) {   // targets of block ti against sources of block si
        for (int q = 0; q < nsub; ++q)
            near.push_back(BItem{(int32_t)(ti * kSymBlock + q * sub), (int32_t)(si * kSymBlock),
                                 (int32_t)((si + 1) * kSymBlock), 0, 0, 0, 0, 0});
    };
    for (int64_t i = 0; i < nb; ++i) {
        near_item(i, i);
        int64_t k = i + 1;
        while (k < nb) {
            if (!far_pair(i, k)) {
                near_item(i, k);
                near_item(k, i);
                ++k;
                continue;
            }
            int64_t k1 = k;
            while (k1 < nb && far_pair(i, k1)) ++k1;
            far_blocks += k1 - k;
            for (int64_t t = k * kSymBlock; t < k1 * kSymBlock; t += (int64_t)kSymTiles * kTile) {
                int64_t e = t + (int64_t)kSymTiles * kTile;
                if (e > k1 * kSymBlock) e = k1 * kSymBlock;
                far.push_back(SymItem{(int32_t)(i * kSymBlock), (int32_t)t, (int32_t)e, 0});
            }
            k = k1;
        }
    }
    pl.rfar2 = rfar2;
    // far pairs (both directions) against all ordered pairs
    if (2.0 * (double)far_blocks < 0.5 * (double)nb * (double)nb) return SSD_OK;
    size_t off = 0;
    auto carve = [&](size_t b) { size_t o = off; off += (b + 255) & ~size_t(255); return o; };
    const size_t o_surf = carve(sizeof(BSurf)), o_c = carve(cbytes);
    const size_t o_near = carve(sizeof(BItem) * near.size()), o_far = carve(sizeof(SymItem) * far.size());
    void *blk = nullptr;
    SSD_TRY(dev_alloc(ctx, off, &blk));
    char *b = static_cast<char *>(blk);
    const BSurf sf{0, n_pad, n, 0, 1, 0, 0, 0};
    std::vector<char> host(off);
    memcpy(host.data() + o_surf, &sf, sizeof(sf));
    memcpy(host.data() + o_c, consts, cbytes);
    memcpy(host.data() + o_near, near.data(), sizeof(BItem) * near.size());
    memcpy(host.data() + o_far, far.data(), sizeof(SymItem) * far.size());
    const int st = cuda_check(ctx, cudaMemcpyAsync(b, host.data(), off, cudaMemcpyHostToDevice, s), "plan copy");
    if (st == SSD_OK) SSD_TRY(cuda_check(ctx, cudaStreamSynchronize(s), "plan sync"));
    if (st != SSD_OK) { dev_free(ctx, blk); return st; }
    pl.block = blk;
    pl.near = (int64_t)near.size();
    pl.far = (int64_t)far.size();
    pl.use = true;
    return SSD_OK;
}

template <int OP>
cudaError_t launch_sym(const Layout &L, const float4 *d0, double *acc, cudaStream_t s) {
    const SymPlan &pl = L.sym[0];
    char *b = static_cast<char *>(pl.block);
    size_t off = 0;
    auto carve = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~size_t(255); return o; };
    const size_t o_surf = carve(sizeof(BSurf)), o_c = carve(sizeof(Consts<float>));
    const size_t o_near = carve(sizeof(BItem) * pl.near);
    const size_t o_far = carve(sizeof(SymItem) * pl.far);
    K32Args ka;
    ka.pos = L.pos32; ka.wn = L.wn32; ka.cbox = L.cbox; ka.d0 = d0; ka.d1 = d0;
    ka.n = L.n; ka.n_pad = L.n_pad; ka.chunk = kSymBlock;
    ka.part = nullptr;
    ka.items = reinterpret_cast<const BItem *>(b + o_near);
    ka.surfs = reinterpret_cast<const BSurf *>(b + o_surf);
    ka.consts = reinterpret_cast<const Consts<float> *>(b + o_c);
    ka.rec_stride = 0; ka.part_stride = 0;
    ka.acc = acc;
    pair32_kernel<OP><<<dim3((unsigned)pl.near, 1), kTPB32, 0, s>>>(ka);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || pl.far == 0) return e;
    SymArgs sa;
    sa.pos = L.pos32; sa.wn = L.wn32; sa.d0 = d0;
    sa.items = reinterpret_cast<const SymItem *>(b + o_far);
    sa.n_pad = L.n_pad; sa.acc = acc;
    sym32_kernel<OP><<<(unsigned)pl.far, kSymTPB32, 0, s>>>(sa);
    return cudaGetLastError();
}

template <int OP>
cudaError_t launch_sym64(const Layout &L, const d4 *d0, double *acc, cudaStream_t s) {
    const SymPlan &pl = L.sym[1];
    char *b = static_cast<char *>(pl.block);
    size_t off = 0;
    auto carve = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~size_t(255); return o; };
    const size_t o_surf = carve(sizeof(BSurf)), o_c = carve(sizeof(Consts<double>));
    const size_t o_near = carve(sizeof(BItem) * pl.near);
    const size_t o_far = carve(sizeof(SymItem) * pl.far);
    KArgs<double> ka;
    ka.pos = L.pos64; ka.wn = L.wn64; ka.d0 = d0; ka.d1 = d0;
    ka.n_pad = L.n_pad; ka.chunk = kSymBlock;
    ka.part = nullptr;
    ka.items = reinterpret_cast<const BItem *>(b + o_near);
    ka.surfs = reinterpret_cast<const BSurf *>(b + o_surf);
    ka.consts = reinterpret_cast<const Consts<double> *>(b + o_c);
    ka.rec_stride = 0; ka.part_stride = 0;
    ka.acc = acc;
    pair_kernel<double, OP, kTPB64, kTPT64><<<dim3((unsigned)pl.near, 1), kTPB64, 0, s>>>(ka);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || pl.far == 0) return e;
    Sym64Args sa;
    sa.pos = L.pos64; sa.wn = L.wn64; sa.d0 = d0;
    sa.items = reinterpret_cast<const SymItem *>(b + o_far);
    sa.n_pad = L.n_pad; sa.acc = acc;
    sym64_kernel<OP><<<(unsigned)pl.far, kTPB64, 0, s>>>(sa);
    return cudaGetLastError();
}

int pair_occupancy(ssd_ctx *ctx) {
    int o32 = 0, o64 = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o32, pair32_kernel<OP_SSLDL>, kTPB32, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o64, pair_kernel<double, OP_SSLDL, kTPB64, kTPT64>,
                                                          kTPB64, 0);
    if (e != cudaSuccess) return cuda_check(ctx, e, "occupancy query");
    ctx->occ32 = o32 > 0 ? o32 : 1;
    ctx->occ64 = o64 > 0 ? o64 : 1;
    return SSD_OK;
}

int pair_apply(ssd_ctx *ctx, const Layout &L, const PairCall &pc, cudaStream_t s) {
    const int op = pc.op;
    const int nc = op_components(op);
    const bool f32 = (pc.prec == SSD_FP32C);
    const int64_t n = L.n, n_pad = L.n_pad;
    const bool transposed = (op == OP_LDLT || op == OP_SDLT);
    const bool packed32 = f32 && !transposed;    // the packed FP32 kernel, else the generic one
    const int tspan = packed32 ? kTPB32 * kTPT32 : kTPB64 * kTPT64;
    const int64_t ntiles_t = n_pad / tspan;
    const int64_t ntiles_s = n_pad / kTile;
    // splits: enough CTAs for several waves of resident CTAs, so that the
    // uneven cost of near and far target tiles evens out (FP32C: tuned on the
    // h = 1/32 sphere, where it reaches one 128-source tile per CTA)
    const int occ = packed32 ? ctx->occ32 : ctx->occ64;
    int64_t want = (int64_t)ctx->num_sms * occ * (packed32 ? ctx->waves32 : ctx->waves64);
    int64_t nsplit = (want + ntiles_t - 1) / ntiles_t;
    if (nsplit < 1) nsplit = 1;
    if (nsplit > ntiles_s) nsplit = ntiles_s;
    const int64_t chunk_tiles = (ntiles_s + nsplit - 1) / nsplit;
    nsplit = (ntiles_s + chunk_tiles - 1) / chunk_tiles;
    const int64_t chunk = chunk_tiles * kTile;

    const size_t rec = f32 ? sizeof(float4) : sizeof(d4);
    // FP32C keeps a (hi, lo) pair per target and split; one slot suffices when
    // every CTA of the packed kernel holds a single source tile (lo stays 0)
    const int nslot = f32 ? ((packed32 && chunk == kTile) ? 1 : 2) : 1;
    const size_t rsz = f32 ? sizeof(float) : sizeof(double);
    const bool two_rec = (op == OP_SSLDL);
    const int pack_blocks = (int)((n_pad + 255) / 256);
    size_t off = 0;
    auto carve = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~size_t(255); return o; };
    const size_t o_d0 = carve(rec * n_pad);
    const size_t o_d1 = two_rec ? carve(rec * n_pad) : 0;
    const size_t o_part = carve(rsz * nslot * nc * nsplit * n_pad);
    const size_t o_wdot = carve(sizeof(double) * pack_blocks);
    // layer operators on a prepared layout: the symmetric plan of the
    // precision when far block pairs are most of the work (FP64 accumulator
    // instead of partials)
    const bool rows_req = pc.row_end >= 0;
    bool use_sym = false;
    if (!transposed && (op == OP_SDL || op == OP_LDL || op == OP_SSL || op == OP_LSL) && !rows_req && ctx->sym &&
        L.order_ok) {
        if (f32) {
            const Consts<float> c = make_consts<float>(pc.delta, kRhoFar32);
            SSD_TRY(sym_plan(ctx, L, 0, c.rfar2, &c, sizeof(c), s));
        } else {
            const Consts<double> c = make_consts<double>(pc.delta, kRhoFar64);
            SSD_TRY(sym_plan(ctx, L, 1, c.rfar2, &c, sizeof(c), s));
        }
        use_sym = L.sym[f32 ? 0 : 1].use;
    }
    const size_t o_acc = use_sym ? carve(sizeof(double) * nc * n_pad) : 0;
    void *ws = nullptr;
    SSD_TRY(dev_alloc(ctx, off, &ws));
    struct Release { ssd_ctx *c; void *p; ~Release() { dev_free(c, p); } } release{ctx, ws};
    char *base = static_cast<char *>(ws);

    // physical constants and record scales
    double scale = 1.0, s0 = 1.0, s1 = 1.0, self_coef = 0.0;
    const double sig1_0 = 16.0 / (3.0 * sqrt(kPi));   // lim s1(rho)/rho at rho = 0
    const double *self_src = nullptr;
    switch (op) {
        case OP_LSL: scale = -1.0 / (4.0 * kPi); self_coef = scale * sig1_0 / pc.delta; self_src = pc.dens0; break;
        case OP_LDL: scale = -1.0 / (4.0 * kPi); break;
        case OP_SSL: scale = 1.0 / (8.0 * kPi * pc.mu); self_coef = scale * sig1_0 / pc.delta; self_src = pc.dens0; break;
        case OP_SDL: scale = 6.0 / (8.0 * kPi); break;
        case OP_SSLDL:
            s0 = pc.beta * 6.0 / (8.0 * kPi);           // u records
            s1 = pc.alpha / (8.0 * kPi * pc.mu);        // w f records
            self_coef = s1 * sig1_0 / pc.delta; self_src = pc.dens1;
            break;
        case OP_LDLT: scale = 1.0 / (4.0 * kPi); break;
        case OP_SDLT: scale = -6.0 / (8.0 * kPi); break;
        default:  // OP_LSLDL
            scale = -1.0 / (4.0 * kPi);
            s0 = pc.beta;                                // p records
            s1 = pc.alpha;                               // w g records
            self_coef = scale * pc.alpha * sig1_0 / pc.delta; self_src = pc.dens1;
            break;
    }
    const bool tsl = pc.transpose_sl && (op == OP_LSL || op == OP_SSL);

    PackArgs pa{};
    pa.perm = L.perm; pa.n = n; pa.n_pad = n_pad; pa.op = op;
    pa.d0 = pc.dens0; pa.d1 = pc.dens1; pa.pos64 = L.pos64; pa.wn64 = L.wn64; pa.s0 = s0; pa.s1 = s1;
    pa.out0 = base + o_d0; pa.out1 = two_rec ? base + o_d1 : nullptr;
    pa.no_weight = tsl ? 1 : 0;
    const bool rank1 = pc.rank1_weight_mean || pc.rank1_nrm != nullptr;
    pa.wdot_part = rank1 ? reinterpret_cast<double *>(base + o_wdot) : nullptr;
    if (f32) pack_kernel<float4, float><<<pack_blocks, 256, 0, s>>>(pa);
    else pack_kernel<d4, double><<<pack_blocks, 256, 0, s>>>(pa);
    ctx->launches++;
    SSD_TRY(launch_check(ctx, "pack kernel"));

    const int cls = kernel_class(op);
    // a row block (layout rows [row_begin, row_end)) launches only the target
    // tiles that cover it, with the splits of the whole operator, so every
    // row's sum is the one the whole operator computes
    const bool rows = pc.row_end >= 0;
    const int64_t tile0 = rows ? pc.row_begin / tspan : 0;
    const int64_t tile1 = rows ? (pc.row_end + tspan - 1) / tspan : ntiles_t;
    if (rows && !(pc.row_begin >= 0 && pc.row_begin < pc.row_end && pc.row_end <= n))
        return set_error(ctx, SSD_EINVAL, "row block must satisfy 0 <= row_begin < row_end <= n");
    cudaEvent_t ev = nullptr;
    double *acc = use_sym ? reinterpret_cast<double *>(base + o_acc) : nullptr;
    if (use_sym)
        SSD_TRY(cuda_check(ctx, cudaMemsetAsync(acc, 0, sizeof(double) * nc * n_pad, s), "accumulator memset"));
    SSD_TRY(timed_begin(ctx, s, &ev));
    dim3 grid((unsigned)(tile1 - tile0), (unsigned)nsplit);
    cudaError_t e;
    if (use_sym && f32) {
        const float4 *d0 = reinterpret_cast<const float4 *>(base + o_d0);
        switch (op) {
            case OP_SDL: e = launch_sym<OP_SDL>(L, d0, acc, s); break;
            case OP_LDL: e = launch_sym<OP_LDL>(L, d0, acc, s); break;
            case OP_SSL: e = launch_sym<OP_SSL>(L, d0, acc, s); break;
            default: e = launch_sym<OP_LSL>(L, d0, acc, s); break;
        }
        if (L.sym[0].far) ctx->launches++;   // near items and far items: two launches
    } else if (use_sym) {
        const d4 *d0 = reinterpret_cast<const d4 *>(base + o_d0);
        switch (op) {
            case OP_SDL: e = launch_sym64<OP_SDL>(L, d0, acc, s); break;
            case OP_LDL: e = launch_sym64<OP_LDL>(L, d0, acc, s); break;
            case OP_SSL: e = launch_sym64<OP_SSL>(L, d0, acc, s); break;
            default: e = launch_sym64<OP_LSL>(L, d0, acc, s); break;
        }
        if (L.sym[1].far) ctx->launches++;
    } else if (f32 && transposed) {
        KArgs<float> ka;
        ka.pos = L.pos32; ka.wn = L.wn32;
        ka.d0 = reinterpret_cast<const float4 *>(base + o_d0);
        ka.d1 = ka.d0;
        ka.n_pad = n_pad; ka.chunk = chunk;
        ka.c = make_consts<float>(pc.delta, kRhoFar32);
        ka.part = reinterpret_cast<float *>(base + o_part);
        ka.items = nullptr; ka.surfs = nullptr; ka.consts = nullptr; ka.rec_stride = 0; ka.part_stride = 0;
        ka.tile0 = tile0;
        e = launch_transpose<float>(op, grid, ka, s);
    } else if (f32) {
        K32Args ka;
        ka.pos = L.pos32; ka.wn = L.wn32; ka.cbox = L.cbox;
        ka.d0 = reinterpret_cast<const float4 *>(base + o_d0);
        ka.d1 = two_rec ? reinterpret_cast<const float4 *>(base + o_d1) : ka.d0;
        ka.n = n; ka.n_pad = n_pad; ka.chunk = chunk;
        ka.c = make_consts<float>(pc.delta, kRhoFar32);
        ka.part = reinterpret_cast<float *>(base + o_part);
        ka.items = nullptr; ka.surfs = nullptr; ka.consts = nullptr; ka.rec_stride = 0; ka.part_stride = 0;
        ka.nslot = nslot;
        ka.tile0 = tile0;
        dim3 g = grid;
        if (ctx->lpt && L.order_ok && !rows) {
            const int2 *ord = nullptr;
            const int st = item_order(ctx, L, 0, kTPB32, kTPT32, ntiles_t, nsplit, chunk, ka.c.rfar2, &ord, s);
            if (st != SSD_OK) return st;
            ka.order = ord;
            g = dim3((unsigned)(ntiles_t * nsplit), 1);
        }
        e = launch_pair_op32(op, g, ka, s);
    } else {
        KArgs<double> ka;
        ka.pos = L.pos64; ka.wn = L.wn64;
        ka.d0 = reinterpret_cast<const d4 *>(base + o_d0);
        ka.d1 = two_rec ? reinterpret_cast<const d4 *>(base + o_d1) : ka.d0;
        ka.n_pad = n_pad; ka.chunk = chunk;
        ka.c = make_consts<double>(pc.delta, kRhoFar64);
        ka.part = reinterpret_cast<double *>(base + o_part);
        ka.items = nullptr; ka.surfs = nullptr; ka.consts = nullptr; ka.rec_stride = 0; ka.part_stride = 0;
        ka.tile0 = tile0;
        dim3 g = grid;
        if (ctx->lpt && L.order_ok && !rows) {
            const int2 *ord = nullptr;
            const int st = item_order(ctx, L, 1, kTPB64, kTPT64, ntiles_t, nsplit, chunk,
                                      (float)ka.c.rfar2, &ord, s);
            if (st != SSD_OK) return st;
            ka.order = ord;
            g = dim3((unsigned)(ntiles_t * nsplit), 1);
        }
        e = transposed ? launch_transpose<double>(op, g, ka, s) : launch_pair_op64(op, g, ka, s);
    }
    ctx->launches++;
    if (e != cudaSuccess) return cuda_check(ctx, e, "pair kernel launch");
    timed_end(ctx, s, ev, cls, pc.prec, (double)(rows ? pc.row_end - pc.row_begin : n) * (double)n);

    EpiArgs ea{};
    ea.perm = L.perm; ea.n = n; ea.n_pad = n_pad; ea.nc = nc; ea.nsplit = (int)nsplit; ea.nslot = nslot;
    ea.part_is_float = f32 ? 1 : 0; ea.part = base + o_part;
    if (use_sym) {   // one FP64 sum per point and component
        ea.nsplit = 1; ea.nslot = 1; ea.part_is_float = 0; ea.part = acc;
    }
    ea.scale = scale; ea.self_coef = self_coef; ea.self_src = self_src; ea.pos64 = L.pos64;
    ea.xin = pc.xin; ea.a_id = pc.a_id; ea.a_op = pc.a_op;
    ea.add0 = pc.add[0]; ea.add1 = pc.add[1]; ea.add2 = pc.add[2]; ea.add_dev = pc.add_dev;
    ea.wdot_part = rank1 ? reinterpret_cast<const double *>(base + o_wdot) : nullptr;
    ea.nwdot = pack_blocks; ea.wdot_scale = rank1 ? 1.0 / L.wsum : 0.0;
    ea.rank1_nrm = pc.rank1_nrm;
    ea.weight_out = tsl ? 1 : 0;
    ea.out = pc.out;
    if (rows) { ea.row0 = pc.row_begin; ea.row1 = pc.row_end; }
    epilogue_kernel<<<(unsigned)((n_pad * nc + 127) / 128), 128, 0, s>>>(ea);
    ctx->launches++;
    return launch_check(ctx, "epilogue kernel");
}


// Near (warp, 32-source chunk) count of each FP32C work item of a batch, as
// item_cost_kernel does for a single surface (smoothing radius per surface).
__global__ void batch_item_cost_kernel(const BItem *items, int64_t nitems, const Consts<float> *consts,
                                       const float4 *cbox, int32_t *key) {
    const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= nitems) return;
    const BItem bi = items[it];
    const float rfar2 = consts[bi.surf].rfar2;
    constexpr int kWarps = kTPB32 / 32;
    const int64_t c0 = bi.tbase / kChunk;
    int cnt = 0;
    for (int w = 0; w < kWarps; ++w) {
        float lo[3] = {1e30f, 1e30f, 1e30f}, hi[3] = {-1e30f, -1e30f, -1e30f};
        for (int k = 0; k < kTPT32; ++k) {
            const int64_t cc = c0 + w + k * kWarps;
            const float4 l = cbox[2 * cc], h = cbox[2 * cc + 1];
            lo[0] = fminf(lo[0], l.x); lo[1] = fminf(lo[1], l.y); lo[2] = fminf(lo[2], l.z);
            hi[0] = fmaxf(hi[0], h.x); hi[1] = fmaxf(hi[1], h.y); hi[2] = fmaxf(hi[2], h.z);
        }
        if (lo[0] > hi[0]) continue;
        for (int64_t sc = bi.s_beg / kChunk; sc < bi.s_end / kChunk; ++sc) {
            const float4 l = cbox[2 * sc], h = cbox[2 * sc + 1];
            const float gx = fmaxf(0.f, fmaxf(l.x - hi[0], lo[0] - h.x));
            const float gy = fmaxf(0.f, fmaxf(l.y - hi[1], lo[1] - h.y));
            const float gz = fmaxf(0.f, fmaxf(l.z - hi[2], lo[2] - h.z));
            cnt += (gx * gx + gy * gy + gz * gz < rfar2) ? 1 : 0;
        }
    }
    key[it] = cnt;
}

int pair_batch_items(ssd_ctx *ctx, BatchLayout *B, cudaStream_t s) {
    const int ns = B->nsurf;
    for (int pr = 0; pr < 2; ++pr) {   // 0: FP32C, 1: FP64
        const int span = pr == 0 ? kTPB32 * kTPT32 : kTPB64 * kTPT64;
        const int occ = pr == 0 ? ctx->occ32 : ctx->occ64;
        const int64_t want = (int64_t)ctx->num_sms * occ * (pr == 0 ? ctx->waves32 : 2);
        // source chunk (multiple of kTile) common to all surfaces: about `want` items
        int64_t pairs_tiles = 0;
        for (int k = 0; k < ns; ++k) pairs_tiles += (B->n_pad[k] / span) * (B->n_pad[k] / kTile);
        int64_t chunk_tiles = pairs_tiles / want;
        if (chunk_tiles < 1) chunk_tiles = 1;
        std::vector<BItem> items;
        std::vector<BSurf> surfs(ns);
        int64_t pb = 0;
        for (int k = 0; k < ns; ++k) {
            const int64_t nts = B->n_pad[k] / kTile;
            const int64_t ct = chunk_tiles < nts ? chunk_tiles : nts;
            const int64_t nsplit = (nts + ct - 1) / ct;
            surfs[k] = BSurf{B->poff[k], B->n_pad[k], B->n[k], pb, nsplit, 0, 0, 0};
            for (int64_t t = 0; t < B->n_pad[k] / span; ++t)
                for (int64_t sp = 0; sp < nsplit; ++sp) {
                    BItem it;
                    it.tbase = (int32_t)(B->poff[k] + t * span);
                    it.s_beg = (int32_t)(B->poff[k] + sp * ct * kTile);
                    int64_t e = B->poff[k] + (sp + 1) * ct * kTile;
                    if (e > B->poff[k] + B->n_pad[k]) e = B->poff[k] + B->n_pad[k];
                    it.s_end = (int32_t)e;
                    it.surf = k;
                    it.split = (int32_t)sp;
                    it.pad0 = it.pad1 = it.pad2 = 0;
                    items.push_back(it);
                }
            pb += nsplit * B->n_pad[k];
        }
        if (items.size() > 0x7fffffff) return set_error(ctx, SSD_EINVAL, "too many work items");
        const size_t csz = pr == 0 ? sizeof(Consts<float>) : sizeof(Consts<double>);
        size_t off = 0;
        auto carve = [&](size_t bb) { size_t o = off; off += (bb + 255) & ~size_t(255); return o; };
        const size_t o_it = carve(sizeof(BItem) * items.size()), o_sf = carve(sizeof(BSurf) * ns),
                     o_c = carve(csz * ns);
        void *blk = nullptr;
        SSD_TRY(dev_alloc(ctx, off, &blk));
        char *bp = static_cast<char *>(blk);
        B->items[pr] = blk;
        B->surfs[pr] = bp + o_sf;
        B->consts[pr] = bp + o_c;
        B->nitems[pr] = (int64_t)items.size();
        B->ptotal[pr] = pb;
        std::vector<char> cbuf(csz * ns);
        for (int k = 0; k < ns; ++k) {
            if (pr == 0) {
                const Consts<float> c = make_consts<float>(B->delta[k], kRhoFar32);
                memcpy(cbuf.data() + k * csz, &c, csz);
            } else {
                const Consts<double> c = make_consts<double>(B->delta[k], kRhoFar64);
                memcpy(cbuf.data() + k * csz, &c, csz);
            }
        }
        SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(bp + o_it, items.data(), sizeof(BItem) * items.size(),
                                                cudaMemcpyHostToDevice, s), "items copy"));
        SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(bp + o_sf, surfs.data(), sizeof(BSurf) * ns,
                                                cudaMemcpyHostToDevice, s), "surfs copy"));
        SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(bp + o_c, cbuf.data(), csz * ns, cudaMemcpyHostToDevice, s),
                           "consts copy"));
        // the host vectors go out of scope: wait for the copies
        SSD_TRY(cuda_check(ctx, cudaStreamSynchronize(s), "items sync"));
        if (pr == 0 && ctx->lpt && !items.empty()) {
            // FP32C items in decreasing order of near work, so that cheap far
            // items fill the last wave; each item keeps its own partial slot
            const int64_t ni = (int64_t)items.size();
            void *kd = nullptr;
            SSD_TRY(dev_alloc(ctx, sizeof(int32_t) * ni, &kd));
            struct Release { ssd_ctx *c; void *p; ~Release() { dev_free(c, p); } } rel{ctx, kd};
            batch_item_cost_kernel<<<(unsigned)((ni + 255) / 256), 256, 0, s>>>(
                reinterpret_cast<const BItem *>(bp + o_it), ni, reinterpret_cast<const Consts<float> *>(bp + o_c),
                B->L.cbox, static_cast<int32_t *>(kd));
            ctx->launches++;
            SSD_TRY(launch_check(ctx, "batch item cost kernel"));
            std::vector<int32_t> hk(ni);
            SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(hk.data(), kd, sizeof(int32_t) * ni, cudaMemcpyDeviceToHost, s),
                               "key copy"));
            SSD_TRY(cuda_check(ctx, cudaStreamSynchronize(s), "key sync"));
            int32_t kmax = 0;
            for (int64_t i = 0; i < ni; ++i) kmax = hk[i] > kmax ? hk[i] : kmax;
            std::vector<int64_t> start(kmax + 2, 0);
            for (int64_t i = 0; i < ni; ++i) start[kmax - hk[i] + 1]++;
            for (int k = 1; k <= kmax + 1; ++k) start[k] += start[k - 1];
            std::vector<BItem> sorted(ni);
            for (int64_t i = 0; i < ni; ++i) sorted[start[kmax - hk[i]]++] = items[i];
            SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(bp + o_it, sorted.data(), sizeof(BItem) * ni,
                                                    cudaMemcpyHostToDevice, s), "items copy"));
            SSD_TRY(cuda_check(ctx, cudaStreamSynchronize(s), "items sync"));
        }
    }
    return SSD_OK;
}

int pair_apply_batch(ssd_ctx *ctx, const BatchLayout &B, const BatchCall &bc, cudaStream_t s) {
    const PairCall &pc = bc.pc;
    const int op = pc.op;
    const int nc = op_components(op);
    const bool f32 = (pc.prec == SSD_FP32C);
    const int pr = f32 ? 0 : 1;
    const int nrhs = bc.nrhs;
    const int64_t n = B.n_total, n_pad = B.n_pad_total;
    const int nslot = f32 ? 2 : 1;
    const size_t rec = f32 ? sizeof(float4) : sizeof(d4);
    const size_t rsz = f32 ? sizeof(float) : sizeof(double);
    const bool two_rec = (op == OP_SSLDL);
    const int pack_blocks = (int)((n_pad + 255) / 256);
    const int64_t part_stride = (int64_t)nc * nslot * B.ptotal[pr];
    size_t off = 0;
    auto carve = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~size_t(255); return o; };
    const size_t o_d0 = carve(rec * n_pad * nrhs);
    const size_t o_d1 = two_rec ? carve(rec * n_pad * nrhs) : 0;
    const size_t o_part = carve(rsz * part_stride * nrhs);
    const size_t o_wdot = carve(sizeof(double) * pack_blocks * nrhs);
    const size_t o_r1 = carve(sizeof(double) * B.nsurf * nrhs);
    void *ws = nullptr;
    SSD_TRY(dev_alloc(ctx, off, &ws));
    struct Release { ssd_ctx *c; void *p; ~Release() { dev_free(c, p); } } release{ctx, ws};
    char *base = static_cast<char *>(ws);

    double scale = 1.0, s0 = 1.0, s1 = 1.0, self_coef = 0.0;
    const double *self_src = nullptr;
    switch (op) {
        case OP_LSL: scale = -1.0 / (4.0 * kPi); self_coef = scale; self_src = pc.dens0; break;
        case OP_LDL: scale = -1.0 / (4.0 * kPi); break;
        case OP_SSL: scale = 1.0 / (8.0 * kPi * pc.mu); self_coef = scale; self_src = pc.dens0; break;
        case OP_SDL: scale = 6.0 / (8.0 * kPi); break;
        case OP_SSLDL:
            s0 = pc.beta * 6.0 / (8.0 * kPi);
            s1 = pc.alpha / (8.0 * kPi * pc.mu);
            self_coef = s1; self_src = pc.dens1;
            break;
        default:
            scale = -1.0 / (4.0 * kPi);
            s0 = pc.beta; s1 = pc.alpha;
            self_coef = scale * pc.alpha; self_src = pc.dens1;
            break;
    }
    const bool rank1 = pc.rank1_weight_mean || pc.rank1_nrm != nullptr;
    BPackArgs pa{};
    pa.perm = B.L.perm; pa.n_total = n; pa.n_pad = n_pad; pa.op = op;
    pa.d0 = pc.dens0; pa.d1 = pc.dens1;
    pa.nc0 = (op == OP_LSL || op == OP_LDL || op == OP_LSLDL) ? 1 : 3;
    pa.nc1 = (op == OP_LSLDL) ? 1 : 3;
    pa.pos64 = B.L.pos64; pa.wn64 = B.L.wn64; pa.s0 = s0; pa.s1 = s1;
    pa.out0 = base + o_d0; pa.out1 = two_rec ? base + o_d1 : nullptr;
    pa.wdot_part = reinterpret_cast<double *>(base + o_wdot);
    pa.want_wdot = rank1 ? 1 : 0;
    const dim3 pg((unsigned)pack_blocks, (unsigned)nrhs);
    if (f32) bpack_kernel<float4, float><<<pg, 256, 0, s>>>(pa);
    else bpack_kernel<d4, double><<<pg, 256, 0, s>>>(pa);
    ctx->launches++;
    SSD_TRY(launch_check(ctx, "batched pack"));
    if (rank1) {
        bwdot_kernel<<<(B.nsurf * nrhs + 127) / 128, 128, 0, s>>>(
            reinterpret_cast<const double *>(base + o_wdot), pack_blocks,
            reinterpret_cast<const BSurf *>(B.surfs[pr]), B.nsurf, nrhs, B.d_wsum,
            reinterpret_cast<double *>(base + o_r1));
        ctx->launches++;
    }

    cudaEvent_t ev = nullptr;
    SSD_TRY(timed_begin(ctx, s, &ev));
    const dim3 grid((unsigned)B.nitems[pr], (unsigned)nrhs);
    cudaError_t e;
    if (f32) {
        K32Args ka;
        ka.pos = B.L.pos32; ka.wn = B.L.wn32; ka.cbox = B.L.cbox;
        ka.d0 = reinterpret_cast<const float4 *>(base + o_d0);
        ka.d1 = two_rec ? reinterpret_cast<const float4 *>(base + o_d1) : ka.d0;
        ka.n = n_pad; ka.n_pad = n_pad; ka.chunk = 0;
        ka.c = make_consts<float>(1.0, kRhoFar32);
        ka.part = reinterpret_cast<float *>(base + o_part);
        ka.items = reinterpret_cast<const BItem *>(B.items[pr]);
        ka.surfs = reinterpret_cast<const BSurf *>(B.surfs[pr]);
        ka.consts = reinterpret_cast<const Consts<float> *>(B.consts[pr]);
        ka.rec_stride = n_pad; ka.part_stride = part_stride;
        e = launch_pair_op32(op, grid, ka, s);
    } else {
        KArgs<double> ka;
        ka.pos = B.L.pos64; ka.wn = B.L.wn64;
        ka.d0 = reinterpret_cast<const d4 *>(base + o_d0);
        ka.d1 = two_rec ? reinterpret_cast<const d4 *>(base + o_d1) : ka.d0;
        ka.n_pad = n_pad; ka.chunk = 0;
        ka.c = make_consts<double>(1.0, kRhoFar64);
        ka.part = reinterpret_cast<double *>(base + o_part);
        ka.items = reinterpret_cast<const BItem *>(B.items[pr]);
        ka.surfs = reinterpret_cast<const BSurf *>(B.surfs[pr]);
        ka.consts = reinterpret_cast<const Consts<double> *>(B.consts[pr]);
        ka.rec_stride = n_pad; ka.part_stride = part_stride;
        e = launch_pair_op64(op, grid, ka, s);
    }
    ctx->launches++;
    if (e != cudaSuccess) return cuda_check(ctx, e, "batched pair kernel launch");
    double pairs = 0.0;
    for (int k = 0; k < B.nsurf; ++k) pairs += (double)B.n[k] * (double)B.n[k];
    timed_end(ctx, s, ev, kernel_class(op), pc.prec, pairs * nrhs);

    BEpiArgs ea{};
    ea.perm = B.L.perm; ea.elem_surf = B.elem_surf; ea.surfs = reinterpret_cast<const BSurf *>(B.surfs[pr]);
    ea.n_total = n; ea.n_pad = n_pad; ea.nc = nc; ea.nslot = nslot; ea.part_is_float = f32 ? 1 : 0;
    ea.nrhs = nrhs; ea.nsurf = B.nsurf; ea.part = base + o_part; ea.part_stride = part_stride;
    ea.scale = scale; ea.self_coef = self_coef; ea.selfc = B.d_selfc; ea.self_src = self_src;
    ea.pos64 = B.L.pos64; ea.xin = pc.xin; ea.a_id = pc.a_id; ea.a_op = pc.a_op;
    for (int r = 0; r < kMaxRhs; ++r)
        for (int q = 0; q < 3; ++q) ea.add[r][q] = (r < nrhs ? bc.add[r][q] : 0.0) + (q < 3 ? 0.0 : 0.0);
    ea.rank1 = rank1 ? reinterpret_cast<const double *>(base + o_r1) : nullptr;
    ea.rank1_nrm = pc.rank1_nrm;
    ea.out = pc.out;
    const int64_t tot = n_pad * nc * nrhs;
    bepilogue_kernel<<<(unsigned)((tot + 127) / 128), 128, 0, s>>>(ea);
    ctx->launches++;
    return launch_check(ctx, "batched epilogue");
}
}  // namespace ssd

// ===================================================================== no-alloc
// Stokes double layer (FP32C) that allocates no device memory: the unsorted
// point layout, the packed density and the per-split partial sums all live in
// one file-scope device array of fixed size, whose device address is looked
// up once per device.  Each call rewrites every region it later reads, so no
// state carries over between calls.  For callers that cannot call cudaMalloc
// (see ssd_stokes_DL_noalloc in include/ssd.h).
namespace ssd {
namespace {

constexpr int64_t kNoAllocMaxN = 32768;                  // points per call (after padding)
constexpr int kNoAllocMaxSplit = 16;
constexpr size_t kNoAllocBytes = 16u << 20;              // 16 MiB per device

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// unsorted layout of the caller's points inside the scratch array
__global__ void noalloc_layout_kernel(const double *xyz, const double *nrm, const double *w, int64_t n,
                                      int64_t n_pad, Layout L) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pad) return;
    if (i < n) {
        const double x = xyz[i], y = xyz[n + i], z = xyz[2 * n + i], ww = w[i];
        const double wx = ww * nrm[i], wy = ww * nrm[n + i], wz = ww * nrm[2 * n + i];
        L.perm[i] = (int32_t)i;
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

__global__ void noalloc_chunk_box_kernel(Layout L) {
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

// Device address of the scratch array on the context's device, looked up
// at the context's first no-alloc call with that device current and kept in
// the ssd_ctx (host code must not pass the symbol itself to a kernel).  The
// address belongs to the CUDA context current at that call, like the rest of
// the ssd_ctx's device state.
int noalloc_scratch(ssd_ctx *ctx, char **out) {
    int dev = 0;
    SSD_TRY(cuda_check(ctx, cudaGetDevice(&dev), "cudaGetDevice"));
    if (dev != ctx->device)
        return set_error(ctx, SSD_EINVAL, "ssd_stokes_DL_noalloc: the current device is not the context's device");
    if (!ctx->noalloc_scratch) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_check(ctx, e, "cudaGetSymbolAddress(no-alloc scratch)");
        ctx->noalloc_scratch = p;
    }
    *out = static_cast<char *>(ctx->noalloc_scratch);
    return SSD_OK;
}

}  // namespace
}  // namespace ssd

extern "C" int ssd_stokes_DL_noalloc(ssd_ctx *ctx, const ssd_points *pts, double delta, const double *u,
                                     double *out, ssd_stream stream) {
    using namespace ssd;
    if (!ctx) return SSD_EINVAL;
    if (!pts || pts->n <= 0 || !pts->xyz || !pts->nrm || !pts->w)
        return set_error(ctx, SSD_EINVAL, "bad point set");
    if (!(delta > 0.0) || !isfinite(delta)) return set_error(ctx, SSD_EINVAL, "delta must be positive");
    if (!u || !out) return set_error(ctx, SSD_EINVAL, "NULL density or output");
    const int64_t n = pts->n;
    const int64_t n_pad = ((n + kRowAlign - 1) / kRowAlign) * kRowAlign;
    if (n_pad > kNoAllocMaxN)
        return set_error(ctx, SSD_EINVAL, "ssd_stokes_DL_noalloc: more than 32768 points (after padding to 512)");
    cudaStream_t s = (cudaStream_t)stream;
    char *base = nullptr;
    SSD_TRY(noalloc_scratch(ctx, &base));

    // carve the scratch array
    size_t off = 0;
    auto carve = [&](size_t b) { size_t o = off; off += (b + 255) & ~size_t(255); return o; };
    Layout L;
    L.n = n;
    L.n_pad = n_pad;
    L.perm = reinterpret_cast<int32_t *>(base + carve(sizeof(int32_t) * n_pad));
    L.pos32 = reinterpret_cast<float4 *>(base + carve(sizeof(float4) * n_pad));
    L.wn32 = reinterpret_cast<float4 *>(base + carve(sizeof(float4) * n_pad));
    L.pos64 = reinterpret_cast<d4 *>(base + carve(sizeof(d4) * n_pad));
    L.wn64 = reinterpret_cast<d4 *>(base + carve(sizeof(d4) * n_pad));
    L.cbox = reinterpret_cast<float4 *>(base + carve(sizeof(float4) * 2 * (n_pad / kChunk)));
    float4 *d0 = reinterpret_cast<float4 *>(base + carve(sizeof(float4) * n_pad));
    const int64_t ntiles_t = n_pad / (kTPB32 * kTPT32);
    const int64_t ntiles_s = n_pad / kTile;
    int64_t nsplit = ((int64_t)ctx->num_sms * ctx->occ32 * ctx->waves32 + ntiles_t - 1) / ntiles_t;
    if (nsplit < 1) nsplit = 1;
    if (nsplit > kNoAllocMaxSplit) nsplit = kNoAllocMaxSplit;
    if (nsplit > ntiles_s) nsplit = ntiles_s;
    const int64_t chunk_tiles = (ntiles_s + nsplit - 1) / nsplit;
    nsplit = (ntiles_s + chunk_tiles - 1) / chunk_tiles;
    float *part = reinterpret_cast<float *>(base + carve(sizeof(float) * 2 * 3 * nsplit * n_pad));
    if (off > kNoAllocBytes) return set_error(ctx, SSD_EINVAL, "no-alloc scratch too small");

    const unsigned nb = (unsigned)((n_pad + 255) / 256);
    noalloc_layout_kernel<<<nb, 256, 0, s>>>(pts->xyz, pts->nrm, pts->w, n, n_pad, L);
    noalloc_chunk_box_kernel<<<(unsigned)((n_pad / kChunk + 127) / 128), 128, 0, s>>>(L);
    PackArgs pa{};
    pa.perm = L.perm; pa.n = n; pa.n_pad = n_pad; pa.op = OP_SDL;
    pa.d0 = u; pa.d1 = nullptr; pa.pos64 = L.pos64; pa.wn64 = L.wn64; pa.s0 = 1.0; pa.s1 = 1.0;
    pa.out0 = d0; pa.out1 = nullptr; pa.wdot_part = nullptr;
    pack_kernel<float4, float><<<nb, 256, 0, s>>>(pa);
    ctx->launches += 3;
    SSD_TRY(launch_check(ctx, "no-alloc layout"));

    K32Args ka;
    ka.pos = L.pos32; ka.wn = L.wn32; ka.cbox = L.cbox; ka.d0 = d0; ka.d1 = d0;
    ka.n = n; ka.n_pad = n_pad; ka.chunk = chunk_tiles * kTile;
    ka.c = make_consts<float>(delta, kRhoFar32);
    ka.part = part;
    ka.items = nullptr; ka.surfs = nullptr; ka.consts = nullptr; ka.rec_stride = 0; ka.part_stride = 0;
    pair32_kernel<OP_SDL><<<dim3((unsigned)ntiles_t, (unsigned)nsplit), kTPB32, 0, s>>>(ka);
    ctx->launches++;
    SSD_TRY(launch_check(ctx, "no-alloc pair kernel"));

    EpiArgs ea{};
    ea.perm = L.perm; ea.n = n; ea.n_pad = n_pad; ea.nc = 3; ea.nsplit = (int)nsplit; ea.nslot = 2;
    ea.part_is_float = 1; ea.part = part;
    ea.scale = 6.0 / (8.0 * kPi); ea.self_coef = 0.0; ea.self_src = nullptr; ea.pos64 = L.pos64;
    ea.xin = nullptr; ea.a_id = 0.0; ea.a_op = 1.0;
    ea.add0 = ea.add1 = ea.add2 = 0.0; ea.add_dev = nullptr;
    ea.wdot_part = nullptr; ea.nwdot = 0; ea.wdot_scale = 0.0; ea.rank1_nrm = nullptr;
    ea.out = out;
    epilogue_kernel<<<(unsigned)((n_pad * 3 + 127) / 128), 128, 0, s>>>(ea);   // one thread per point and component
    ctx->launches++;
    return launch_check(ctx, "no-alloc epilogue");
}
