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

#include "internal.h"
#include "series_coef.h"

namespace ssd {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kRhoSeries = 0.5;   // series branch below this rho (both precisions)
constexpr double kRhoFar32 = 5.5;    // 1 - s_i(rho) < 2^-25 beyond this (FP32)
constexpr double kRhoFar64 = 8.0;    // 1 - s_i(rho) < 1e-21 beyond this (FP64)

template <int OP> struct OpInfo;
template <> struct OpInfo<OP_LSL>   { enum { NC = 1, WN = 0, D1 = 0, SL = 1, DL = 0 }; };
template <> struct OpInfo<OP_LDL>   { enum { NC = 1, WN = 1, D1 = 0, SL = 0, DL = 1 }; };
template <> struct OpInfo<OP_SSL>   { enum { NC = 3, WN = 0, D1 = 0, SL = 1, DL = 0 }; };
template <> struct OpInfo<OP_SDL>   { enum { NC = 3, WN = 1, D1 = 0, SL = 0, DL = 1 }; };
template <> struct OpInfo<OP_SSLDL> { enum { NC = 3, WN = 1, D1 = 1, SL = 1, DL = 1 }; };
template <> struct OpInfo<OP_LSLDL> { enum { NC = 1, WN = 1, D1 = 0, SL = 1, DL = 1 }; };

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
    static __device__ __forceinline__ double rsq(double x) { return 1.0 / sqrt(x); }
    static __device__ __forceinline__ double erf_(double x) { return erf(x); }
    static __device__ __forceinline__ double exp_(double x) { return exp(x); }
    static __device__ __forceinline__ double ser(int i, double t) {
        double s = kSeries[i][SSD_NSER - 1];
#pragma unroll
        for (int k = SSD_NSER - 2; k >= 0; --k) s = fma(s, t, kSeries[i][k]);
        return s;
    }
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
};

// Smoothed radial factors k1 = s1/r, k2 = s2/r^3, k3 = s3/r^3, k4 = s4/r^5
// (Section 5.3).  `ser` selects the Taylor branch (rho < rho_series); the
// closed forms are evaluated otherwise.
template <typename R, int OP>
__device__ __forceinline__ void smooth(R r2, const Consts<R> &c, bool anyser, R &k1, R &k2, R &k3, R &k4) {
    typedef Prec<R> P;
    const R rinv = P::rsq(r2);
    const R t = r2 * c.inv_d2;
    const R rho = r2 * rinv * c.inv_d;
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
    if (OP == OP_LDL || OP == OP_LSLDL) {
        const R s2 = er + ce * ((R(2) * t - R(3)) * third);
        k2 = s2 * rinv3;
    }
    if (OP == OP_SDL || OP == OP_SSLDL) {
        const R s4 = er - ce * ((t * (t * (R(8) * t - R(36)) + R(6)) + R(9)) * (R(1) / R(9)));
        k4 = s4 * rinv3 * rinv2;
    }
    if (anyser && t < c.tser) {
        if (OpInfo<OP>::SL) {
            k1 = P::ser(0, t) * c.inv_d;
            k3 = P::ser(2, t) * c.inv_d3;
        }
        if (OP == OP_LDL || OP == OP_LSLDL) k2 = P::ser(1, t) * c.inv_d3;
        if (OP == OP_SDL || OP == OP_SSLDL) k4 = P::ser(3, t) * c.inv_d5;
    }
}

// Adds the pair (target with position y and density dt, source record s)
// into acc.  Near = smoothed kernels.  `self` removes the single-layer self
// term (added in FP64 by the epilogue).
template <typename R, int OP, bool NEAR>
__device__ __forceinline__ void pair_term(const R d[3], const R r2, const R dt[3], const typename Prec<R>::V4 &sw,
                                          const typename Prec<R>::V4 &s0, const typename Prec<R>::V4 &s1,
                                          const Consts<R> &c, bool anyser, bool self, R acc[3]) {
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

    const int64_t tbase = (int64_t)blockIdx.x * (TPB * TPT);
    R y[TPT][3], dt[TPT][3];
    Acc<R> acc[TPT][NC];
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int64_t i = tbase + threadIdx.x + t * TPB;   // < n_pad by construction
        const V4 p = a.pos[i];
        y[t][0] = p.x; y[t][1] = p.y; y[t][2] = p.z;
        const V4 d = a.d0[i];
        dt[t][0] = d.x; dt[t][1] = d.y; dt[t][2] = d.z;
    }
    const int64_t s_beg = (int64_t)blockIdx.y * a.chunk;
    int64_t s_end = s_beg + a.chunk;
    if (s_end > a.n_pad) s_end = a.n_pad;
    const Consts<R> c = a.c;

    for (int64_t tile = s_beg; tile < s_end; tile += kTile) {
        __syncthreads();
        for (int k = threadIdx.x; k < kTile; k += TPB) {
            sm_pos[k] = a.pos[tile + k];
            if (OpInfo<OP>::WN) sm_wn[k] = a.wn[tile + k];
            sm_d0[k] = a.d0[tile + k];
            if (OpInfo<OP>::D1) sm_d1[k] = a.d1[tile + k];
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
                    pair_term<R, OP, true>(d[t], r2[t], dt[t], sw, s0, s1, c, anyser, self, part[t]);
                }
            } else {
#pragma unroll
                for (int t = 0; t < TPT; ++t)
                    pair_term<R, OP, false>(d[t], r2[t], dt[t], sw, s0, s1, c, false, false, part[t]);
            }
        }
#pragma unroll
        for (int t = 0; t < TPT; ++t)
#pragma unroll
            for (int q = 0; q < NC; ++q) acc[t][q].add(part[t][q]);
    }
    // partial layout: [split][comp][slot][n_pad], slot = hi (and lo for FP32)
    constexpr int NS = sizeof(Acc<R>) / sizeof(R);
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int64_t i = tbase + threadIdx.x + t * TPB;
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            R *dst = a.part + (((int64_t)blockIdx.y * NC + q) * NS) * a.n_pad + i;
            dst[0] = acc[t][q].hi;
            if (NS == 2) dst[a.n_pad] = reinterpret_cast<const R *>(&acc[t][q])[1];
        }
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
            const double w = a.pos64[i].w;
            switch (a.op) {
                case OP_LSL: r0.x = R(a.s0 * w * a.d0[o]); break;
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
};

__global__ void epilogue_kernel(const EpiArgs a) {
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
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_pad) return;
    const int32_t o = a.perm[i];
    if (o < 0) return;
    for (int q = 0; q < a.nc; ++q) {
        double s = 0.0;
        for (int sp = 0; sp < a.nsplit; ++sp) {
            const int64_t base = (((int64_t)sp * a.nc + q) * a.nslot) * a.n_pad + i;
            if (a.part_is_float) {
                const float *pf = reinterpret_cast<const float *>(a.part);
                s += (double)pf[base];
                if (a.nslot == 2) s += (double)pf[base + a.n_pad];
            } else {
                s += reinterpret_cast<const double *>(a.part)[base];
            }
        }
        double v = a.scale * s;
        if (a.self_src) v += a.self_coef * a.pos64[i].w * a.self_src[(int64_t)q * a.n + o];
        double r = a.a_op * v + extra + (q == 0 ? a.add0 : (q == 1 ? a.add1 : a.add2));
        if (a.rank1_nrm) r += rank1 * a.rank1_nrm[(int64_t)q * a.n + o];
        if (a.xin) r += a.a_id * a.xin[(int64_t)q * a.n + o];
        a.out[(int64_t)q * a.n + o] = r;
    }
}

template <typename R, int OP>
cudaError_t launch_pair(dim3 grid, int tpb, const KArgs<R> &ka, cudaStream_t s) {
    if (sizeof(R) == 4) {
        pair_kernel<R, OP, kTPB32, kTPT32><<<grid, kTPB32, 0, s>>>(ka);
    } else {
        pair_kernel<R, OP, kTPB64, kTPT64><<<grid, kTPB64, 0, s>>>(ka);
    }
    (void)tpb;
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_pair_op(int op, dim3 grid, const KArgs<R> &ka, cudaStream_t s) {
    switch (op) {
        case OP_LSL: return launch_pair<R, OP_LSL>(grid, 0, ka, s);
        case OP_LDL: return launch_pair<R, OP_LDL>(grid, 0, ka, s);
        case OP_SSL: return launch_pair<R, OP_SSL>(grid, 0, ka, s);
        case OP_SDL: return launch_pair<R, OP_SDL>(grid, 0, ka, s);
        case OP_SSLDL: return launch_pair<R, OP_SSLDL>(grid, 0, ka, s);
        default: return launch_pair<R, OP_LSLDL>(grid, 0, ka, s);
    }
}

int kernel_class(int op) {
    switch (op) {
        case OP_LSL: return SSD_K_LAPLACE_SL;
        case OP_LDL: return SSD_K_LAPLACE_DL;
        case OP_SSL: return SSD_K_STOKES_SL;
        case OP_SDL: return SSD_K_STOKES_DL;
        case OP_SSLDL: return SSD_K_STOKES_SLDL;
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

}  // namespace

int pair_occupancy(ssd_ctx *ctx) {
    int o32 = 0, o64 = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &o32, pair_kernel<float, OP_SSLDL, kTPB32, kTPT32>, kTPB32, 0);
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
    const int tspan = f32 ? kTPB32 * kTPT32 : kTPB64 * kTPT64;
    const int64_t ntiles_t = n_pad / tspan;
    const int64_t ntiles_s = n_pad / kTile;
    // splits: enough CTAs for about two waves of resident CTAs
    const int occ = f32 ? ctx->occ32 : ctx->occ64;
    int64_t want = (int64_t)ctx->num_sms * occ * 2;
    int64_t nsplit = (want + ntiles_t - 1) / ntiles_t;
    if (nsplit < 1) nsplit = 1;
    if (nsplit > ntiles_s) nsplit = ntiles_s;
    const int64_t chunk_tiles = (ntiles_s + nsplit - 1) / nsplit;
    nsplit = (ntiles_s + chunk_tiles - 1) / chunk_tiles;
    const int64_t chunk = chunk_tiles * kTile;

    const size_t rec = f32 ? sizeof(float4) : sizeof(d4);
    const int nslot = f32 ? 2 : 1;
    const size_t rsz = f32 ? sizeof(float) : sizeof(double);
    const bool two_rec = (op == OP_SSLDL);
    const int pack_blocks = (int)((n_pad + 255) / 256);
    size_t off = 0;
    auto carve = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~size_t(255); return o; };
    const size_t o_d0 = carve(rec * n_pad);
    const size_t o_d1 = two_rec ? carve(rec * n_pad) : 0;
    const size_t o_part = carve(rsz * nslot * nc * nsplit * n_pad);
    const size_t o_wdot = carve(sizeof(double) * pack_blocks);
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
        default:  // OP_LSLDL
            scale = -1.0 / (4.0 * kPi);
            s0 = pc.beta;                                // p records
            s1 = pc.alpha;                               // w g records
            self_coef = scale * pc.alpha * sig1_0 / pc.delta; self_src = pc.dens1;
            break;
    }

    PackArgs pa;
    pa.perm = L.perm; pa.n = n; pa.n_pad = n_pad; pa.op = op;
    pa.d0 = pc.dens0; pa.d1 = pc.dens1; pa.pos64 = L.pos64; pa.wn64 = L.wn64; pa.s0 = s0; pa.s1 = s1;
    pa.out0 = base + o_d0; pa.out1 = two_rec ? base + o_d1 : nullptr;
    const bool rank1 = pc.rank1_weight_mean || pc.rank1_nrm != nullptr;
    pa.wdot_part = rank1 ? reinterpret_cast<double *>(base + o_wdot) : nullptr;
    if (f32) pack_kernel<float4, float><<<pack_blocks, 256, 0, s>>>(pa);
    else pack_kernel<d4, double><<<pack_blocks, 256, 0, s>>>(pa);
    ctx->launches++;
    SSD_TRY(launch_check(ctx, "pack kernel"));

    const int cls = kernel_class(op);
    cudaEvent_t ev = nullptr;
    SSD_TRY(timed_begin(ctx, s, &ev));
    dim3 grid((unsigned)ntiles_t, (unsigned)nsplit);
    cudaError_t e;
    if (f32) {
        KArgs<float> ka;
        ka.pos = L.pos32; ka.wn = L.wn32;
        ka.d0 = reinterpret_cast<const float4 *>(base + o_d0);
        ka.d1 = two_rec ? reinterpret_cast<const float4 *>(base + o_d1) : ka.d0;
        ka.n_pad = n_pad; ka.chunk = chunk;
        ka.c = make_consts<float>(pc.delta, kRhoFar32);
        ka.part = reinterpret_cast<float *>(base + o_part);
        e = launch_pair_op<float>(op, grid, ka, s);
    } else {
        KArgs<double> ka;
        ka.pos = L.pos64; ka.wn = L.wn64;
        ka.d0 = reinterpret_cast<const d4 *>(base + o_d0);
        ka.d1 = two_rec ? reinterpret_cast<const d4 *>(base + o_d1) : ka.d0;
        ka.n_pad = n_pad; ka.chunk = chunk;
        ka.c = make_consts<double>(pc.delta, kRhoFar64);
        ka.part = reinterpret_cast<double *>(base + o_part);
        e = launch_pair_op<double>(op, grid, ka, s);
    }
    ctx->launches++;
    if (e != cudaSuccess) return cuda_check(ctx, e, "pair kernel launch");
    timed_end(ctx, s, ev, cls, pc.prec, (double)n * (double)n);

    EpiArgs ea;
    ea.perm = L.perm; ea.n = n; ea.n_pad = n_pad; ea.nc = nc; ea.nsplit = (int)nsplit; ea.nslot = nslot;
    ea.part_is_float = f32 ? 1 : 0; ea.part = base + o_part;
    ea.scale = scale; ea.self_coef = self_coef; ea.self_src = self_src; ea.pos64 = L.pos64;
    ea.xin = pc.xin; ea.a_id = pc.a_id; ea.a_op = pc.a_op;
    ea.add0 = pc.add[0]; ea.add1 = pc.add[1]; ea.add2 = pc.add[2]; ea.add_dev = pc.add_dev;
    ea.wdot_part = rank1 ? reinterpret_cast<const double *>(base + o_wdot) : nullptr;
    ea.nwdot = pack_blocks; ea.wdot_scale = rank1 ? 1.0 / L.wsum : 0.0;
    ea.rank1_nrm = pc.rank1_nrm;
    ea.out = pc.out;
    epilogue_kernel<<<(unsigned)((n_pad + 255) / 256), 256, 0, s>>>(ea);
    ctx->launches++;
    return launch_check(ctx, "epilogue kernel");
}

}  // namespace ssd
