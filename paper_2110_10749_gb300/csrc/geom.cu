// Geometric derivatives of the layer operators (FP64).
//
// For a bilinear form B(a, b) = sum_i a_i . (K b)_i, with K one of the four
// pair sums of Sections 5.1-5.3 (Laplace single / double layer, Stokes single
// / double layer, including the subtraction of the double layers and the
// single-layer self terms), the kernels below add to each point k the
// derivatives dB/dx_k [3], dB/dn_k [3] and dB/dw_k.  A pair (i, j) depends on
// x_i - x_j, on the source normal n_j and weight w_j, so point k collects the
// terms where it is the target and those where it is the source; every term
// is a function of the partner's data and of d = x_k - x_m, so one target
// loop over all partners m computes them without scatter or atomics.
//
// Radial kernels k_1 = s1/r, k_2 = s2/r^3, k_3 = s3/r^3, k_4 = s4/r^5 and
// q_i = (1/r) dk_i/dr.  With t = rho^2, rho = r/delta, E = exp(-t):
//   s1' = 2/(3 sqrt(pi)) E (4 t^2 - 16 t + 8),   s2' = 8/(3 sqrt(pi)) t (3 - t) E,
//   s3' = 16/(3 sqrt(pi)) t (t^2 - 6 t + 6) E,   s4' = 32/(9 sqrt(pi)) t^2 (t^2 - 8 t + 12) E,
// (derivatives of the closed forms of Section 5.3 in rho), so
//   q_1 = (s1'/delta - s1/r)/r^2,   q_2 = (s2'/delta - 3 s2/r)/r^4,
//   q_3 = (s3'/delta - 3 s3/r)/r^4, q_4 = (s4'/delta - 5 s4/r)/r^6.
// Below rho = 0.5 the Taylor series of sigma_i(t) = s_i/rho^p gives
// k_i = sigma_i(t)/delta^p and q_i = 2 sigma_i'(t)/delta^(p+2).
#include <math.h>

#include "internal.h"
#include "series_coef.h"

namespace ssd {
namespace {

constexpr int kGeoTPB = 128;
constexpr double kPiG = 3.14159265358979323846;

struct GeoArgs {
    int64_t n;
    int op;
    const double *xyz, *nrm, *w;   // [3][n], [3][n], [n]
    const double *a, *b;           // target-side and source-side densities ([c][n])
    double delta, scale, selfc;    // pair-sum scale, single-layer self coefficient
    double *gx, *gn, *gw;          // accumulated outputs [3][n], [3][n], [n]
};

__device__ __forceinline__ double ser_val(int i, double t) {
    double s = kSeries[i][SSD_NSER - 1];
    for (int k = SSD_NSER - 2; k >= 0; --k) s = fma(s, t, kSeries[i][k]);
    return s;
}
__device__ __forceinline__ double ser_der(int i, double t) {
    double s = (SSD_NSER - 1) * kSeries[i][SSD_NSER - 1];
    for (int k = SSD_NSER - 2; k >= 1; --k) s = fma(s, t, k * kSeries[i][k]);
    return s;
}

// k_i and q_i of the pair at squared distance r2
__device__ void radial(double r2, double delta, double k[4], double q[4]) {
    const double id = 1.0 / delta;
    const double t = r2 * id * id;
    if (t < 0.25) {
        const double id2 = id * id, id3 = id2 * id, id5 = id3 * id2;
        k[0] = ser_val(0, t) * id;
        k[1] = ser_val(1, t) * id3;
        k[2] = ser_val(2, t) * id3;
        k[3] = ser_val(3, t) * id5;
        q[0] = 2.0 * ser_der(0, t) * id3;
        q[1] = 2.0 * ser_der(1, t) * id5;
        q[2] = 2.0 * ser_der(2, t) * id5;
        q[3] = 2.0 * ser_der(3, t) * id5 * id2;
        return;
    }
    const double r = sqrt(r2);
    const double ir = 1.0 / r, ir2 = ir * ir;
    double s[4], sp[4];
    if (t < 64.0) {
        const double rho = r * id;
        const double E = exp(-t);
        const double er = erf(rho);
        const double c = 2.0 / sqrt(kPiG);
        const double ce = c * rho * E;
        s[0] = er - ce * (2.0 * t - 5.0) / 3.0;
        s[1] = er + ce * (2.0 * t - 3.0) / 3.0;
        s[2] = er - ce * (t * (4.0 * t - 14.0) + 3.0) / 3.0;
        s[3] = er - ce * (t * (t * (8.0 * t - 36.0) + 6.0) + 9.0) / 9.0;
        sp[0] = c / 3.0 * E * (t * (4.0 * t - 16.0) + 8.0);
        sp[1] = 4.0 * c / 3.0 * t * (3.0 - t) * E;
        sp[2] = 8.0 * c / 3.0 * t * (t * (t - 6.0) + 6.0) * E;
        sp[3] = 16.0 * c / 9.0 * t * t * (t * (t - 8.0) + 12.0) * E;
    } else {
        for (int i = 0; i < 4; ++i) { s[i] = 1.0; sp[i] = 0.0; }
    }
    const double ir3 = ir2 * ir, ir4 = ir2 * ir2, ir5 = ir4 * ir, ir6 = ir4 * ir2;
    k[0] = s[0] * ir;
    k[1] = s[1] * ir3;
    k[2] = s[2] * ir3;
    k[3] = s[3] * ir5;
    q[0] = (sp[0] * id - s[0] * ir) * ir2;
    q[1] = (sp[1] * id - 3.0 * s[1] * ir) * ir4;
    q[2] = (sp[2] * id - 3.0 * s[2] * ir) * ir4;
    q[3] = (sp[3] * id - 5.0 * s[3] * ir) * ir6;
}

__device__ __forceinline__ double dot3(const double *u, const double *v) { return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]; }

// Adds the terms of partner m to the sums of point k.  Source data of the
// partner: pm (position), nm, wm, am, bm; of k: nk, wk, ak, bk; d = x_k - x_m.
template <int OP>
__device__ __forceinline__ void geo_pair(const double d[3], double r2, double delta, const double *nk, double wk,
                                         const double *ak, const double *bk, const double *nm, double wm,
                                         const double *am, const double *bm, double gx[3], double gn[3],
                                         double &gw) {
    double k[4], q[4];
    radial(r2, delta, k, q);
    if (OP == OP_LSL) {
        // sum_{i != j} a_i w_j k1 b_j
        const double c = ak[0] * wm * bm[0] + am[0] * wk * bk[0];
        for (int e = 0; e < 3; ++e) gx[e] += q[0] * d[e] * c;
        gw += bk[0] * am[0] * k[0];
    } else if (OP == OP_LDL) {
        // sum_{i,j} a_i (b_j - b_i) w_j k2 (d_ij . n_j)
        const double dn_m = dot3(d, nm), dn_k = dot3(d, nk);
        const double c1 = ak[0] * (bm[0] - bk[0]) * wm;     // k as target
        const double c2 = am[0] * (bk[0] - bm[0]) * wk;     // k as source (d_mk = -d)
        for (int e = 0; e < 3; ++e)
            gx[e] += c1 * (q[1] * d[e] * dn_m + k[1] * nm[e]) - c2 * (q[1] * d[e] * dn_k + k[1] * nk[e]);
        for (int e = 0; e < 3; ++e) gn[e] -= c2 * k[1] * d[e];
        gw -= am[0] * (bk[0] - bm[0]) * k[1] * dn_k;
    } else if (OP == OP_SSL) {
        // sum_{i != j} w_j [k1 (a_i . b_j) + k3 (a_i . d)(d . b_j)]
        const double akbm = dot3(ak, bm), ambk = dot3(am, bk);
        const double akd = dot3(ak, d), dbm = dot3(d, bm), amd = dot3(am, d), dbk = dot3(d, bk);
        for (int e = 0; e < 3; ++e) {
            const double g1 = q[0] * d[e] * akbm + q[2] * d[e] * akd * dbm + k[2] * (ak[e] * dbm + bm[e] * akd);
            const double g2 = q[0] * d[e] * ambk + q[2] * d[e] * amd * dbk + k[2] * (am[e] * dbk + bk[e] * amd);
            gx[e] += wm * g1 + wk * g2;
        }
        gw += k[0] * ambk + k[2] * amd * dbk;
    } else {  // OP_SDL
        // sum_{i,j} w_j k4 (a_i . d)(d . (b_j - b_i))(d . n_j)
        double v1[3], v2[3];
        for (int e = 0; e < 3; ++e) { v1[e] = bm[e] - bk[e]; v2[e] = bk[e] - bm[e]; }
        const double akd = dot3(ak, d), dv1 = dot3(d, v1), dnm = dot3(d, nm);
        const double amd = dot3(am, d), dv2 = dot3(d, v2), dnk = dot3(d, nk);
        for (int e = 0; e < 3; ++e) {
            const double g1 = q[3] * d[e] * akd * dv1 * dnm + k[3] * (ak[e] * dv1 * dnm + v1[e] * akd * dnm +
                                                                     nm[e] * akd * dv1);
            const double g2 = q[3] * d[e] * amd * dv2 * dnk + k[3] * (am[e] * dv2 * dnk + v2[e] * amd * dnk +
                                                                     nk[e] * amd * dv2);
            gx[e] += wm * g1 - wk * g2;
            gn[e] -= wk * k[3] * amd * dv2 * d[e];
        }
        gw -= k[3] * amd * dv2 * dnk;
    }
}

template <int OP>
__global__ void __launch_bounds__(kGeoTPB) geo_kernel(const GeoArgs A) {
    constexpr int NC = (OP == OP_LSL || OP == OP_LDL) ? 1 : 3;
    __shared__ double sx[3][kGeoTPB], sn[3][kGeoTPB], sw[kGeoTPB], sa[NC][kGeoTPB], sb[NC][kGeoTPB];
    const int64_t n = A.n;
    const int64_t k = (int64_t)blockIdx.x * kGeoTPB + threadIdx.x;
    const bool act = k < n;
    double xk[3] = {0, 0, 0}, nk[3] = {0, 0, 0}, ak[3] = {0, 0, 0}, bk[3] = {0, 0, 0}, wk = 0.0;
    if (act) {
        for (int e = 0; e < 3; ++e) { xk[e] = A.xyz[e * n + k]; nk[e] = A.nrm[e * n + k]; }
        wk = A.w[k];
        for (int e = 0; e < NC; ++e) { ak[e] = A.a[e * n + k]; bk[e] = A.b[e * n + k]; }
    }
    double gx[3] = {0, 0, 0}, gn[3] = {0, 0, 0}, gw = 0.0;
    for (int64_t base = 0; base < n; base += kGeoTPB) {
        const int64_t m = base + threadIdx.x;
        __syncthreads();
        if (m < n) {
            for (int e = 0; e < 3; ++e) { sx[e][threadIdx.x] = A.xyz[e * n + m]; sn[e][threadIdx.x] = A.nrm[e * n + m]; }
            sw[threadIdx.x] = A.w[m];
            for (int e = 0; e < NC; ++e) { sa[e][threadIdx.x] = A.a[e * n + m]; sb[e][threadIdx.x] = A.b[e * n + m]; }
        }
        __syncthreads();
        const int cnt = (int)((n - base) < kGeoTPB ? (n - base) : kGeoTPB);
        if (!act) continue;
        for (int j = 0; j < cnt; ++j) {
            if (base + j == k) continue;
            const double d[3] = {xk[0] - sx[0][j], xk[1] - sx[1][j], xk[2] - sx[2][j]};
            const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            const double nm[3] = {sn[0][j], sn[1][j], sn[2][j]};
            double am[3] = {0, 0, 0}, bm[3] = {0, 0, 0};
            for (int e = 0; e < NC; ++e) { am[e] = sa[e][j]; bm[e] = sb[e][j]; }
            geo_pair<OP>(d, r2, A.delta, nk, wk, ak, bk, nm, sw[j], am, bm, gx, gn, gw);
        }
    }
    if (!act) return;
    // single-layer self term selfc * w_k (a_k . b_k)
    double self = 0.0;
    if (OP == OP_LSL || OP == OP_SSL)
        for (int e = 0; e < NC; ++e) self += ak[e] * bk[e];
    for (int e = 0; e < 3; ++e) {
        A.gx[e * n + k] += A.scale * gx[e];
        A.gn[e * n + k] += A.scale * gn[e];
    }
    A.gw[k] += A.scale * gw + A.selfc * self;
}

}  // namespace

int geometry_gradient(ssd_ctx *ctx, const ssd_points *pts, int op, double delta, double mu, double alpha,
                      const double *a, const double *b, double *gx, double *gn, double *gw, cudaStream_t s) {
    GeoArgs A;
    A.n = pts->n;
    A.op = op;
    A.xyz = pts->xyz; A.nrm = pts->nrm; A.w = pts->w;
    A.a = a; A.b = b;
    A.delta = delta;
    A.gx = gx; A.gn = gn; A.gw = gw;
    const double sig1_0 = 16.0 / (3.0 * sqrt(kPiG));   // lim s1(rho)/rho at rho = 0
    switch (op) {
        case OP_LSL: A.scale = -1.0 / (4.0 * kPiG); A.selfc = A.scale * sig1_0 / delta; break;
        case OP_LDL: A.scale = -1.0 / (4.0 * kPiG); A.selfc = 0.0; break;
        case OP_SSL: A.scale = 1.0 / (8.0 * kPiG * mu); A.selfc = A.scale * sig1_0 / delta; break;
        case OP_SDL: A.scale = 6.0 / (8.0 * kPiG); A.selfc = 0.0; break;
        default: return set_error(ctx, SSD_EINVAL, "geometry gradient: unknown operator");
    }
    A.scale *= alpha;
    A.selfc *= alpha;
    const unsigned grid = (unsigned)((A.n + kGeoTPB - 1) / kGeoTPB);
    switch (op) {
        case OP_LSL: geo_kernel<OP_LSL><<<grid, kGeoTPB, 0, s>>>(A); break;
        case OP_LDL: geo_kernel<OP_LDL><<<grid, kGeoTPB, 0, s>>>(A); break;
        case OP_SSL: geo_kernel<OP_SSL><<<grid, kGeoTPB, 0, s>>>(A); break;
        default: geo_kernel<OP_SDL><<<grid, kGeoTPB, 0, s>>>(A); break;
    }
    ctx->launches++;
    return launch_check(ctx, "geometry gradient kernel");
}

}  // namespace ssd
