// Off-surface evaluation (FP64): the Darcy pressure inside the body from
// Green's representation (eq. Greens), the Stokes velocity outside from the
// Stokes representation (eq. Stokes) and the Stokes pressure outside from the
// pressures that go with its two kernels, given the boundary data of a D-N
// solve.  Bare kernels: the surface quadrature is accurate for field points a
// few grid spacings away from the surface.
//
// One thread per field point; the surface points stream through shared
// memory in 128-point tiles.
#include <math.h>

#include "internal.h"

namespace ssd {
namespace {

constexpr int kFieldTPB = 128;
constexpr double kPiF = 3.14159265358979323846;

struct FieldArgs {
    int64_t n, nt;
    const double *xyz, *nrm, *w;   // surface [3][n], [3][n], [n]
    const double *a, *b;           // Darcy: q [n], p [n]; Stokes: f [3][n], u [3][n]
    const double *y;               // field points [3][nt]
    double ca, cb;                 // coefficients of the single and double layer sums
    double u0, u1, u2;             // far field (Stokes)
    double *out;                   // Darcy [nt]; Stokes [3][nt]
};

// p(y) = ca sum_j w_j q_j / r + cb sum_j w_j p_j (yh . n_j) / r^3,  yh = y - x_j,
// ca = (mu/kappa)(-1/(4 pi)) (from -dp/dn G with dp/dn = -(mu/kappa) q), cb = -1/(4 pi)
__global__ void __launch_bounds__(kFieldTPB) darcy_field_kernel(const FieldArgs A) {
    __shared__ double sx[3][kFieldTPB], sn[3][kFieldTPB], sw[kFieldTPB], sa[kFieldTPB], sb[kFieldTPB];
    const int64_t t = (int64_t)blockIdx.x * kFieldTPB + threadIdx.x;
    const bool act = t < A.nt;
    double y[3] = {0.0, 0.0, 0.0};
    if (act)
        for (int e = 0; e < 3; ++e) y[e] = A.y[e * A.nt + t];
    double s1 = 0.0, s2 = 0.0;
    for (int64_t base = 0; base < A.n; base += kFieldTPB) {
        const int64_t m = base + threadIdx.x;
        __syncthreads();
        if (m < A.n) {
            for (int e = 0; e < 3; ++e) { sx[e][threadIdx.x] = A.xyz[e * A.n + m]; sn[e][threadIdx.x] = A.nrm[e * A.n + m]; }
            sw[threadIdx.x] = A.w[m];
            sa[threadIdx.x] = A.a[m];
            sb[threadIdx.x] = A.b[m];
        }
        __syncthreads();
        const int cnt = (int)((A.n - base) < kFieldTPB ? (A.n - base) : kFieldTPB);
        for (int j = 0; j < cnt; ++j) {
            const double d0 = y[0] - sx[0][j], d1 = y[1] - sx[1][j], d2 = y[2] - sx[2][j];
            const double ri = 1.0 / sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            const double dn = d0 * sn[0][j] + d1 * sn[1][j] + d2 * sn[2][j];
            s1 += sw[j] * sa[j] * ri;
            s2 += sw[j] * sb[j] * dn * ri * ri * ri;
        }
    }
    if (act) A.out[t] = A.ca * s1 + A.cb * s2;
}

// u(y) = U + ca sum_j w_j [f_j / r + yh (yh . f_j) / r^3]
//          + cb sum_j w_j (u_j . yh)(yh . n_j) yh / r^5,
// ca = -1/(8 pi mu), cb = 6/(8 pi) (the stresslet -6 yh yh yh / r^5 against n_S = -n)
__global__ void __launch_bounds__(kFieldTPB) stokes_field_kernel(const FieldArgs A) {
    __shared__ double sx[3][kFieldTPB], sn[3][kFieldTPB], sw[kFieldTPB], sf[3][kFieldTPB], su[3][kFieldTPB];
    const int64_t t = (int64_t)blockIdx.x * kFieldTPB + threadIdx.x;
    const bool act = t < A.nt;
    double y[3] = {0.0, 0.0, 0.0};
    if (act)
        for (int e = 0; e < 3; ++e) y[e] = A.y[e * A.nt + t];
    double s1[3] = {0.0, 0.0, 0.0}, s2[3] = {0.0, 0.0, 0.0};
    for (int64_t base = 0; base < A.n; base += kFieldTPB) {
        const int64_t m = base + threadIdx.x;
        __syncthreads();
        if (m < A.n) {
            for (int e = 0; e < 3; ++e) {
                sx[e][threadIdx.x] = A.xyz[e * A.n + m];
                sn[e][threadIdx.x] = A.nrm[e * A.n + m];
                sf[e][threadIdx.x] = A.a[e * A.n + m];
                su[e][threadIdx.x] = A.b[e * A.n + m];
            }
            sw[threadIdx.x] = A.w[m];
        }
        __syncthreads();
        const int cnt = (int)((A.n - base) < kFieldTPB ? (A.n - base) : kFieldTPB);
        for (int j = 0; j < cnt; ++j) {
            const double d[3] = {y[0] - sx[0][j], y[1] - sx[1][j], y[2] - sx[2][j]};
            const double ri = 1.0 / sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            const double ri2 = ri * ri, ri3 = ri2 * ri;
            const double df = d[0] * sf[0][j] + d[1] * sf[1][j] + d[2] * sf[2][j];
            const double du = d[0] * su[0][j] + d[1] * su[1][j] + d[2] * su[2][j];
            const double dn = d[0] * sn[0][j] + d[1] * sn[1][j] + d[2] * sn[2][j];
            const double wj = sw[j];
            const double bs = wj * df * ri3;
            const double bd = wj * du * dn * ri3 * ri2;
            for (int e = 0; e < 3; ++e) {
                s1[e] += wj * sf[e][j] * ri + d[e] * bs;
                s2[e] += d[e] * bd;
            }
        }
    }
    if (!act) return;
    const double u0[3] = {A.u0, A.u1, A.u2};
    for (int e = 0; e < 3; ++e) A.out[e * A.nt + t] = u0[e] + A.ca * s1[e] + A.cb * s2[e];
}

// p(y) = ca sum_j w_j (yh . f_j) / r^3
//        + cb sum_j w_j [(u_j . n_j) / r^3 - 3 (yh . u_j)(yh . n_j) / r^5],
// from -1/(8 pi) (Stokeslet pressure 2 yh / r^3) . f and -mu/(8 pi) u . (stresslet
// pressure 4(-I/r^3 + 3 yh yh / r^5)) . n_S with n_S = -n: ca = -2/(8 pi),
// cb = -4 mu/(8 pi); far-field pressure 0
__global__ void __launch_bounds__(kFieldTPB) stokes_pressure_kernel(const FieldArgs A) {
    __shared__ double sx[3][kFieldTPB], sn[3][kFieldTPB], sw[kFieldTPB], sf[3][kFieldTPB], su[3][kFieldTPB];
    const int64_t t = (int64_t)blockIdx.x * kFieldTPB + threadIdx.x;
    const bool act = t < A.nt;
    double y[3] = {0.0, 0.0, 0.0};
    if (act)
        for (int e = 0; e < 3; ++e) y[e] = A.y[e * A.nt + t];
    double s1 = 0.0, s2 = 0.0;
    for (int64_t base = 0; base < A.n; base += kFieldTPB) {
        const int64_t m = base + threadIdx.x;
        __syncthreads();
        if (m < A.n) {
            for (int e = 0; e < 3; ++e) {
                sx[e][threadIdx.x] = A.xyz[e * A.n + m];
                sn[e][threadIdx.x] = A.nrm[e * A.n + m];
                sf[e][threadIdx.x] = A.a[e * A.n + m];
                su[e][threadIdx.x] = A.b[e * A.n + m];
            }
            sw[threadIdx.x] = A.w[m];
        }
        __syncthreads();
        const int cnt = (int)((A.n - base) < kFieldTPB ? (A.n - base) : kFieldTPB);
        for (int j = 0; j < cnt; ++j) {
            const double d[3] = {y[0] - sx[0][j], y[1] - sx[1][j], y[2] - sx[2][j]};
            const double ri = 1.0 / sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            const double ri2 = ri * ri, ri3 = ri2 * ri;
            const double df = d[0] * sf[0][j] + d[1] * sf[1][j] + d[2] * sf[2][j];
            const double du = d[0] * su[0][j] + d[1] * su[1][j] + d[2] * su[2][j];
            const double dn = d[0] * sn[0][j] + d[1] * sn[1][j] + d[2] * sn[2][j];
            const double un = su[0][j] * sn[0][j] + su[1][j] * sn[1][j] + su[2][j] * sn[2][j];
            const double wj = sw[j];
            s1 += wj * df * ri3;
            s2 += wj * ri3 * (un - 3.0 * du * dn * ri2);   // n_S = -n flips both terms
        }
    }
    if (act) A.out[t] = A.ca * s1 + A.cb * s2;
}

int field_common(ssd_ctx *ctx, const ssd_points *pts, int64_t nt, const double *targets, double *out) {
    SSD_TRY(check_points(ctx, pts));
    if (nt < 0) return set_error(ctx, SSD_EINVAL, "negative field-point count");
    if (nt > 0 && (!targets || !out)) return set_error(ctx, SSD_EINVAL, "NULL field points or output");
    return SSD_OK;
}

}  // namespace
}  // namespace ssd

using namespace ssd;

extern "C" {

int ssd_darcy_pressure_field(ssd_ctx *ctx, const ssd_points *pts, double mu, double kappa, const double *q,
                             const double *p, int64_t nt, const double *targets, double *out, ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    ctx->err.clear();
    SSD_TRY(field_common(ctx, pts, nt, targets, out));
    if (!(mu > 0.0) || !(kappa > 0.0) || !isfinite(mu) || !isfinite(kappa))
        return set_error(ctx, SSD_EINVAL, "mu and kappa must be positive");
    if (!q || !p) return set_error(ctx, SSD_EINVAL, "NULL boundary data");
    if (nt == 0) return SSD_OK;
    FieldArgs A;
    A.n = pts->n; A.nt = nt; A.xyz = pts->xyz; A.nrm = pts->nrm; A.w = pts->w;
    A.a = q; A.b = p; A.y = targets; A.out = out;
    A.ca = -(mu / kappa) / (4.0 * kPiF);
    A.cb = -1.0 / (4.0 * kPiF);
    A.u0 = A.u1 = A.u2 = 0.0;
    darcy_field_kernel<<<(unsigned)((nt + kFieldTPB - 1) / kFieldTPB), kFieldTPB, 0, (cudaStream_t)stream>>>(A);
    ctx->launches++;
    return launch_check(ctx, "darcy field kernel");
}

int ssd_stokes_velocity_field(ssd_ctx *ctx, const ssd_points *pts, double mu, const double uinf[3], const double *f,
                              const double *u, int64_t nt, const double *targets, double *out, ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    ctx->err.clear();
    SSD_TRY(field_common(ctx, pts, nt, targets, out));
    if (!(mu > 0.0) || !isfinite(mu)) return set_error(ctx, SSD_EINVAL, "mu must be positive");
    if (!f || !u || !uinf) return set_error(ctx, SSD_EINVAL, "NULL boundary data or far field");
    if (nt == 0) return SSD_OK;
    FieldArgs A;
    A.n = pts->n; A.nt = nt; A.xyz = pts->xyz; A.nrm = pts->nrm; A.w = pts->w;
    A.a = f; A.b = u; A.y = targets; A.out = out;
    A.ca = -1.0 / (8.0 * kPiF * mu);
    A.cb = 6.0 / (8.0 * kPiF);
    A.u0 = uinf[0]; A.u1 = uinf[1]; A.u2 = uinf[2];
    stokes_field_kernel<<<(unsigned)((nt + kFieldTPB - 1) / kFieldTPB), kFieldTPB, 0, (cudaStream_t)stream>>>(A);
    ctx->launches++;
    return launch_check(ctx, "stokes field kernel");
}

int ssd_stokes_pressure_field(ssd_ctx *ctx, const ssd_points *pts, double mu, const double *f, const double *u,
                              int64_t nt, const double *targets, double *out, ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    ctx->err.clear();
    SSD_TRY(field_common(ctx, pts, nt, targets, out));
    if (!(mu > 0.0) || !isfinite(mu)) return set_error(ctx, SSD_EINVAL, "mu must be positive");
    if (!f || !u) return set_error(ctx, SSD_EINVAL, "NULL boundary data");
    if (nt == 0) return SSD_OK;
    FieldArgs A;
    A.n = pts->n; A.nt = nt; A.xyz = pts->xyz; A.nrm = pts->nrm; A.w = pts->w;
    A.a = f; A.b = u; A.y = targets; A.out = out;
    A.ca = -2.0 / (8.0 * kPiF);
    A.cb = -4.0 * mu / (8.0 * kPiF);
    A.u0 = A.u1 = A.u2 = 0.0;
    stokes_pressure_kernel<<<(unsigned)((nt + kFieldTPB - 1) / kFieldTPB), kFieldTPB, 0, (cudaStream_t)stream>>>(A);
    ctx->launches++;
    return launch_check(ctx, "stokes pressure kernel");
}

}  // extern "C"
