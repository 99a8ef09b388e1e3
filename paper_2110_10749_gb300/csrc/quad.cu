// Quadrature points of Section 5.4 (eq. Quadrature) on spheres, ellipsoids,
// the four-atom molecule (eq. Molecule) and star-shaped surfaces
// r(xi) = 1 + sum_{l<=4} c_lm Y_lm(xi).
//
// One thread per grid line.  A first pass counts the kept intersections per
// line, an exclusive scan turns counts into output offsets, and a second pass
// writes points, normals, weights and (axis, j1, j2, root ordinal).  Points
// and normals use correctly rounded +, -, *, /, sqrt only, in the order
// stated next to each line (this file is compiled without FMA contraction),
// so that they are reproducible bit for bit by any implementation of the
// same definition.
#include <math.h>

#include "internal.h"

namespace ssd {
namespace {

constexpr int kStarCoef = 25;
constexpr int kMaxRoots = 8;        // crossings of one grid line (star surfaces)

struct QuadGeo {
    int kind;
    double A[3], c[3];
    double h, ct, theta;
    int64_t j0[3][2];     // first index of the two in-plane coordinates per axis
    int64_t nj[3][2];     // counts
    int64_t line0[4];     // first line id of each axis
    // star surfaces
    double a[kStarCoef];  // c_k K_k
    double K[kStarCoef];  // normalisation constants of the real Y_lm
    double rb;            // bound of r: 1 + sum |c_k| B_l
    double tlo[3], dt[3]; // sample grid along the lines of each axis
    int nk;               // sample intervals per line
    // molecule (eq. Molecule): atom centres, Gaussian width r, level c, reach D
    double mol[4][3];
    double mr, mc, mD;
    int nka[3];           // sample intervals per line of each axis
    int *overflow;        // set when a line has more than kMaxRoots crossings
};

__device__ __forceinline__ void line_coords(const QuadGeo &g, int64_t line, int &ax, int64_t &ja, int64_t &jb) {
    ax = line >= g.line0[2] ? 2 : (line >= g.line0[1] ? 1 : 0);
    const int64_t l = line - g.line0[ax];
    ja = g.j0[ax][0] + l / g.nj[ax][1];
    jb = g.j0[ax][1] + l % g.nj[ax][1];
}

__device__ __forceinline__ double bump(double r) {
    if (!(fabs(r) < 1.0)) return 0.0;
    const double r2 = r * r;
    return exp(r2 / (r2 - 1.0));
}

// Evaluates the line; returns the number of kept roots and fills them.
__device__ int eval_line(const QuadGeo &g, int ax, int64_t ja, int64_t jb, double P[kMaxRoots][3],
                         double N[kMaxRoots][3], int br[kMaxRoots]) {
    const int a = ax == 0 ? 1 : 0;
    const int b = ax == 2 ? 1 : 2;
    const double xa = __dmul_rn((double)ja, g.h);
    const double xb = __dmul_rn((double)jb, g.h);
    const double u = __ddiv_rn(__dsub_rn(xa, g.c[a]), g.A[a]);
    const double v = __ddiv_rn(__dsub_rn(xb, g.c[b]), g.A[b]);
    const double s = __dsub_rn(__dsub_rn(1.0, __dmul_rn(u, u)), __dmul_rn(v, v));   // (1 - u^2) - v^2
    if (!(s > 0.0)) return 0;
    const double rt = __dsqrt_rn(s);
    const double Art = __dmul_rn(g.A[ax], rt);
    int kept = 0;
    for (int k = 0; k < 2; ++k) {
        double x[3];
        x[ax] = k == 0 ? __dsub_rn(g.c[ax], Art) : __dadd_rn(g.c[ax], Art);
        x[a] = xa;
        x[b] = xb;
        double gr[3];
        for (int q = 0; q < 3; ++q)   // (x_q - c_q) / (A_q A_q)
            gr[q] = __ddiv_rn(__dsub_rn(x[q], g.c[q]), __dmul_rn(g.A[q], g.A[q]));
        const double gn = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(gr[0], gr[0]), __dmul_rn(gr[1], gr[1])),
                                               __dmul_rn(gr[2], gr[2])));
        double nv[3];
        for (int q = 0; q < 3; ++q) nv[q] = __ddiv_rn(gr[q], gn);
        if (fabs(nv[ax]) >= g.ct) {
            for (int q = 0; q < 3; ++q) { P[kept][q] = x[q]; N[kept][q] = nv[q]; }
            br[kept] = k;
            ++kept;
        }
    }
    return kept;
}

// ------------------------------------------------------------ star surfaces
// Real orthonormal Y_lm (l <= 4) as Cartesian polynomials p_k in the unit
// direction xi, Y_k = K_k p_k, k = l^2 + l + m.  P(xi) = sum_k a_k p_k with
// a_k = c_k K_k, summed over k ascending; the gradient components are the
// sums of a_k times the R^3 partial derivatives of p_k, over the k whose
// partial does not vanish identically, k ascending.  T is double, or Dual
// for forward-mode derivatives.
struct Dual {
    double v, d;
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) { return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; }
__device__ __forceinline__ Dual operator*(double a, Dual b) { return {a * b.v, a * b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, double b) { return {a.v - b, a.d}; }
__device__ __forceinline__ Dual operator+(Dual a, double b) { return {a.v + b, a.d}; }
__device__ __forceinline__ Dual dsqrt(Dual a) {
    const double r = sqrt(a.v);
    return {r, a.d / (2.0 * r)};
}
__device__ __forceinline__ double dsqrt(double a) { return sqrt(a); }

template <typename T, bool GRAD = true>
__device__ void star_eval(const T *a, T x, T y, T z, T &P, T g[3]) {
    const T x2 = x * x, y2 = y * y, z2 = z * z;
    const T xy = x * y, yz = y * z, xz = x * z;
    const T u = x2 - y2;
    const T v3x = 3.0 * x2 - y2;
    const T w3y = x2 - 3.0 * y2;
    const T z5 = 5.0 * z2 - 1.0;
    const T z53 = 5.0 * z2 - 3.0;
    const T z7 = 7.0 * z2 - 1.0;
    const T z73 = 7.0 * z2 - 3.0;
    T s = a[0];
    s = s + a[1] * y;
    s = s + a[2] * z;
    s = s + a[3] * x;
    s = s + a[4] * xy;
    s = s + a[5] * yz;
    s = s + a[6] * (3.0 * z2 - 1.0);
    s = s + a[7] * xz;
    s = s + a[8] * u;
    s = s + a[9] * (y * v3x);
    s = s + a[10] * (xy * z);
    s = s + a[11] * (y * z5);
    s = s + a[12] * (z * z53);
    s = s + a[13] * (x * z5);
    s = s + a[14] * (z * u);
    s = s + a[15] * (x * w3y);
    s = s + a[16] * (xy * u);
    s = s + a[17] * (yz * v3x);
    s = s + a[18] * (xy * z7);
    s = s + a[19] * (yz * z73);
    s = s + a[20] * ((35.0 * z2 - 30.0) * z2 + 3.0);
    s = s + a[21] * (xz * z73);
    s = s + a[22] * (u * z7);
    s = s + a[23] * (xz * w3y);
    s = s + a[24] * (x2 * w3y - y2 * v3x);
    P = s;
    if (!GRAD) return;
    T gx = a[3];
    gx = gx + a[4] * y;
    gx = gx + a[7] * z;
    gx = gx + a[8] * (2.0 * x);
    gx = gx + a[9] * (6.0 * xy);
    gx = gx + a[10] * yz;
    gx = gx + a[13] * z5;
    gx = gx + a[14] * (2.0 * xz);
    gx = gx + a[15] * (3.0 * u);
    gx = gx + a[16] * (y * v3x);
    gx = gx + a[17] * ((6.0 * xy) * z);
    gx = gx + a[18] * (y * z7);
    gx = gx + a[21] * (z * z73);
    gx = gx + a[22] * ((2.0 * x) * z7);
    gx = gx + a[23] * ((3.0 * z) * u);
    gx = gx + a[24] * ((4.0 * x) * w3y);
    T gy = a[1];
    gy = gy + a[4] * x;
    gy = gy + a[5] * z;
    gy = gy + a[8] * (-2.0 * y);
    gy = gy + a[9] * (3.0 * u);
    gy = gy + a[10] * xz;
    gy = gy + a[11] * z5;
    gy = gy + a[14] * (-2.0 * yz);
    gy = gy + a[15] * (-6.0 * xy);
    gy = gy + a[16] * (x * w3y);
    gy = gy + a[17] * ((3.0 * z) * u);
    gy = gy + a[18] * (x * z7);
    gy = gy + a[19] * (z * z73);
    gy = gy + a[22] * ((-2.0 * y) * z7);
    gy = gy + a[23] * ((-6.0 * xy) * z);
    gy = gy + a[24] * ((-4.0 * y) * v3x);
    T gz = a[2];
    gz = gz + a[5] * y;
    gz = gz + a[6] * (6.0 * z);
    gz = gz + a[7] * x;
    gz = gz + a[10] * xy;
    gz = gz + a[11] * (10.0 * yz);
    gz = gz + a[12] * (15.0 * z2 - 3.0);
    gz = gz + a[13] * (10.0 * xz);
    gz = gz + a[14] * u;
    gz = gz + a[17] * (y * v3x);
    gz = gz + a[18] * ((14.0 * xy) * z);
    gz = gz + a[19] * (y * (21.0 * z2 - 3.0));
    gz = gz + a[20] * (z * (140.0 * z2 - 60.0));
    gz = gz + a[21] * (x * (21.0 * z2 - 3.0));
    gz = gz + a[22] * ((14.0 * z) * u);
    gz = gz + a[23] * (x * w3y);
    g[0] = gx;
    g[1] = gy;
    g[2] = gz;
}

// phi(x) = (|x - c| - 1) - P(xi), xi = (x - c)/|x - c|
__device__ double star_phi(const QuadGeo &g, const double X[3]) {
    const double d0 = X[0] - g.c[0], d1 = X[1] - g.c[1], d2 = X[2] - g.c[2];
    const double rho = sqrt((d0 * d0 + d1 * d1) + d2 * d2);
    double P, gr[3];
    star_eval<double, false>(g.a, d0 / rho, d1 / rho, d2 / rho, P, gr);
    return (rho - 1.0) - P;
}

// grad phi = xi - (g - (xi . g) xi)/rho (unnormalised); returns it in G
template <typename T>
__device__ void star_grad(const T *a, const QuadGeo &g, const T X[3], T G[3]) {
    const T d0 = X[0] - g.c[0], d1 = X[1] - g.c[1], d2 = X[2] - g.c[2];
    const T rho = dsqrt((d0 * d0 + d1 * d1) + d2 * d2);
    const T xi[3] = {d0 / rho, d1 / rho, d2 / rho};
    T P, gr[3];
    star_eval<T>(a, xi[0], xi[1], xi[2], P, gr);
    const T gxi = (gr[0] * xi[0] + gr[1] * xi[1]) + gr[2] * xi[2];
    for (int k = 0; k < 3; ++k) G[k] = xi[k] - (gr[k] - gxi * xi[k]) / rho;
}

template <typename T>
__device__ void star_normal(const T *a, const QuadGeo &g, const T X[3], T nv[3]) {
    T G[3];
    star_grad<T>(a, g, X, G);
    const T gn = dsqrt((G[0] * G[0] + G[1] * G[1]) + G[2] * G[2]);
    for (int k = 0; k < 3; ++k) nv[k] = G[k] / gn;
}

// Crossings of one grid line with the star surface (sampling + bisection).
__device__ int eval_line_star(const QuadGeo &g, int ax, int64_t ja, int64_t jb, double P[kMaxRoots][3],
                              double N[kMaxRoots][3], int br[kMaxRoots]) {
    const int a = ax == 0 ? 1 : 0;
    const int b = ax == 2 ? 1 : 2;
    const double xa = (double)ja * g.h;
    const double xb = (double)jb * g.h;
    const double da = xa - g.c[a], db = xb - g.c[b];
    if (!(da * da + db * db < g.rb * g.rb)) return 0;
    double X[3];
    X[a] = xa;
    X[b] = xb;
    X[ax] = g.tlo[ax];
    double fprev = star_phi(g, X);
    double tprev = g.tlo[ax];
    int kept = 0, ordinal = 0;
    for (int k = 1; k <= g.nk; ++k) {
        const double t = g.tlo[ax] + (double)k * g.dt[ax];
        X[ax] = t;
        const double f = star_phi(g, X);
        if ((fprev > 0.0) != (f > 0.0)) {
            double lo = tprev, hi = t, flo = fprev, fhi = f;
            const bool slo = flo > 0.0;
            for (int it = 0; it < 200; ++it) {
                const double mid = 0.5 * (lo + hi);
                if (mid == lo || mid == hi) break;
                X[ax] = mid;
                const double fm = star_phi(g, X);
                if ((fm > 0.0) == slo) { lo = mid; flo = fm; }
                else { hi = mid; fhi = fm; }
            }
            X[ax] = fabs(flo) <= fabs(fhi) ? lo : hi;
            double nv[3];
            star_normal<double>(g.a, g, X, nv);
            if (fabs(nv[ax]) >= g.ct) {
                if (kept == kMaxRoots) {
                    atomicExch(g.overflow, 1);
                } else {
                    for (int q = 0; q < 3; ++q) { P[kept][q] = X[q]; N[kept][q] = nv[q]; }
                    br[kept] = ordinal;
                    ++kept;
                }
            }
            ++ordinal;
        }
        fprev = f;
        tprev = t;
    }
    return kept;
}

// ----------------------------------------------------------------- molecule
// e^x for the Gaussians of the level set (x <= 0), by one stated method so
// that the point set does not depend on a math library's last bits: Cody and
// Waite's additive reduction x = k ln2 + r (k = floor(x/ln2 + 1/2), ln2 split
// into a 32-bit head, exact when multiplied by k, and its tail), the
// degree-13 Taylor polynomial of e^r (|r| <= ln2/2, truncation < 5e-18) by
// Horner's rule with the coefficients 1/j! rounded to double, then scaling by
// 2^k.  Each operation is rounded once (this file compiles without FMA
// contraction).  Zero below x = -700.
__device__ double gauss_exp(double x) {
    if (x < -700.0) return 0.0;
    const double k = floor(x * 1.4426950408889634 + 0.5);
    const double r = (x - k * 0.6931471803691238) - k * 1.9082149292705877e-10;
    const double c[14] = {1.0, 1.0, 0.5, 0.16666666666666666, 0.041666666666666664, 0.008333333333333333,
                          0.001388888888888889, 0.0001984126984126984, 2.48015873015873e-05,
                          2.7557319223985893e-06, 2.755731922398589e-07, 2.505210838544172e-08,
                          2.08767569878681e-09, 1.6059043836821613e-10};
    double p = c[13];
    for (int j = 12; j >= 0; --j) p = p * r + c[j];
    return ldexp(p, (int)k);
}

// phi = c - sum_k e^{-|x - x_k|^2 / r^2} (phi > 0 outside), grad phi =
// sum_k e^{-|x - x_k|^2 / r^2} 2 (x - x_k) / r^2 (e^x by gauss_exp); the same
// sampling and bisection as the star surfaces.
__device__ double mol_phi(const QuadGeo &g, const double X[3]) {
    double s = 0.0;
    for (int k = 0; k < 4; ++k) {
        const double d0 = X[0] - g.mol[k][0], d1 = X[1] - g.mol[k][1], d2 = X[2] - g.mol[k][2];
        const double r2 = (d0 * d0 + d1 * d1) + d2 * d2;
        s = s + gauss_exp(-r2 / (g.mr * g.mr));
    }
    return g.mc - s;
}

__device__ void mol_normal(const QuadGeo &g, const double X[3], double nv[3]) {
    double G[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 4; ++k) {
        const double d[3] = {X[0] - g.mol[k][0], X[1] - g.mol[k][1], X[2] - g.mol[k][2]};
        const double e = gauss_exp(-((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]) / (g.mr * g.mr));
        for (int q = 0; q < 3; ++q) G[q] = G[q] + e * (2.0 * d[q] / (g.mr * g.mr));
    }
    const double gn = sqrt((G[0] * G[0] + G[1] * G[1]) + G[2] * G[2]);
    for (int q = 0; q < 3; ++q) nv[q] = G[q] / gn;
}

__device__ int eval_line_molecule(const QuadGeo &g, int ax, int64_t ja, int64_t jb, double P[kMaxRoots][3],
                                  double N[kMaxRoots][3], int br[kMaxRoots]) {
    const int a = ax == 0 ? 1 : 0;
    const int b = ax == 2 ? 1 : 2;
    const double xa = (double)ja * g.h;
    const double xb = (double)jb * g.h;
    bool near = false;
    for (int k = 0; k < 4; ++k) {
        const double da = xa - g.mol[k][a], db = xb - g.mol[k][b];
        near |= da * da + db * db < g.mD * g.mD;
    }
    if (!near) return 0;
    double X[3];
    X[a] = xa;
    X[b] = xb;
    X[ax] = g.tlo[ax];
    double fprev = mol_phi(g, X);
    double tprev = g.tlo[ax];
    int kept = 0, ordinal = 0;
    for (int k = 1; k <= g.nka[ax]; ++k) {
        const double t = g.tlo[ax] + (double)k * g.dt[ax];
        X[ax] = t;
        const double f = mol_phi(g, X);
        if ((fprev > 0.0) != (f > 0.0)) {
            double lo = tprev, hi = t, flo = fprev, fhi = f;
            const bool slo = flo > 0.0;
            for (int it = 0; it < 200; ++it) {
                const double mid = 0.5 * (lo + hi);
                if (mid == lo || mid == hi) break;
                X[ax] = mid;
                const double fm = mol_phi(g, X);
                if ((fm > 0.0) == slo) { lo = mid; flo = fm; }
                else { hi = mid; fhi = fm; }
            }
            X[ax] = fabs(flo) <= fabs(fhi) ? lo : hi;
            double nv[3];
            mol_normal(g, X, nv);
            if (fabs(nv[ax]) >= g.ct) {
                if (kept == kMaxRoots) {
                    atomicExch(g.overflow, 1);
                } else {
                    for (int q = 0; q < 3; ++q) { P[kept][q] = X[q]; N[kept][q] = nv[q]; }
                    br[kept] = ordinal;
                    ++kept;
                }
            }
            ++ordinal;
        }
        fprev = f;
        tprev = t;
    }
    return kept;
}

__device__ __forceinline__ int eval_any(const QuadGeo &g, int ax, int64_t ja, int64_t jb, double P[kMaxRoots][3],
                                        double N[kMaxRoots][3], int br[kMaxRoots]) {
    if (g.kind == SSD_STAR) return eval_line_star(g, ax, ja, jb, P, N, br);
    if (g.kind == SSD_MOLECULE) return eval_line_molecule(g, ax, ja, jb, P, N, br);
    return eval_line(g, ax, ja, jb, P, N, br);
}

__global__ void quad_count_kernel(const QuadGeo g, int64_t nlines, int32_t *count) {
    const int64_t line = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= nlines) return;
    int ax;
    int64_t ja, jb;
    line_coords(g, line, ax, ja, jb);
    double P[kMaxRoots][3], N[kMaxRoots][3];
    int br[kMaxRoots];
    count[line] = eval_any(g, ax, ja, jb, P, N, br);
}

// Exclusive scan, three phases: per-block scan, scan of block totals (one
// block, sequential over totals), add block offsets.
__global__ void scan_block_kernel(const int32_t *in, int64_t n, int64_t *out, int64_t *blocksum) {
    __shared__ int64_t buf[1024];
    const int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    const int64_t v = i < n ? in[i] : 0;
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int64_t t = threadIdx.x >= off ? buf[threadIdx.x - off] : 0;
        __syncthreads();
        buf[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i] = buf[threadIdx.x] - v;
    if (threadIdx.x == 1023) blocksum[blockIdx.x] = buf[1023];
}

__global__ void scan_totals_kernel(int64_t *blocksum, int64_t nb, int64_t *total) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t run = 0;
    for (int64_t k = 0; k < nb; ++k) {
        const int64_t t = blocksum[k];
        blocksum[k] = run;
        run += t;
    }
    *total = run;
}

__global__ void scan_add_kernel(int64_t *out, int64_t n, const int64_t *blocksum) {
    const int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    if (i < n) out[i] += blocksum[blockIdx.x];
}

__global__ void quad_write_kernel(const QuadGeo g, int64_t nlines, const int64_t *offs, int64_t n, double *xyz,
                                  double *nrm, double *w, int32_t *meta) {
    const int64_t line = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= nlines) return;
    int ax;
    int64_t ja, jb;
    line_coords(g, line, ax, ja, jb);
    double P[kMaxRoots][3], N[kMaxRoots][3];
    int br[kMaxRoots];
    const int kept = eval_any(g, ax, ja, jb, P, N, br);
    for (int k = 0; k < kept; ++k) {
        const int64_t o = offs[line] + k;
        for (int q = 0; q < 3; ++q) {
            xyz[q * n + o] = P[k][q];
            nrm[q * n + o] = N[k][q];
        }
        // psi_i = b(acos|n_i|/theta) / sum_j b(acos|n_j|/theta); w = psi_i h^2 / |n_i|
        double beta[3];
        for (int q = 0; q < 3; ++q) beta[q] = bump(acos(fabs(N[k][q])) / g.theta);
        const double psi = beta[ax] / ((beta[0] + beta[1]) + beta[2]);
        w[o] = (psi * (g.h * g.h)) / fabs(N[k][ax]);
        if (meta) {
            meta[o] = ax;
            meta[n + o] = (int32_t)ja;
            meta[2 * n + o] = (int32_t)jb;
            meta[3 * n + o] = br[k];
        }
    }
}

// Derivatives of the points, normals and weights of a star surface with
// respect to its 25 coefficients.  A point on the line of axis i moves along
// e_i: phi(x(c), c) = 0 gives dt/dc_k = K_k p_k(xi) / (d phi/d x_i).  The
// normal's derivative is forward-mode (Dual) through the normal formula with
// the seed (dx, da_k = K_k); the weight's derivative differentiates
// w = psi_i(n) h^2 / |n_i| with psi_i = beta_i / sum_j beta_j,
// beta_j = b(acos|n_j| / theta):
//   d beta_j = beta_j 2 (alpha/sin alpha) / (theta^2 (r^2 - 1)^2) d|n_j|,
//   alpha = acos|n_j|, r = alpha/theta  (alpha/sin alpha -> 1 as alpha -> 0).
__device__ void pou_derivative(const QuadGeo &g, int ax, const double nv[3], const double dn[3], double &w,
                               double &dw) {
    double beta[3], dbeta[3];
    for (int j = 0; j < 3; ++j) {
        const double u = fabs(nv[j]);
        const double du = nv[j] < 0.0 ? -dn[j] : dn[j];
        const double al = acos(fmin(u, 1.0));
        const double r = al / g.theta;
        if (!(r < 1.0)) { beta[j] = 0.0; dbeta[j] = 0.0; continue; }
        const double r2 = r * r;
        beta[j] = exp(r2 / (r2 - 1.0));
        const double f = al > 1e-8 ? al / sin(al) : 1.0;
        dbeta[j] = beta[j] * 2.0 * f / (g.theta * g.theta * (r2 - 1.0) * (r2 - 1.0)) * du;
    }
    const double sb = (beta[0] + beta[1]) + beta[2];
    const double dsb = (dbeta[0] + dbeta[1]) + dbeta[2];
    const double psi = beta[ax] / sb;
    const double dpsi = (dbeta[ax] * sb - beta[ax] * dsb) / (sb * sb);
    const double ui = fabs(nv[ax]);
    const double dui = nv[ax] < 0.0 ? -dn[ax] : dn[ax];
    const double h2 = g.h * g.h;
    w = psi * h2 / ui;
    dw = h2 * (dpsi / ui - psi * dui / (ui * ui));
}

__global__ void quad_jacobian_kernel(const QuadGeo g, int64_t nlines, const int64_t *offs, int64_t n, double *dxyz,
                                     double *dnrm, double *dw) {
    const int64_t line = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= nlines) return;
    int ax;
    int64_t ja, jb;
    line_coords(g, line, ax, ja, jb);
    double P[kMaxRoots][3], N[kMaxRoots][3];
    int br[kMaxRoots];
    const int kept = eval_any(g, ax, ja, jb, P, N, br);
    for (int r = 0; r < kept; ++r) {
        const int64_t o = offs[line] + r;
        const double *X = P[r];
        double G[3];
        star_grad<double>(g.a, g, X, G);
        const double d0 = X[0] - g.c[0], d1 = X[1] - g.c[1], d2 = X[2] - g.c[2];
        const double rho = sqrt((d0 * d0 + d1 * d1) + d2 * d2);
        const double xi[3] = {d0 / rho, d1 / rho, d2 / rho};
        for (int k = 0; k < kStarCoef; ++k) {
            double e[kStarCoef];
            for (int j = 0; j < kStarCoef; ++j) e[j] = j == k ? 1.0 : 0.0;
            double pk, gdum[3];
            star_eval<double, false>(e, xi[0], xi[1], xi[2], pk, gdum);
            const double dt = g.K[k] * pk / G[ax];
            Dual ad[kStarCoef], Xd[3], nd[3];
            for (int j = 0; j < kStarCoef; ++j) ad[j] = {g.a[j], j == k ? g.K[k] : 0.0};
            for (int q = 0; q < 3; ++q) Xd[q] = {X[q], q == ax ? dt : 0.0};
            star_normal<Dual>(ad, g, Xd, nd);
            double dn[3], wv, dwv;
            for (int q = 0; q < 3; ++q) {
                dn[q] = nd[q].d;
                dxyz[((int64_t)k * 3 + q) * n + o] = q == ax ? dt : 0.0;
                dnrm[((int64_t)k * 3 + q) * n + o] = dn[q];
            }
            pou_derivative(g, ax, N[r], dn, wv, dwv);
            dw[(int64_t)k * n + o] = dwv;
        }
    }
}

// Host setup of the surface description (all kinds).
int quad_geometry(ssd_ctx *ctx, const ssd_surface *surf, double h, double angle_deg, QuadGeo *out) {
    QuadGeo &g = *out;
    memset(&g, 0, sizeof(g));
    g.kind = surf->kind;
    if (surf->kind == SSD_SPHERE) {
        for (int k = 0; k < 3; ++k) g.A[k] = surf->abc[0];
    } else if (surf->kind == SSD_ELLIPSOID) {
        for (int k = 0; k < 3; ++k) g.A[k] = surf->abc[k];
    } else if (surf->kind == SSD_STAR) {
        if (!surf->clm) return set_error(ctx, SSD_EINVAL, "star surface without coefficients");
        const double pi = M_PI;
        const double K[kStarCoef] = {
            0.5 * sqrt(1.0 / pi),
            sqrt(3.0 / (4.0 * pi)), sqrt(3.0 / (4.0 * pi)), sqrt(3.0 / (4.0 * pi)),
            0.5 * sqrt(15.0 / pi), 0.5 * sqrt(15.0 / pi), 0.25 * sqrt(5.0 / pi), 0.5 * sqrt(15.0 / pi),
            0.25 * sqrt(15.0 / pi),
            0.25 * sqrt(35.0 / (2.0 * pi)), 0.5 * sqrt(105.0 / pi), 0.25 * sqrt(21.0 / (2.0 * pi)),
            0.25 * sqrt(7.0 / pi), 0.25 * sqrt(21.0 / (2.0 * pi)), 0.25 * sqrt(105.0 / pi),
            0.25 * sqrt(35.0 / (2.0 * pi)),
            0.75 * sqrt(35.0 / pi), 0.75 * sqrt(35.0 / (2.0 * pi)), 0.75 * sqrt(5.0 / pi),
            0.75 * sqrt(5.0 / (2.0 * pi)), (3.0 / 16.0) * sqrt(1.0 / pi), 0.75 * sqrt(5.0 / (2.0 * pi)),
            0.375 * sqrt(5.0 / pi), 0.75 * sqrt(35.0 / (2.0 * pi)), (3.0 / 16.0) * sqrt(35.0 / pi)};
        double rb = 1.0;
        for (int k = 0; k < kStarCoef; ++k) {
            const double ck = surf->clm[k];
            if (!isfinite(ck)) return set_error(ctx, SSD_EINVAL, "non-finite star coefficient");
            const int l = k < 1 ? 0 : (k < 4 ? 1 : (k < 9 ? 2 : (k < 16 ? 3 : 4)));
            g.K[k] = K[k];
            g.a[k] = ck * K[k];
            rb = rb + fabs(ck) * sqrt((2.0 * l + 1.0) / (4.0 * pi));
        }
        if (!(rb < 2.0)) return set_error(ctx, SSD_EINVAL, "star coefficients too large: sum |c_lm| B_l must be < 1");
        g.rb = rb;
        for (int k = 0; k < 3; ++k) g.A[k] = rb;
        const double ds = 1.0 / 64.0;
        g.nk = (int)ceil(2.125 * rb / ds);
    } else if (surf->kind == SSD_MOLECULE) {
        // the four-atom molecule of Section 5.4 about surf->center
        const double r = surf->abc[0] > 0.0 ? surf->abc[0] : 0.5;
        const double c = surf->abc[1] > 0.0 ? surf->abc[1] : 0.6;
        if (!isfinite(r) || !isfinite(c) || !(c < 4.0))
            return set_error(ctx, SSD_EINVAL, "molecule width r must be positive and level c in (0, 4)");
        const double s3 = sqrt(3.0), s6 = sqrt(6.0);
        const double cen[4][3] = {{s3 / 3.0, 0.0, -s6 / 12.0}, {-s3 / 6.0, 0.5, -s6 / 12.0},
                                  {-s3 / 6.0, -0.5, -s6 / 12.0}, {0.0, 0.0, s6 / 4.0}};
        g.mr = r;
        g.mc = c;
        g.mD = 1.0625 * r * sqrt(log(4.0 / c));
        const double ds = 1.0 / 64.0;
        for (int k = 0; k < 3; ++k) {
            double lo = 1e300, hi = -1e300;
            for (int a = 0; a < 4; ++a) {
                g.mol[a][k] = cen[a][k] + surf->center[k];
                lo = fmin(lo, g.mol[a][k]);
                hi = fmax(hi, g.mol[a][k]);
            }
            lo = lo - g.mD;
            hi = hi + g.mD;
            g.nka[k] = (int)ceil((hi - lo) / ds);
            g.tlo[k] = lo;
            g.dt[k] = (hi - lo) / g.nka[k];
            g.c[k] = 0.5 * (lo + hi);      // line ranges only
            g.A[k] = 0.5 * (hi - lo) + 1e-9;   // covers [lo, hi] despite rounding
        }
    } else {
        return set_error(ctx, SSD_EINVAL, "unknown surface kind");
    }
    for (int k = 0; k < 3; ++k) {
        if (g.kind == SSD_MOLECULE) continue;
        g.c[k] = surf->center[k];
        if (!(g.A[k] > 0.0) || !isfinite(g.A[k]) || !isfinite(g.c[k]))
            return set_error(ctx, SSD_EINVAL, "semi-axes must be positive and finite");
        if (g.kind == SSD_STAR) {
            g.tlo[k] = g.c[k] - 1.0625 * g.rb;
            const double thi = g.c[k] + 1.0625 * g.rb;
            g.dt[k] = (thi - g.tlo[k]) / g.nk;
        }
    }
    g.h = h;
    g.ct = cos(angle_deg * (M_PI / 180.0));
    g.theta = angle_deg * (M_PI / 180.0);
    return SSD_OK;
}

}  // namespace

int quadrature_impl(ssd_ctx *ctx, const ssd_surface *surf, double h, double angle_deg, int64_t capacity,
                    int64_t *n_out, double *xyz, double *nrm, double *w, int32_t *meta, double *jx, double *jn,
                    double *jw, cudaStream_t s) {
    if (!surf || !n_out) return set_error(ctx, SSD_EINVAL, "surface or n_out is NULL");
    if (!(h > 0.0) || !isfinite(h)) return set_error(ctx, SSD_EINVAL, "h must be positive");
    if (!(angle_deg > 0.0 && angle_deg < 90.0)) return set_error(ctx, SSD_EINVAL, "angle must be in (0, 90)");
    QuadGeo g;
    SSD_TRY(quad_geometry(ctx, surf, h, angle_deg, &g));
    int64_t nlines = 0;
    for (int ax = 0; ax < 3; ++ax) {
        const int a = ax == 0 ? 1 : 0, b = ax == 2 ? 1 : 2;
        const int oth[2] = {a, b};
        g.line0[ax] = nlines;
        int64_t cnt = 1;
        for (int q = 0; q < 2; ++q) {
            const int k = oth[q];
            const int64_t lo = (int64_t)floor((g.c[k] - g.A[k]) / h) - 1;
            const int64_t hi = (int64_t)ceil((g.c[k] + g.A[k]) / h) + 1;
            if (hi - lo > 2000000) return set_error(ctx, SSD_EINVAL, "grid too fine for the surface");
            g.j0[ax][q] = lo;
            g.nj[ax][q] = hi - lo + 1;
            cnt *= g.nj[ax][q];
        }
        nlines += cnt;
    }
    g.line0[3] = nlines;
    if (nlines > (int64_t)1 << 31) return set_error(ctx, SSD_EINVAL, "grid too fine for the surface");

    const int64_t nb = (nlines + 1023) / 1024;
    size_t off = 0;
    auto carve = [&](size_t bb) { size_t o = off; off += (bb + 255) & ~size_t(255); return o; };
    const size_t o_cnt = carve(sizeof(int32_t) * nlines), o_off = carve(sizeof(int64_t) * nlines);
    const size_t o_bs = carve(sizeof(int64_t) * nb), o_tot = carve(sizeof(int64_t));
    const size_t o_ovf = carve(sizeof(int));
    void *tmp = nullptr;
    SSD_TRY(dev_alloc(ctx, off, &tmp));
    struct Release { ssd_ctx *c; void *p; ~Release() { dev_free(c, p); } } release{ctx, tmp};
    char *tb = static_cast<char *>(tmp);
    int32_t *cnt = reinterpret_cast<int32_t *>(tb + o_cnt);
    int64_t *offs = reinterpret_cast<int64_t *>(tb + o_off);
    int64_t *bs = reinterpret_cast<int64_t *>(tb + o_bs);
    int64_t *tot = reinterpret_cast<int64_t *>(tb + o_tot);
    g.overflow = reinterpret_cast<int *>(tb + o_ovf);
    SSD_TRY(cuda_check(ctx, cudaMemsetAsync(g.overflow, 0, sizeof(int), s), "memset"));
    const unsigned lb = (unsigned)((nlines + 255) / 256);
    quad_count_kernel<<<lb, 256, 0, s>>>(g, nlines, cnt);
    scan_block_kernel<<<(unsigned)nb, 1024, 0, s>>>(cnt, nlines, offs, bs);
    scan_totals_kernel<<<1, 32, 0, s>>>(bs, nb, tot);
    scan_add_kernel<<<(unsigned)nb, 1024, 0, s>>>(offs, nlines, bs);
    ctx->launches += 4;
    SSD_TRY(launch_check(ctx, "quadrature count"));
    SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(ctx->hbuf, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s),
                       "count copy"));
    SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(reinterpret_cast<char *>(ctx->hbuf) + 8, g.overflow, sizeof(int),
                                            cudaMemcpyDeviceToHost, s), "flag copy"));
    SSD_TRY(cuda_check(ctx, cudaStreamSynchronize(s), "quadrature sync"));
    int64_t total;
    int ovf;
    memcpy(&total, ctx->hbuf, sizeof(int64_t));
    memcpy(&ovf, reinterpret_cast<char *>(ctx->hbuf) + 8, sizeof(int));
    if (ovf) return set_error(ctx, SSD_EINVAL, "a grid line crosses the surface more than 8 times");
    *n_out = total;
    if (jx) {
        if (g.kind != SSD_STAR) return set_error(ctx, SSD_EINVAL, "shape derivatives need a STAR surface");
        if (capacity != total) return set_error(ctx, SSD_EINVAL, "n differs from the point count");
        if (!jn || !jw) return set_error(ctx, SSD_EINVAL, "NULL output array");
        quad_jacobian_kernel<<<lb, 256, 0, s>>>(g, nlines, offs, total, jx, jn, jw);
        ctx->launches += 1;
        SSD_TRY(launch_check(ctx, "quadrature jacobian"));
        return cuda_check(ctx, cudaStreamSynchronize(s), "quadrature sync");
    }
    if (!xyz) return SSD_OK;
    if (capacity < total) return set_error(ctx, SSD_EINVAL, "capacity smaller than the point count");
    if (!nrm || !w) return set_error(ctx, SSD_EINVAL, "NULL output array");
    quad_write_kernel<<<lb, 256, 0, s>>>(g, nlines, offs, total, xyz, nrm, w, meta);
    ctx->launches += 1;
    SSD_TRY(launch_check(ctx, "quadrature write"));
    return cuda_check(ctx, cudaStreamSynchronize(s), "quadrature sync");
}

int quadrature_points(ssd_ctx *ctx, const ssd_surface *surf, double h, double angle_deg, int64_t capacity,
                      int64_t *n_out, double *xyz, double *nrm, double *w, int32_t *meta, cudaStream_t s) {
    return quadrature_impl(ctx, surf, h, angle_deg, capacity, n_out, xyz, nrm, w, meta, nullptr, nullptr, nullptr, s);
}

int quadrature_jacobian(ssd_ctx *ctx, const ssd_surface *surf, double h, double angle_deg, int64_t n, double *dxyz,
                        double *dnrm, double *dw, cudaStream_t s) {
    if (!dxyz) return set_error(ctx, SSD_EINVAL, "NULL output array");
    int64_t total = 0;
    return quadrature_impl(ctx, surf, h, angle_deg, n, &total, nullptr, nullptr, nullptr, nullptr, dxyz, dnrm, dw, s);
}

}  // namespace ssd
