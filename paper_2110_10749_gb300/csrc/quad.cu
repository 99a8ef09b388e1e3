// Quadrature points of Section 5.4 (eq. Quadrature) on sphere and ellipsoid.
//
// One thread per grid line.  A first pass counts the kept intersections per
// line, an exclusive scan turns counts into output offsets, and a second pass
// writes points, normals, weights and (axis, j1, j2, branch).  Points and
// normals use explicitly rounded +, -, *, /, sqrt (no contraction), in the
// order stated next to each line, so that they are reproducible bit for bit
// by any implementation of the same definition.
#include <math.h>

#include "internal.h"

namespace ssd {
namespace {

struct QuadGeo {
    double A[3], c[3];
    double h, ct, theta;
    int64_t j0[3][2];     // first index of the two in-plane coordinates per axis
    int64_t nj[3][2];     // counts
    int64_t line0[4];     // first line id of each axis
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
__device__ int eval_line(const QuadGeo &g, int ax, int64_t ja, int64_t jb, double P[2][3], double N[2][3],
                         int br[2]) {
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

__global__ void quad_count_kernel(const QuadGeo g, int64_t nlines, int32_t *count) {
    const int64_t line = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= nlines) return;
    int ax;
    int64_t ja, jb;
    line_coords(g, line, ax, ja, jb);
    double P[2][3], N[2][3];
    int br[2];
    count[line] = eval_line(g, ax, ja, jb, P, N, br);
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
    double P[2][3], N[2][3];
    int br[2];
    const int kept = eval_line(g, ax, ja, jb, P, N, br);
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

}  // namespace

int quadrature_points(ssd_ctx *ctx, const ssd_surface *surf, double h, double angle_deg, int64_t capacity,
                      int64_t *n_out, double *xyz, double *nrm, double *w, int32_t *meta, cudaStream_t s) {
    if (!surf || !n_out) return set_error(ctx, SSD_EINVAL, "surface or n_out is NULL");
    if (!(h > 0.0) || !isfinite(h)) return set_error(ctx, SSD_EINVAL, "h must be positive");
    if (!(angle_deg > 0.0 && angle_deg < 90.0)) return set_error(ctx, SSD_EINVAL, "angle must be in (0, 90)");
    QuadGeo g;
    if (surf->kind == SSD_SPHERE) {
        for (int k = 0; k < 3; ++k) g.A[k] = surf->abc[0];
    } else if (surf->kind == SSD_ELLIPSOID) {
        for (int k = 0; k < 3; ++k) g.A[k] = surf->abc[k];
    } else {
        return set_error(ctx, SSD_EINVAL, "unknown surface kind");
    }
    for (int k = 0; k < 3; ++k) {
        g.c[k] = surf->center[k];
        if (!(g.A[k] > 0.0) || !isfinite(g.A[k]) || !isfinite(g.c[k]))
            return set_error(ctx, SSD_EINVAL, "semi-axes must be positive and finite");
    }
    g.h = h;
    g.ct = cos(angle_deg * (M_PI / 180.0));
    g.theta = angle_deg * (M_PI / 180.0);
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
    void *tmp = nullptr;
    SSD_TRY(dev_alloc(ctx, off, &tmp));
    struct Release { ssd_ctx *c; void *p; ~Release() { dev_free(c, p); } } release{ctx, tmp};
    char *tb = static_cast<char *>(tmp);
    int32_t *cnt = reinterpret_cast<int32_t *>(tb + o_cnt);
    int64_t *offs = reinterpret_cast<int64_t *>(tb + o_off);
    int64_t *bs = reinterpret_cast<int64_t *>(tb + o_bs);
    int64_t *tot = reinterpret_cast<int64_t *>(tb + o_tot);
    const unsigned lb = (unsigned)((nlines + 255) / 256);
    quad_count_kernel<<<lb, 256, 0, s>>>(g, nlines, cnt);
    scan_block_kernel<<<(unsigned)nb, 1024, 0, s>>>(cnt, nlines, offs, bs);
    scan_totals_kernel<<<1, 32, 0, s>>>(bs, nb, tot);
    scan_add_kernel<<<(unsigned)nb, 1024, 0, s>>>(offs, nlines, bs);
    ctx->launches += 4;
    SSD_TRY(launch_check(ctx, "quadrature count"));
    SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(ctx->hbuf, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s),
                       "count copy"));
    SSD_TRY(cuda_check(ctx, cudaStreamSynchronize(s), "quadrature sync"));
    int64_t total;
    memcpy(&total, ctx->hbuf, sizeof(int64_t));
    *n_out = total;
    if (!xyz) return SSD_OK;
    if (capacity < total) return set_error(ctx, SSD_EINVAL, "capacity smaller than the point count");
    if (!nrm || !w) return set_error(ctx, SSD_EINVAL, "NULL output array");
    quad_write_kernel<<<lb, 256, 0, s>>>(g, nlines, offs, total, xyz, nrm, w, meta);
    ctx->launches += 1;
    SSD_TRY(launch_check(ctx, "quadrature write"));
    return cuda_check(ctx, cudaStreamSynchronize(s), "quadrature sync");
}

}  // namespace ssd
