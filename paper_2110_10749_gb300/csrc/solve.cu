// Local boundary-integral solves, the Dirichlet-Neumann iteration and the
// C ABI of the layer operators.  All Krylov and interface arithmetic is FP64
// on the device; the host only sequences launches and reads one residual per
// iteration.
#include <math.h>
#include <string.h>

#include <functional>

#include "internal.h"

namespace ssd {
namespace {


// ------------------------------------------------------------ vector kernels
constexpr int kMaxRestart = 512;
constexpr int kDotMaxBlocks = 512;

// One warp per vector: partial[v * gridDim.x + bx] = V[v][rows of bx] . w
// over the block's row chunk (lanes stride 32 rows, four accumulators,
// shuffle reduction in a fixed pattern).  Blocks hold 8 warps = 8 vectors.
__global__ void multidot_warp_kernel(const double *V, int64_t ldv, const double *w, int64_t n, int64_t chunk,
                                     int nv, double *partial, const double *cond) {
    const int lane = threadIdx.x & 31;
    const int v = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (v >= nv) return;
    double *dst = partial + (int64_t)v * gridDim.x + blockIdx.x;
    if (cond && *cond == 0.0) {
        if (lane == 0) *dst = 0.0;
        return;
    }
    const double *a = V + (int64_t)v * ldv;
    const int64_t beg = (int64_t)blockIdx.x * chunk;
    int64_t end = beg + chunk;
    if (end > n) end = n;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int64_t k = beg + lane;
    for (; k + 96 < end; k += 128) {
        s0 += a[k] * w[k];
        s1 += a[k + 32] * w[k + 32];
        s2 += a[k + 64] * w[k + 64];
        s3 += a[k + 96] * w[k + 96];
    }
    for (; k < end; k += 32) s0 += a[k] * w[k];
    double t = (s0 + s1) + (s2 + s3);
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if (lane == 0) *dst = t;
}

// out[v] = sum_b partial[v * nbx + b], one warp per vector
__global__ void multidot_finish_warp_kernel(const double *partial, int nbx, int nv, double *out) {
    const int lane = threadIdx.x & 31;
    const int v = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (v >= nv) return;
    double t = 0.0;
    for (int b = lane; b < nbx; b += 32) t += partial[(int64_t)v * nbx + b];
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if (lane == 0) out[v] = t;
}

// w += sign * sum_v coef[v] V[v] (skipped when cond is set and *cond == 0);
// eight interleaved accumulators per row, combined in a fixed order
__global__ void vupdate_kernel(const double *V, int64_t ldv, int nv, const double *coef, double sign, double *w,
                               int64_t n, const double *cond = nullptr) {
    if (cond && *cond == 0.0) return;
    __shared__ double c[kMaxRestart + 4];
    for (int v = threadIdx.x; v < nv; v += blockDim.x) c[v] = sign * coef[v];
    __syncthreads();
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        double a[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        int v = 0;
        for (; v + 7 < nv; v += 8) {
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] += c[v + u] * V[(int64_t)(v + u) * ldv + k];
        }
        for (; v < nv; ++v) a[0] += c[v] * V[(int64_t)v * ldv + k];
        w[k] += ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    }
}

// Reorthogonalisation test of Daniel, Gragg, Kaufman and Stewart: after the
// first Gram-Schmidt pass h = V^T w (h[0..j]) with h[j+1] = w . w, the
// remaining norm is ||w||^2 - sum h_i^2; a second pass runs when more than
// half of ||w||^2 was removed.  Writes the decision to h[j+2] (1 or 0).
__global__ void dgks_kernel(double *h, int j) {
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i <= j; i += 256) s += h[i] * h[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) h[j + 2] = (red[0] > 0.5 * h[j + 1]) ? 1.0 : 0.0;
}

// y = a x + b y
__global__ void axpby_kernel(int64_t n, double a, const double *x, double b, double *y) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        y[k] = a * x[k] + b * y[k];
}

// y = x * (1 / *d) (or y = x if *d == 0)
__global__ void scale_inv_kernel(int64_t n, const double *x, const double *d, double *y) {
    const double dd = *d;
    const double f = dd != 0.0 ? 1.0 / dd : 1.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        y[k] = x[k] * f;
}

// y -= (*s) * f
__global__ void sub_dev_scalar_kernel(int64_t n, const double *s, double f, double *y) {
    const double v = (*s) * f;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        y[k] -= v;
}

// GMRES bookkeeping: H(:, j) = h1 + h2, H(j+1, j) = sqrt(nrm2), previous
// rotations applied, new rotation formed, residual estimate updated.
// Applying rotations 0..j-1 to the new column is the affine recurrence
// a_{i+1} = -s_i a_i + c_i b_i (a_0 = col_0, b_i = col_{i+1}), after which
// col_i = c_i a_i + s_i b_i.  The recurrence is evaluated as an inclusive
// scan of the affine maps (Hillis-Steele, fixed order), so the FP64
// dependency chain is log2(j) steps long instead of j.  Block of kMaxRestart
// threads (one per rotation).
__global__ void givens_kernel(double *H, int ldh, double *cs, double *sn, double *g, const double *h1,
                              const double *h2, const double *nrm2, int j, double *out) {
    __shared__ double col[kMaxRestart + 2], al[2][kMaxRestart], be[2][kMaxRestart];
    const int t = threadIdx.x;
    for (int i = t; i <= j; i += blockDim.x) col[i] = h1[i] + h2[i];
    __syncthreads();
    double ci = 0.0, si = 0.0, bi = 0.0;
    if (t < j) {
        ci = cs[t];
        si = sn[t];
        bi = col[t + 1];
        al[0][t] = -si;
        be[0][t] = ci * bi;
    }
    __syncthreads();
    int cur = 0;
    for (int off = 1; off < j; off <<= 1) {
        if (t < j) {
            if (t >= off) {
                const double a = al[cur][t], b = be[cur][t];
                al[cur ^ 1][t] = a * al[cur][t - off];
                be[cur ^ 1][t] = a * be[cur][t - off] + b;
            } else {
                al[cur ^ 1][t] = al[cur][t];
                be[cur ^ 1][t] = be[cur][t];
            }
        }
        cur ^= 1;
        __syncthreads();
    }
    const double a0 = col[0];
    __syncthreads();
    if (t < j) {
        const double ai = t == 0 ? a0 : al[cur][t - 1] * a0 + be[cur][t - 1];
        col[t] = ci * ai + si * bi;
    }
    if (t == 0 && j > 0) col[j] = al[cur][j - 1] * a0 + be[cur][j - 1];
    __syncthreads();
    double *hc = H + (int64_t)j * ldh;
    if (t == 0) {
        const double hn = sqrt(fmax(*nrm2, 0.0));
        const double den = hypot(col[j], hn);
        double cj = 1.0, sj = 0.0;
        if (den != 0.0) {
            cj = col[j] / den;
            sj = hn / den;
        }
        cs[j] = cj;
        sn[j] = sj;
        col[j] = den;
        col[j + 1] = 0.0;
        const double gj = g[j];
        g[j + 1] = -sj * gj;
        g[j] = cj * gj;
        out[0] = fabs(g[j + 1]);
        out[1] = hn;
    }
    __syncthreads();
    for (int i = t; i <= j + 1; i += blockDim.x) hc[i] = col[i];
}

// Back substitution H(0:k, 0:k) y = g(0:k), column by column: y_i is fixed,
// then every earlier right-hand side entry drops H(l, i) y_i in parallel.
__global__ void backsolve_kernel(const double *H, int ldh, const double *g, int k, double *y) {
    __shared__ double b[kMaxRestart];
    for (int i = threadIdx.x; i < k; i += blockDim.x) b[i] = g[i];
    __syncthreads();
    for (int i = k - 1; i >= 0; --i) {
        const double *hc = H + (int64_t)i * ldh;
        const double yi = b[i] / hc[i];
        __syncthreads();
        for (int l = threadIdx.x; l < i; l += blockDim.x) b[l] -= hc[l] * yi;
        if (threadIdx.x == 0) y[i] = yi;
        __syncthreads();
    }
}

__global__ void gmres_init_kernel(double *g, int m, const double *beta) {
    for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = i == 0 ? *beta : 0.0;
}

__global__ void sqrt_kernel(double *v) {
    if (threadIdx.x == 0) *v = sqrt(fmax(*v, 0.0));
}

// q_new = (1 - theta) q + theta (u . n)
__global__ void q_update_kernel(int64_t n, double theta, const double *q, const double *u, const double *nrm,
                                double *qn) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double un = u[i] * nrm[i] + u[n + i] * nrm[n + i] + u[2 * n + i] * nrm[2 * n + i];
        qn[i] = (1.0 - theta) * q[i] + theta * un;
    }
}

// BJS traction (eq. f): f = -p n + s (gamma/sqrt(kappa)) (u - (u.n) n)
__global__ void traction_bjs_kernel(int64_t n, const double *p, const double *u, const double *nrm, double coef,
                                    double *f) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double n0 = nrm[i], n1 = nrm[n + i], n2 = nrm[2 * n + i];
        double u0 = 0, u1 = 0, u2 = 0;
        if (u) { u0 = u[i]; u1 = u[n + i]; u2 = u[2 * n + i]; }
        const double un = u0 * n0 + u1 * n1 + u2 * n2;
        f[i] = -p[i] * n0 + coef * (u0 - un * n0);
        f[n + i] = -p[i] * n1 + coef * (u1 - un * n1);
        f[2 * n + i] = -p[i] * n2 + coef * (u2 - un * n2);
    }
}

// Porous-sphere benchmark traction (Section 7.3, eqs. f_r, f_theta): the
// computed Darcy pressure plus the exact velocity-derivative terms,
// f = (-p + 2 mu du_r/dr) e_r + f_theta e_theta, with sin(theta) e_theta =
// cos(theta) e_r - e for the flow direction e and c = 2 + kappa/R^2:
//   2 mu du_r/dr = -12 mu U kappa cos(theta) / (R^3 c),
//   f_theta      = -(3 mu U/(R c)) (1 + 2 kappa/R^2) sin(theta).
__global__ void traction_jt_kernel(int64_t n, const double *p, const double *xyz, double R, double kappa, double mu,
                                   double U, double e0, double e1, double e2, double *f) {
    const double c = 2.0 + kappa / (R * R);
    const double bcoef = -(3.0 * mu * U / (R * c)) * (1.0 + 2.0 * kappa / (R * R));
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = xyz[i], y = xyz[n + i], z = xyz[2 * n + i];
        const double r = sqrt(x * x + y * y + z * z);
        const double er0 = x / r, er1 = y / r, er2 = z / r;
        const double ct = (e0 * x + e1 * y + e2 * z) / r;
        const double a = -12.0 * mu * U * kappa * ct / (R * R * R * c);
        const double fr = -p[i] + a;
        f[i] = fr * er0 + bcoef * (ct * er0 - e0);
        f[n + i] = fr * er1 + bcoef * (ct * er1 - e1);
        f[2 * n + i] = fr * er2 + bcoef * (ct * er2 - e2);
    }
}

// pn = p n
__global__ void scalar_times_normal_kernel(int64_t n, const double *p, const double *nrm, double *pn) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int k = 0; k < 3; ++k) pn[k * n + i] = p[i] * nrm[k * n + i];
}

// tangential part u - (u . n) n
__global__ void tangential_kernel(int64_t n, const double *u, const double *nrm, double *t) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double un = u[i] * nrm[i] + u[n + i] * nrm[n + i] + u[2 * n + i] * nrm[2 * n + i];
        for (int k = 0; k < 3; ++k) t[k * n + i] = u[k * n + i] - un * nrm[k * n + i];
    }
}

inline unsigned grid_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > 4096) b = 4096;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// ------------------------------------------------------------------- helpers
struct Buf {
    ssd_ctx *ctx = nullptr;
    void *p = nullptr;
    Buf() {}
    Buf(const Buf &) = delete;
    Buf &operator=(const Buf &) = delete;
    ~Buf() { if (ctx) dev_free(ctx, p); }
    int alloc(ssd_ctx *c, size_t bytes) {
        ctx = c;
        return dev_alloc(c, bytes, &p);
    }
    double *d() const { return static_cast<double *>(p); }
};

struct Dots {
    ssd_ctx *ctx;
    cudaStream_t s;
    Buf partial;
    int init(ssd_ctx *c, cudaStream_t st, int maxv) {
        ctx = c;
        s = st;
        return partial.alloc(c, sizeof(double) * kDotMaxBlocks * (maxv + 1));
    }
    // out[v] = V[v] . w, v < nv (deterministic); out = 0 when cond && *cond == 0
    int multi(const double *V, int64_t ldv, int nv, const double *w, int64_t n, double *out,
              const double *cond = nullptr) {
        // row chunks of at least 1024 (a multiple of 128), at most kDotMaxBlocks of them
        int64_t chunk = (n + kDotMaxBlocks - 1) / kDotMaxBlocks;
        if (chunk < 1024) chunk = 1024;
        chunk = (chunk + 127) / 128 * 128;
        const int64_t nbx = (n + chunk - 1) / chunk;
        multidot_warp_kernel<<<dim3((unsigned)nbx, (unsigned)((nv + 7) / 8)), 256, 0, s>>>(V, ldv, w, n, chunk, nv,
                                                                                          partial.d(), cond);
        multidot_finish_warp_kernel<<<(nv + 7) / 8, 256, 0, s>>>(partial.d(), (int)nbx, nv, out);
        ctx->launches += 2;
        return launch_check(ctx, "dot kernels");
    }
};

int read_scalars(ssd_ctx *ctx, const double *dev, int k, double *host, cudaStream_t s) {
    SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(ctx->hbuf, dev, sizeof(double) * k, cudaMemcpyDeviceToHost, s),
                       "scalar copy"));
    SSD_TRY(cuda_check(ctx, cudaStreamSynchronize(s), "stream sync"));
    memcpy(host, ctx->hbuf, sizeof(double) * k);
    return SSD_OK;
}

// ---------------------------------------------------------------------- GMRES
typedef std::function<int(const double *in, double *out)> MatVec;

struct GmresResult {
    int iters = 0;
    double relres = 1.0;
};

// Restarted GMRES (Saad) with classical Gram-Schmidt and a second
// (re)orthogonalisation pass when the DGKS test calls for it, x0 = 0 unless
// `warm`.  Stops when the residual
// estimate falls to tol * ||b|| or after maxit Arnoldi steps.
// `trace`, when given, receives the residual estimate of every step read.
int gmres(ssd_ctx *ctx, cudaStream_t s, int64_t n, const MatVec &A, const double *b, double *x, double tol,
          int restart, int maxit, bool warm, GmresResult *res, bool pipeline = true,
          std::vector<double> *trace = nullptr) {
    const int m = restart;
    // residual estimates come back through a pinned frame: with `pipeline`
    // the next Arnoldi step is queued before the previous one's residual is
    // read (while that residual is still above 30 tol), so the host never
    // leaves the GPU idle between steps; a step queued past convergence is
    // discarded
    double *slot = nullptr;
    cudaEvent_t ev[2];
    SSD_TRY(frame_acquire(ctx, &slot, ev));
    struct FrameGuard { ssd_ctx *c; ~FrameGuard() { frame_release(c); } } frame_guard{ctx};
    Buf V, small;
    SSD_TRY(V.alloc(ctx, sizeof(double) * (size_t)(m + 1) * n));
    const int ldh = m + 1;
    // small: H[(m+1)*m], cs[m], sn[m], g[m+1], h1[m+3], h2[m+3], y[m], scal[8]
    const size_t nsmall = (size_t)ldh * m + 2 * m + (m + 1) + 2 * (m + 3) + m + 8;
    SSD_TRY(small.alloc(ctx, sizeof(double) * nsmall));
    double *H = small.d(), *cs = H + (size_t)ldh * m, *sn = cs + m, *g = sn + m, *h1 = g + m + 1,
           *h2 = h1 + m + 3, *y = h2 + m + 3, *scal = y + m;
    Dots dots;
    SSD_TRY(dots.init(ctx, s, m + 2));
    const unsigned gb = grid_for(n);

    // ||b||
    SSD_TRY(dots.multi(b, 0, 1, b, n, scal));
    double hb[2];
    SSD_TRY(read_scalars(ctx, scal, 1, hb, s));
    const double bnorm = sqrt(hb[0]);
    if (!isfinite(bnorm)) return set_error(ctx, SSD_ENUMERIC, "non-finite right-hand side");
    if (!warm) SSD_TRY(cuda_check(ctx, cudaMemsetAsync(x, 0, sizeof(double) * n, s), "memset"));
    res->iters = 0;
    res->relres = 0.0;
    if (bnorm == 0.0) {
        SSD_TRY(cuda_check(ctx, cudaMemsetAsync(x, 0, sizeof(double) * n, s), "memset"));
        return SSD_OK;
    }
    int total = 0;
    bool first = true;
    for (;;) {
        // r = b - A x  (r = b when x = 0 on the first cycle)
        double *v0 = V.d();
        if (first && !warm) {
            SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(v0, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s),
                               "copy"));
        } else {
            SSD_TRY(A(x, v0));
            axpby_kernel<<<gb, 256, 0, s>>>(n, 1.0, b, -1.0, v0);
            ctx->launches++;
        }
        first = false;
        SSD_TRY(dots.multi(v0, 0, 1, v0, n, scal));
        sqrt_kernel<<<1, 32, 0, s>>>(scal);
        gmres_init_kernel<<<1, 128, 0, s>>>(g, m, scal);
        scale_inv_kernel<<<gb, 256, 0, s>>>(n, v0, scal, v0);
        ctx->launches += 3;
        SSD_TRY(read_scalars(ctx, scal, 1, hb, s));
        double rel = hb[0] / bnorm;
        res->relres = rel;
        if (!isfinite(rel)) return set_error(ctx, SSD_ENUMERIC, "non-finite residual");
        if (rel <= tol || total >= maxit || hb[0] == 0.0) break;
        int k = 0;
        bool done = false;
        double prev_rel = rel;
        int pending = -1;      // queued step whose residual has not been read yet
        auto fetch = [&](int step) -> int {
            SSD_TRY(cuda_check(ctx, cudaEventSynchronize(ev[step & 1]), "event sync"));
            hb[0] = slot[2 * (step & 1)];
            hb[1] = slot[2 * (step & 1) + 1];
            return SSD_OK;
        };
        for (int j = 0; j < m; ++j) {
            double *vj = V.d() + (size_t)j * n;
            double *w = V.d() + (size_t)(j + 1) * n;    // the new vector is built in its slot
            SSD_TRY(A(vj, w));
            ++total;
            // Gram-Schmidt pass (h1[j+1] = w . w from the same sweep), the
            // DGKS test, and a second pass only when the test asks for it
            SSD_TRY(dots.multi(V.d(), n, j + 2, w, n, h1));
            vupdate_kernel<<<gb, 256, 0, s>>>(V.d(), n, j + 1, h1, -1.0, w, n);
            dgks_kernel<<<1, 256, 0, s>>>(h1, j);
            ctx->launches += 2;
            SSD_TRY(dots.multi(V.d(), n, j + 1, w, n, h2, h1 + j + 2));
            vupdate_kernel<<<gb, 256, 0, s>>>(V.d(), n, j + 1, h2, -1.0, w, n, h1 + j + 2);
            ctx->launches++;
            SSD_TRY(dots.multi(w, 0, 1, w, n, scal + 2));
            givens_kernel<<<1, kMaxRestart, 0, s>>>(H, ldh, cs, sn, g, h1, h2, scal + 2, j, scal);
            scale_inv_kernel<<<gb, 256, 0, s>>>(n, w, scal + 1, w);
            ctx->launches += 2;
            SSD_TRY(launch_check(ctx, "arnoldi step"));
            SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(slot + 2 * (j & 1), scal, 2 * sizeof(double),
                                                    cudaMemcpyDeviceToHost, s), "residual copy"));
            SSD_TRY(cuda_check(ctx, cudaEventRecord(ev[j & 1], s), "event record"));
            if (pending >= 0) {
                // step j was queued ahead: read step j - 1 now
                SSD_TRY(fetch(pending));
                rel = hb[0] / bnorm;
                res->relres = rel;
                if (trace) trace->push_back(rel);
                if (!isfinite(rel)) return set_error(ctx, SSD_ENUMERIC, "non-finite residual");
                if (rel <= tol || hb[1] == 0.0) {
                    k = pending + 1;      // discard step j
                    --total;
                    done = true;
                    break;
                }
                prev_rel = rel;
                pending = -1;
            }
            const bool last = (j + 1 >= m) || (total >= maxit);
            if (pipeline && !last && prev_rel > 30.0 * tol) {
                pending = j;
                continue;
            }
            SSD_TRY(fetch(j));
            k = j + 1;
            rel = hb[0] / bnorm;
            res->relres = rel;
            if (trace) trace->push_back(rel);
            if (!isfinite(rel)) return set_error(ctx, SSD_ENUMERIC, "non-finite residual");
            if (rel <= tol || total >= maxit || hb[1] == 0.0) { done = true; break; }
            prev_rel = rel;
        }
        backsolve_kernel<<<1, 256, 0, s>>>(H, ldh, g, k, y);
        vupdate_kernel<<<gb, 256, 0, s>>>(V.d(), n, k, y, 1.0, x, n);
        ctx->launches += 2;
        SSD_TRY(launch_check(ctx, "gmres update"));
        if (done && (rel <= tol || hb[1] == 0.0)) break;
        if (total >= maxit) break;
    }
    res->iters = total;
    SSD_TRY(cuda_check(ctx, cudaStreamSynchronize(s), "gmres sync"));
    if (res->relres > tol) return set_error(ctx, SSD_ENOTCONV, "GMRES reached its iteration limit");
    return SSD_OK;
}

// Successive approximations x <- step(x) until ||x_k - x_{k-1}|| <= tol ||x_k||.
int successive(ssd_ctx *ctx, cudaStream_t s, int64_t n, const std::function<int(const double *, double *)> &step,
               double *x, double tol, int maxit, GmresResult *res, bool warm = false) {
    Buf xn, scal;
    SSD_TRY(xn.alloc(ctx, sizeof(double) * n));
    SSD_TRY(scal.alloc(ctx, sizeof(double) * 4));
    Dots dots;
    SSD_TRY(dots.init(ctx, s, 2));
    if (!warm) SSD_TRY(cuda_check(ctx, cudaMemsetAsync(x, 0, sizeof(double) * n, s), "memset"));
    const unsigned gb = grid_for(n);
    for (int it = 1; it <= maxit; ++it) {
        SSD_TRY(step(x, xn.d()));
        SSD_TRY(dots.multi(xn.d(), 0, 1, xn.d(), n, scal.d()));
        axpby_kernel<<<gb, 256, 0, s>>>(n, 1.0, xn.d(), -1.0, x);   // x = xn - x
        ctx->launches++;
        SSD_TRY(dots.multi(x, 0, 1, x, n, scal.d() + 1));
        SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(x, xn.d(), sizeof(double) * n, cudaMemcpyDeviceToDevice, s),
                           "copy"));
        double h[2];
        SSD_TRY(read_scalars(ctx, scal.d(), 2, h, s));
        const double rel = h[0] > 0 ? sqrt(h[1] / h[0]) : 0.0;
        res->iters = it;
        res->relres = rel;
        if (!isfinite(rel)) return set_error(ctx, SSD_ENUMERIC, "non-finite iterate");
        if (rel <= tol) return SSD_OK;
    }
    return set_error(ctx, SSD_ENOTCONV, "successive approximations reached the iteration limit");
}

bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

// Mixed-precision iterative refinement of one local system A x = b
// (Wilkinson's scheme, as in Moler 1967): the residual r = b - A x with the
// FP64 operator `A_hi`, the correction from A_lo e = r by GMRES with the
// FP32C operator `A_lo`, x += e, until ||r|| <= tol ||b||.  The correction
// only has to take the residual down by tol ||b|| / ||r||: the operators
// differ by the FP32 pair-term rounding (about 1e-7 relative), so from a start
// that is already FP32C-accurate one correction and one check suffice, i.e.
// two FP64 applications instead of one per Krylov step.  res->iters counts
// the FP32C correction steps; res->relres is the last FP64 residual.
int ir_solve(ssd_ctx *ctx, cudaStream_t s, int64_t n, const MatVec &A_hi, const MatVec &A_lo, const double *b,
             double *x, double tol, int restart, int maxit, bool warm, GmresResult *res, int max_ref = 4) {
    Buf r, e, scal;
    SSD_TRY(r.alloc(ctx, sizeof(double) * n));
    SSD_TRY(e.alloc(ctx, sizeof(double) * n));
    SSD_TRY(scal.alloc(ctx, sizeof(double) * 2));
    Dots dots;
    SSD_TRY(dots.init(ctx, s, 1));
    const unsigned gb = grid_for(n);
    SSD_TRY(dots.multi(b, 0, 1, b, n, scal.d()));
    double h[1];
    SSD_TRY(read_scalars(ctx, scal.d(), 1, h, s));
    const double bnorm = sqrt(h[0]);
    if (!isfinite(bnorm)) return set_error(ctx, SSD_ENUMERIC, "non-finite right-hand side");
    res->iters = 0;
    res->relres = 0.0;
    if (!warm || bnorm == 0.0) SSD_TRY(cuda_check(ctx, cudaMemsetAsync(x, 0, sizeof(double) * n, s), "memset"));
    if (bnorm == 0.0) return SSD_OK;
    for (int k = 0;; ++k) {
        if (k == 0 && !warm) {
            SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(r.d(), b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s),
                               "copy"));
        } else {
            SSD_TRY(A_hi(x, r.d()));
            axpby_kernel<<<gb, 256, 0, s>>>(n, 1.0, b, -1.0, r.d());   // r = b - A x
            ctx->launches++;
        }
        SSD_TRY(dots.multi(r.d(), 0, 1, r.d(), n, scal.d()));
        SSD_TRY(read_scalars(ctx, scal.d(), 1, h, s));
        const double rel = sqrt(h[0]) / bnorm;
        res->relres = rel;
        if (!isfinite(rel)) return set_error(ctx, SSD_ENUMERIC, "non-finite refinement residual");
        if (rel <= tol) return SSD_OK;
        if (k >= max_ref || res->iters >= maxit)
            return set_error(ctx, SSD_ENOTCONV, "local refinement reached its iteration limit");
        GmresResult ge;
        const double tc = fmax(0.5 * tol / rel, 1e-6);
        const int st = gmres(ctx, s, n, A_lo, r.d(), e.d(), tc, restart, maxit - res->iters, false, &ge);
        if (st != SSD_OK && st != SSD_ENOTCONV) return st;
        res->iters += ge.iters;
        axpby_kernel<<<gb, 256, 0, s>>>(n, 1.0, e.d(), 1.0, x);
        ctx->launches++;
        SSD_TRY(launch_check(ctx, "refinement update"));
    }
}


int check_krylov(ssd_ctx *ctx, const ssd_krylov *kr) {
    if (!kr) return set_error(ctx, SSD_EINVAL, "krylov settings are NULL");
    if (!(kr->tol > 0.0) || !isfinite(kr->tol)) return set_error(ctx, SSD_EINVAL, "tolerance must be positive");
    if (kr->maxit < 1) return set_error(ctx, SSD_EINVAL, "maxit must be >= 1");
    if (!kr->use_sa && (kr->restart < 1 || kr->restart > kMaxRestart))
        return set_error(ctx, SSD_EINVAL, "restart must be in 1..512");
    if (kr->prec != SSD_FP64 && kr->prec != SSD_FP32C) return set_error(ctx, SSD_EINVAL, "unknown precision");
    return SSD_OK;
}

// ------------------------------------------------------------- local solves
int darcy_solve_impl(ssd_ctx *ctx, const ssd_points *pts, const Layout &L, double delta, double mu, double kappa,
                     const double *q, double *p, const ssd_krylov &kr, GmresResult *res, cudaStream_t s,
                     bool gauge = true, bool warm = false, bool mixed = false) {
    const int64_t n = pts->n;
    Buf b, scal;
    SSD_TRY(b.alloc(ctx, sizeof(double) * n));
    SSD_TRY(scal.alloc(ctx, sizeof(double) * 2));
    // b_D = (mu / kappa) L q  (eq. Darcy_final)
    PairCall pc;
    pc.op = OP_LSL; pc.prec = kr.prec; pc.delta = delta; pc.dens0 = q; pc.a_op = mu / kappa; pc.out = b.d();
    SSD_TRY(pair_apply(ctx, L, pc, s));
    int st;
    if (kr.use_sa) {
        // p <- p + D^L p + b, projected to zero weighted mean (eq. Darcy_BIEM_iter)
        Dots dots;
        SSD_TRY(dots.init(ctx, s, 1));
        auto step = [&](const double *x, double *y) -> int {
            PairCall a;
            a.op = OP_LDL; a.prec = kr.prec; a.delta = delta; a.dens0 = x; a.xin = x; a.a_id = 1.0; a.a_op = 1.0;
            a.out = y;
            SSD_TRY(pair_apply(ctx, L, a, s));
            axpby_kernel<<<grid_for(n), 256, 0, s>>>(n, 1.0, b.d(), 1.0, y);
            ctx->launches++;
            SSD_TRY(dots.multi(pts->w, 0, 1, y, n, scal.d()));
            sub_dev_scalar_kernel<<<grid_for(n), 256, 0, s>>>(n, scal.d(), 1.0 / L.wsum, y);
            ctx->launches++;
            return launch_check(ctx, "darcy sa step");
        };
        st = successive(ctx, s, n, step, p, kr.tol, kr.maxit, res, warm);
    } else {
        // -D^L p + (w . p)/sum(w): nonsingular, same solution for consistent b
        auto Ap = [&](int prec) {
            return [&, prec](const double *x, double *y) -> int {
                PairCall a;
                a.op = OP_LDL; a.prec = prec; a.delta = delta; a.dens0 = x; a.a_op = -1.0;
                a.rank1_weight_mean = true; a.out = y;
                return pair_apply(ctx, L, a, s);
            };
        };
        if (mixed && kr.prec == SSD_FP64)
            st = ir_solve(ctx, s, n, Ap(SSD_FP64), Ap(SSD_FP32C), b.d(), p, kr.tol, kr.restart, kr.maxit, warm, res);
        else
            st = gmres(ctx, s, n, Ap(kr.prec), b.d(), p, kr.tol, kr.restart, kr.maxit, warm, res);
    }
    if (st != SSD_OK && st != SSD_ENOTCONV) return st;
    if (!gauge) return st;
    // zero weighted mean
    Dots dots;
    SSD_TRY(dots.init(ctx, s, 1));
    SSD_TRY(dots.multi(pts->w, 0, 1, p, n, scal.d()));
    sub_dev_scalar_kernel<<<grid_for(n), 256, 0, s>>>(n, scal.d(), 1.0 / L.wsum, p);
    ctx->launches++;
    SSD_TRY(launch_check(ctx, "darcy gauge"));
    return st;
}

int stokes_solve_impl(ssd_ctx *ctx, const ssd_points *pts, const Layout &L, double delta, double mu,
                      const double *f, const double uinf[3], double *u, const ssd_krylov &kr, GmresResult *res,
                      cudaStream_t s, bool warm = false, bool mixed = false) {
    const int64_t n = pts->n;
    Buf b;
    SSD_TRY(b.alloc(ctx, sizeof(double) * 3 * n));
    // b_S = U_inf - M f  (eq. Stokes_final)
    PairCall pc;
    pc.op = OP_SSL; pc.prec = kr.prec; pc.delta = delta; pc.mu = mu; pc.dens0 = f; pc.a_op = -1.0;
    pc.add[0] = uinf[0]; pc.add[1] = uinf[1]; pc.add[2] = uinf[2]; pc.out = b.d();
    SSD_TRY(pair_apply(ctx, L, pc, s));
    if (kr.use_sa) {
        // u <- D^S u + b (eq. Stokes_BIEM_iter)
        auto step = [&](const double *x, double *y) -> int {
            PairCall a;
            a.op = OP_SDL; a.prec = kr.prec; a.delta = delta; a.dens0 = x; a.a_op = 1.0; a.out = y;
            SSD_TRY(pair_apply(ctx, L, a, s));
            axpby_kernel<<<grid_for(3 * n), 256, 0, s>>>(3 * n, 1.0, b.d(), 1.0, y);
            ctx->launches++;
            return launch_check(ctx, "stokes sa step");
        };
        return successive(ctx, s, 3 * n, step, u, kr.tol, kr.maxit, res, warm);
    }
    // (I - D^S) u  [+ n (w . (u.n))/sum(w) when deflating]
    auto Ap = [&](int prec) {
        return [&, prec](const double *x, double *y) -> int {
            PairCall a;
            a.op = OP_SDL; a.prec = prec; a.delta = delta; a.dens0 = x; a.xin = x; a.a_id = 1.0; a.a_op = -1.0;
            a.rank1_nrm = kr.deflate ? pts->nrm : nullptr;
            a.out = y;
            return pair_apply(ctx, L, a, s);
        };
    };
    if (mixed && kr.prec == SSD_FP64)
        return ir_solve(ctx, s, 3 * n, Ap(SSD_FP64), Ap(SSD_FP32C), b.d(), u, kr.tol, kr.restart, kr.maxit, warm, res);
    return gmres(ctx, s, 3 * n, Ap(kr.prec), b.d(), u, kr.tol, kr.restart, kr.maxit, warm, res);
}

// Stokes step with the BJS slip at its own velocity: with f = -p n + c P u
// (c = s gamma/sqrt(kappa), P u = u - (u.n) n), u = D^S u + U_inf - M f reads
//   (I - D^S) u + c M(P u) = U_inf + M(p n);
// the matvec is one fused single+double layer pass.
int stokes_solve_bjs_impl(ssd_ctx *ctx, const ssd_points *pts, const Layout &L, double delta, double mu,
                          const double *p, const double uinf[3], double c, double *u, const ssd_krylov &kr,
                          GmresResult *res, cudaStream_t s, bool warm = false, bool mixed = false) {
    const int64_t n = pts->n;
    Buf b, tmp;
    SSD_TRY(b.alloc(ctx, sizeof(double) * 3 * n));
    SSD_TRY(tmp.alloc(ctx, sizeof(double) * 3 * n));
    scalar_times_normal_kernel<<<grid_for(n), 256, 0, s>>>(n, p, pts->nrm, tmp.d());
    ctx->launches++;
    PairCall pc;
    pc.op = OP_SSL; pc.prec = kr.prec; pc.delta = delta; pc.mu = mu; pc.dens0 = tmp.d(); pc.a_op = 1.0;
    pc.add[0] = uinf[0]; pc.add[1] = uinf[1]; pc.add[2] = uinf[2]; pc.out = b.d();
    SSD_TRY(pair_apply(ctx, L, pc, s));
    auto Ap = [&](int prec) {
        return [&, prec](const double *x, double *y) -> int {
            tangential_kernel<<<grid_for(n), 256, 0, s>>>(n, x, pts->nrm, tmp.d());
            ctx->launches++;
            PairCall a;
            a.op = OP_SSLDL; a.prec = prec; a.delta = delta; a.mu = mu; a.dens0 = x; a.dens1 = tmp.d();
            a.alpha = c; a.beta = -1.0; a.xin = x; a.a_id = 1.0; a.a_op = 1.0; a.out = y;
            a.rank1_nrm = kr.deflate ? pts->nrm : nullptr;
            return pair_apply(ctx, L, a, s);
        };
    };
    if (mixed && kr.prec == SSD_FP64)
        return ir_solve(ctx, s, 3 * n, Ap(SSD_FP64), Ap(SSD_FP32C), b.d(), u, kr.tol, kr.restart, kr.maxit, warm, res);
    return gmres(ctx, s, 3 * n, Ap(kr.prec), b.d(), u, kr.tol, kr.restart, kr.maxit, warm, res);
}

// ------------------------------------------------------------------ D-N solve
struct Ddm {
    ssd_ctx *ctx;
    const ssd_points *pts;
    const Layout *L;
    ssd_ddm_params P;
    cudaStream_t s;
    int64_t n;
    Buf f, scal;
    std::vector<int> inner;   // (darcy, stokes) per sweep
    int nonconv = 0;
    bool start_from_outputs = false;   // local solves start from the contents of p and u
    bool mixed = false;                // FP64 local solves by refinement with FP32C corrections (ir_solve)

    // one sweep: (q, uprev) -> (qn, u); p and f are left in pbuf and f
    int sweep(const double *q, const double *uprev, double *qn, double *u, double *p) {
        GmresResult rd, rs;
        // relaxed sweeps may start each local solve from the previous sweep's
        // solution (p keeps it; u starts from uprev); the refinement's FP64
        // sweeps start from an FP32C sweep's solutions already in p and u
        const bool warm = (P.inner.warm && !P.outer_gmres) || start_from_outputs;
        if (warm && !start_from_outputs && u != uprev)
            SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(u, uprev, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s),
                               "warm start copy"));
        int st = darcy_solve_impl(ctx, pts, *L, P.delta, P.mu, P.kappa, q, p, P.inner, &rd, s, true, warm, mixed);
        if (st == SSD_ENOTCONV) { nonconv++; st = SSD_OK; }
        SSD_TRY(st);
        if (P.traction_mode == SSD_TRACTION_BJS && P.bjs_implicit) {
            const double coef = P.bjs_sign * P.gamma / sqrt(P.kappa);
            st = stokes_solve_bjs_impl(ctx, pts, *L, P.delta, P.mu, p, P.uinf, coef, u, P.inner, &rs, s, warm,
                                       mixed);
            if (st == SSD_ENOTCONV) { nonconv++; st = SSD_OK; }
            SSD_TRY(st);
            traction_bjs_kernel<<<grid_for(n), 256, 0, s>>>(n, p, u, pts->nrm, coef, f.d());
            q_update_kernel<<<grid_for(n), 256, 0, s>>>(n, P.theta, q, u, pts->nrm, qn);
            ctx->launches += 2;
            inner.push_back(rd.iters);
            inner.push_back(rs.iters);
            return launch_check(ctx, "implicit BJS sweep");
        }
        if (P.traction_mode == SSD_TRACTION_BJS) {
            const double coef = P.bjs_sign * P.gamma / sqrt(P.kappa);
            traction_bjs_kernel<<<grid_for(n), 256, 0, s>>>(n, p, P.gamma != 0.0 ? uprev : nullptr, pts->nrm, coef,
                                                            f.d());
        } else {
            const double U = sqrt(P.uinf[0] * P.uinf[0] + P.uinf[1] * P.uinf[1] + P.uinf[2] * P.uinf[2]);
            const double e0 = U > 0 ? P.uinf[0] / U : 0.0, e1 = U > 0 ? P.uinf[1] / U : 0.0,
                         e2 = U > 0 ? P.uinf[2] / U : 1.0;
            traction_jt_kernel<<<grid_for(n), 256, 0, s>>>(n, p, pts->xyz, P.radius, P.kappa, P.mu, U, e0, e1, e2,
                                                           f.d());
        }
        ctx->launches++;
        SSD_TRY(launch_check(ctx, "traction"));
        st = stokes_solve_impl(ctx, pts, *L, P.delta, P.mu, f.d(), P.uinf, u, P.inner, &rs, s, warm, mixed);
        if (st == SSD_ENOTCONV) { nonconv++; st = SSD_OK; }
        SSD_TRY(st);
        q_update_kernel<<<grid_for(n), 256, 0, s>>>(n, P.theta, q, u, pts->nrm, qn);
        ctx->launches++;
        inner.push_back(rd.iters);
        inner.push_back(rs.iters);
        return launch_check(ctx, "q update");
    }
};

int check_ddm(ssd_ctx *ctx, const ssd_ddm_params *P) {
    if (!P) return set_error(ctx, SSD_EINVAL, "parameters are NULL");
    if (!finite_pos(P->mu) || !finite_pos(P->kappa) || !finite_pos(P->delta))
        return set_error(ctx, SSD_EINVAL, "mu, kappa and delta must be positive");
    if (!(P->theta > 0.0 && P->theta <= 1.0)) return set_error(ctx, SSD_EINVAL, "theta must be in (0, 1]");
    if (!isfinite(P->gamma) || P->gamma < 0.0) return set_error(ctx, SSD_EINVAL, "gamma must be >= 0");
    for (int k = 0; k < 3; ++k)
        if (!isfinite(P->uinf[k])) return set_error(ctx, SSD_EINVAL, "non-finite far-field velocity");
    if (!finite_pos(P->tol_outer) || P->maxit_outer < 1) return set_error(ctx, SSD_EINVAL, "bad outer settings");
    if (P->traction_mode != SSD_TRACTION_BJS && P->traction_mode != SSD_TRACTION_JOSEPH_TAO)
        return set_error(ctx, SSD_EINVAL, "unknown traction mode");
    if (P->traction_mode == SSD_TRACTION_BJS && !(P->bjs_sign == 1.0 || P->bjs_sign == -1.0))
        return set_error(ctx, SSD_EINVAL, "bjs_sign must be +1 or -1");
    if (P->traction_mode == SSD_TRACTION_JOSEPH_TAO && !finite_pos(P->radius))
        return set_error(ctx, SSD_EINVAL, "radius must be positive");
    return check_krylov(ctx, &P->inner);
}

int ddm_impl(ssd_ctx *ctx, const ssd_points *pts, const ssd_ddm_params *prm, double *q_out, double *p_out,
             double *u_out, double *f_out, double drag[3], int *outer_its, int *inner_its, double *res_hist,
             cudaStream_t s) {
    SSD_TRY(check_ddm(ctx, prm));
    LayoutRef lref;
    SSD_TRY(get_layout(ctx, pts, &lref, s));
    Ddm D;
    D.ctx = ctx; D.pts = pts; D.L = lref.L; D.P = *prm; D.s = s; D.n = pts->n;
    const int64_t n = pts->n;
    const bool stacked = prm->traction_mode == SSD_TRACTION_BJS && prm->gamma != 0.0 && !prm->bjs_implicit;
    const int64_t nz = stacked ? 4 * n : n;
    SSD_TRY(D.f.alloc(ctx, sizeof(double) * 3 * n));
    SSD_TRY(D.scal.alloc(ctx, sizeof(double) * 8));
    Buf z, zn, p, u, c;
    SSD_TRY(z.alloc(ctx, sizeof(double) * 4 * n));
    SSD_TRY(zn.alloc(ctx, sizeof(double) * 4 * n));
    SSD_TRY(p.alloc(ctx, sizeof(double) * n));
    SSD_TRY(u.alloc(ctx, sizeof(double) * 3 * n));
    SSD_TRY(cuda_check(ctx, cudaMemsetAsync(z.d(), 0, sizeof(double) * 4 * n, s), "memset"));
    SSD_TRY(cuda_check(ctx, cudaMemsetAsync(p.d(), 0, sizeof(double) * n, s), "memset"));
    Dots dots;
    SSD_TRY(dots.init(ctx, s, 2));
    int its = 0;
    int status = SSD_OK;
    std::vector<double> hist;
    Ddm D64;                        // FP64 sweeps of the refinement (unused otherwise)
    D64.ctx = nullptr;
    const double *fsrc = nullptr;   // traction of the returned state
    if (!prm->outer_gmres) {
        // relaxed sweeps; z = (q, u_prev) with u_prev kept in z + n
        for (its = 1; its <= prm->maxit_outer; ++its) {
            SSD_TRY(D.sweep(z.d(), z.d() + n, zn.d(), zn.d() + n, p.d()));
            SSD_TRY(dots.multi(zn.d(), 0, 1, zn.d(), n, D.scal.d()));
            axpby_kernel<<<grid_for(n), 256, 0, s>>>(n, 1.0, zn.d(), -1.0, z.d());   // z = qn - q
            ctx->launches++;
            SSD_TRY(dots.multi(z.d(), 0, 1, z.d(), n, D.scal.d() + 1));
            SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(z.d(), zn.d(), sizeof(double) * 4 * n, cudaMemcpyDeviceToDevice,
                                                    s), "copy"));
            double h[2];
            SSD_TRY(read_scalars(ctx, D.scal.d(), 2, h, s));
            const double res = h[0] > 0 ? sqrt(h[1] / h[0]) : 0.0;
            hist.push_back(res);
            if (!isfinite(res)) return set_error(ctx, SSD_ENUMERIC, "non-finite DDM residual");
            if (res <= prm->tol_outer) break;
        }
        if (its > prm->maxit_outer) { its = prm->maxit_outer; status = SSD_ENOTCONV; }
    } else {
        // GMRES on D (I - G) z = D c, c = F(0).  In the stacked (lagged BJS)
        // form D divides the q rows, theta (q - u.n), by theta: the operator is
        // then the unrelaxed interface map, independent of theta, and the q
        // block (of size O(kappa)) is not swamped by the u block's residual.
        // With z = q alone D = I (a global scale would not change GMRES).
        SSD_TRY(c.alloc(ctx, sizeof(double) * 4 * n));
        SSD_TRY(D.sweep(z.d(), z.d() + n, c.d(), c.d() + n, p.d()));
        const double qscale = stacked ? 1.0 / prm->theta : 1.0;
        Buf cs;
        SSD_TRY(cs.alloc(ctx, sizeof(double) * 4 * n));
        SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(cs.d(), c.d(), sizeof(double) * nz, cudaMemcpyDeviceToDevice, s),
                           "copy"));
        if (stacked) {
            axpby_kernel<<<grid_for(n), 256, 0, s>>>(n, 0.0, cs.d(), qscale, cs.d());   // D c
            ctx->launches++;
        }
        auto F = [&](const double *v, double *out) -> int {
            // out = D (v - (F(v) - c)); F(v) = (q_new, u) of one sweep from v
            const double *uprev = stacked ? v + n : z.d() + n;   // z + n stays zero here
            SSD_TRY(D.sweep(v, uprev, zn.d(), zn.d() + n, p.d()));
            SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(out, c.d(), sizeof(double) * nz, cudaMemcpyDeviceToDevice, s),
                               "copy"));
            axpby_kernel<<<grid_for(nz), 256, 0, s>>>(nz, -1.0, zn.d(), 1.0, out);  // c - F(v)
            axpby_kernel<<<grid_for(nz), 256, 0, s>>>(nz, 1.0, v, 1.0, out);        // + v
            ctx->launches += 2;
            if (stacked) {
                axpby_kernel<<<grid_for(n), 256, 0, s>>>(n, 0.0, out, qscale, out);
                ctx->launches++;
            }
            return launch_check(ctx, "outer matvec");
        };
        GmresResult gr;
        // the lagged BJS interface needs a few hundred steps at small kappa and
        // large gamma; a restart there stalls, so the cycle is as long as allowed
        const int m_out = prm->maxit_outer < kMaxRestart ? prm->maxit_outer : kMaxRestart;
        // with refinement the FP32C solve only needs to get below the pair-sum
        // rounding (about 1e-7 relative); the FP64 residuals take it further
        const bool refine = prm->refine > 0 && prm->inner.prec == SSD_FP32C;
        const double tol1 = refine && prm->tol_outer < 1e-6 ? 1e-6 : prm->tol_outer;
        // each matvec is a whole sweep: no step is queued ahead of its check
        int st = gmres(ctx, s, nz, F, cs.d(), z.d(), tol1, m_out, prm->maxit_outer, false, &gr, false, &hist);
        if (st == SSD_ENOTCONV) status = SSD_ENOTCONV;
        else SSD_TRY(st);
        its = gr.iters;
        if (!stacked) SSD_TRY(cuda_check(ctx, cudaMemsetAsync(z.d() + n, 0, sizeof(double) * 3 * n, s), "memset"));
        if (!refine) {
            // final sweep from the solution gives the returned fields
            SSD_TRY(D.sweep(z.d(), z.d() + n, zn.d(), zn.d() + n, p.d()));
            SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(z.d() + n, zn.d() + n, sizeof(double) * 3 * n,
                                                    cudaMemcpyDeviceToDevice, s), "copy"));
        } else {
            // iterative refinement: r = F64(z) - z is the true residual of
            // (I - G) z = c, from one plain-FP64 sweep; D (I - G) e = D r is
            // solved with the FP32C sweeps and z += e
            D64.ctx = ctx; D64.pts = pts; D64.L = lref.L; D64.P = *prm; D64.P.inner.prec = SSD_FP64;
            D64.P.outer_gmres = 1; D64.s = s; D64.n = n; D64.start_from_outputs = true; D64.mixed = true;
            SSD_TRY(D64.f.alloc(ctx, sizeof(double) * 3 * n));
            Buf rb, eb;
            SSD_TRY(rb.alloc(ctx, sizeof(double) * 4 * n));
            SSD_TRY(eb.alloc(ctx, sizeof(double) * 4 * n));
            SSD_TRY(dots.multi(cs.d(), 0, 1, cs.d(), nz, D.scal.d()));
            double hc[1];
            SSD_TRY(read_scalars(ctx, D.scal.d(), 1, hc, s));
            const double cnorm = sqrt(hc[0]);
            for (int k = 0;; ++k) {
                // an FP32C sweep from z gives the FP64 local solves their start
                SSD_TRY(D.sweep(z.d(), z.d() + n, zn.d(), zn.d() + n, p.d()));
                SSD_TRY(D64.sweep(z.d(), z.d() + n, zn.d(), zn.d() + n, p.d()));
                SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(rb.d(), zn.d(), sizeof(double) * nz, cudaMemcpyDeviceToDevice,
                                                        s), "copy"));
                axpby_kernel<<<grid_for(nz), 256, 0, s>>>(nz, -1.0, z.d(), 1.0, rb.d());   // F64(z) - z
                ctx->launches++;
                if (stacked) {
                    axpby_kernel<<<grid_for(n), 256, 0, s>>>(n, 0.0, rb.d(), qscale, rb.d());
                    ctx->launches++;
                }
                SSD_TRY(dots.multi(rb.d(), 0, 1, rb.d(), nz, D.scal.d()));
                SSD_TRY(read_scalars(ctx, D.scal.d(), 1, hc, s));
                const double rel = cnorm > 0.0 ? sqrt(hc[0]) / cnorm : 0.0;
                if (!isfinite(rel)) return set_error(ctx, SSD_ENUMERIC, "non-finite refinement residual");
                hist.push_back(rel);
                if (rel <= prm->tol_outer) { status = SSD_OK; break; }
                if (k >= prm->refine) { status = SSD_ENOTCONV; break; }
                GmresResult ge;
                const double tcorr = fmax(0.5 * prm->tol_outer / rel, 1e-4);
                st = gmres(ctx, s, nz, F, rb.d(), eb.d(), tcorr, m_out, prm->maxit_outer, false, &ge, false);
                if (st != SSD_ENOTCONV) SSD_TRY(st);
                its += ge.iters;
                axpby_kernel<<<grid_for(nz), 256, 0, s>>>(nz, 1.0, eb.d(), 1.0, z.d());
                ctx->launches++;
            }
            // the returned fields are those of the last FP64 sweep
            SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(z.d() + n, zn.d() + n, sizeof(double) * 3 * n,
                                                    cudaMemcpyDeviceToDevice, s), "copy"));
            fsrc = D64.f.d();
        }
    }
    // outputs: q (the interface variable at convergence), p_D, u_S, f_S
    if (q_out) SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(q_out, z.d(), sizeof(double) * n, cudaMemcpyDeviceToDevice, s),
                                  "copy"));
    if (p_out) SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(p_out, p.d(), sizeof(double) * n, cudaMemcpyDeviceToDevice, s),
                                  "copy"));
    if (u_out) SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(u_out, z.d() + n, sizeof(double) * 3 * n,
                                                       cudaMemcpyDeviceToDevice, s), "copy"));
    if (!fsrc) fsrc = D.f.d();
    if (f_out) SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(f_out, fsrc, sizeof(double) * 3 * n,
                                                       cudaMemcpyDeviceToDevice, s), "copy"));
    // drag = sum_x w f (eq. drag_int)
    SSD_TRY(dots.multi(fsrc, n, 3, pts->w, n, D.scal.d()));
    double dh[3];
    SSD_TRY(read_scalars(ctx, D.scal.d(), 3, dh, s));
    if (drag) for (int k = 0; k < 3; ++k) drag[k] = dh[k];
    if (outer_its) *outer_its = its;
    if (inner_its) {
        const size_t cap = 2 * (size_t)(prm->maxit_outer + 2);
        for (size_t k = 0; k < D.inner.size() && k < cap; ++k) inner_its[k] = D.inner[k];
    }
    if (res_hist) {
        size_t k = 0;
        for (; k < hist.size() && k < (size_t)prm->maxit_outer; ++k) res_hist[k] = hist[k];
        if (k < (size_t)prm->maxit_outer) res_hist[k] = -1.0;   // end of the history
    }
    if (D64.ctx && D64.nonconv && status == SSD_OK) status = SSD_ENOTCONV;
    if (D.nonconv && status == SSD_OK && !D64.ctx) status = SSD_ENOTCONV;
    if (status == SSD_ENOTCONV) set_error(ctx, SSD_ENOTCONV, "iteration limit reached in the D-N solve");
    return status;
}

// One D-N sweep from a given interface state (q, u_prev).
int ddm_sweep_impl(ssd_ctx *ctx, const ssd_points *pts, const ssd_ddm_params *prm, const double *q,
                   const double *u_prev, double *q_out, double *p_out, double *u_out, double *f_out,
                   int *inner_its, cudaStream_t s) {
    SSD_TRY(check_ddm(ctx, prm));
    if (!q || !q_out) return set_error(ctx, SSD_EINVAL, "q and q_out are required");
    LayoutRef lref;
    SSD_TRY(get_layout(ctx, pts, &lref, s));
    Ddm D;
    D.ctx = ctx; D.pts = pts; D.L = lref.L; D.P = *prm; D.P.outer_gmres = 1; D.s = s; D.n = pts->n;
    const int64_t n = pts->n;
    SSD_TRY(D.f.alloc(ctx, sizeof(double) * 3 * n));
    Buf pb, ub, zb;
    double *p = p_out, *u = u_out;
    if (!p) { SSD_TRY(pb.alloc(ctx, sizeof(double) * n)); p = pb.d(); }
    if (!u) { SSD_TRY(ub.alloc(ctx, sizeof(double) * 3 * n)); u = ub.d(); }
    const double *up = u_prev;
    if (!up) {
        SSD_TRY(zb.alloc(ctx, sizeof(double) * 3 * n));
        SSD_TRY(cuda_check(ctx, cudaMemsetAsync(zb.d(), 0, sizeof(double) * 3 * n, s), "memset"));
        up = zb.d();
    }
    SSD_TRY(D.sweep(q, up, q_out, u, p));
    if (f_out) SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(f_out, D.f.d(), sizeof(double) * 3 * n,
                                                       cudaMemcpyDeviceToDevice, s), "copy"));
    SSD_TRY(cuda_check(ctx, cudaStreamSynchronize(s), "sweep sync"));
    if (inner_its && D.inner.size() >= 2) { inner_its[0] = D.inner[0]; inner_its[1] = D.inner[1]; }
    if (D.nonconv) return set_error(ctx, SSD_ENOTCONV, "a local solve reached its iteration limit");
    return SSD_OK;
}

// ------------------------------------------------- discrete iteration matrix
// Eigenvalues of a real upper Hessenberg matrix a (n x n, column-major,
// overwritten) by the implicitly double-shifted QR iteration: deflate at
// negligible subdiagonal entries (normwise against the neighbouring diagonal,
// refined by the neighbour-gap test, and, for windows stuck on clustered
// eigenvalues, 1e-11 relative after 30 sweeps), read off 1x1 and 2x2 blocks,
// otherwise
// chase a bulge started from the first column of (H - s1)(H - s2), s1, s2 the
// eigenvalues of the trailing 2x2 block (ad hoc shifts every tenth step).
// Only the active window is transformed (enough for eigenvalues).
static int hessenberg_eigenvalues(int n, double *a, double *wr, double *wi) {
    auto A = [&](int i, int j) -> double & { return a[i + (size_t)j * n]; };
    double anorm = 0.0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i <= (j + 1 < n ? j + 1 : n - 1); ++i) anorm += fabs(A(i, j));
    if (anorm == 0.0) anorm = 1.0;
    const double eps = 2.220446049250313e-16;
    int hi = n - 1, iter = 0, total = 0;
    while (hi >= 0) {
        int l = hi;
        for (; l > 0; --l) {
            const double h = fabs(A(l, l - 1));
            if (h <= 1e-300) { A(l, l - 1) = 0.0; break; }
            double sc = fabs(A(l - 1, l - 1)) + fabs(A(l, l));
            if (sc == 0.0) {
                if (l >= 2) sc += fabs(A(l - 1, l - 2));
                if (l + 1 <= hi) sc += fabs(A(l + 1, l));
            }
            if (sc == 0.0) sc = anorm;
            // normwise negligible, and (the test of Ahues and Tisseur) the
            // off-diagonal pair's product also small against the gap of the
            // neighbouring diagonal entries, which keeps small eigenvalues of
            // graded matrices accurate; a stricter test than the first alone
            if (h <= eps * sc) {
                const double ab = fmax(h, fabs(A(l - 1, l))), ba = fmin(h, fabs(A(l - 1, l)));
                const double gap = fabs(A(l - 1, l - 1) - A(l, l));
                const double aa = fmax(fabs(A(l, l)), gap), bb = fmin(fabs(A(l, l)), gap);
                const double s2 = aa + ab;
                if (ba * (ab / s2) <= fmax(1e-300, eps * (bb * (aa / s2)))) { A(l, l - 1) = 0.0; break; }
            }
            // clustered eigenvalues can leave a window stuck at rounding level
            if (iter >= 30 && h <= 1e-11 * sc) { A(l, l - 1) = 0.0; break; }
        }
        if (l == hi) {
            wr[hi] = A(hi, hi);
            wi[hi] = 0.0;
            --hi;
            iter = 0;
            continue;
        }
        if (l == hi - 1) {
            const double p = A(hi - 1, hi - 1), q = A(hi - 1, hi), r = A(hi, hi - 1), t = A(hi, hi);
            const double m = 0.5 * (p + t), d = 0.5 * (p - t);
            const double disc = d * d + q * r;
            if (disc >= 0.0) {
                const double sq = sqrt(disc);
                const double e1 = m + (m >= 0.0 ? sq : -sq);
                const double det = p * t - q * r;
                const double e2 = e1 != 0.0 ? det / e1 : m - sq;
                wr[hi - 1] = e1; wr[hi] = e2;
                wi[hi - 1] = wi[hi] = 0.0;
            } else {
                const double sq = sqrt(-disc);
                wr[hi - 1] = wr[hi] = m;
                wi[hi - 1] = sq;
                wi[hi] = -sq;
            }
            hi -= 2;
            iter = 0;
            continue;
        }
        if (++total > 100 * n) return -1;
        ++iter;
        // shifts s1, s2 (complex: s1r +- i s1i)
        double s1r, s1i = 0.0, s2r, s2i = 0.0;
        if (iter % 10 == 0) {
            const double w = fabs(A(hi, hi - 1)) + fabs(A(hi - 1, hi - 2));
            s1r = A(hi, hi) + 0.75 * w;
            s2r = A(hi, hi) - 0.4375 * w;
        } else {
            // eigenvalues of the trailing 2x2 block; a real pair is replaced
            // by the eigenvalue nearer A(hi, hi), taken twice
            const double p = A(hi - 1, hi - 1), q = A(hi - 1, hi), r = A(hi, hi - 1), t = A(hi, hi);
            const double m = 0.5 * (p + t), d = 0.5 * (p - t);
            const double disc = d * d + q * r;
            if (disc >= 0.0) {
                const double sq = sqrt(disc);
                const double e1 = m + sq, e2 = m - sq;
                s1r = s2r = fabs(e1 - t) <= fabs(e2 - t) ? e1 : e2;
            } else {
                s1r = s2r = m;
                s1i = sqrt(-disc);
                s2i = -s1i;
            }
        }
        // first column of (H - s1)(H - s2) in product form, scaled: no
        // cancellation of O(|H|^2) terms when the spectrum is clustered
        const double d1 = A(l, l) - s1r, d2 = A(l, l) - s2r;
        const double sc = fabs(d2) + fabs(s2i) + fabs(A(l + 1, l));
        const double h21 = A(l + 1, l) / sc;
        double x = h21 * A(l, l + 1) + d1 * (d2 / sc) - s1i * (s2i / sc);
        double y = h21 * (d1 + (A(l + 1, l + 1) - s2r));
        double z = h21 * A(l + 2, l + 1);
        for (int k = l; k <= hi - 2; ++k) {
            // reflector I - 2 v v^T / (v^T v) taking (x, y, z) to (alpha, 0, 0);
            // (x, y, z) normalised first against over- and underflow
            const double s3 = fabs(x) + fabs(y) + fabs(z);
            if (s3 != 0.0) { x /= s3; y /= s3; z /= s3; }
            const double nv = sqrt(x * x + y * y + z * z);
            if (nv != 0.0) {
                const double alpha = x >= 0.0 ? -nv : nv;
                const double v0 = x - alpha, v1 = y, v2 = z;
                const double beta = 2.0 / (v0 * v0 + v1 * v1 + v2 * v2);
                const int c0 = k > l ? k - 1 : l;
                for (int j = c0; j <= hi; ++j) {
                    const double f = beta * (v0 * A(k, j) + v1 * A(k + 1, j) + v2 * A(k + 2, j));
                    A(k, j) -= f * v0;
                    A(k + 1, j) -= f * v1;
                    A(k + 2, j) -= f * v2;
                }
                const int r1 = k + 3 < hi ? k + 3 : hi;
                for (int i = l; i <= r1; ++i) {
                    const double f = beta * (v0 * A(i, k) + v1 * A(i, k + 1) + v2 * A(i, k + 2));
                    A(i, k) -= f * v0;
                    A(i, k + 1) -= f * v1;
                    A(i, k + 2) -= f * v2;
                }
            }
            x = A(k + 1, k);
            y = A(k + 2, k);
            if (k < hi - 2) z = A(k + 3, k);
        }
        // last rotation on rows/columns hi-1, hi
        const double nr = hypot(x, y);
        if (nr != 0.0) {
            const double c = x / nr, sn = y / nr;
            for (int j = hi - 2; j <= hi; ++j) {
                const double u = A(hi - 1, j), v = A(hi, j);
                A(hi - 1, j) = c * u + sn * v;
                A(hi, j) = -sn * u + c * v;
            }
            for (int i = l; i <= hi; ++i) {
                const double u = A(i, hi - 1), v = A(i, hi);
                A(i, hi - 1) = c * u + sn * v;
                A(i, hi) = -sn * u + c * v;
            }
        }
    }
    return 0;
}

// v_i = frac(i g) - 1/2 (g = 0.6180339887498949): a start vector with every mode present
__global__ void golden_fill_kernel(int64_t n, double *v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double t = (double)i * 0.6180339887498949;
        v[i] = (t - floor(t)) - 0.5;
    }
}

// Ritz values of the discrete iteration matrix A~ v = F(v) - F(0), F one D-N
// sweep (eq. A_mat), from m Arnoldi steps (Gram-Schmidt twice).
// e = unit vector of index j (length n)
__global__ void unit_vector_kernel(int64_t n, int64_t j, double *e) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        e[k] = k == j ? 1.0 : 0.0;
}

// The discrete iteration matrix of eq. A_mat, column by column: column j is
// F(e_j) - F(0) for the sweep F on the interface variable q.
int ddm_iteration_matrix_impl(ssd_ctx *ctx, const ssd_points *pts, const ssd_ddm_params *prm, int64_t col0,
                              int64_t ncol, double *A, cudaStream_t s) {
    SSD_TRY(check_ddm(ctx, prm));
    if (!A) return set_error(ctx, SSD_EINVAL, "NULL output");
    if (!pts || col0 < 0 || ncol < 1 || col0 + ncol > pts->n)
        return set_error(ctx, SSD_EINVAL, "columns must satisfy 0 <= col0 < col0 + ncol <= n");
    if (prm->traction_mode == SSD_TRACTION_BJS && prm->gamma != 0.0 && !prm->bjs_implicit)
        return set_error(ctx, SSD_EINVAL, "the iteration matrix acts on q alone: lagged slip with gamma != 0 "
                                          "is not supported");
    LayoutRef lref;
    SSD_TRY(get_layout(ctx, pts, &lref, s));
    Ddm D;
    D.ctx = ctx; D.pts = pts; D.L = lref.L; D.P = *prm; D.P.outer_gmres = 1; D.s = s; D.n = pts->n;
    const int64_t n = pts->n;
    SSD_TRY(D.f.alloc(ctx, sizeof(double) * 3 * n));
    Buf c, zero, e, u, p;
    SSD_TRY(c.alloc(ctx, sizeof(double) * n));
    SSD_TRY(zero.alloc(ctx, sizeof(double) * 4 * n));
    SSD_TRY(e.alloc(ctx, sizeof(double) * n));
    SSD_TRY(u.alloc(ctx, sizeof(double) * 3 * n));
    SSD_TRY(p.alloc(ctx, sizeof(double) * n));
    SSD_TRY(cuda_check(ctx, cudaMemsetAsync(zero.d(), 0, sizeof(double) * 4 * n, s), "memset"));
    SSD_TRY(D.sweep(zero.d(), zero.d() + n, c.d(), u.d(), p.d()));      // c = F(0)
    const unsigned gb = grid_for(n);
    for (int64_t j = 0; j < ncol; ++j) {
        double *col = A + (size_t)j * n;
        unit_vector_kernel<<<gb, 256, 0, s>>>(n, col0 + j, e.d());
        ctx->launches++;
        SSD_TRY(D.sweep(e.d(), zero.d() + n, col, u.d(), p.d()));
        axpby_kernel<<<gb, 256, 0, s>>>(n, -1.0, c.d(), 1.0, col);     // F(e_j) - F(0)
        ctx->launches++;
    }
    SSD_TRY(cuda_check(ctx, cudaStreamSynchronize(s), "iteration matrix sync"));
    if (D.nonconv) return set_error(ctx, SSD_ENOTCONV, "a local solve reached its iteration limit");
    return SSD_OK;
}

int ddm_spectrum_impl(ssd_ctx *ctx, const ssd_points *pts, const ssd_ddm_params *prm, int m, int *m_out,
                      double *re, double *im, double *Hout, cudaStream_t s) {
    SSD_TRY(check_ddm(ctx, prm));
    if (m < 1 || m > kMaxRestart) return set_error(ctx, SSD_EINVAL, "m must be in 1..512");
    if (!m_out || !re || !im) return set_error(ctx, SSD_EINVAL, "NULL output");
    if (prm->traction_mode == SSD_TRACTION_BJS && prm->gamma != 0.0 && !prm->bjs_implicit)
        return set_error(ctx, SSD_EINVAL, "the iteration matrix acts on q alone: lagged slip with gamma != 0 "
                                          "is not supported");
    LayoutRef lref;
    SSD_TRY(get_layout(ctx, pts, &lref, s));
    Ddm D;
    D.ctx = ctx; D.pts = pts; D.L = lref.L; D.P = *prm; D.P.outer_gmres = 1; D.s = s; D.n = pts->n;
    const int64_t n = pts->n;
    SSD_TRY(D.f.alloc(ctx, sizeof(double) * 3 * n));
    SSD_TRY(D.scal.alloc(ctx, sizeof(double) * 8));
    Buf V, c, zero, u, p, small;
    SSD_TRY(V.alloc(ctx, sizeof(double) * (size_t)(m + 1) * n));
    SSD_TRY(c.alloc(ctx, sizeof(double) * n));
    SSD_TRY(zero.alloc(ctx, sizeof(double) * 4 * n));
    SSD_TRY(u.alloc(ctx, sizeof(double) * 3 * n));
    SSD_TRY(p.alloc(ctx, sizeof(double) * n));
    SSD_TRY(small.alloc(ctx, sizeof(double) * (2 * (m + 3) + 8)));
    double *h1 = small.d(), *h2 = h1 + m + 3, *scal = h2 + m + 3;
    SSD_TRY(cuda_check(ctx, cudaMemsetAsync(zero.d(), 0, sizeof(double) * 4 * n, s), "memset"));
    SSD_TRY(cuda_check(ctx, cudaMemsetAsync(p.d(), 0, sizeof(double) * n, s), "memset"));
    SSD_TRY(D.sweep(zero.d(), zero.d() + n, c.d(), u.d(), p.d()));      // c = F(0)
    Dots dots;
    SSD_TRY(dots.init(ctx, s, m + 2));
    const unsigned gb = grid_for(n);
    golden_fill_kernel<<<gb, 256, 0, s>>>(n, V.d());
    ctx->launches++;
    SSD_TRY(dots.multi(V.d(), 0, 1, V.d(), n, scal));
    sqrt_kernel<<<1, 32, 0, s>>>(scal);
    scale_inv_kernel<<<gb, 256, 0, s>>>(n, V.d(), scal, V.d());
    ctx->launches += 2;
    std::vector<double> hh((size_t)(m + 1) * m, 0.0), c1(m + 2), c2(m + 2);
    int mm = m;
    for (int j = 0; j < m; ++j) {
        double *vj = V.d() + (size_t)j * n, *w = V.d() + (size_t)(j + 1) * n;
        SSD_TRY(D.sweep(vj, zero.d() + n, w, u.d(), p.d()));
        axpby_kernel<<<gb, 256, 0, s>>>(n, -1.0, c.d(), 1.0, w);       // w = F(v_j) - F(0)
        ctx->launches++;
        SSD_TRY(dots.multi(V.d(), n, j + 1, w, n, h1));
        vupdate_kernel<<<gb, 256, 0, s>>>(V.d(), n, j + 1, h1, -1.0, w, n);
        ctx->launches++;
        SSD_TRY(dots.multi(V.d(), n, j + 1, w, n, h2));
        vupdate_kernel<<<gb, 256, 0, s>>>(V.d(), n, j + 1, h2, -1.0, w, n);
        ctx->launches++;
        SSD_TRY(dots.multi(w, 0, 1, w, n, scal));
        SSD_TRY(read_scalars(ctx, h1, j + 1, c1.data(), s));
        SSD_TRY(read_scalars(ctx, h2, j + 1, c2.data(), s));
        double nrm2;
        SSD_TRY(read_scalars(ctx, scal, 1, &nrm2, s));
        double cmax = 0.0;
        for (int i = 0; i <= j; ++i) {
            hh[i + (size_t)j * (m + 1)] = c1[i] + c2[i];
            cmax = fmax(cmax, fabs(c1[i] + c2[i]));
        }
        const double hn = sqrt(fmax(nrm2, 0.0));
        hh[(j + 1) + (size_t)j * (m + 1)] = hn;
        if (!isfinite(hn)) return set_error(ctx, SSD_ENUMERIC, "non-finite Arnoldi vector");
        if (hn <= 1e-12 * cmax) { mm = j + 1; break; }      // invariant subspace
        axpby_kernel<<<gb, 256, 0, s>>>(n, 1.0 / hn, w, 0.0, w);
        ctx->launches++;
        SSD_TRY(launch_check(ctx, "arnoldi step"));
    }
    SSD_TRY(cuda_check(ctx, cudaStreamSynchronize(s), "arnoldi sync"));
    if (Hout)
        for (size_t k = 0; k < hh.size(); ++k) Hout[k] = hh[k];
    std::vector<double> sq((size_t)mm * mm);
    for (int j = 0; j < mm; ++j)
        for (int i = 0; i < mm; ++i) sq[i + (size_t)j * mm] = hh[i + (size_t)j * (m + 1)];
    if (hessenberg_eigenvalues(mm, sq.data(), re, im) != 0)
        return set_error(ctx, SSD_ENUMERIC, "Hessenberg QR iteration did not converge");
    *m_out = mm;
    return D.nonconv ? set_error(ctx, SSD_ENOTCONV, "a local solve reached its iteration limit") : SSD_OK;
}

// ------------------------------------------------------------------- adjoint
// Discrete adjoint of the interface solve.  With the sweep written as
//   p = P_g A_D^{-1} (mu/kappa) L q            (Darcy, gauge projection P_g)
//   u = A_S^{-1} (U_inf + M(n p) - M f_x)      (Stokes, f_x = explicit traction part)
//   q = n . u                                  (fixed point of the interface map)
// the interface map is q = T q + t0 with T = N^T A_S^{-1} M N P_g A_D^{-1} (mu/kappa) L.
// For a functional J(q, p, u; theta) the derivative in a parameter theta is
//   dJ/dtheta = dJ/dtheta|explicit + g_p . dp/dtheta|_q + nu . X_theta,
//   X_theta = d(U_inf + M(n p) - M f_x)/dtheta|_q - (dA_S/dtheta) u,
//   nu = A_S^{-T} (n lambda) + mu_u,  (I - T)^T lambda = zeta,
// where mu_u = A_S^{-T} g_u and zeta collects dJ/dq and the adjoint Darcy
// term (mu/kappa) L^T A_D^{-T} P_g^T (g_p + N^T M^T mu_u).  All transposes are
// those of the weighted discrete operators (transposed pair kernels).

// y = v n (scalar field times the normal field)
__global__ void scal_normal_kernel(int64_t n, const double *v, const double *nrm, double *y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int k = 0; k < 3; ++k) y[k * n + i] = v[i] * nrm[k * n + i];
}
// s = n . y (vector field dotted with the normal)
__global__ void dot_normal_kernel(int64_t n, const double *y, const double *nrm, double *s) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s[i] = y[i] * nrm[i] + y[n + i] * nrm[n + i] + y[2 * n + i] * nrm[2 * n + i];
}
// y += f * (*d) * x  (device scalar)
__global__ void axpy_dev_kernel(int64_t n, const double *d, double f, const double *x, double *y) {
    const double a = f * (*d);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += a * x[i];
}
__global__ void fill_kernel(int64_t n, double v, double *y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = v;
}
// kind 0: y = w (e . x)   (weights of the flux moment)
// kind 1: y = -w (n . e)  (pressure weights of the drag along e)
__global__ void weight_field_kernel(int64_t n, const double *w, const double *xyz, const double *nrm, double e0,
                                    double e1, double e2, int kind, double *y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (kind == 0) y[i] = w[i] * (e0 * xyz[i] + e1 * xyz[n + i] + e2 * xyz[2 * n + i]);
        else y[i] = -w[i] * (e0 * nrm[i] + e1 * nrm[n + i] + e2 * nrm[2 * n + i]);
    }
}
// y = c w (e - (e . n) n)
__global__ void weighted_tangent_kernel(int64_t n, const double *w, const double *nrm, double c, double e0, double e1,
                                        double e2, double *y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double en = e0 * nrm[i] + e1 * nrm[n + i] + e2 * nrm[2 * n + i];
        y[i] = c * w[i] * (e0 - en * nrm[i]);
        y[n + i] = c * w[i] * (e1 - en * nrm[n + i]);
        y[2 * n + i] = c * w[i] * (e2 - en * nrm[2 * n + i]);
    }
}
// d/dlog(kappa) of the exact-velocity part a e_r + f_theta e_theta of the
// porous-sphere benchmark traction (traction_jt_kernel), c = 2 + kappa/R^2:
//   da/dlog(kappa)      = -24 mu U kappa cos(theta) / (R^3 c^2),
//   d(b)/dlog(kappa)    = -(3 mu U/R) 3 kappa/(R^2 c^2)  for f_theta = b sin(theta).
__global__ void jt_dtraction_kernel(int64_t n, const double *xyz, double R, double kappa, double mu, double U, double e0,
                                    double e1, double e2, double *y) {
    const double c = 2.0 + kappa / (R * R);
    const double db = -(3.0 * mu * U / R) * 3.0 * kappa / (R * R * c * c);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = xyz[i], yy = xyz[n + i], z = xyz[2 * n + i];
        const double r = sqrt(x * x + yy * yy + z * z);
        const double er0 = x / r, er1 = yy / r, er2 = z / r;
        const double ct = (e0 * x + e1 * yy + e2 * z) / r;
        const double da = -24.0 * mu * U * kappa * ct / (R * R * R * c * c);
        y[i] = da * er0 + db * (ct * er0 - e0);
        y[n + i] = da * er1 + db * (ct * er1 - e1);
        y[2 * n + i] = da * er2 + db * (ct * er2 - e2);
    }
}

struct Adjoint {
    ssd_ctx *ctx;
    const ssd_points *pts;
    const Layout *L;
    ssd_ddm_params P;
    cudaStream_t s;
    int64_t n;
    double c;          // BJS slip coefficient of A_S (0 unless implicit BJS)
    int nonconv = 0;
    Dots dots;
    Buf scal, ones, t3a, t3b, t1a, w3, w3b, w1, w1b;

    int init() {
        SSD_TRY(dots.init(ctx, s, 1));
        SSD_TRY(scal.alloc(ctx, sizeof(double) * 8));
        SSD_TRY(ones.alloc(ctx, sizeof(double) * n));
        SSD_TRY(t3a.alloc(ctx, sizeof(double) * 3 * n));
        SSD_TRY(t3b.alloc(ctx, sizeof(double) * 3 * n));
        SSD_TRY(t1a.alloc(ctx, sizeof(double) * n));
        SSD_TRY(w3.alloc(ctx, sizeof(double) * 3 * n));
        SSD_TRY(w3b.alloc(ctx, sizeof(double) * 3 * n));
        SSD_TRY(w1.alloc(ctx, sizeof(double) * n));
        SSD_TRY(w1b.alloc(ctx, sizeof(double) * n));
        fill_kernel<<<grid_for(n), 256, 0, s>>>(n, 1.0, ones.d());
        ctx->launches++;
        return launch_check(ctx, "adjoint init");
    }
    // y = a_op * op(x) [+ a_id * xin]; tsl: transposed single layer
    int apply(int op, bool tsl, const double *x, double *y, double a_op = 1.0, const double *xin = nullptr,
              double a_id = 0.0) {
        PairCall pc;
        pc.op = op; pc.transpose_sl = tsl; pc.prec = P.inner.prec; pc.delta = P.delta; pc.mu = P.mu;
        pc.dens0 = x; pc.a_op = a_op; pc.xin = xin; pc.a_id = a_id; pc.out = y;
        return pair_apply(ctx, *L, pc, s);
    }
    // *dst = sum_i v_i
    int sum(const double *v, double *dst) { return dots.multi(v, 0, 1, ones.d(), n, dst); }
    // a . b to the host
    int hdot(const double *a, const double *b, int64_t m, double *host) {
        SSD_TRY(dots.multi(a, 0, 1, b, m, scal.d() + 4));
        return read_scalars(ctx, scal.d() + 4, 1, host, s);
    }
    // A_S^T y = y - (D^S)^T y + c P M^T y [+ (w n)(sum_i n_i . y_i)/W when deflating]
    int AsT(const double *y, double *out) {
        SSD_TRY(apply(OP_SDLT, false, y, out, -1.0, y, 1.0));
        if (c != 0.0) {
            SSD_TRY(apply(OP_SSL, true, y, t3a.d()));
            tangential_kernel<<<grid_for(n), 256, 0, s>>>(n, t3a.d(), pts->nrm, t3b.d());
            axpby_kernel<<<grid_for(3 * n), 256, 0, s>>>(3 * n, c, t3b.d(), 1.0, out);
            ctx->launches += 2;
        }
        if (P.inner.deflate) {
            dot_normal_kernel<<<grid_for(n), 256, 0, s>>>(n, y, pts->nrm, t1a.d());
            ctx->launches++;
            SSD_TRY(sum(t1a.d(), scal.d()));
            scal_normal_kernel<<<grid_for(n), 256, 0, s>>>(n, pts->w, pts->nrm, t3b.d());
            axpy_dev_kernel<<<grid_for(3 * n), 256, 0, s>>>(3 * n, scal.d(), 1.0 / L->wsum, t3b.d(), out);
            ctx->launches += 2;
        }
        return launch_check(ctx, "A_S^T");
    }
    // A_D^T v = -(D^L)^T v + w (sum_j v_j)/W
    int AdT(const double *v, double *out) {
        SSD_TRY(apply(OP_LDLT, false, v, out, -1.0));
        SSD_TRY(sum(v, scal.d() + 1));
        axpy_dev_kernel<<<grid_for(n), 256, 0, s>>>(n, scal.d() + 1, 1.0 / L->wsum, pts->w, out);
        ctx->launches++;
        return launch_check(ctx, "A_D^T");
    }
    int solve(int64_t m, const MatVec &A, const double *rhs, double *x) {
        GmresResult r;
        const int st = gmres(ctx, s, m, A, rhs, x, P.inner.tol, P.inner.restart, P.inner.maxit, false, &r);
        if (st == SSD_ENOTCONV) { nonconv++; return SSD_OK; }
        return st;
    }
    int solveAsT(const double *rhs, double *x) {
        return solve(3 * n, [&](const double *in, double *o) -> int { return AsT(in, o); }, rhs, x);
    }
    int solveAdT(const double *rhs, double *x) {
        return solve(n, [&](const double *in, double *o) -> int { return AdT(in, o); }, rhs, x);
    }
    // P_g^T v = v - w (sum_j v_j)/W  (in place)
    int PgT(double *v) {
        SSD_TRY(sum(v, scal.d() + 2));
        axpy_dev_kernel<<<grid_for(n), 256, 0, s>>>(n, scal.d() + 2, -1.0 / L->wsum, pts->w, v);
        ctx->launches++;
        return launch_check(ctx, "P_g^T");
    }
    // out = (mu/kappa) L^T A_D^{-T} P_g^T N^T h   (h: a 3n field, N^T h = n . h)
    int darcy_adjoint(const double *h3, double *out) {
        dot_normal_kernel<<<grid_for(n), 256, 0, s>>>(n, h3, pts->nrm, w1.d());
        ctx->launches++;
        SSD_TRY(PgT(w1.d()));
        SSD_TRY(solveAdT(w1.d(), w1b.d()));
        return apply(OP_LSL, true, w1b.d(), out, P.mu / P.kappa);
    }
    // out = v - T^T v, T^T v = (mu/kappa) L^T A_D^{-T} P_g^T N^T M^T A_S^{-T} (n v)
    int interface_matvec(const double *v, double *out) {
        scal_normal_kernel<<<grid_for(n), 256, 0, s>>>(n, v, pts->nrm, w3.d());
        ctx->launches++;
        SSD_TRY(solveAsT(w3.d(), w3b.d()));
        SSD_TRY(apply(OP_SSL, true, w3b.d(), w3.d()));
        SSD_TRY(darcy_adjoint(w3.d(), out));
        axpby_kernel<<<grid_for(n), 256, 0, s>>>(n, 1.0, v, -1.0, out);
        ctx->launches++;
        return launch_check(ctx, "adjoint interface matvec");
    }
};

// Pointwise geometric terms of the adjoint (derivatives in n_k, w_k, x_k of
// the terms that are not pair sums).  Scalars: W = sum w, S1 = sum nu . n,
// S2 = sum w n . u, S3 = sum (M^T nu) . n, sa = sum alpha, sg = sum g_p.
struct GeoPoint {
    int64_t n;
    const double *xyz, *nrm, *w, *u, *p, *q, *lam, *nu, *mtnu;
    double c, W, S1, S2, S3, sa, sg, e[3];
    int deflate, functional;
    double *gx, *gn, *gw;
};
__global__ void geo_point_kernel(const GeoPoint a) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.n; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = a.n;
        double nk[3], uk[3], vk[3], nu[3];
        for (int e = 0; e < 3; ++e) {
            nk[e] = a.nrm[e * n + k]; uk[e] = a.u[e * n + k]; vk[e] = a.mtnu[e * n + k]; nu[e] = a.nu[e * n + k];
        }
        const double wk = a.w[k], pk = a.p[k];
        const double vn = vk[0] * nk[0] + vk[1] * nk[1] + vk[2] * nk[2];
        const double un = uk[0] * nk[0] + uk[1] * nk[1] + uk[2] * nk[2];
        const double en = a.e[0] * nk[0] + a.e[1] * nk[1] + a.e[2] * nk[2];
        double gn[3], gx[3] = {0, 0, 0};
        // interface q = n . u, Stokes source M(n p), slip -c M(P u)
        for (int e = 0; e < 3; ++e) gn[e] = a.lam[k] * uk[e] + pk * vk[e] + a.c * (vn * uk[e] + un * vk[e]);
        // gauge projections of p in M(n p) and in -A_D's rank-one term
        double gw = -pk * (a.S3 + a.sa) / a.W;
        if (a.deflate) {
            for (int e = 0; e < 3; ++e) gn[e] -= (nu[e] * a.S2 + a.S1 * wk * uk[e]) / a.W;
            gw -= a.S1 * (un - a.S2 / a.W) / a.W;
        }
        if (a.functional == SSD_FUNC_DRAG) {
            // J = sum_k w_k f_k . e, f = -p n + c (u - (u.n) n)
            const double ue = uk[0] * a.e[0] + uk[1] * a.e[1] + uk[2] * a.e[2];
            gw += -pk * en + a.c * (ue - un * en) - pk * a.sg / a.W;
            for (int e = 0; e < 3; ++e) gn[e] += -wk * pk * a.e[e] - a.c * wk * (en * uk[e] + un * a.e[e]);
        } else {
            // J = sum_k w_k q_k (e . x_k)
            const double ex = a.e[0] * a.xyz[k] + a.e[1] * a.xyz[n + k] + a.e[2] * a.xyz[2 * n + k];
            gw += a.q[k] * ex;
            for (int e = 0; e < 3; ++e) gx[e] += wk * a.q[k] * a.e[e];
        }
        for (int e = 0; e < 3; ++e) {
            a.gx[e * n + k] = gx[e];
            a.gn[e * n + k] = gn[e];
        }
        a.gw[k] = gw;
    }
}

int ddm_gradient_impl(ssd_ctx *ctx, const ssd_points *pts, const ssd_ddm_params *prm, int functional, double *value,
                      double grad[2], double *geo_x, double *geo_n, double *geo_w, cudaStream_t s) {
    SSD_TRY(check_ddm(ctx, prm));
    if (!prm->outer_gmres) return set_error(ctx, SSD_EINVAL, "gradients need the interface GMRES (outer_gmres = 1)");
    const bool jt = prm->traction_mode == SSD_TRACTION_JOSEPH_TAO;
    const bool implicit = prm->traction_mode == SSD_TRACTION_BJS && prm->bjs_implicit;
    if (!jt && !implicit && prm->gamma != 0.0)
        return set_error(ctx, SSD_EINVAL, "gradients need bjs_implicit = 1 in BJS mode with gamma != 0");
    const bool geo = geo_x || geo_n || geo_w;
    if (geo && !(geo_x && geo_n && geo_w)) return set_error(ctx, SSD_EINVAL, "geometry outputs must all be given");
    if (geo && jt) return set_error(ctx, SSD_EINVAL, "geometry gradients need the BJS traction");
    if (functional != SSD_FUNC_DRAG && functional != SSD_FUNC_FLUX)
        return set_error(ctx, SSD_EINVAL, "unknown functional");
    if (prm->inner.use_sa) return set_error(ctx, SSD_EINVAL, "gradients need GMRES local solves (use_sa = 0)");
    const int64_t n = pts->n;
    // forward solve
    Buf q, p, u;
    SSD_TRY(q.alloc(ctx, sizeof(double) * n));
    SSD_TRY(p.alloc(ctx, sizeof(double) * n));
    SSD_TRY(u.alloc(ctx, sizeof(double) * 3 * n));
    double drag[3];
    int its = 0;
    int status = ddm_impl(ctx, pts, prm, q.d(), p.d(), u.d(), nullptr, drag, &its, nullptr, nullptr, s);
    if (status != SSD_OK && status != SSD_ENOTCONV) return status;
    LayoutRef lref;
    SSD_TRY(get_layout(ctx, pts, &lref, s));
    Adjoint A;
    A.ctx = ctx; A.pts = pts; A.L = lref.L; A.P = *prm; A.s = s; A.n = n;
    A.c = implicit ? prm->bjs_sign * prm->gamma / sqrt(prm->kappa) : 0.0;
    SSD_TRY(A.init());
    const double U = sqrt(prm->uinf[0] * prm->uinf[0] + prm->uinf[1] * prm->uinf[1] + prm->uinf[2] * prm->uinf[2]);
    const double e0 = U > 0 ? prm->uinf[0] / U : 0.0, e1 = U > 0 ? prm->uinf[1] / U : 0.0,
                 e2 = U > 0 ? prm->uinf[2] / U : 1.0;
    double h = 0.0, g0 = 0.0, g1 = 0.0, val = 0.0;

    // X_theta for theta = log(kappa) (X0) and gamma (X1).  At fixed q the
    // Darcy pressure scales as 1/kappa, so dp/dlog(kappa)|_q = -p.
    Buf X0, X1, t3, t3b, pu;
    SSD_TRY(X0.alloc(ctx, sizeof(double) * 3 * n));
    SSD_TRY(X1.alloc(ctx, sizeof(double) * 3 * n));
    SSD_TRY(t3.alloc(ctx, sizeof(double) * 3 * n));
    SSD_TRY(t3b.alloc(ctx, sizeof(double) * 3 * n));
    SSD_TRY(pu.alloc(ctx, sizeof(double) * 3 * n));
    scal_normal_kernel<<<grid_for(n), 256, 0, s>>>(n, p.d(), pts->nrm, t3.d());
    ctx->launches++;
    SSD_TRY(A.apply(OP_SSL, false, t3.d(), X0.d(), -1.0));                 // -M(n p)
    SSD_TRY(cuda_check(ctx, cudaMemsetAsync(X1.d(), 0, sizeof(double) * 3 * n, s), "memset"));
    if (A.c != 0.0) {
        // dA_S/dlog(kappa) = -(c/2) M P,  dA_S/dgamma = (c/gamma) M P
        tangential_kernel<<<grid_for(n), 256, 0, s>>>(n, u.d(), pts->nrm, pu.d());
        ctx->launches++;
        SSD_TRY(A.apply(OP_SSL, false, pu.d(), t3b.d()));                  // M P u
        axpby_kernel<<<grid_for(3 * n), 256, 0, s>>>(3 * n, 0.5 * A.c, t3b.d(), 1.0, X0.d());
        axpby_kernel<<<grid_for(3 * n), 256, 0, s>>>(3 * n, -A.c / prm->gamma, t3b.d(), 0.0, X1.d());
        ctx->launches += 2;
    }
    if (jt) {
        // the benchmark right-hand side holds -M(a e_r + f_theta e_theta)
        jt_dtraction_kernel<<<grid_for(n), 256, 0, s>>>(n, pts->xyz, prm->radius, prm->kappa, prm->mu, U, e0, e1, e2,
                                                       t3.d());
        ctx->launches++;
        SSD_TRY(A.apply(OP_SSL, false, t3.d(), X0.d(), -1.0, X0.d(), 1.0));
    }
    SSD_TRY(launch_check(ctx, "adjoint sources"));

    // zeta = dJ/dq + Darcy adjoint of the pressure sensitivity; nu_extra = mu_u
    Buf zeta, lam, nu, mu_u;
    SSD_TRY(zeta.alloc(ctx, sizeof(double) * n));
    SSD_TRY(lam.alloc(ctx, sizeof(double) * n));
    SSD_TRY(nu.alloc(ctx, sizeof(double) * 3 * n));
    SSD_TRY(mu_u.alloc(ctx, sizeof(double) * 3 * n));
    if (functional == SSD_FUNC_FLUX) {
        // J = sum_i w_i q_i (e . x_i)
        weight_field_kernel<<<grid_for(n), 256, 0, s>>>(n, pts->w, pts->xyz, pts->nrm, e0, e1, e2, 0, zeta.d());
        ctx->launches++;
        SSD_TRY(A.hdot(zeta.d(), q.d(), n, &val));
        SSD_TRY(cuda_check(ctx, cudaMemsetAsync(mu_u.d(), 0, sizeof(double) * 3 * n, s), "memset"));
    } else {
        // J = e . sum_i w_i f_i = g_p . p + g_u . u + explicit terms
        val = drag[0] * e0 + drag[1] * e1 + drag[2] * e2;
        Buf gp;
        SSD_TRY(gp.alloc(ctx, sizeof(double) * n));
        weight_field_kernel<<<grid_for(n), 256, 0, s>>>(n, pts->w, pts->xyz, pts->nrm, e0, e1, e2, 1, gp.d());
        ctx->launches++;
        SSD_TRY(A.hdot(gp.d(), p.d(), n, &h));
        g0 -= h;                                                             // g_p . dp/dlog(kappa)|_q
        if (A.c != 0.0) {
            // g_u = c w P e;  explicit: (dc/dtheta) sum_i w_i (P u_i) . e
            weighted_tangent_kernel<<<grid_for(n), 256, 0, s>>>(n, pts->w, pts->nrm, A.c, e0, e1, e2, t3.d());
            ctx->launches++;
            SSD_TRY(A.solveAsT(t3.d(), mu_u.d()));
            SSD_TRY(A.hdot(pu.d(), t3.d(), 3 * n, &h));                     // c sum w (P u) . e
            g0 += -0.5 * h;
            g1 += h / prm->gamma;
        } else {
            SSD_TRY(cuda_check(ctx, cudaMemsetAsync(mu_u.d(), 0, sizeof(double) * 3 * n, s), "memset"));
        }
        if (jt) {
            // explicit: e . sum_i w_i d(a e_r + f_theta e_theta)/dlog(kappa)
            jt_dtraction_kernel<<<grid_for(n), 256, 0, s>>>(n, pts->xyz, prm->radius, prm->kappa, prm->mu, U, e0, e1,
                                                           e2, t3.d());
            ctx->launches++;
            const double ek[3] = {e0, e1, e2};
            for (int k = 0; k < 3; ++k) {
                if (ek[k] == 0.0) continue;
                SSD_TRY(A.hdot(t3.d() + k * n, pts->w, n, &h));
                g0 += ek[k] * h;
            }
        }
        // zeta = (mu/kappa) L^T A_D^{-T} P_g^T (g_p + N^T M^T mu_u)
        SSD_TRY(A.apply(OP_SSL, true, mu_u.d(), t3b.d()));
        scal_normal_kernel<<<grid_for(n), 256, 0, s>>>(n, gp.d(), pts->nrm, t3.d());
        axpby_kernel<<<grid_for(3 * n), 256, 0, s>>>(3 * n, 1.0, t3.d(), 1.0, t3b.d());   // n g_p + M^T mu_u
        ctx->launches += 2;
        SSD_TRY(A.darcy_adjoint(t3b.d(), zeta.d()));
    }
    // interface adjoint (I - T)^T lambda = zeta, then nu = A_S^{-T}(n lambda) + mu_u
    {
        GmresResult r;
        const int m = prm->maxit_outer < 128 ? prm->maxit_outer : 128;
        auto M = [&](const double *v, double *o) -> int { return A.interface_matvec(v, o); };
        const int st = gmres(ctx, s, n, M, zeta.d(), lam.d(), prm->tol_outer, m, prm->maxit_outer, false, &r,
                             false);
        if (st == SSD_ENOTCONV) A.nonconv++;
        else SSD_TRY(st);
        scal_normal_kernel<<<grid_for(n), 256, 0, s>>>(n, lam.d(), pts->nrm, t3.d());
        ctx->launches++;
        SSD_TRY(A.solveAsT(t3.d(), nu.d()));
        axpby_kernel<<<grid_for(3 * n), 256, 0, s>>>(3 * n, 1.0, mu_u.d(), 1.0, nu.d());
        ctx->launches++;
    }
    SSD_TRY(A.hdot(nu.d(), X0.d(), 3 * n, &h)); g0 += h;
    SSD_TRY(A.hdot(nu.d(), X1.d(), 3 * n, &h)); g1 += h;
    if (geo) {
        // alpha = A_D^{-T} P_g^T (g_p + N^T M^T nu), p~ = the Darcy solution before its gauge projection
        Buf mtnu, al, pt, gp2, b3, t1;
        SSD_TRY(t1.alloc(ctx, sizeof(double) * n));
        SSD_TRY(mtnu.alloc(ctx, sizeof(double) * 3 * n));
        SSD_TRY(al.alloc(ctx, sizeof(double) * n));
        SSD_TRY(pt.alloc(ctx, sizeof(double) * n));
        SSD_TRY(gp2.alloc(ctx, sizeof(double) * n));
        SSD_TRY(b3.alloc(ctx, sizeof(double) * 3 * n));
        SSD_TRY(A.apply(OP_SSL, true, nu.d(), mtnu.d()));
        dot_normal_kernel<<<grid_for(n), 256, 0, s>>>(n, mtnu.d(), pts->nrm, gp2.d());
        ctx->launches++;
        double sg = 0.0;
        if (functional == SSD_FUNC_DRAG) {
            weight_field_kernel<<<grid_for(n), 256, 0, s>>>(n, pts->w, pts->xyz, pts->nrm, e0, e1, e2, 1, t1.d());
            axpby_kernel<<<grid_for(n), 256, 0, s>>>(n, 1.0, t1.d(), 1.0, gp2.d());
            ctx->launches += 2;
            SSD_TRY(A.sum(t1.d(), A.scal.d() + 6));
            SSD_TRY(read_scalars(ctx, A.scal.d() + 6, 1, &sg, s));
        }
        double S3 = 0.0;
        SSD_TRY(A.hdot(mtnu.d(), pts->nrm, 3 * n, &S3));
        SSD_TRY(A.PgT(gp2.d()));
        SSD_TRY(A.solveAdT(gp2.d(), al.d()));
        GmresResult rd;
        int sd = darcy_solve_impl(ctx, pts, *lref.L, prm->delta, prm->mu, prm->kappa, q.d(), pt.d(), prm->inner, &rd,
                                  s, false);
        if (sd == SSD_ENOTCONV) A.nonconv++;
        else SSD_TRY(sd);
        double sa = 0.0, S1 = 0.0, S2 = 0.0;
        SSD_TRY(A.sum(al.d(), A.scal.d() + 6));
        SSD_TRY(read_scalars(ctx, A.scal.d() + 6, 1, &sa, s));
        SSD_TRY(A.hdot(nu.d(), pts->nrm, 3 * n, &S1));
        scal_normal_kernel<<<grid_for(n), 256, 0, s>>>(n, pts->w, pts->nrm, t3.d());
        ctx->launches++;
        SSD_TRY(A.hdot(t3.d(), u.d(), 3 * n, &S2));
        GeoPoint gpk;
        gpk.n = n; gpk.xyz = pts->xyz; gpk.nrm = pts->nrm; gpk.w = pts->w; gpk.u = u.d(); gpk.p = p.d();
        gpk.q = q.d(); gpk.lam = lam.d(); gpk.nu = nu.d(); gpk.mtnu = mtnu.d();
        gpk.c = A.c; gpk.W = lref.L->wsum; gpk.S1 = S1; gpk.S2 = S2; gpk.S3 = S3; gpk.sa = sa; gpk.sg = sg;
        gpk.e[0] = e0; gpk.e[1] = e1; gpk.e[2] = e2;
        gpk.deflate = prm->inner.deflate; gpk.functional = functional;
        gpk.gx = geo_x; gpk.gn = geo_n; gpk.gw = geo_w;
        geo_point_kernel<<<grid_for(n), 256, 0, s>>>(gpk);
        ctx->launches++;
        SSD_TRY(launch_check(ctx, "geometry point terms"));
        // pair terms: (mu/kappa) B_L(alpha, q) + B_DL(alpha, p~) + B_M(nu, n p - c P u) + B_DS(nu, u)
        SSD_TRY(geometry_gradient(ctx, pts, OP_LSL, prm->delta, prm->mu, prm->mu / prm->kappa, al.d(), q.d(), geo_x,
                                  geo_n, geo_w, s));
        SSD_TRY(geometry_gradient(ctx, pts, OP_LDL, prm->delta, prm->mu, 1.0, al.d(), pt.d(), geo_x, geo_n, geo_w,
                                  s));
        scal_normal_kernel<<<grid_for(n), 256, 0, s>>>(n, p.d(), pts->nrm, b3.d());
        ctx->launches++;
        if (A.c != 0.0) {
            axpby_kernel<<<grid_for(3 * n), 256, 0, s>>>(3 * n, -A.c, pu.d(), 1.0, b3.d());
            ctx->launches++;
        }
        SSD_TRY(geometry_gradient(ctx, pts, OP_SSL, prm->delta, prm->mu, 1.0, nu.d(), b3.d(), geo_x, geo_n, geo_w,
                                  s));
        SSD_TRY(geometry_gradient(ctx, pts, OP_SDL, prm->delta, prm->mu, 1.0, nu.d(), u.d(), geo_x, geo_n, geo_w,
                                  s));
        SSD_TRY(cuda_check(ctx, cudaStreamSynchronize(s), "geometry sync"));
    }
    if (value) *value = val;
    grad[0] = g0;
    grad[1] = g1;
    if (A.nonconv && status == SSD_OK) status = set_error(ctx, SSD_ENOTCONV, "iteration limit reached in an adjoint solve");
    return status;
}

int op_entry(ssd_ctx *ctx, const ssd_points *pts, const PairCall &pc, cudaStream_t s) {
    if (!finite_pos(pc.delta)) return set_error(ctx, SSD_EINVAL, "delta must be positive and finite");
    if (!finite_pos(pc.mu)) return set_error(ctx, SSD_EINVAL, "mu must be positive and finite");
    if (!isfinite(pc.alpha) || !isfinite(pc.beta)) return set_error(ctx, SSD_EINVAL, "non-finite alpha or beta");
    if (pc.prec != SSD_FP64 && pc.prec != SSD_FP32C) return set_error(ctx, SSD_EINVAL, "unknown precision");
    if (!pc.dens0 || !pc.out) return set_error(ctx, SSD_EINVAL, "NULL density or output");
    LayoutRef lref;
    SSD_TRY(get_layout(ctx, pts, &lref, s));
    return pair_apply(ctx, *lref.L, pc, s);
}

}  // namespace

int dot(ssd_ctx *ctx, const double *a, const double *b, int64_t n, double *dev_out, cudaStream_t s) {
    Dots d;
    SSD_TRY(d.init(ctx, s, 1));
    return d.multi(a, 0, 1, b, n, dev_out);
}

}  // namespace ssd

using namespace ssd;

extern "C" {

int ssd_laplace_SL(ssd_ctx *ctx, const ssd_points *pts, double delta, const double *g, double *out, int prec,
                   ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    PairCall pc;
    pc.op = OP_LSL; pc.prec = prec; pc.delta = delta; pc.dens0 = g; pc.out = out;
    return op_entry(ctx, pts, pc, (cudaStream_t)stream);
}

int ssd_laplace_DL(ssd_ctx *ctx, const ssd_points *pts, double delta, const double *p, double *out, int prec,
                   ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    PairCall pc;
    pc.op = OP_LDL; pc.prec = prec; pc.delta = delta; pc.dens0 = p; pc.out = out;
    return op_entry(ctx, pts, pc, (cudaStream_t)stream);
}

int ssd_stokes_SL(ssd_ctx *ctx, const ssd_points *pts, double delta, double mu, const double *f, double *out,
                  int prec, ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    PairCall pc;
    pc.op = OP_SSL; pc.prec = prec; pc.delta = delta; pc.mu = mu; pc.dens0 = f; pc.out = out;
    return op_entry(ctx, pts, pc, (cudaStream_t)stream);
}

int ssd_stokes_DL(ssd_ctx *ctx, const ssd_points *pts, double delta, const double *u, double *out, int prec,
                  ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    PairCall pc;
    pc.op = OP_SDL; pc.prec = prec; pc.delta = delta; pc.dens0 = u; pc.out = out;
    return op_entry(ctx, pts, pc, (cudaStream_t)stream);
}

int ssd_apply_rows(ssd_ctx *ctx, const ssd_points *pts, int op, double delta, double mu, const double *dens,
                   int64_t row_begin, int64_t row_end, double *out, int prec, ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    ctx->err.clear();
    if (op < OP_LSL || op > OP_SDL) return set_error(ctx, SSD_EINVAL, "op must be one of the four layer operators");
    if (!pts || row_begin < 0 || row_end <= row_begin || row_end > pts->n)
        return set_error(ctx, SSD_EINVAL, "row block must satisfy 0 <= row_begin < row_end <= n");
    PairCall pc;
    pc.op = op; pc.prec = prec; pc.delta = delta; pc.mu = mu; pc.dens0 = dens; pc.out = out;
    pc.row_begin = row_begin; pc.row_end = row_end;
    return op_entry(ctx, pts, pc, (cudaStream_t)stream);
}

int ssd_points_order(ssd_ctx *ctx, const ssd_points *pts, int32_t *order, ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    ctx->err.clear();
    if (!order) return set_error(ctx, SSD_EINVAL, "NULL output");
    SSD_TRY(check_points(ctx, pts));
    cudaStream_t s = (cudaStream_t)stream;
    LayoutRef lref;
    SSD_TRY(get_layout(ctx, pts, &lref, s));
    SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(order, lref.L->perm, sizeof(int32_t) * pts->n, cudaMemcpyDeviceToHost, s),
                       "order copy"));
    return cuda_check(ctx, cudaStreamSynchronize(s), "order sync");
}

int ssd_stokes_SLDL(ssd_ctx *ctx, const ssd_points *pts, double delta, double mu, const double *f, const double *u,
                    double alpha, double beta, double *out, int prec, ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    if (!f) return set_error(ctx, SSD_EINVAL, "NULL traction");
    PairCall pc;
    pc.op = OP_SSLDL; pc.prec = prec; pc.delta = delta; pc.mu = mu; pc.dens0 = u; pc.dens1 = f;
    pc.alpha = alpha; pc.beta = beta; pc.out = out;
    return op_entry(ctx, pts, pc, (cudaStream_t)stream);
}

int ssd_laplace_SLDL(ssd_ctx *ctx, const ssd_points *pts, double delta, const double *g, const double *p,
                     double alpha, double beta, double *out, int prec, ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    if (!g) return set_error(ctx, SSD_EINVAL, "NULL single-layer density");
    PairCall pc;
    pc.op = OP_LSLDL; pc.prec = prec; pc.delta = delta; pc.dens0 = p; pc.dens1 = g;
    pc.alpha = alpha; pc.beta = beta; pc.out = out;
    return op_entry(ctx, pts, pc, (cudaStream_t)stream);
}

int ssd_apply_transpose(ssd_ctx *ctx, const ssd_points *pts, int op, double delta, double mu, const double *dens,
                        double *out, int prec, ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    PairCall pc;
    switch (op) {
        case SSD_OP_LAPLACE_SL: pc.op = OP_LSL; pc.transpose_sl = true; break;
        case SSD_OP_LAPLACE_DL: pc.op = OP_LDLT; break;
        case SSD_OP_STOKES_SL: pc.op = OP_SSL; pc.transpose_sl = true; break;
        case SSD_OP_STOKES_DL: pc.op = OP_SDLT; break;
        default: return set_error(ctx, SSD_EINVAL, "transpose: op must be a single or double layer");
    }
    pc.prec = prec; pc.delta = delta; pc.mu = mu; pc.dens0 = dens; pc.out = out;
    return op_entry(ctx, pts, pc, (cudaStream_t)stream);
}

int ssd_darcy_solve(ssd_ctx *ctx, const ssd_points *pts, double delta, double mu, double kappa, const double *q,
                    double *p_out, const ssd_krylov *kr, int *iters, double *relres, ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    ctx->err.clear();
    if (!finite_pos(delta) || !finite_pos(mu) || !finite_pos(kappa))
        return set_error(ctx, SSD_EINVAL, "delta, mu and kappa must be positive");
    if (!q || !p_out) return set_error(ctx, SSD_EINVAL, "NULL q or p");
    SSD_TRY(check_krylov(ctx, kr));
    cudaStream_t s = (cudaStream_t)stream;
    LayoutRef lref;
    SSD_TRY(get_layout(ctx, pts, &lref, s));
    GmresResult r;
    const int st = darcy_solve_impl(ctx, pts, *lref.L, delta, mu, kappa, q, p_out, *kr, &r, s, true, kr->warm != 0);
    if (iters) *iters = r.iters;
    if (relres) *relres = r.relres;
    if (st == SSD_OK || st == SSD_ENOTCONV) cudaStreamSynchronize(s);
    return st;
}

int ssd_stokes_solve(ssd_ctx *ctx, const ssd_points *pts, double delta, double mu, const double *f,
                     const double uinf[3], double *u_out, const ssd_krylov *kr, int *iters, double *relres,
                     ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    ctx->err.clear();
    if (!finite_pos(delta) || !finite_pos(mu)) return set_error(ctx, SSD_EINVAL, "delta and mu must be positive");
    if (!f || !u_out || !uinf) return set_error(ctx, SSD_EINVAL, "NULL f, u or uinf");
    for (int k = 0; k < 3; ++k)
        if (!isfinite(uinf[k])) return set_error(ctx, SSD_EINVAL, "non-finite far-field velocity");
    SSD_TRY(check_krylov(ctx, kr));
    cudaStream_t s = (cudaStream_t)stream;
    LayoutRef lref;
    SSD_TRY(get_layout(ctx, pts, &lref, s));
    GmresResult r;
    const int st = stokes_solve_impl(ctx, pts, *lref.L, delta, mu, f, uinf, u_out, *kr, &r, s, kr->warm != 0);
    if (iters) *iters = r.iters;
    if (relres) *relres = r.relres;
    if (st == SSD_OK || st == SSD_ENOTCONV) cudaStreamSynchronize(s);
    return st;
}

int ssd_ddm_solve(ssd_ctx *ctx, const ssd_points *pts, const ssd_ddm_params *prm, double *q, double *p_D,
                  double *u_S, double *f_S, double drag[3], int *outer_its, int *inner_its, double *res_hist,
                  ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    ctx->err.clear();
    return ddm_impl(ctx, pts, prm, q, p_D, u_S, f_S, drag, outer_its, inner_its, res_hist, (cudaStream_t)stream);
}

int ssd_ddm_sweep(ssd_ctx *ctx, const ssd_points *pts, const ssd_ddm_params *prm, const double *q,
                  const double *u_prev, double *q_out, double *p_D, double *u_S, double *f_S, int inner_its[2],
                  ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    ctx->err.clear();
    return ddm_sweep_impl(ctx, pts, prm, q, u_prev, q_out, p_D, u_S, f_S, inner_its, (cudaStream_t)stream);
}

int ssd_ddm_iteration_matrix(ssd_ctx *ctx, const ssd_points *pts, const ssd_ddm_params *prm, int64_t col0,
                             int64_t ncol, double *A, ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    ctx->err.clear();
    return ddm_iteration_matrix_impl(ctx, pts, prm, col0, ncol, A, (cudaStream_t)stream);
}

int ssd_ddm_spectrum(ssd_ctx *ctx, const ssd_points *pts, const ssd_ddm_params *prm, int m, int *m_out,
                     double *ritz_re, double *ritz_im, double *H, ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    ctx->err.clear();
    return ddm_spectrum_impl(ctx, pts, prm, m, m_out, ritz_re, ritz_im, H, (cudaStream_t)stream);
}

int ssd_hessenberg_eigenvalues(int n, const double *h, int ldh, double *wr, double *wi) {
    if (n < 1 || n > 4096 || ldh < n || !h || !wr || !wi) return SSD_EINVAL;
    try {
        std::vector<double> a((size_t)n * n, 0.0);     // entries below the subdiagonal start at 0
        for (int j = 0; j < n; ++j) {
            const int iend = j + 1 < n ? j + 1 : n - 1;
            for (int i = 0; i <= iend; ++i) {
                const double v = h[i + (size_t)j * ldh];
                if (!isfinite(v)) return SSD_EINVAL;
                a[i + (size_t)j * n] = v;
            }
        }
        return hessenberg_eigenvalues(n, a.data(), wr, wi) == 0 ? SSD_OK : SSD_ENUMERIC;
    } catch (...) {
        return SSD_ENOMEM;
    }
}

int ssd_ddm_gradient(ssd_ctx *ctx, const ssd_points *pts, const ssd_ddm_params *prm, int functional, double *value,
                     double grad[2], ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    ctx->err.clear();
    if (!grad) return set_error(ctx, SSD_EINVAL, "grad is NULL");
    return ddm_gradient_impl(ctx, pts, prm, functional, value, grad, nullptr, nullptr, nullptr, (cudaStream_t)stream);
}

int ssd_ddm_gradient_geometry(ssd_ctx *ctx, const ssd_points *pts, const ssd_ddm_params *prm, int functional,
                              double *value, double grad[2], double *gx, double *gn, double *gw, ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    ctx->err.clear();
    if (!grad) return set_error(ctx, SSD_EINVAL, "grad is NULL");
    if (!gx || !gn || !gw) return set_error(ctx, SSD_EINVAL, "geometry outputs are NULL");
    return ddm_gradient_impl(ctx, pts, prm, functional, value, grad, gx, gn, gw, (cudaStream_t)stream);
}

int ssd_geometry_gradient(ssd_ctx *ctx, const ssd_points *pts, int op, double delta, double mu, double alpha,
                          const double *a, const double *b, double *gx, double *gn, double *gw, ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    ctx->err.clear();
    SSD_TRY(check_points(ctx, pts));
    if (!(delta > 0.0) || !isfinite(delta) || !(mu > 0.0) || !isfinite(mu) || !isfinite(alpha))
        return set_error(ctx, SSD_EINVAL, "delta and mu must be positive, alpha finite");
    if (!a || !b || !gx || !gn || !gw) return set_error(ctx, SSD_EINVAL, "NULL array");
    int iop;
    switch (op) {
        case SSD_OP_LAPLACE_SL: iop = OP_LSL; break;
        case SSD_OP_LAPLACE_DL: iop = OP_LDL; break;
        case SSD_OP_STOKES_SL: iop = OP_SSL; break;
        case SSD_OP_STOKES_DL: iop = OP_SDL; break;
        default: return set_error(ctx, SSD_EINVAL, "op must be a single or double layer");
    }
    return geometry_gradient(ctx, pts, iop, delta, mu, alpha, a, b, gx, gn, gw, (cudaStream_t)stream);
}

int ssd_shape_contract(ssd_ctx *ctx, int64_t n, int ncoef, const double *dxyz, const double *dnrm, const double *dw,
                       const double *gx, const double *gn, const double *gw, double *out, ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    ctx->err.clear();
    if (n < 1 || ncoef < 1 || ncoef > 512) return set_error(ctx, SSD_EINVAL, "n >= 1 and 1 <= ncoef <= 512");
    if (!dxyz || !dnrm || !dw || !gx || !gn || !gw || !out) return set_error(ctx, SSD_EINVAL, "NULL array");
    cudaStream_t s = (cudaStream_t)stream;
    Dots dots;
    SSD_TRY(dots.init(ctx, s, ncoef));
    Buf r;
    SSD_TRY(r.alloc(ctx, sizeof(double) * 3 * ncoef));
    SSD_TRY(dots.multi(dxyz, 3 * n, ncoef, gx, 3 * n, r.d()));
    SSD_TRY(dots.multi(dnrm, 3 * n, ncoef, gn, 3 * n, r.d() + ncoef));
    SSD_TRY(dots.multi(dw, n, ncoef, gw, n, r.d() + 2 * ncoef));
    std::vector<double> h(3 * (size_t)ncoef);
    for (int part = 0; part < 3; ++part)
        SSD_TRY(read_scalars(ctx, r.d() + part * ncoef, ncoef, h.data() + part * ncoef, s));
    for (int k = 0; k < ncoef; ++k) out[k] = (h[k] + h[ncoef + k]) + h[2 * ncoef + k];
    return SSD_OK;
}

int ssd_ddm_solve_host(ssd_ctx *ctx, int64_t n, const double *xyz, const double *nrm, const double *w,
                       const ssd_ddm_params *prm, double *q, double *p_D, double *u_S, double *f_S, double drag[3],
                       int *outer_its, int *inner_its, double *res_hist, ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    ctx->err.clear();
    if (n <= 0 || !xyz || !nrm || !w) return set_error(ctx, SSD_EINVAL, "bad host point arrays");
    cudaStream_t s = (cudaStream_t)stream;
    Buf dx, dn, dw, dout;
    SSD_TRY(dx.alloc(ctx, sizeof(double) * 3 * n));
    SSD_TRY(dn.alloc(ctx, sizeof(double) * 3 * n));
    SSD_TRY(dw.alloc(ctx, sizeof(double) * n));
    SSD_TRY(dout.alloc(ctx, sizeof(double) * 8 * n));
    SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(dx.d(), xyz, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s), "h2d"));
    SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(dn.d(), nrm, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s), "h2d"));
    SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(dw.d(), w, sizeof(double) * n, cudaMemcpyHostToDevice, s), "h2d"));
    ssd_points pts;
    pts.n = n; pts.xyz = dx.d(); pts.nrm = dn.d(); pts.w = dw.d(); pts.layout = nullptr;
    SSD_TRY(ssd_points_prepare(ctx, &pts, stream));
    double *o = dout.d();
    const int st = ddm_impl(ctx, &pts, prm, o, o + n, o + 2 * n, o + 5 * n, drag, outer_its, inner_its, res_hist, s);
    ssd_points_release(ctx, &pts);
    if (st != SSD_OK && st != SSD_ENOTCONV) return st;
    if (q) SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(q, o, sizeof(double) * n, cudaMemcpyDeviceToHost, s), "d2h"));
    if (p_D) SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(p_D, o + n, sizeof(double) * n, cudaMemcpyDeviceToHost, s), "d2h"));
    if (u_S) SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(u_S, o + 2 * n, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s),
                                "d2h"));
    if (f_S) SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(f_S, o + 5 * n, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s),
                                "d2h"));
    SSD_TRY(cuda_check(ctx, cudaStreamSynchronize(s), "sync"));
    return st;
}

}  // extern "C"
