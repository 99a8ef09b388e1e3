// Batched local solves and Dirichlet-Neumann iterations over many surfaces
// and right-hand sides.  Every operator application of a sweep is one
// batched launch (pair.cu); GMRES keeps one Hessenberg matrix, rotation set
// and stopping test per system (right-hand side r, surface s), advances all
// systems together and freezes each one once it has converged.
#include <math.h>
#include <string.h>

#include <functional>
#include <vector>

#include "internal.h"

namespace ssd {
namespace {

constexpr int kSegBlock = 2048;   // elements per reduction block (within one system segment)
constexpr int kMaxM = 256;        // Krylov dimension limit

inline unsigned gridn(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > 8192) b = 8192;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// A vector of the batch: [nrhs][nc][n_total] in caller order.  System of
// element e: r * nsurf + elem_surf[e % n_total], r = e / (nc * n_total).
struct VecShape {
    int nrhs, nc, nsurf;
    int64_t n_total;
    int64_t len() const { return (int64_t)nrhs * nc * n_total; }
    int nsys() const { return nrhs * nsurf; }
};

__device__ __forceinline__ int sys_of(int64_t e, int nc, int nsurf, int64_t n_total, const int32_t *esurf) {
    const int64_t per = (int64_t)nc * n_total;
    const int r = (int)(e / per);
    return r * nsurf + esurf[e % n_total];
}

// Reduction blocks: block b covers [beg[b], end[b]) of one system; blocks of a
// system are contiguous, system k owns blocks [first[k], first[k + 1]).
struct SegTable {
    int64_t nb = 0;
    int64_t *beg = nullptr, *end = nullptr;
    int32_t *first = nullptr;
    void *block = nullptr;
};

int seg_table(ssd_ctx *ctx, const BatchLayout &B, const VecShape &v, SegTable *T, cudaStream_t s) {
    std::vector<int64_t> hb, he;
    std::vector<int32_t> hf;
    for (int r = 0; r < v.nrhs; ++r)
        for (int k = 0; k < B.nsurf; ++k) {
            hf.push_back((int32_t)hb.size());
            for (int c = 0; c < v.nc; ++c) {
                const int64_t base = ((int64_t)r * v.nc + c) * v.n_total + B.off[k];
                for (int64_t x = 0; x < B.n[k]; x += kSegBlock) {
                    hb.push_back(base + x);
                    he.push_back(base + (x + kSegBlock < B.n[k] ? x + kSegBlock : B.n[k]));
                }
            }
        }
    hf.push_back((int32_t)hb.size());
    T->nb = (int64_t)hb.size();
    size_t off = 0;
    auto carve = [&](size_t bb) { size_t o = off; off += (bb + 255) & ~size_t(255); return o; };
    const size_t o_b = carve(sizeof(int64_t) * hb.size()), o_e = carve(sizeof(int64_t) * he.size()),
                 o_f = carve(sizeof(int32_t) * hf.size());
    SSD_TRY(dev_alloc(ctx, off, &T->block));
    char *bp = static_cast<char *>(T->block);
    T->beg = reinterpret_cast<int64_t *>(bp + o_b);
    T->end = reinterpret_cast<int64_t *>(bp + o_e);
    T->first = reinterpret_cast<int32_t *>(bp + o_f);
    SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(T->beg, hb.data(), sizeof(int64_t) * hb.size(), cudaMemcpyHostToDevice, s),
                       "seg copy"));
    SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(T->end, he.data(), sizeof(int64_t) * he.size(), cudaMemcpyHostToDevice, s),
                       "seg copy"));
    SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(T->first, hf.data(), sizeof(int32_t) * hf.size(), cudaMemcpyHostToDevice, s),
                       "seg copy"));
    return cuda_check(ctx, cudaStreamSynchronize(s), "seg sync");
}

// partial[v * nb + b] = sum over block b of V[v][e] * w[e]
__global__ void bdot_kernel(const double *V, int64_t ldv, const double *w, const int64_t *beg, const int64_t *end,
                            int64_t nb, double *partial) {
    __shared__ double red[256];
    const int v = blockIdx.y;
    const int64_t b = blockIdx.x;
    const double *a = V + (int64_t)v * ldv;
    double acc = 0.0;
    for (int64_t e = beg[b] + threadIdx.x; e < end[b]; e += blockDim.x) acc += a[e] * w[e];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[(int64_t)v * nb + b] = red[0];
}

// out[k * ldo + v] = sum of the blocks of system k (fixed order)
__global__ void bdot_finish_kernel(const double *partial, int64_t nb, const int32_t *first, int nsys, int nv,
                                   double *out, int ldo) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nsys * nv) return;
    const int k = g / nv, v = g % nv;
    double acc = 0.0;
    for (int32_t b = first[k]; b < first[k + 1]; ++b) acc += partial[(int64_t)v * nb + b];
    out[(int64_t)k * ldo + v] = acc;
}

// w[e] += sign * sum_v coef[sys(e) * ldc + v] V[v][e]
__global__ void bvupdate_kernel(const double *V, int64_t ldv, int nv, const double *coef, int ldc, double sign,
                                double *w, int64_t len, int nc, int nsurf, int64_t n_total, const int32_t *esurf) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
        const double *c = coef + (int64_t)sys_of(e, nc, nsurf, n_total, esurf) * ldc;
        double acc = 0.0;
        for (int v = 0; v < nv; ++v) acc += c[v] * V[(int64_t)v * ldv + e];
        w[e] += sign * acc;
    }
}

// y[e] = x[e] / d[sys(e) * ldd] (copy where d is zero)
__global__ void bscale_inv_kernel(const double *x, const double *d, int ldd, double *y, int64_t len, int nc,
                                  int nsurf, int64_t n_total, const int32_t *esurf) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
        const double dd = d[(int64_t)sys_of(e, nc, nsurf, n_total, esurf) * ldd];
        y[e] = dd != 0.0 ? x[e] / dd : x[e];
    }
}

// y[e] -= d[sys(e)] * f
__global__ void bsub_kernel(double *y, const double *d, double f, int64_t len, int nc, int nsurf, int64_t n_total,
                            const int32_t *esurf) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x)
        y[e] -= f * d[sys_of(e, nc, nsurf, n_total, esurf)];
}

__global__ void axpby_kernel(int64_t n, double a, const double *x, double b, double *y) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        y[k] = a * x[k] + b * y[k];
}

// per-system GMRES state: H [m+1][m] column-major, cs, sn, g, bnorm, k, active
struct SysState {
    double *H, *cs, *sn, *g, *bnorm, *h1, *h2, *nrm, *y, *resid;
    int32_t *k, *active, *nactive;
};

__global__ void binit_kernel(SysState S, int nsys, int m, double tol) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nsys) return;
    const double b = sqrt(fmax(S.nrm[q], 0.0));   // nrm holds ||b||^2 here
    S.bnorm[q] = b;
    for (int i = 0; i <= m; ++i) S.g[(int64_t)q * (m + 1) + i] = 0.0;
    S.g[(int64_t)q * (m + 1)] = b;
    S.nrm[q] = b;
    S.k[q] = 0;
    S.active[q] = (b > 0.0 && isfinite(b)) ? 1 : 0;
    S.resid[q] = b > 0.0 ? 1.0 : 0.0;
}

__global__ void bgivens_kernel(SysState S, int nsys, int m, int j, double tol) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nsys) return;
    const int ldh = m + 1;
    const double hn = sqrt(fmax(S.nrm[q], 0.0));
    S.nrm[q] = hn;
    if (!S.active[q]) return;
    double *col = S.H + ((int64_t)q * m + j) * ldh;
    double *cs = S.cs + (int64_t)q * m, *sn = S.sn + (int64_t)q * m, *g = S.g + (int64_t)q * (m + 1);
    const double *h1 = S.h1 + (int64_t)q * (m + 2), *h2 = S.h2 + (int64_t)q * (m + 2);
    for (int i = 0; i <= j; ++i) col[i] = h1[i] + h2[i];
    col[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
        const double t = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = t;
    }
    const double den = hypot(col[j], col[j + 1]);
    cs[j] = den == 0.0 ? 1.0 : col[j] / den;
    sn[j] = den == 0.0 ? 0.0 : col[j + 1] / den;
    col[j] = den;
    col[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    const double rel = fabs(g[j + 1]) / S.bnorm[q];
    S.resid[q] = rel;
    S.k[q] = j + 1;
    if (!(rel > tol) || hn == 0.0 || !isfinite(rel)) S.active[q] = 0;
    else atomicAdd(S.nactive, 1);
}

__global__ void bbacksolve_kernel(SysState S, int nsys, int m) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nsys) return;
    const int ldh = m + 1, k = S.k[q];
    const double *H = S.H + (int64_t)q * m * ldh, *g = S.g + (int64_t)q * (m + 1);
    double *y = S.y + (int64_t)q * (m + 2);
    for (int i = 0; i < m + 2; ++i) y[i] = 0.0;
    for (int i = k - 1; i >= 0; --i) {
        double s = g[i];
        for (int l = i + 1; l < k; ++l) s -= H[(int64_t)l * ldh + i] * y[l];
        y[i] = s / H[(int64_t)i * ldh + i];
    }
}

struct Buf {
    ssd_ctx *ctx = nullptr;
    void *p = nullptr;
    Buf() {}
    Buf(const Buf &) = delete;
    Buf &operator=(const Buf &) = delete;
    ~Buf() { if (ctx) dev_free(ctx, p); }
    int alloc(ssd_ctx *c, size_t bytes) { ctx = c; return dev_alloc(c, bytes, &p); }
    double *d() const { return static_cast<double *>(p); }
};

typedef std::function<int(const double *, double *)> BMatVec;

struct BResult {
    std::vector<int> iters;
    std::vector<double> relres;
};

// Per-system GMRES, one Krylov cycle of at most m steps, x0 = 0.
int bgmres(ssd_ctx *ctx, cudaStream_t s, const BatchLayout &B, const VecShape &v, const BMatVec &A,
           const double *b, double *x, double tol, int m, BResult *res) {
    const int64_t len = v.len();
    const int nsys = v.nsys();
    SegTable T;
    SSD_TRY(seg_table(ctx, B, v, &T, s));
    struct TRel { ssd_ctx *c; void *p; ~TRel() { dev_free(c, p); } } trel{ctx, T.block};
    Buf V, w, part, st;
    SSD_TRY(V.alloc(ctx, sizeof(double) * (size_t)(m + 1) * len));
    SSD_TRY(w.alloc(ctx, sizeof(double) * len));
    SSD_TRY(part.alloc(ctx, sizeof(double) * T.nb * (m + 2)));
    const int ldh = m + 1;
    const size_t nst = (size_t)nsys * ((size_t)ldh * m + 2 * m + (m + 1) + 3 * (m + 2) + 4) + 8;
    SSD_TRY(st.alloc(ctx, sizeof(double) * nst + sizeof(int32_t) * (3 * nsys + 8)));
    SysState S;
    double *p = st.d();
    S.H = p; p += (size_t)nsys * ldh * m;
    S.cs = p; p += (size_t)nsys * m;
    S.sn = p; p += (size_t)nsys * m;
    S.g = p; p += (size_t)nsys * (m + 1);
    S.h1 = p; p += (size_t)nsys * (m + 2);
    S.h2 = p; p += (size_t)nsys * (m + 2);
    S.y = p; p += (size_t)nsys * (m + 2);
    S.bnorm = p; p += nsys;
    S.nrm = p; p += nsys;
    S.resid = p; p += nsys;
    p += nsys;
    int32_t *ip = reinterpret_cast<int32_t *>(p + 8);
    S.k = ip; S.active = ip + nsys; S.nactive = ip + 2 * nsys;
    const unsigned sb = (unsigned)((nsys + 127) / 128);
    auto dots = [&](const double *VV, int64_t ldv, int nv, const double *ww, double *out, int ldo) -> int {
        bdot_kernel<<<dim3((unsigned)T.nb, (unsigned)nv), 256, 0, s>>>(VV, ldv, ww, T.beg, T.end, T.nb, part.d());
        bdot_finish_kernel<<<(unsigned)((nsys * nv + 127) / 128), 128, 0, s>>>(part.d(), T.nb, T.first, nsys, nv, out,
                                                                               ldo);
        ctx->launches += 2;
        return launch_check(ctx, "batched dots");
    };
    // V0 = b / ||b|| per system
    SSD_TRY(dots(b, 0, 1, b, S.nrm, 1));
    binit_kernel<<<sb, 128, 0, s>>>(S, nsys, m, tol);
    bscale_inv_kernel<<<gridn(len), 256, 0, s>>>(b, S.nrm, 1, V.d(), len, v.nc, v.nsurf, v.n_total, B.elem_surf);
    ctx->launches += 2;
    SSD_TRY(cuda_check(ctx, cudaMemsetAsync(x, 0, sizeof(double) * len, s), "memset"));
    int j = 0;
    for (j = 0; j < m; ++j) {
        double *vj = V.d() + (size_t)j * len;
        SSD_TRY(A(vj, w.d()));
        SSD_TRY(dots(V.d(), len, j + 1, w.d(), S.h1, m + 2));
        bvupdate_kernel<<<gridn(len), 256, 0, s>>>(V.d(), len, j + 1, S.h1, m + 2, -1.0, w.d(), len, v.nc, v.nsurf,
                                                   v.n_total, B.elem_surf);
        ctx->launches++;
        SSD_TRY(dots(V.d(), len, j + 1, w.d(), S.h2, m + 2));
        bvupdate_kernel<<<gridn(len), 256, 0, s>>>(V.d(), len, j + 1, S.h2, m + 2, -1.0, w.d(), len, v.nc, v.nsurf,
                                                   v.n_total, B.elem_surf);
        ctx->launches++;
        SSD_TRY(dots(w.d(), 0, 1, w.d(), S.nrm, 1));
        SSD_TRY(cuda_check(ctx, cudaMemsetAsync(S.nactive, 0, sizeof(int32_t), s), "memset"));
        bgivens_kernel<<<sb, 128, 0, s>>>(S, nsys, m, j, tol);   // also turns nrm into ||w||
        ctx->launches++;
        SSD_TRY(launch_check(ctx, "batched arnoldi"));
        // next basis vector w / ||w|| per system
        bscale_inv_kernel<<<gridn(len), 256, 0, s>>>(w.d(), S.nrm, 1, V.d() + (size_t)(j + 1) * len, len, v.nc,
                                                     v.nsurf, v.n_total, B.elem_surf);
        ctx->launches++;
        int32_t nact = 0;
        SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(ctx->hbuf, S.nactive, sizeof(int32_t), cudaMemcpyDeviceToHost, s),
                           "active copy"));
        SSD_TRY(cuda_check(ctx, cudaStreamSynchronize(s), "sync"));
        memcpy(&nact, ctx->hbuf, sizeof(int32_t));
        if (nact == 0) { ++j; break; }
    }
    // j Arnoldi steps ran: basis vectors 0..j-1 enter the update (y is zero
    // beyond each system's own step count)
    bbacksolve_kernel<<<sb, 128, 0, s>>>(S, nsys, m);
    bvupdate_kernel<<<gridn(len), 256, 0, s>>>(V.d(), len, j, S.y, m + 2, 1.0, x, len, v.nc, v.nsurf, v.n_total,
                                               B.elem_surf);
    ctx->launches += 2;
    SSD_TRY(launch_check(ctx, "batched gmres update"));
    std::vector<int32_t> hk(nsys);
    res->relres.assign(nsys, 0.0);
    res->iters.assign(nsys, 0);
    SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(res->relres.data(), S.resid, sizeof(double) * nsys, cudaMemcpyDeviceToHost, s),
                       "resid copy"));
    SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(hk.data(), S.k, sizeof(int32_t) * nsys, cudaMemcpyDeviceToHost, s),
                       "k copy"));
    SSD_TRY(cuda_check(ctx, cudaStreamSynchronize(s), "sync"));
    bool ok = true;
    for (int q = 0; q < nsys; ++q) {
        res->iters[q] = hk[q];
        if (!isfinite(res->relres[q])) return set_error(ctx, SSD_ENUMERIC, "non-finite residual in a batched solve");
        if (res->relres[q] > tol) ok = false;
    }
    return ok ? SSD_OK : SSD_ENOTCONV;
}

}  // namespace
}  // namespace ssd

namespace ssd {
namespace {

// ------------------------------------------------------ batched sweep kernels
struct RhsVec {
    double v[kMaxRhs][3];
};

// q_new = (1 - theta) q + theta u . n, per right-hand side
__global__ void bq_update_kernel(int64_t n, int nrhs, double theta, const double *q, const double *u,
                                 const double *nrm, double *qn) {
    const int64_t len = (int64_t)nrhs * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / n, o = e % n;
        const double *ur = u + r * 3 * n;
        const double un = ur[o] * nrm[o] + ur[n + o] * nrm[n + o] + ur[2 * n + o] * nrm[2 * n + o];
        qn[e] = (1.0 - theta) * q[e] + theta * un;
    }
}

// BJS traction f = -p n + coef (u - (u.n) n) (u may be NULL)
__global__ void btraction_bjs_kernel(int64_t n, int nrhs, const double *p, const double *u, const double *nrm,
                                     double coef, double *f) {
    const int64_t len = (int64_t)nrhs * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / n, o = e % n;
        const double n0 = nrm[o], n1 = nrm[n + o], n2 = nrm[2 * n + o];
        double u0 = 0, u1 = 0, u2 = 0;
        if (u) { const double *ur = u + r * 3 * n; u0 = ur[o]; u1 = ur[n + o]; u2 = ur[2 * n + o]; }
        const double un = u0 * n0 + u1 * n1 + u2 * n2;
        double *fr = f + r * 3 * n;
        fr[o] = -p[e] * n0 + coef * (u0 - un * n0);
        fr[n + o] = -p[e] * n1 + coef * (u1 - un * n1);
        fr[2 * n + o] = -p[e] * n2 + coef * (u2 - un * n2);
    }
}

// porous-sphere benchmark traction (Section 7.3) per right-hand side: flow
// direction e_r = uinf_r / |uinf_r|, speed |uinf_r|
__global__ void btraction_jt_kernel(int64_t n, int nrhs, const double *p, const double *xyz, double R, double kappa,
                                    double mu, const RhsVec dir, const double *speed, double *f) {
    const int64_t len = (int64_t)nrhs * n;
    const double c = 2.0 + kappa / (R * R);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / n);
        const int64_t o = e % n;
        const double U = speed[r];
        const double e0 = dir.v[r][0], e1 = dir.v[r][1], e2 = dir.v[r][2];
        const double bcoef = -(3.0 * mu * U / (R * c)) * (1.0 + 2.0 * kappa / (R * R));
        const double x = xyz[o], y = xyz[n + o], z = xyz[2 * n + o];
        const double rr = sqrt(x * x + y * y + z * z);
        const double er0 = x / rr, er1 = y / rr, er2 = z / rr;
        const double ct = (e0 * x + e1 * y + e2 * z) / rr;
        const double a = -12.0 * mu * U * kappa * ct / (R * R * R * c);
        const double fr = -p[e] + a;
        double *f_r = f + (int64_t)r * 3 * n;
        f_r[o] = fr * er0 + bcoef * (ct * er0 - e0);
        f_r[n + o] = fr * er1 + bcoef * (ct * er1 - e1);
        f_r[2 * n + o] = fr * er2 + bcoef * (ct * er2 - e2);
    }
}

// pn = p n per right-hand side
__global__ void bpn_kernel(int64_t n, int nrhs, const double *p, const double *nrm, double *pn) {
    const int64_t len = (int64_t)nrhs * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / n, o = e % n;
        for (int k = 0; k < 3; ++k) pn[(r * 3 + k) * n + o] = p[e] * nrm[k * n + o];
    }
}

// tangential part u - (u.n) n per right-hand side
__global__ void btangential_kernel(int64_t n, int nrhs, const double *u, const double *nrm, double *t) {
    const int64_t len = (int64_t)nrhs * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / n, o = e % n;
        const double *ur = u + r * 3 * n;
        const double un = ur[o] * nrm[o] + ur[n + o] * nrm[n + o] + ur[2 * n + o] * nrm[2 * n + o];
        for (int k = 0; k < 3; ++k) t[(r * 3 + k) * n + o] = ur[k * n + o] - un * nrm[k * n + o];
    }
}

// out[(r * nsurf + s) * 3 + c] = sum over surface s of w f_c (right-hand side r), one block each
__global__ void bdrag_kernel(const double *f, const double *w, const int64_t *off, int nsurf, int64_t n, double *out) {
    __shared__ double red[256];
    const int g = blockIdx.x;              // (r * nsurf + s) * 3 + c
    const int c = g % 3, sys = g / 3;
    const int r = sys / nsurf, sidx = sys % nsurf;
    const double *fr = f + ((int64_t)r * 3 + c) * n;
    double acc = 0.0;
    for (int64_t o = off[sidx] + threadIdx.x; o < off[sidx + 1]; o += blockDim.x) acc += w[o] * fr[o];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[g] = red[0];
}

// weights repeated for every right-hand side: wrep[r][o] = w[o]
__global__ void brepeat_kernel(const double *w, int64_t n, int nrhs, double *wrep) {
    const int64_t len = (int64_t)nrhs * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x)
        wrep[e] = w[e % n];
}

struct BDdm {
    ssd_ctx *ctx;
    const ssd_batch *b;
    const BatchLayout *B;
    ssd_ddm_params P;
    cudaStream_t s;
    int nrhs;
    int64_t n;
    double uinf[kMaxRhs][3];
    Buf f, tmp, pn, wrep, mean, speed;
    SegTable T1;   // scalar segments (for the Darcy gauge)
    int nonconv = 0;
    std::vector<int> inner_max;

    int darcy(const double *q, double *p) {
        const VecShape v{nrhs, 1, B->nsurf, n};
        BatchCall bc;
        bc.nrhs = nrhs;
        bc.pc.op = OP_LSL; bc.pc.prec = P.inner.prec; bc.pc.dens0 = q; bc.pc.a_op = P.mu / P.kappa;
        bc.pc.out = tmp.d();
        SSD_TRY(pair_apply_batch(ctx, *B, bc, s));
        auto A = [&](const double *x, double *y) -> int {
            BatchCall a;
            a.nrhs = nrhs;
            a.pc.op = OP_LDL; a.pc.prec = P.inner.prec; a.pc.dens0 = x; a.pc.a_op = -1.0;
            a.pc.rank1_weight_mean = true; a.pc.out = y;
            return pair_apply_batch(ctx, *B, a, s);
        };
        BResult r;
        int st = bgmres(ctx, s, *B, v, A, tmp.d(), p, P.inner.tol, P.inner.restart, &r);
        if (st == SSD_ENOTCONV) { nonconv++; st = SSD_OK; }
        SSD_TRY(st);
        track(r);
        // zero weighted mean per system
        bdot_kernel<<<dim3((unsigned)T1.nb, 1), 256, 0, s>>>(p, 0, wrep.d(), T1.beg, T1.end, T1.nb, pn.d());
        bdot_finish_kernel<<<(unsigned)((v.nsys() + 127) / 128), 128, 0, s>>>(pn.d(), T1.nb, T1.first, v.nsys(), 1,
                                                                               mean.d(), 1);
        ctx->launches += 2;
        // mean = (w . p)_sys / W_s: divide per system on the host-known sums
        std::vector<double> hm(v.nsys());
        SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(hm.data(), mean.d(), sizeof(double) * v.nsys(), cudaMemcpyDeviceToHost, s),
                           "mean copy"));
        SSD_TRY(cuda_check(ctx, cudaStreamSynchronize(s), "sync"));
        for (int r2 = 0; r2 < nrhs; ++r2)
            for (int k = 0; k < B->nsurf; ++k) hm[r2 * B->nsurf + k] /= B->wsum[k];
        SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(mean.d(), hm.data(), sizeof(double) * v.nsys(), cudaMemcpyHostToDevice, s),
                           "mean copy"));
        bsub_kernel<<<gridn(v.len()), 256, 0, s>>>(p, mean.d(), 1.0, v.len(), 1, B->nsurf, n, B->elem_surf);
        ctx->launches++;
        SSD_TRY(cuda_check(ctx, cudaStreamSynchronize(s), "sync"));
        return launch_check(ctx, "batched darcy gauge");
    }

    void track(const BResult &r) {
        int mx = 0;
        for (int k : r.iters) mx = k > mx ? k : mx;
        inner_max.push_back(mx);
    }

    int stokes(const double *p, const double *uprev, double *u) {
        const VecShape v{nrhs, 3, B->nsurf, n};
        const bool implicit = P.traction_mode == SSD_TRACTION_BJS && P.bjs_implicit;
        const double coef = P.bjs_sign * P.gamma / sqrt(P.kappa);
        BatchCall bc;
        bc.nrhs = nrhs;
        for (int r = 0; r < nrhs; ++r)
            for (int k = 0; k < 3; ++k) bc.add[r][k] = uinf[r][k];
        bc.pc.prec = P.inner.prec; bc.pc.mu = P.mu; bc.pc.out = tmp.d();
        if (implicit) {
            // (I - D^S) u + c M(P u) = U_inf + M(p n)
            bpn_kernel<<<gridn((int64_t)nrhs * n), 256, 0, s>>>(n, nrhs, p, b->nrm, pn.d());
            ctx->launches++;
            bc.pc.op = OP_SSL; bc.pc.dens0 = pn.d(); bc.pc.a_op = 1.0;
        } else {
            if (P.traction_mode == SSD_TRACTION_BJS) {
                btraction_bjs_kernel<<<gridn((int64_t)nrhs * n), 256, 0, s>>>(n, nrhs, p, nullptr, b->nrm, coef, f.d());
            } else {
                RhsVec dir;
                std::vector<double> sp(nrhs);
                for (int r = 0; r < nrhs; ++r) {
                    const double U = sqrt(uinf[r][0] * uinf[r][0] + uinf[r][1] * uinf[r][1] + uinf[r][2] * uinf[r][2]);
                    sp[r] = U;
                    for (int k = 0; k < 3; ++k) dir.v[r][k] = U > 0 ? uinf[r][k] / U : (k == 2 ? 1.0 : 0.0);
                }
                SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(speed.d(), sp.data(), sizeof(double) * nrhs,
                                                        cudaMemcpyHostToDevice, s), "speed copy"));
                btraction_jt_kernel<<<gridn((int64_t)nrhs * n), 256, 0, s>>>(n, nrhs, p, b->xyz, P.radius, P.kappa,
                                                                             P.mu, dir, speed.d(), f.d());
                SSD_TRY(cuda_check(ctx, cudaStreamSynchronize(s), "sync"));
            }
            ctx->launches++;
            bc.pc.op = OP_SSL; bc.pc.dens0 = f.d(); bc.pc.a_op = -1.0;
        }
        SSD_TRY(pair_apply_batch(ctx, *B, bc, s));
        Buf t2;
        if (implicit) SSD_TRY(t2.alloc(ctx, sizeof(double) * v.len()));
        auto A = [&](const double *x, double *y) -> int {
            BatchCall a;
            a.nrhs = nrhs;
            a.pc.prec = P.inner.prec; a.pc.mu = P.mu; a.pc.xin = x; a.pc.a_id = 1.0; a.pc.out = y;
            a.pc.rank1_nrm = P.inner.deflate ? b->nrm : nullptr;
            if (implicit) {
                btangential_kernel<<<gridn((int64_t)nrhs * n), 256, 0, s>>>(n, nrhs, x, b->nrm, t2.d());
                ctx->launches++;
                a.pc.op = OP_SSLDL; a.pc.dens0 = x; a.pc.dens1 = t2.d(); a.pc.alpha = coef; a.pc.beta = -1.0;
                a.pc.a_op = 1.0;
            } else {
                a.pc.op = OP_SDL; a.pc.dens0 = x; a.pc.a_op = -1.0;
            }
            return pair_apply_batch(ctx, *B, a, s);
        };
        BResult r;
        int st = bgmres(ctx, s, *B, v, A, tmp.d(), u, P.inner.tol, P.inner.restart, &r);
        if (st == SSD_ENOTCONV) { nonconv++; st = SSD_OK; }
        SSD_TRY(st);
        track(r);
        if (implicit) {
            btraction_bjs_kernel<<<gridn((int64_t)nrhs * n), 256, 0, s>>>(n, nrhs, p, u, b->nrm, coef, f.d());
            ctx->launches++;
        }
        (void)uprev;
        return launch_check(ctx, "batched stokes");
    }

    int sweep(const double *q, double *qn, double *u, double *p) {
        SSD_TRY(darcy(q, p));
        SSD_TRY(stokes(p, nullptr, u));
        bq_update_kernel<<<gridn((int64_t)nrhs * n), 256, 0, s>>>(n, nrhs, P.theta, q, u, b->nrm, qn);
        ctx->launches++;
        return launch_check(ctx, "batched q update");
    }
};

int check_batch(ssd_ctx *ctx, const ssd_batch *b) {
    if (!b) return set_error(ctx, SSD_EINVAL, "batch is NULL");
    if (!b->layout) return set_error(ctx, SSD_EINVAL, "batch has no layout (call ssd_batch_prepare)");
    return SSD_OK;
}

}  // namespace
}  // namespace ssd

using namespace ssd;

extern "C" {

int ssd_batch_apply(ssd_ctx *ctx, const ssd_batch *b, int op, int nrhs, double mu, double alpha, double beta,
                    const double *dens0, const double *dens1, double *out, int prec, ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    SSD_TRY(check_batch(ctx, b));
    if (op < 0 || op > 5) return set_error(ctx, SSD_EINVAL, "unknown operator");
    if (nrhs < 1 || nrhs > kMaxRhs) return set_error(ctx, SSD_EINVAL, "nrhs must be in 1..16");
    if (!(mu > 0.0) || !isfinite(mu) || !isfinite(alpha) || !isfinite(beta))
        return set_error(ctx, SSD_EINVAL, "bad mu, alpha or beta");
    if (prec != SSD_FP64 && prec != SSD_FP32C) return set_error(ctx, SSD_EINVAL, "unknown precision");
    if (!dens0 || !out || ((op == OP_SSLDL || op == OP_LSLDL) && !dens1))
        return set_error(ctx, SSD_EINVAL, "NULL density or output");
    BatchCall bc;
    bc.nrhs = nrhs;
    bc.pc.op = op; bc.pc.prec = prec; bc.pc.mu = mu; bc.pc.alpha = alpha; bc.pc.beta = beta;
    bc.pc.dens0 = dens0; bc.pc.dens1 = dens1; bc.pc.out = out;
    return pair_apply_batch(ctx, b->layout->B, bc, (cudaStream_t)stream);
}

int ssd_batch_ddm_solve(ssd_ctx *ctx, const ssd_batch *b, const ssd_ddm_params *prm, int nrhs, const double *uinf,
                        double *q, double *p_D, double *u_S, double *f_S, double *drag, int *outer_its,
                        double *relres, ssd_stream stream) {
    if (!ctx) return SSD_EINVAL;
    ctx->err.clear();
    SSD_TRY(check_batch(ctx, b));
    if (!prm || !uinf) return set_error(ctx, SSD_EINVAL, "NULL parameters or far-field velocities");
    if (nrhs < 1 || nrhs > kMaxRhs) return set_error(ctx, SSD_EINVAL, "nrhs must be in 1..16");
    if (!(prm->mu > 0.0) || !(prm->kappa > 0.0) || !isfinite(prm->mu) || !isfinite(prm->kappa))
        return set_error(ctx, SSD_EINVAL, "mu and kappa must be positive");
    if (!(prm->theta > 0.0 && prm->theta <= 1.0)) return set_error(ctx, SSD_EINVAL, "theta must be in (0, 1]");
    if (!(prm->tol_outer > 0.0) || prm->maxit_outer < 1 || prm->maxit_outer > kMaxM)
        return set_error(ctx, SSD_EINVAL, "bad outer tolerance or maxit_outer (1..256)");
    if (!prm->outer_gmres) return set_error(ctx, SSD_EINVAL, "batched solves use the interface GMRES");
    if (prm->traction_mode == SSD_TRACTION_BJS && prm->gamma != 0.0 && !prm->bjs_implicit)
        return set_error(ctx, SSD_EINVAL, "batched BJS solves need bjs_implicit = 1 (or gamma = 0)");
    if (prm->traction_mode == SSD_TRACTION_JOSEPH_TAO && !(prm->radius > 0.0))
        return set_error(ctx, SSD_EINVAL, "radius must be positive");
    if (prm->inner.use_sa || prm->inner.restart < 1 || prm->inner.restart > kMaxM || !(prm->inner.tol > 0.0) ||
        (prm->inner.prec != SSD_FP64 && prm->inner.prec != SSD_FP32C))
        return set_error(ctx, SSD_EINVAL, "batched local solves use GMRES with restart (Krylov length) 1..256");
    for (int r = 0; r < nrhs; ++r)
        for (int k = 0; k < 3; ++k)
            if (!isfinite(uinf[3 * r + k])) return set_error(ctx, SSD_EINVAL, "non-finite far-field velocity");
    cudaStream_t s = (cudaStream_t)stream;
    const BatchLayout &B = b->layout->B;
    const int64_t n = B.n_total;
    BDdm D;
    D.ctx = ctx; D.b = b; D.B = &B; D.P = *prm; D.s = s; D.nrhs = nrhs; D.n = n;
    for (int r = 0; r < nrhs; ++r)
        for (int k = 0; k < 3; ++k) D.uinf[r][k] = uinf[3 * r + k];
    const int64_t ls = (int64_t)nrhs * n, lv = 3 * ls;
    SSD_TRY(D.f.alloc(ctx, sizeof(double) * lv));
    SSD_TRY(D.tmp.alloc(ctx, sizeof(double) * lv));
    SSD_TRY(D.pn.alloc(ctx, sizeof(double) * lv));
    SSD_TRY(D.wrep.alloc(ctx, sizeof(double) * ls));
    SSD_TRY(D.mean.alloc(ctx, sizeof(double) * nrhs * B.nsurf));
    SSD_TRY(D.speed.alloc(ctx, sizeof(double) * kMaxRhs));
    SSD_TRY(seg_table(ctx, B, VecShape{nrhs, 1, B.nsurf, n}, &D.T1, s));
    struct TRel { ssd_ctx *c; void *p; ~TRel() { dev_free(c, p); } } trel{ctx, D.T1.block};
    brepeat_kernel<<<gridn(ls), 256, 0, s>>>(b->w, n, nrhs, D.wrep.d());
    ctx->launches++;
    Buf z, zn, c0, u, p;
    SSD_TRY(z.alloc(ctx, sizeof(double) * ls));
    SSD_TRY(zn.alloc(ctx, sizeof(double) * ls));
    SSD_TRY(c0.alloc(ctx, sizeof(double) * ls));
    SSD_TRY(u.alloc(ctx, sizeof(double) * lv));
    SSD_TRY(p.alloc(ctx, sizeof(double) * ls));
    SSD_TRY(cuda_check(ctx, cudaMemsetAsync(z.d(), 0, sizeof(double) * ls, s), "memset"));
    // c = F(0)
    SSD_TRY(D.sweep(z.d(), c0.d(), u.d(), p.d()));
    auto F = [&](const double *v, double *out) -> int {
        SSD_TRY(D.sweep(v, zn.d(), u.d(), p.d()));
        SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(out, c0.d(), sizeof(double) * ls, cudaMemcpyDeviceToDevice, s), "copy"));
        axpby_kernel<<<gridn(ls), 256, 0, s>>>(ls, -1.0, zn.d(), 1.0, out);
        axpby_kernel<<<gridn(ls), 256, 0, s>>>(ls, 1.0, v, 1.0, out);
        ctx->launches += 2;
        return launch_check(ctx, "batched outer matvec");
    };
    BResult orr;
    int st = bgmres(ctx, s, B, VecShape{nrhs, 1, B.nsurf, n}, F, c0.d(), z.d(), prm->tol_outer, prm->maxit_outer, &orr);
    int status = SSD_OK;
    if (st == SSD_ENOTCONV) status = SSD_ENOTCONV;
    else SSD_TRY(st);
    // final sweep from the solution
    SSD_TRY(D.sweep(z.d(), zn.d(), u.d(), p.d()));
    if (q) SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(q, z.d(), sizeof(double) * ls, cudaMemcpyDeviceToDevice, s), "copy"));
    if (p_D) SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(p_D, p.d(), sizeof(double) * ls, cudaMemcpyDeviceToDevice, s), "copy"));
    if (u_S) SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(u_S, u.d(), sizeof(double) * lv, cudaMemcpyDeviceToDevice, s), "copy"));
    if (f_S) SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(f_S, D.f.d(), sizeof(double) * lv, cudaMemcpyDeviceToDevice, s),
                                "copy"));
    if (drag) {
        Buf dd, offs;
        SSD_TRY(dd.alloc(ctx, sizeof(double) * 3 * nrhs * B.nsurf));
        SSD_TRY(offs.alloc(ctx, sizeof(int64_t) * (B.nsurf + 1)));
        std::vector<int64_t> ho(B.off);
        ho.push_back(n);
        SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(offs.p, ho.data(), sizeof(int64_t) * ho.size(), cudaMemcpyHostToDevice, s),
                           "offs copy"));
        bdrag_kernel<<<(unsigned)(3 * nrhs * B.nsurf), 256, 0, s>>>(D.f.d(), b->w, static_cast<int64_t *>(offs.p),
                                                                    B.nsurf, n, dd.d());
        ctx->launches++;
        SSD_TRY(cuda_check(ctx, cudaMemcpyAsync(drag, dd.d(), sizeof(double) * 3 * nrhs * B.nsurf,
                                                cudaMemcpyDeviceToHost, s), "drag copy"));
    }
    SSD_TRY(cuda_check(ctx, cudaStreamSynchronize(s), "sync"));
    for (int k = 0; k < nrhs * B.nsurf; ++k) {
        if (outer_its) outer_its[k] = orr.iters[k];
        if (relres) relres[k] = orr.relres[k];
    }
    if (D.nonconv && status == SSD_OK) status = SSD_ENOTCONV;
    if (status == SSD_ENOTCONV) set_error(ctx, SSD_ENOTCONV, "iteration limit reached in a batched D-N solve");
    return status;
}

}  // extern "C"
