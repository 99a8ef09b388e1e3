"""Local boundary-integral solves and the Dirichlet-Neumann iteration (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Conventions: n is the outward unit normal of the porous body (it points into
the fluid); q = u . n on the interface (the paper's q = -u_S . n_S with
n_S = -n).  Operators are those of ``oracle/__init__.py``:
D^L = H - I/2 (eq. H_subtr) and D^S = K + I/2 (eq. K_subtr).

Darcy (eq. Darcy_final):  1/2 p = H p + b_D  <=>  -D^L p = b_D,
                          b_D = (mu/kappa) L q.
Stokes (eq. Stokes_final): 1/2 u = K u + b_S  <=>  (I - D^S) u = b_S,
                          b_S = U_inf - M f.

Readings where the paper is silent (each is listed with its reason in the
design notes): GMRES restarts after ``restart`` steps, orthogonalises by
modified Gram-Schmidt, starts from x0 = 0 and stops when the residual
estimate falls to tol * ||b||; the Darcy pressure, which the operator
determines only up to a constant, is returned with zero quadrature-weighted
mean; successive approximations stop on the relative change between sweeps.
"""
from __future__ import annotations

import math

import numpy as np

import oracle
from oracle import analytic


def gmres(A, b, tol=1e-9, restart=50, maxit=1000, x0=None):
    """Restarted GMRES with modified Gram-Schmidt and Givens rotations.

    Returns (x, iterations, estimated relative residual).  ``iterations``
    counts Arnoldi steps, i.e. applications of A inside the Krylov loop.
    """
    b = np.asarray(b, dtype=np.float64)
    shape = b.shape
    bv = b.ravel()
    bnorm = float(np.linalg.norm(bv))
    x = np.zeros_like(bv) if x0 is None else np.array(x0, dtype=np.float64).ravel()
    if bnorm == 0.0:
        return x.reshape(shape), 0, 0.0
    Av = (lambda v: np.asarray(A(v.reshape(shape)), dtype=np.float64).ravel())
    total = 0
    rel = 1.0
    while True:
        r = bv - Av(x) if (x0 is not None or total > 0) else bv.copy()
        beta = float(np.linalg.norm(r))
        rel = beta / bnorm
        if rel <= tol or total >= maxit or beta == 0.0:
            return x.reshape(shape), total, rel
        m = restart
        V = np.zeros((m + 1, bv.size))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            w = Av(V[j])
            total += 1
            for i in range(j + 1):
                H[i, j] = float(V[i] @ w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = float(np.linalg.norm(w))
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            rel = abs(g[j + 1]) / bnorm
            nxt = np.linalg.norm(w)
            if nxt > 0.0:
                V[j + 1] = w / nxt
            if rel <= tol or total >= maxit or nxt == 0.0:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + V[:k].T @ y
        if rel <= tol or total >= maxit:
            return x.reshape(shape), total, rel


def successive_approx(step, x0, tol=1e-9, maxit=1000):
    """x <- step(x) until ||x_new - x|| / ||x_new|| <= tol (eqs. *_BIEM_iter)."""
    x = np.array(x0, dtype=np.float64)
    rel = 1.0
    for it in range(1, maxit + 1):
        xn = step(x)
        nn = float(np.linalg.norm(xn))
        rel = float(np.linalg.norm(xn - x)) / nn if nn > 0 else 0.0
        x = xn
        if rel <= tol:
            return x, it, rel
    return x, maxit, rel


def weighted_mean(pts, v):
    return float(pts["w"] @ v) / float(pts["w"].sum())


def darcy_solve(pts, delta, mu, kappa, q, tol=1e-9, restart=50, maxit=1000, use_sa=False, x0=None):
    """Solve -D^L p = (mu/kappa) L q for the Darcy pressure on the interface.

    Returns (p, iterations, relres).  p has zero quadrature-weighted mean.
    x0: initial iterate (zero when None).
    """
    b = (mu / kappa) * oracle.laplace_sl(pts, delta, q)
    if use_sa:
        # eq. Darcy_BIEM_iter: p <- p/2 + H p + b = p + D^L p + b, each sweep
        # projected to zero weighted mean (the constant mode is not damped)
        def step(p):
            pn = p + oracle.laplace_dl(pts, delta, p) + b
            return pn - weighted_mean(pts, pn)
        p, its, rel = successive_approx(step, np.zeros_like(b) if x0 is None else x0, tol, maxit)
    else:
        # -D^L annihilates constants.  The rank-one term 1 (w . p) / sum(w)
        # makes the operator nonsingular; for a right-hand side in the range
        # of D^L the solution is unchanged (the zero-mean one).
        W = float(pts["w"].sum())
        wv = pts["w"]
        p, its, rel = gmres(lambda p: -oracle.laplace_dl(pts, delta, p) + float(wv @ p) / W,
                            b, tol, restart, maxit, x0=x0)
    return p - weighted_mean(pts, p), its, rel


def normal_flux_term(pts, u):
    """n (w . (u . n)) / sum(w): rank-one term on the normal mode."""
    n = pts["nrm"]
    return n * (float(pts["w"] @ (u * n).sum(0)) / float(pts["w"].sum()))


def stokes_solve(pts, delta, mu, f, uinf, tol=1e-9, restart=50, maxit=1000, use_sa=False, deflate=False,
                 x0=None):
    """Solve (I - D^S) u = U_inf - M f for the interface velocity [3][N].

    deflate: the continuous I/2 - K has the normal field n in its null space,
    so the discrete I - D^S has a near-null vector (eigenvalue O(h^5)).  With
    deflate, GMRES runs on (I - D^S) u + n (w . (u.n))/sum(w): nonsingular,
    and its solution is the one with zero net flux  int u.n dS = 0 (the
    Darcy compatibility condition on q = u.n).
    """
    b = np.asarray(uinf, dtype=np.float64)[:, None] - oracle.stokes_sl(pts, delta, mu, f)
    if use_sa:
        # eq. Stokes_BIEM_iter: u <- u/2 + K u + b = D^S u + b
        return successive_approx(lambda u: oracle.stokes_dl(pts, delta, u) + b,
                                 np.zeros_like(b) if x0 is None else x0, tol, maxit)
    if deflate:
        return gmres(lambda u: u - oracle.stokes_dl(pts, delta, u) + normal_flux_term(pts, u), b, tol,
                     restart, maxit, x0=x0)
    return gmres(lambda u: u - oracle.stokes_dl(pts, delta, u), b, tol, restart, maxit, x0=x0)


def stokes_solve_bjs_implicit(pts, delta, mu, p, uinf, kappa, gamma, sign=1.0, tol=1e-9, restart=50,
                              maxit=1000, deflate=False, x0=None):
    """Stokes solve with the BJS slip term taken at the current velocity.

    With f = -p n + s c P u (c = gamma/sqrt(kappa), P u = u - (u.n) n),
    u = D^S u + U_inf - M f becomes
        (I - D^S) u + s c M(P u) = U_inf + M(p n).
    """
    n = pts["nrm"]
    c = sign * gamma / math.sqrt(kappa)
    b = np.asarray(uinf, dtype=np.float64)[:, None] + oracle.stokes_sl(pts, delta, mu, p * n)

    def A(u):
        Pu = u - (u * n).sum(0) * n
        v = u - oracle.stokes_dl(pts, delta, u) + c * oracle.stokes_sl(pts, delta, mu, Pu)
        return v + normal_flux_term(pts, u) if deflate else v
    return gmres(A, b, tol, restart, maxit, x0=x0)


def traction_bjs(pts, p, u_prev, kappa, gamma, sign=1.0):
    """f = -p n + sign (gamma/sqrt(kappa)) (u - (u.n) n)   (eq. f, sign read as +1)."""
    n = pts["nrm"]
    un = (u_prev * n).sum(0)
    return -p * n + sign * (gamma / math.sqrt(kappa)) * (u_prev - un * n)


def traction_joseph_tao(pts, p, R, kappa, mu, uinf):
    """f = (-p_D + 2 mu du_r/dr) e_r + f_theta e_theta (eqs. f_r, f_theta, Section 7.3).

    The pressure is the computed Darcy pressure; the velocity terms are exact.
    """
    a, tang = analytic.jt_traction_exact_velocity_terms(pts["xyz"], R, kappa, mu, uinf)
    er = pts["xyz"] / np.sqrt((pts["xyz"] ** 2).sum(0))
    return (-p + a) * er + tang


def ddm_solve(pts, delta, mu, kappa, gamma, uinf, theta, tol=1e-9, maxit=100,
              outer="sa", traction="bjs", R=1.0, bjs_sign=1.0,
              inner_tol=None, restart=50, inner_maxit=1000, use_sa=False, bjs_implicit=False,
              deflate=False, warm_inner=False, arnoldi=0):
    """Dirichlet-Neumann iteration of Sections 3 and 6.

    One sweep G maps (q, u_prev) to (q_new, u): Darcy solve with Neumann data
    q, traction from p_D (and u_prev in BJS mode), Stokes solve, relaxed update
    q_new = (1 - theta) q + theta u . n  (eq. q_update).
    outer="sa": repeat the sweep until the DDM residual (eq. DDM_residual)
    ||q_k - q_{k-1}|| / ||q_k|| <= tol.
    outer="gmres": the sweep is affine, z -> G z + c with z = q (or
    (q, u_prev) in BJS mode with gamma != 0); GMRES solves D (I - G) z = D c
    with relative residual tol, D dividing the q rows by theta (the unrelaxed
    map), and one final sweep from the solution gives the returned fields.
    bjs_implicit: the Stokes step imposes the BJS slip at its own velocity
    (see stokes_solve_bjs_implicit) instead of the previous sweep's, so the
    interface state is q alone.
    deflate: Stokes solves remove the near-null normal mode (see stokes_solve).
    warm_inner: with outer="sa", each local solve starts from the previous
    sweep's solution (Darcy from p, Stokes from u) instead of zero.
    arnoldi > 0: no solve; instead `arnoldi` Arnoldi steps (modified
    Gram-Schmidt) on the discrete iteration matrix A~ v = F(v) - F(0)
    (eq. A_mat, Section 6) from the start vector frac(i g) - 1/2 (normalised,
    i the point index, g = 0.6180339887498949), with Gram-Schmidt twice;
    returns {"H": Hessenberg [m+1][m], "ritz": eigenvalues of H[:m, :m]}.
    Returns a dict with q, p, u, f, drag, outer iteration count, inner counts
    and the residual history.
    """
    n = pts["nrm"]
    N = n.shape[1]
    uinf = np.asarray(uinf, dtype=np.float64)
    if inner_tol is None:
        inner_tol = tol if outer == "sa" else 0.1 * tol
    stacked = (traction == "bjs" and gamma != 0.0 and not bjs_implicit)
    inner_its = []

    warm = {"p": None}

    def sweep(q, u_prev):
        wstart = warm_inner and outer == "sa"
        p, itd, _ = darcy_solve(pts, delta, mu, kappa, q, inner_tol, restart, inner_maxit, use_sa,
                                x0=warm["p"] if wstart else None)
        if wstart:
            warm["p"] = p
        u0 = u_prev if wstart else None
        if traction == "bjs" and bjs_implicit:
            u, its, _ = stokes_solve_bjs_implicit(pts, delta, mu, p, uinf, kappa, gamma, bjs_sign,
                                                  inner_tol, restart, inner_maxit, deflate, x0=u0)
            f = traction_bjs(pts, p, u, kappa, gamma, bjs_sign)
        else:
            if traction == "bjs":
                f = traction_bjs(pts, p, u_prev, kappa, gamma, bjs_sign)
            else:
                f = traction_joseph_tao(pts, p, R, kappa, mu, uinf)
            u, its, _ = stokes_solve(pts, delta, mu, f, uinf, inner_tol, restart, inner_maxit, use_sa,
                                     deflate, x0=u0)
        inner_its.append((itd, its))
        qn = (1.0 - theta) * q + theta * (u * n).sum(0)
        return qn, u, p, f

    hist = []
    q = np.zeros(N)
    u_prev = np.zeros((3, N))
    if outer == "sa":
        k = 0
        for k in range(1, maxit + 1):
            qn, u, p, f = sweep(q, u_prev)
            nq = float(np.linalg.norm(qn))
            res = float(np.linalg.norm(qn - q)) / nq if nq > 0 else 0.0
            hist.append(res)
            q, u_prev = qn, u
            if res <= tol:
                break
        its = k
    else:
        def F(z):
            if stacked:
                qq, uu = z[:N], z[N:].reshape(3, N)
            else:
                qq, uu = z, np.zeros((3, N))
            qn, u, _, _ = sweep(qq, uu)
            return np.concatenate([qn, u.ravel()]) if stacked else qn

        z0 = np.zeros(4 * N if stacked else N)
        c = F(z0)
        if arnoldi > 0:
            assert not stacked, "the iteration matrix acts on q alone"
            # start vector with every mode present: v_i = frac(i g) - 1/2, g the golden section
            v = np.mod(np.arange(N, dtype=np.float64) * 0.6180339887498949, 1.0) - 0.5
            V = [v / np.linalg.norm(v)]
            H = np.zeros((arnoldi + 1, arnoldi))
            m = arnoldi
            for j in range(arnoldi):
                w = F(V[j]) - c
                for _ in range(2):           # Gram-Schmidt twice (orthogonality to working precision)
                    for i in range(j + 1):
                        hij = float(V[i] @ w)
                        H[i, j] += hij
                        w = w - hij * V[i]
                H[j + 1, j] = float(np.linalg.norm(w))
                if H[j + 1, j] <= 1e-12 * float(np.abs(H[:j + 1, j]).max()):
                    m = j + 1          # an invariant subspace: its Ritz values are eigenvalues
                    break
                V.append(w / H[j + 1, j])
            return {"H": H[:m + 1, :m], "ritz": np.linalg.eigvals(H[:m, :m])}
        # GMRES on the unrelaxed interface map: the q rows of the stacked
        # system, theta (q - u.n), are divided by theta, so the operator and
        # the iterates do not depend on theta (as the equal counts for
        # theta = 0.5 kappa and 0.75 kappa in Table 2 show) and the q block,
        # whose size is O(kappa), is not swamped by the u block's residual.
        # With z = q alone this is a global scaling, which GMRES ignores.
        D = np.ones(z0.size)
        D[:N] = 1.0 / theta
        z, its, rel = gmres(lambda v: D * (v - (F(v) - c)), D * c, tol, restart=max(restart, maxit), maxit=maxit)
        hist.append(rel)
        if stacked:
            q, u_prev = z[:N], z[N:].reshape(3, N)
        else:
            q = z
        _, u, p, f = sweep(q, u_prev)
    drag = (f * pts["w"]).sum(1)
    return {"q": q, "p": p, "u": u, "f": f, "drag": drag, "outer_its": its,
            "inner_its": inner_its, "hist": hist}


def iteration_matrix(pts, delta, mu, kappa, theta, deflate=False):
    """The discrete iteration matrix of the D-N sweeps (eq. A_mat, Section 6),
    assembled from the dense operator matrices:

        A~ = (1 - theta) I + theta N^T (I - D^S)^{-1} M N G,
        G  = (mu/kappa) P0 (-D^L + 1 w^T / W)^{-1} L,

    with N p = p n (so f = -p n and b_S = M N p for u_inf = 0, gamma = 0), N^T u
    = u . n, P0 = I - 1 w^T / W the projection to zero weighted mean.  G is the
    Darcy solve with the gauge of darcy_solve: the printed (I/2 - H~)^{-1} does
    not exist (constants are in the kernel of D^L = H - I/2).  The signs are
    those of eq. q_update with n the body normal (q = u . n); eq. A_mat writes
    the same matrix as I - theta {I + (mu/kappa) [...] . n_S [...]}.
    deflate: the Stokes matrix carries the rank-one normal-mode term
    n (w . (u . n)) / W of stokes_solve.  Returns A~ (n x n).
    """
    n = pts["nrm"]
    N = n.shape[1]
    w = pts["w"]
    W = float(w.sum())
    L = oracle.operator_matrix(pts, delta, "L")
    DL = oracle.operator_matrix(pts, delta, "DL")
    M = oracle.operator_matrix(pts, delta, "M", mu)
    DS = oracle.operator_matrix(pts, delta, "DS")
    one = np.ones(N)
    Gd = np.linalg.solve(-DL + np.outer(one, w) / W, (mu / kappa) * L)
    Gd -= np.outer(one, w @ Gd) / W
    Nm = np.concatenate([np.diag(n[0]), np.diag(n[1]), np.diag(n[2])])      # 3N x N
    S = np.eye(3 * N) - DS
    if deflate:
        S += np.outer(n.ravel(), (w[None, :] * n).ravel()) / W
    U = np.linalg.solve(S, M @ (Nm @ Gd))
    return (1.0 - theta) * np.eye(N) + theta * (Nm.T @ U)


def rms(v):
    """Unweighted RMS over points (eqs. error_Darcy, error_Stokes): v is [N] or [3][N]."""
    v = np.asarray(v)
    if v.ndim == 2:
        return float(np.sqrt((v * v).sum(0).mean()))
    return float(np.sqrt((v * v).mean()))
