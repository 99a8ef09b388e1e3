"""Writes bjs_lagged_sphere_h16.txt: the oracle's lagged BJS D-N solve
(Section 3, step 2 with the slip of eq. f taken from the previous sweep) on
the unit sphere at h = 1/16 (N = 4302), delta = 3h, mu = 1, U = e_z,
kappa = 1e-4, gamma = 1, theta = kappa/2, interface GMRES on (q, u_prev) to
1e-11 with local GMRES to 1e-13.  Calls only oracle/.  Stores the drag, the
outer iteration count and q, p_D, u_S at every 16th point.

    python tests/golden/make_bjs_lagged.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import quadrature as Q  # noqa: E402
from oracle import solvers as S  # noqa: E402

H, KAPPA, GAMMA, STRIDE = 1.0 / 16, 1e-4, 1.0, 16


def main():
    pts = Q.sphere_points(1.0, H)
    r = S.ddm_solve(pts, 3 * H, 1.0, KAPPA, GAMMA, (0.0, 0.0, 1.0), 0.5 * KAPPA, tol=1e-11, maxit=600,
                    outer="gmres", traction="bjs", inner_tol=1e-13, restart=200)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "bjs_lagged_sphere_h16.txt")
    with open(out, "w") as fh:
        fh.write("# oracle lagged BJS D-N solve: unit sphere h=1/16 (N=%d), delta=3h, mu=1, U=e_z, kappa=%g, "
                 "gamma=%g, theta=%g\n" % (pts["w"].size, KAPPA, GAMMA, 0.5 * KAPPA))
        fh.write("# interface GMRES to 1e-11 (local 1e-13); written by tests/golden/make_bjs_lagged.py\n")
        fh.write("drag %.17e %.17e %.17e\n" % tuple(r["drag"]))
        fh.write("outer_its %d\n" % r["outer_its"])
        fh.write("# index q p u_x u_y u_z (every %dth point)\n" % STRIDE)
        for i in range(0, pts["w"].size, STRIDE):
            fh.write("%d %.17e %.17e %.17e %.17e %.17e\n" % (i, r["q"][i], r["p"][i], r["u"][0, i], r["u"][1, i],
                                                           r["u"][2, i]))
    print("wrote", out, "outer its", r["outer_its"])


if __name__ == "__main__":
    main()
