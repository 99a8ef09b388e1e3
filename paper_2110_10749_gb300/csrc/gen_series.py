"""Write series_coef.h: Taylor coefficients of sigma_i(rho) = s_i(rho) / rho^p_i.

s_1..s_4 are the smoothing factors of Section 5.3; p = 1, 3, 3, 5.  The
coefficients are those of powers of t = rho^2, derived exactly with sympy
from the closed forms and printed to 17 significant digits.
Run:  python gen_series.py > series_coef.h
"""
import sympy as sp

r = sp.symbols("r", positive=True)
c = 2 / sp.sqrt(sp.pi)
S = {
    1: sp.erf(r) - c / 3 * r * (2 * r**2 - 5) * sp.exp(-r**2),
    2: sp.erf(r) + c / 3 * r * (2 * r**2 - 3) * sp.exp(-r**2),
    3: sp.erf(r) - c / 3 * r * (4 * r**4 - 14 * r**2 + 3) * sp.exp(-r**2),
    4: sp.erf(r) - c / 9 * r * (8 * r**6 - 36 * r**4 + 6 * r**2 + 9) * sp.exp(-r**2),
}
P = {1: 1, 2: 3, 3: 3, 4: 5}
NT = 18
print("// Generated by gen_series.py: Taylor coefficients of sigma_i(rho) = s_i(rho)/rho^p_i")
print("// in powers of t = rho^2 (s_i of Section 5.3; p = 1, 3, 3, 5).  Do not edit.")
print("#pragma once")
print("#define SSD_NSER %d" % NT)
NT32 = 9
rows = []
for i in range(1, 5):
    ser = sp.series(S[i] / r**P[i], r, 0, 2 * NT + 1).removeO()
    assert all(ser.coeff(r, 2 * k + 1) == 0 for k in range(NT))
    rows.append([float(sp.N(ser.coeff(r, 2 * k), 30)) for k in range(NT)])
print("#define SSD_NSER32 %d" % NT32)
print("static __device__ __constant__ double kSeries[4][SSD_NSER] = {")
for row in rows:
    print("  {" + ", ".join("%.17e" % v for v in row) + "},")
print("};")
print("static __device__ __constant__ float kSeries32[4][SSD_NSER32] = {")
for row in rows:
    print("  {" + ", ".join("%.9ef" % v for v in row[:NT32]) + "},")
print("};")
