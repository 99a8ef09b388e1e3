"""Write erfcx_coef.h: polynomial fit of erfcx(rho) = e^{rho^2} erfc(rho) on [0.5, 5.5].

Used by the FP32C pair kernels to write the smoothing factors of Section 5.3
as s_i(rho) = 1 - e^{-rho^2} (erfcx(rho) - (2/sqrt(pi)) rho Q_i(rho^2)).
Only e^{-rho^2} (erfcx - fit) enters s_i, so the fit is a least-squares
Chebyshev fit weighted by e^{-rho^2}, in the variable z = 1/(1 + rho) mapped
to [-1, 1], converted to monomials in that variable; reference values come
from mpmath at 40 digits.  Weighted error of the degree-7 fit: 1.2e-9 in
exact arithmetic, about 1e-7 when evaluated in FP32 (the rounding level).
Run:  python gen_erfcx.py > erfcx_coef.h
"""
import mpmath as mp
import numpy as np

mp.mp.dps = 40
A, B, DEG = 0.5, 5.5, 7
xs = np.linspace(A, B, 20001)
f = np.array([float(mp.erfc(x) * mp.exp(x * x)) for x in xs])
wgt = np.exp(-xs ** 2)
za, zb = 1.0 / (1.0 + B), 1.0 / (1.0 + A)
zz = (2.0 / (1.0 + xs) - (za + zb)) / (zb - za)
V = np.polynomial.chebyshev.chebvander(zz, DEG)
c, *_ = np.linalg.lstsq(V * wgt[:, None], f * wgt, rcond=None)
pc = np.polynomial.chebyshev.cheb2poly(c)
print("// Generated by gen_erfcx.py: erfcx(rho) ~ sum_k kErfcx[k] w^k on [0.5, 5.5], with")
print("// w = kErfcxA / (1 + rho) - kErfcxB.  Do not edit.")
print("#pragma once")
print("#define SSD_ERFCX_DEG %d" % DEG)
print("static constexpr float kErfcxA = %.9ef;" % (2.0 / (zb - za)))
print("static constexpr float kErfcxB = %.9ef;" % ((za + zb) / (zb - za)))
for k, v in enumerate(pc):
    print("static constexpr float kErfcx%d = %.9ef;" % (k, v))
print("// Horner evaluation for a packed pair of arguments")
print("static __device__ __forceinline__ float2 erfcx_fit2(float2 w) {")
print("    float2 p = make_float2(kErfcx%d, kErfcx%d);" % (DEG, DEG))
for k in range(DEG - 1, -1, -1):
    print("    p = __ffma2_rn(p, w, make_float2(kErfcx%d, kErfcx%d));" % (k, k))
print("    return p;")
print("}")
