"""Generate csrc/rules_table.h: the quadrature tables of the CUDA library.

- 7-point triangle rule of Sec. 3.1 (barycentre, vertices, mid-sides; weights
  27/60, 3/60, 8/60 times 1/2);
- 16-point degree-7 conical product rule (4-point Gauss-Jacobi with weight
  (1 - u) times 4-point Gauss-Legendre on [0, 1]);
- Gauss-Legendre points on (0, 1) for the regularising transforms.

Values are computed with sympy at 60 digits and written as correctly rounded
hexadecimal double literals. Run: python -m paper_2207_03921_gb300.gen_rules
"""
import os

import sympy as sp

HERE = os.path.dirname(os.path.abspath(__file__))
DIG = 60


def hexd(x) -> str:
    return float(sp.Float(x, DIG)).hex()


def gauss_jacobi_01(n, alpha):
    """Nodes/weights on [0, 1] for weight (1 - u)^alpha, from the roots of P_n^{(alpha,0)}(2u - 1)."""
    u = sp.symbols("u")
    P = sp.jacobi(n, alpha, 0, 2 * u - 1)
    roots = sorted(sp.Poly(sp.expand(P), u).nroots(n=DIG, maxsteps=200))
    # weights: solve the moment equations sum_i w_i u_i^m = int_0^1 (1-u)^alpha u^m du, m < n
    mom = [sp.integrate((1 - u) ** alpha * u ** m, (u, 0, 1)) for m in range(n)]
    V = sp.Matrix([[r ** m for r in roots] for m in range(n)])
    w = V.LUsolve(sp.Matrix(mom))
    return [sp.Float(r, DIG) for r in roots], [sp.Float(x, DIG) for x in w]


def main():
    lines = ["// Generated by gen_rules.py: quadrature tables (barycentric l0, l1, l2, weight).",
             "#pragma once", ""]
    third = sp.Rational(1, 3)
    r7 = [(third, third, third, sp.Rational(27, 120))]
    r7 += [(1, 0, 0, sp.Rational(3, 120)), (0, 1, 0, sp.Rational(3, 120)), (0, 0, 1, sp.Rational(3, 120))]
    h = sp.Rational(1, 2)
    r7 += [(h, h, 0, sp.Rational(8, 120)), (0, h, h, sp.Rational(8, 120)), (h, 0, h, sp.Rational(8, 120))]
    lines.append("static const double NLFEM_RULE7[7][4] = {")
    for p in r7:
        lines.append("  {" + ", ".join(hexd(v) for v in p) + "},")
    lines.append("};")
    uj, wj = gauss_jacobi_01(4, 1)
    vl, wl = gauss_jacobi_01(4, 0)
    lines.append("static const double NLFEM_RULE16[16][4] = {")
    for ui, wui in zip(uj, wj):
        for vi, wvi in zip(vl, wl):
            l1 = ui
            l2 = (1 - ui) * vi
            l0 = (1 - ui) * (1 - vi)
            lines.append("  {" + ", ".join(hexd(v) for v in (l0, l1, l2, wui * wvi)) + "},")
    lines.append("};")
    for n in (5,):
        x, w = gauss_jacobi_01(n, 0)
        lines.append(f"static const double NLFEM_GAUSS{n}_X[{n}] = {{" + ", ".join(hexd(v) for v in x) + "};")
        lines.append(f"static const double NLFEM_GAUSS{n}_W[{n}] = {{" + ", ".join(hexd(v) for v in w) + "};")
    out = os.path.join(HERE, "csrc", "rules_table.h")
    open(out, "w").write("\n".join(lines) + "\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
