"""Write exp2_table.inc: the constants of the table-driven exponential used by
the integrator (Tang's method, ACM TOMS 15 (1989) 144-157).

  T[j] = 2^(j/256), j = 0..255, each correctly rounded to double
  kExpInvL = 256 / ln 2 (rounded), kExpL1 + kExpL2 = ln 2 / 256 (head + tail)

Values are computed with 60-digit decimal arithmetic and rounded once.
Run: python gen_exp_table.py  (rewrites exp2_table.inc next to this file)."""
import os
from decimal import Decimal, getcontext

getcontext().prec = 60
LN2 = Decimal(2).ln()


def dbl(x: Decimal) -> float:
    return float(x)          # decimal -> nearest double (correctly rounded)


def main():
    lines = ["// Generated by gen_exp_table.py: 2^(j/256) correctly rounded, and the",
             "// reduction constants of the table-driven exponential.  Do not edit."]
    inv_l = dbl(Decimal(256) / LN2)
    l1 = dbl(LN2 / 256)
    l2 = dbl(LN2 / 256 - Decimal(l1))
    lines.append(f"constexpr double kExpInvL = {inv_l.hex()};   // 256 / ln 2")
    lines.append(f"constexpr double kExpL1 = {l1.hex()};    // ln 2 / 256, head")
    lines.append(f"constexpr double kExpL2 = {l2.hex()};    // ln 2 / 256, tail")
    lines.append("__device__ const double kExp2Table[256] = {")
    for j in range(256):
        v = dbl((LN2 * j / 256).exp())
        lines.append(f"    {v.hex()},")
    lines.append("};")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "exp2_table.inc")
    with open(out, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print(out)


if __name__ == "__main__":
    main()
