"""Write exp2_table.inc: the constants of the table-driven exponential used by
the integrator and the product analysis (Tang's method, ACM TOMS 15 (1989)
144-157), with N = 2048 table entries.

  T[j] = 2^(j/N), j = 0..N-1, each correctly rounded to double
  kExpInvL = N / ln 2 (rounded), kExpL1 + kExpL2 = ln 2 / N (head + tail)

Values are computed with 60-digit decimal arithmetic and rounded once.
Run: python gen_exp_table.py  (rewrites exp2_table.inc next to this file)."""
import os
from decimal import Decimal, getcontext

getcontext().prec = 60
LN2 = Decimal(2).ln()
N = 2048


def dbl(x: Decimal) -> float:
    return float(x)          # decimal -> nearest double (correctly rounded)


def main():
    lines = [f"// Generated by gen_exp_table.py: 2^(j/{N}) correctly rounded, and the",
             "// reduction constants of the table-driven exponential.  Do not edit."]
    inv_l = dbl(Decimal(N) / LN2)
    l1 = dbl(LN2 / N)
    l2 = dbl(LN2 / N - Decimal(l1))
    lines.append(f"constexpr int kExpTableSize = {N};")
    lines.append(f"constexpr double kExpInvL = {inv_l.hex()};   // {N} / ln 2")
    lines.append(f"constexpr double kExpL1 = {l1.hex()};    // ln 2 / {N}, head")
    lines.append(f"constexpr double kExpL2 = {l2.hex()};    // ln 2 / {N}, tail")
    lines.append(f"__device__ const double kExp2Table[{N}] = {{")
    for j in range(N):
        v = dbl((LN2 * j / N).exp())
        lines.append(f"    {v.hex()},")
    lines.append("};")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "exp2_table.inc")
    with open(out, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print(out)


if __name__ == "__main__":
    main()
