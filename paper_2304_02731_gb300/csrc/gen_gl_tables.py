"""Write gl_tables.inc: Gauss-Legendre rules for the action and period
integrals, in the sine-mapped form the kernels use: 32 points for the
product analysis (at the rounding floor of the action integral for the
Morse and LJ wells of the studies; within 4e-11 in v' 1e-8 below a
centrifugal barrier top), 128 for the level solver.

The integrals over [r-, r+] are taken after r = c + d sin(pi x / 2),
x in [-1, 1] (dr = d (pi/2) cos(pi x / 2) dx), with the n-point
Gauss-Legendre rule on x.  The rule is symmetric, so each table holds the
n/2 positive nodes only, as

  S[k]  = sin(pi x_k / 2)            (node position: r = c +- d S[k])
  WC[k] = w_k cos(pi x_k / 2)        (weight times the map's Jacobian factor)

Nodes are the roots of P_n found by Newton's method from the standard
cosine guess, with P_n and P_n' from the three-term recurrence; weights are
w = 2 / ((1 - x^2) P_n'(x)^2).  Everything is computed with 50-digit mpmath
arithmetic and rounded once to double.
Run: python gen_gl_tables.py  (rewrites gl_tables.inc next to this file)."""
import os

import mpmath as mp

mp.mp.dps = 50


def legendre_rule(n: int):
    """Positive nodes and weights of the n-point Gauss-Legendre rule (n even)."""
    out = []
    for i in range(n // 2):
        x = mp.cos(mp.pi * (i + mp.mpf(3) / 4) / (n + mp.mpf(1) / 2))
        for _ in range(100):
            p0, p1 = mp.mpf(1), x
            for k in range(2, n + 1):
                p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
            dp = n * (x * p1 - p0) / (x * x - 1)
            dx = p1 / dp
            x -= dx
            if abs(dx) < mp.mpf(10) ** -45:
                break
        w = 2 / ((1 - x * x) * dp * dp)
        out.append((x, w))
    return out


def table(name: str, n: int):
    rule = legendre_rule(n)
    s = [float(mp.sin(mp.pi * x / 2)) for x, _ in rule]
    wc = [float(w * mp.cos(mp.pi * x / 2)) for x, w in rule]
    lines = [f"__constant__ double {name}S[{n // 2}] = {{"]
    lines += [f"    {v.hex()}," for v in s]
    lines.append("};")
    lines.append(f"__constant__ double {name}WC[{n // 2}] = {{")
    lines += [f"    {v.hex()}," for v in wc]
    lines.append("};")
    return lines


def main():
    lines = ["// Generated by gen_gl_tables.py: sine-mapped Gauss-Legendre rules",
             "// (positive half of the symmetric nodes).  Do not edit."]
    lines += table("kGL32", 32)
    lines += table("kGL128", 128)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gl_tables.inc")
    with open(out, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print(out)


if __name__ == "__main__":
    main()
