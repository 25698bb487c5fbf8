"""Write sincos_table.inc: cos and sin of 2 pi k / 256 for k = -128 .. 128,
each correctly rounded to float64 (evaluated with mpmath at 50 digits).

The float64 predictors evaluate exp(i 2 pi t), |t| <= 1/2, by table-driven
argument reduction (the classic table-lookup method, e.g. P. T. P. Tang,
ACM TOMS 15(2), 1989): t = k/256 + f with |f| <= 1/512, then
exp(i 2 pi t) = exp(i 2 pi k/256) * exp(i 2 pi f), the second factor from short
Taylor series. This script only produces the table entries.

    python paper_1909_03956_gb300/csrc/gen_sincos_table.py
"""
import os

import mpmath

mpmath.mp.dps = 50
HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    lines = ["// Generated by gen_sincos_table.py: {cos, sin}(2 pi k / 256), k = -128 .. 128,",
             "// correctly rounded to float64.",
             "{"]
    for k in range(-128, 129):
        x = mpmath.mpf(k) / 128          # 2 k / 256, in half-turns: exact
        c, s = float(mpmath.cospi(x)), float(mpmath.sinpi(x))
        lines.append("    {%s, %s}," % (repr(c), repr(s)))
    lines.append("}")
    with open(os.path.join(HERE, "sincos_table.inc"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
