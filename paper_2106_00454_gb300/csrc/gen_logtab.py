"""Writes logtab.h: the table of the T kernel's logarithm.

For F_j = 1 + j/256, j = 0 .. 255: log F_j as an unevaluated sum hi + lo of two
doubles (hi the double nearest to log F_j, lo the double nearest to the
remainder) and 1/F_j rounded to nearest; log 2 split the same way.  The values
come from Python's decimal module at 60 significant digits (its ln is
correctly rounded at that precision), so the table is the same on every
machine.  Run from this directory: python gen_logtab.py
"""
from decimal import Decimal, getcontext
import os

getcontext().prec = 60


def split(d: Decimal):
    hi = float(d)
    lo = float(d - Decimal(hi))
    return hi, lo


def main():
    lines = [
        "// Generated by gen_logtab.py (decimal arithmetic, 60 digits); do not edit.",
        "// kLogTab[j] = {hi, lo, inv, 0}: log(1 + j/256) = hi + lo, inv = RN(1 / (1 + j/256)).",
        "#pragma once",
        "",
        "namespace wpcd {",
        "",
        "struct __align__(32) LogEntry {",
        "    double hi, lo, inv, pad;",
        "};",
        "",
    ]
    l2h, l2l = split(Decimal(2).ln())
    lines.append(f"constexpr double kLn2Hi = {l2h.hex()};")
    lines.append(f"constexpr double kLn2Lo = {l2l.hex()};")
    lines.append("")
    lines.append("__device__ const LogEntry kLogTab[256] = {")
    for j in range(256):
        F = Decimal(1) + Decimal(j) / Decimal(256)
        hi, lo = split(F.ln()) if j else (0.0, 0.0)
        inv = float(Decimal(1) / F)
        lines.append(f"    {{{hi.hex()}, {lo.hex()}, {inv.hex()}, 0.0}},")
    lines.append("};")
    lines.append("")
    lines.append("}  // namespace wpcd")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "logtab.h")
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
