"""The resolvent kernel's logarithm table (csrc/logtab.h): the committed file is
what gen_logtab.py writes, and every entry is right to far below a double's
rounding — hi is the double nearest to log(1 + j/256), hi + lo agrees with it
to 2^-100 relative, inv is the double nearest to 1/(1 + j/256), and log 2 is
split the same way.  Checked with exact rational / 60-digit decimal arithmetic,
independently of the generator's code path (math.log and fractions)."""
import math
import os
import re
import subprocess
import sys
from decimal import Decimal, getcontext
from fractions import Fraction

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2106_00454_gb300", "csrc")


def _entries():
    src = open(os.path.join(CSRC, "logtab.h")).read()
    rows = re.findall(r"\{([^{}]*)\},", src)
    vals = [[float.fromhex(v.strip()) if "0x" in v else float(v) for v in r.split(",")] for r in rows]
    ln2 = [float.fromhex(re.search(rf"{k} = ([^;]+);", src).group(1)) for k in ("kLn2Hi", "kLn2Lo")]
    return vals, ln2


def test_table_is_generator_output(tmp_path):
    before = open(os.path.join(CSRC, "logtab.h")).read()
    gen = open(os.path.join(CSRC, "gen_logtab.py")).read()
    script = tmp_path / "gen_logtab.py"
    script.write_text(gen)
    subprocess.run([sys.executable, str(script)], check=True, cwd=tmp_path)
    assert (tmp_path / "logtab.h").read_text() == before


def test_table_values():
    getcontext().prec = 60
    vals, (l2h, l2l) = _entries()
    assert len(vals) == 256
    for j, (hi, lo, inv, pad) in enumerate(vals):
        F = Fraction(256 + j, 256)
        exact = Decimal(256 + j).ln() - Decimal(256).ln()  # log F from two independent logs
        assert abs(hi - math.log(float(F))) <= 2 * math.ulp(hi) if j else hi == 0.0
        assert hi == float(exact)
        assert abs((Decimal(hi) + Decimal(lo)) - exact) <= abs(exact) * Decimal(2) ** -100
        assert inv == float(1 / F)  # Fraction -> float rounds to nearest
        assert pad == 0.0
    ln2 = Decimal(2).ln()
    assert l2h == float(ln2) and abs(Decimal(l2h) + Decimal(l2l) - ln2) <= ln2 * Decimal(2) ** -100
