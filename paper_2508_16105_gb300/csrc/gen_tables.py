"""Write fastmath_tables.h: the constant tables of the table-driven exp and log.

Values are computed with Python's decimal module at 60 significant digits and
rounded once to binary64, so the header is identical on every host.

  exp: T_j = 2^(j/1024), j = 0..1023
  log: for j = 0..127 the interval [1 + j/128, 1 + (j+1)/128) of the mantissa,
       invc_j = 1/c_j rounded to binary64 with c_j the interval centre, and
       logc_j = -ln(invc_j) of that rounded value (so ln m = logc_j + ln(m invc_j)
       holds exactly in real arithmetic).
  Cody-Waite splits of ln2/1024 (for exp) and ln2 (for log): the high parts have
  at most 32 significant bits, so k * hi is exact for |k| < 2^21.
"""
import os
from decimal import Decimal, getcontext
from fractions import Fraction

getcontext().prec = 60
HERE = os.path.dirname(os.path.abspath(__file__))


def to_double(d: Decimal) -> float:
    # correctly rounded conversion via an exact rational
    return float(Fraction(d))


def ln2() -> Decimal:
    return Decimal(2).ln()


def hi_part(x: Decimal, bits: int = 32) -> float:
    """x rounded to `bits` significant bits (exactly representable)."""
    f = Fraction(x)
    e = 0
    while f >= 1:
        f /= 2
        e += 1
    while f < Fraction(1, 2):
        f *= 2
        e -= 1
    m = round(f * (1 << bits))
    return float(Fraction(m, 1 << bits) * (Fraction(2) ** e))


def main():
    L2 = ln2()
    exp_tab = [to_double(Decimal(2) ** (Decimal(j) / Decimal(1024))) for j in range(1024)]
    c = ln2() / Decimal(1024)
    e_hi = hi_part(c)
    e_lo = to_double(c - Decimal(Fraction(e_hi).numerator) / Decimal(Fraction(e_hi).denominator))
    l_hi = hi_part(L2)
    l_lo = to_double(L2 - Decimal(Fraction(l_hi).numerator) / Decimal(Fraction(l_hi).denominator))
    log2e_1024 = to_double(Decimal(1024) / L2)
    ln2_54 = to_double(Decimal(54) * L2)
    invc, logc = [], []
    for j in range(128):
        centre = Decimal(1) + (Decimal(j) + Decimal("0.5")) / Decimal(128)
        ic = to_double(Decimal(1) / centre)
        icd = Decimal(Fraction(ic).numerator) / Decimal(Fraction(ic).denominator)
        invc.append(ic)
        logc.append(to_double(-icd.ln()))
    out = []
    out.append("// Generated by gen_tables.py: constant tables of the table-driven exp and log.")
    out.append("#pragma once")
    out.append("namespace rde {")
    out.append("constexpr double kExpLog2e1024 = %s;  // 1024 / ln 2" % log2e_1024.hex())
    out.append("constexpr double kExpLn2Hi = %s;      // ln2/1024, high 32 bits" % e_hi.hex())
    out.append("constexpr double kExpLn2Lo = %s;      // ln2/1024 - high part" % e_lo.hex())
    out.append("constexpr double kLogLn2Hi = %s;      // ln 2, high 32 bits" % l_hi.hex())
    out.append("constexpr double kLogLn2Lo = %s;      // ln 2 - high part" % l_lo.hex())
    out.append("constexpr double kLog54Ln2 = %s;      // 54 ln 2 (subnormal log)" % ln2_54.hex())
    out.append("constexpr int kExpTabSize = 1024;")
    out.append("constexpr int kLogTabSize = 128;")
    out.append("inline const double* exp2_table_host() {")
    out.append("  static const double t[1024] = {")
    for i in range(0, 1024, 4):
        out.append("    " + ", ".join(v.hex() for v in exp_tab[i:i + 4]) + ",")
    out.append("  };")
    out.append("  return t;")
    out.append("}")
    out.append("inline const double* log_table_host() {")
    out.append("  // pairs (invc_j, logc_j)")
    out.append("  static const double t[256] = {")
    for j in range(128):
        out.append("    %s, %s," % (invc[j].hex(), logc[j].hex()))
    out.append("  };")
    out.append("  return t;")
    out.append("}")
    out.append("}  // namespace rde")
    with open(os.path.join(HERE, "fastmath_tables.h"), "w") as f:
        f.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
