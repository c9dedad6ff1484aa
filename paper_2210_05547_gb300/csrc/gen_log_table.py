"""Write log_table.h: the constants of the table-driven logarithm in fp64_fast.cuh.

The method follows Tang's table-driven logarithm (P. T. P. Tang, "Table-driven implementation of
the logarithm function in IEEE floating-point arithmetic", ACM TOMS 16(4), 1990) in the
reciprocal form: x = 2^m y with y in [1, 2), j = the top 7 fraction bits of y, c_j = 1 + (j + 1/2)
/ 128 the centre of y's interval, and

    log x = m ln2 - log(inv_j) + log1p(y inv_j - 1),

inv_j being the binary64 nearest to 1 / c_j, so that |y inv_j - 1| < 2^-8. This script computes,
in 60-digit decimal arithmetic,
  * inv_j for j = 0..127;
  * -log(inv_j) of that binary64 value, split into a binary64 head and the binary64 nearest to the
    remainder;
  * ln2 split as LN2_HI (42 significant bits, so that m * LN2_HI is exact for |m| < 2^11) and the
    binary64 nearest to the remainder.
Usage: python gen_log_table.py  (rewrites log_table.h beside this file).
"""
from __future__ import annotations

import decimal
import os
import struct

D = decimal.Decimal
decimal.getcontext().prec = 60
N = 128


def trunc_bits(x: float, bits: int) -> float:
    """x with its significand cut to `bits` bits (towards zero)."""
    u = struct.unpack("<Q", struct.pack("<d", x))[0]
    drop = 53 - bits
    u &= ~((1 << drop) - 1)
    return struct.unpack("<d", struct.pack("<Q", u))[0]


def tables():
    """(rows, LN2_HI, LN2_LO): rows[j] = (inv_j, -log(inv_j) head, remainder) as binary64."""
    rows = []
    for j in range(N):
        c = 1 + (D(j) + D("0.5")) / N
        v = float(1 / c)                       # Decimal -> binary64 rounds to nearest
        t = -D(v).ln()
        h = float(t)
        rows.append((v, h, float(t - D(h))))
    ln2 = D(2).ln()
    ln2_hi = trunc_bits(float(ln2), 42)
    return rows, ln2_hi, float(ln2 - D(ln2_hi))


def render() -> str:
    rows, ln2_hi, ln2_lo = tables()
    out = ["// Generated by gen_log_table.py: constants of the table-driven logarithm\n",
           "// (Tang 1990, reciprocal form) in fp64_fast.cuh. Do not edit.\n#pragma once\n\n",
           "namespace hyp {\n\n",
           f"constexpr int LOG_TABLE_N = {N};\n",
           f"constexpr double LOG_LN2_HI = {ln2_hi.hex()};   // ln2, 42 bits\n",
           f"constexpr double LOG_LN2_LO = {ln2_lo.hex()};   // ln2 - LOG_LN2_HI\n",
           "// per j: the binary64 nearest to 1 / (1 + (j + 1/2) / 128), then -log of that value\n",
           "// as a head and the binary64 nearest to the remainder\n",
           "__device__ const double LOG_TABLE[LOG_TABLE_N][3] = {\n"]
    for v, h, lo in rows:
        out.append(f"    {{{v.hex()}, {h.hex()}, {lo.hex()}}},\n")
    out.append("};\n\n}  // namespace hyp\n")
    return "".join(out)


def main() -> None:
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "log_table.h")
    with open(out, "w") as fh:
        fh.write(render())


if __name__ == "__main__":
    main()
