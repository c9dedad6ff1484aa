"""Write exp_table.h: the constants of the table-driven exponential in fp64_fast.cuh.

The method is Tang's (P. T. P. Tang, "Table-driven implementation of the exponential function in
IEEE floating-point arithmetic", ACM TOMS 15(2), 1989): x = (256 m + j) ln2/256 + r with
|r| <= ln2/512, exp(x) = 2^m 2^(j/256) exp(r). This script computes, in 60-digit decimal
arithmetic,
  * 2^(j/256) for j = 0..255, each rounded to the nearest binary64;
  * ln2/256 split as C_HI + C_LO (Cody and Waite's technique), C_HI with 33 significant bits so
    that n * C_HI is exact for |n| < 2^20, C_LO the binary64 nearest to the remainder;
  * 256/ln2 rounded to binary32 (the reduction index comes from a binary32 product).
Usage: python gen_exp_table.py  (rewrites exp_table.h beside this file).
"""
from __future__ import annotations

import decimal
import os
import struct

D = decimal.Decimal
decimal.getcontext().prec = 60
LN2 = D(2).ln()
L = 256


def trunc_bits(x: float, bits: int) -> float:
    """x with its significand cut to `bits` bits (towards zero)."""
    u = struct.unpack("<Q", struct.pack("<d", x))[0]
    drop = 53 - bits
    u &= ~((1 << drop) - 1)
    return struct.unpack("<d", struct.pack("<Q", u))[0]


def f32(x: D) -> float:
    return struct.unpack("<f", struct.pack("<f", float(x)))[0]


def tables():
    """(table, C_HI, C_LO, INV_C): 2^(j/256) for j = 0..255 as binary64, the Cody-Waite split of
    ln2/256 and 256/ln2 as a binary32 value (held in a Python float)."""
    table = [float((D(j) / L * LN2).exp()) for j in range(L)]
    c = LN2 / L
    c_hi = trunc_bits(float(c), 33)
    c_lo = float(c - D(c_hi))
    inv = f32(D(L) / LN2)
    return table, c_hi, c_lo, inv


def render() -> str:
    table, c_hi, c_lo, inv = tables()
    out = ["// Generated by gen_exp_table.py: constants of the table-driven exponential\n",
           "// (Tang 1989) in fp64_fast.cuh. Do not edit.\n#pragma once\n\n",
           "namespace hyp {\n\n",
           f"constexpr int EXP_TABLE_N = {L};\n",
           f"constexpr double EXP_C_HI = {c_hi.hex()};   // ln2/256, 33 bits\n",
           f"constexpr double EXP_C_LO = {c_lo.hex()};   // ln2/256 - EXP_C_HI\n",
           f"constexpr float EXP_INV_C = {inv.hex()}f;   // 256/ln2 in binary32\n",
           "// 2^(j/256), j = 0..255, each the binary64 nearest to the exact value\n",
           "__device__ const double EXP_TABLE[EXP_TABLE_N] = {\n"]
    for j in range(0, L, 3):
        row = ", ".join(t.hex() for t in table[j:j + 3])
        out.append(f"    {row},\n")
    out.append("};\n\n}  // namespace hyp\n")
    return "".join(out)


def main() -> None:
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "exp_table.h")
    with open(out, "w") as fh:
        fh.write(render())
    print(out)


if __name__ == "__main__":
    main()
