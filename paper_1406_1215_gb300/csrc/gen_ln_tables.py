"""Writes ln_tables.h: the reduction tables of the logarithms (ln(64/J) for
J = 32..64, and for J = 65..128 ln(128/J); ln(1024/J) for J = 512..1024) and
the atanh-series coefficients 1/(2k+1) and the multiples e ln2, split into float-float and
double-double pairs.

Values come from Python's decimal module at 80 significant digits (its ln is
correctly rounded), so each split is exact to the precision of the pair.
Run: python gen_ln_tables.py  (rewrites ln_tables.h beside this file).
"""
import decimal
import os
import struct

decimal.getcontext().prec = 80
D = decimal.Decimal


def f32(x: D) -> float:
    # round-to-nearest float32 of a Decimal (via float64 rounding of an
    # already very close value, then float32 of the remainder-corrected value)
    if x == 0:
        return 0.0
    v = struct.unpack("f", struct.pack("f", float(x)))[0]
    # correct a possible double rounding: pick the nearest of v and its neighbours
    best = v
    bits = struct.unpack("I", struct.pack("f", v))[0]
    for d in (-1, 1):
        cand = struct.unpack("f", struct.pack("I", (bits + d) & 0xFFFFFFFF))[0]
        if cand == cand and abs(D(cand) - x) < abs(D(best) - x):
            best = cand
    return best


def f64(x: D) -> float:
    return float(x)  # Decimal -> float is correctly rounded


def hexf(x: float) -> str:
    return float(x).hex()


def split_ff(x: D):
    hi = f32(x)
    lo = f32(x - D(hi))
    return hi, lo


def split_dd(x: D):
    hi = f64(x)
    lo = f64(x - D(hi))
    return hi, lo


def main():
    lines = [
        "// Generated by gen_ln_tables.py -- do not edit.",
        "// CL_LNT2_FF[J - 32] = ln(64 / J) for J = 32..64 and ln(128 / J) for",
        "// J = 65..128 (never negative), as float-float pairs (one 8-byte load);",
        "// CL_LNT_DD[J - 32] = ln(64 / J), J = 32..64, as double-double pairs;",
        "// ATANH_DD[k] = 1 / (2k + 1) as double-double pairs, k = 0..9.",
        "// Global (not constant) memory: lanes index the table divergently, which",
        "// the constant cache would serialise; reads go through L1.",
        "#pragma once",
        "",
        "static __device__ __align__(8) float2 CL_LNT2_FF[97] = {",
    ]
    for J in range(32, 129):
        num = 64 if J <= 64 else 128
        hi, lo = split_ff((D(num) / D(J)).ln())
        lines.append(f"  {{{hexf(hi)}f, {hexf(lo)}f}},  // J = {J}")
    lines.append("};")
    lines.append("// CL_LNR_FF[J - 512] = ln(1024 / J), J = 512..1024: the finer table of -ln r")
    lines.append("static __device__ __align__(8) float2 CL_LNR_FF[513] = {")
    for J in range(512, 1025):
        hi, lo = split_ff((D(1024) / D(J)).ln())
        lines.append(f"  {{{hexf(hi)}f, {hexf(lo)}f}},")
    lines.append("};")
    lines.append("static __device__ double CL_LNT_DD[33][2] = {")
    for J in range(32, 65):
        hi, lo = split_dd((D(64) / D(J)).ln())
        lines.append(f"  {{{hexf(hi)}, {hexf(lo)}}},  // J = {J}")
    lines.append("};")
    ln2 = D(2).ln()
    lines.append("// CL_ELN2_FF[e] = e ln2, e = 0..63, as float-float pairs (the exponent term of -ln r)")
    lines.append("static __device__ __align__(8) float2 CL_ELN2_FF[64] = {")
    for e in range(64):
        hi, lo = split_ff(D(e) * ln2)
        lines.append(f"  {{{hexf(hi)}f, {hexf(lo)}f}},")
    lines.append("};")
    hi, lo = split_ff(ln2)
    lines.append(f"#define CL_LN2_FF_HI {hexf(hi)}f")
    lines.append(f"#define CL_LN2_FF_LO {hexf(lo)}f")
    hi, lo = split_dd(ln2)
    lines.append(f"#define CL_LN2_DD_HI {hexf(hi)}")
    lines.append(f"#define CL_LN2_DD_LO {hexf(lo)}")
    hi, lo = split_ff(D(1) / D(3))
    lines.append(f"#define CL_THIRD_FF_HI {hexf(hi)}f")
    lines.append(f"#define CL_THIRD_FF_LO {hexf(lo)}f")
    lines.append("static __device__ double CL_ATANH_DD[10][2] = {")
    for k in range(10):
        hi, lo = split_dd(D(1) / D(2 * k + 1))
        lines.append(f"  {{{hexf(hi)}, {hexf(lo)}}},  // 1/{2 * k + 1}")
    lines.append("};")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ln_tables.h")
    text = "\n".join(lines) + "\n"
    with open(out, "w") as f:
        f.write(text)
    return text


if __name__ == "__main__":
    main()
