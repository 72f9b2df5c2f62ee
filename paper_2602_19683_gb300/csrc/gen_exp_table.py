"""Writes exp_table.cuh: the constants of the table-driven exponential of se_kernel.cuh (Tang's method,
ACM TOMS 15(2), 1989), computed here in 60-digit decimal arithmetic and rounded once to FP64.

    python paper_2602_19683_gb300/csrc/gen_exp_table.py > paper_2602_19683_gb300/csrc/exp_table.cuh

exp(x) = 2^m * 2^(j/1024) * exp(r) with x = (1024 m + j) ln2/1024 + r, |r| <= ln2/2048. Emitted:
1024/ln2 (FP64), ln2/1024 split into a head with 32 significant bits (so that N * head is exact for
|N| < 2^21) and the FP64-rounded remainder, and 2^(j/1024), j = 0..1023, as a head (FP64-rounded) and
a tail (the FP64-rounded remainder), so that head + tail carries the table value to about 2^-106.
"""
from decimal import Decimal, getcontext
import math

getcontext().prec = 60
BITS = 10
NT = 1 << BITS


def d_ln2() -> Decimal:
    return Decimal(2).ln()


def to_double(x: Decimal) -> float:
    """Correctly rounded FP64 value of a decimal (via the exact rational of a float neighbour)."""
    f = float(x)  # Python's Decimal -> float conversion rounds correctly
    return f


def hexd(f: float) -> str:
    return f"{f.hex()}"


def head32(x: Decimal) -> float:
    """x truncated to 32 significant bits (exactly representable in FP64)."""
    e = math.floor(math.log2(float(x)))
    scale = Decimal(2) ** (31 - e)
    return float(int(x * scale)) / float(2 ** (31 - e))


def main():
    ln2 = d_ln2()
    inv = to_double(Decimal(NT) / ln2)
    c = ln2 / NT
    c1 = head32(c)
    c2 = to_double(c - Decimal(c1))
    print("// Generated by gen_exp_table.py: constants of the table-driven exponential in se_kernel.cuh")
    print("// (Tang's method). Do not edit by hand.")
    print("#pragma once")
    print("namespace gpk {")
    print(f"constexpr int kExpTableBits = {BITS};  // table of 2^(j/{NT}), j < {NT}")
    print(f"constexpr double kExpInvLn2xN = {hexd(inv)};  // {NT} / ln 2")
    print(f"constexpr double kExpLn2byNHi = {hexd(c1)};  // ln 2 / {NT}, first 32 significant bits")
    print(f"constexpr double kExpLn2byNLo = {hexd(c2)};  // ln 2 / {NT} - kExpLn2byNHi")
    heads, tails = [], []
    for j in range(NT):
        v = (Decimal(j) / NT * ln2).exp()  # 2^(j/NT)
        h = to_double(v)
        t = to_double(v - Decimal(h))
        heads.append(h)
        tails.append(t)
    print(f"// 2^(j/{NT}) = kExp2Head[j] + kExp2Tail[j]")
    print(f"__device__ const double kExp2Head[{NT}] = {{")
    for j in range(0, NT, 4):
        print("    " + ", ".join(hexd(x) for x in heads[j:j + 4]) + ",")
    print("};")
    print(f"__device__ const double kExp2Tail[{NT}] = {{")
    for j in range(0, NT, 4):
        print("    " + ", ".join(hexd(x) for x in tails[j:j + 4]) + ",")
    print("};")
    print("}  // namespace gpk")


if __name__ == "__main__":
    main()
