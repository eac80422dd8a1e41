"""Generate log_table.inc: the constants of the kernels' table-driven logarithm.

Method (Tang, "Table-driven implementation of the logarithm function in IEEE
floating-point arithmetic", ACM TOMS 16(4), 1990): write the argument as
2^k * m with m in [1, 2), pick the table point F_j = 1 + j/256 nearest to m,
and use log(2^k m) = k log 2 + log F_j + log(1 + (m - F_j)/F_j), the last
term by a short series since |(m - F_j)/F_j| <= 2^-9.

The leading parts k * LN2_HI + LOG_HI[j] are kept as integers in units of
2^-42 so that their sum is exact; the trailing parts (LN2_LO, LOG_LO[j]) are
doubles.  Values are computed here with 60-digit decimal arithmetic.

  python paper_1606_08281_gb300/csrc/gen_log_table.py > paper_1606_08281_gb300/csrc/log_table.inc
"""
from decimal import ROUND_HALF_EVEN, Decimal, getcontext

getcontext().prec = 60
SCALE = Decimal(2) ** 42


def split(x: Decimal):
    hi = int((x * SCALE).to_integral_value(rounding=ROUND_HALF_EVEN))
    lo = float(x - Decimal(hi) / SCALE)
    return hi, lo


def main():
    ln2_hi, ln2_lo = split(Decimal(2).ln())
    print("// Generated by gen_log_table.py -- do not edit.")
    print("// LOG_HI in units of 2^-42; LOG_LO and INV_F are doubles; F_j = 1 + j/256.")
    print(f"constexpr long long kLn2HiUnits = {ln2_hi}LL;")
    print(f"constexpr double kLn2Lo = {ln2_lo.hex()};")
    his, los, invs = [], [], []
    for j in range(257):
        F = Decimal(256 + j) / 256
        hi, lo = split(F.ln())
        his.append(f"{hi}LL")
        los.append(lo.hex())
        invs.append(float(1 / F).hex())
    for name, ty, vals in (("kLogHiUnits", "long long", his), ("kLogLo", "double", los),
                           ("kInvF", "double", invs)):
        print(f"__device__ const {ty} {name}[257] = {{")
        for i in range(0, 257, 4):
            print("    " + ", ".join(vals[i:i + 4]) + ",")
        print("};")


if __name__ == "__main__":
    main()
