"""Writes mg_log_table.h, the tables of the binary64 logarithm that the
binary64 mode applies to its uniforms u = (2w + 1) 2^-33 (mg_em_step.cuh,
ln_u01):

* c_j = 64 / (64 + j), j = 0..64, rounded to binary64, and -ln(c_j) of that
  rounded value to 50 significant digits, as a pair of binary64 numbers
  (hi = the nearest binary64, lo = the nearest to the rest): then
  ln f = -ln(c_j) + ln(f c_j) holds exactly for the stored c_j;
* -k ln 2, k = 0..33, as the same kind of pair.

Run from this directory:  python gen_log_table.py > mg_log_table.h
"""
import mpmath

mpmath.mp.dps = 50


def pair(v):
    hi = float(v)
    return hi, float(v - mpmath.mpf(hi))


def main():
    c, thi, tlo = [], [], []
    for j in range(65):
        cj = float(mpmath.mpf(64) / (64 + j))  # correctly rounded
        h, l = pair(-mpmath.log(mpmath.mpf(cj)))
        c.append(cj)
        thi.append(h)
        tlo.append(l)
    ehi, elo = zip(*(pair(-k * mpmath.log(2)) for k in range(34)))

    def arr(name, vals):
        body = ",\n".join("    " + ", ".join(v.hex() for v in vals[i:i + 3])
                          for i in range(0, len(vals), 3))
        return f"__device__ const double {name}[{len(vals)}] = {{\n{body}}};\n"

    print("// mg_log_table.h -- written by gen_log_table.py (do not edit): the tables")
    print("// of the binary64 logarithm of the binary64 mode's uniforms.")
    print("#pragma once\n\nnamespace mg {\n")
    print("// c_j = 64 / (64 + j) rounded to binary64; -ln(c_j) = kLogTHi[j] + kLogTLo[j]")
    print(arr("kLogC", c))
    print(arr("kLogTHi", thi))
    print(arr("kLogTLo", tlo))
    print("// -k ln 2 = kLn2Hi[k] + kLn2Lo[k], k = 0..33")
    print(arr("kLn2Hi", list(ehi)))
    print(arr("kLn2Lo", list(elo)))
    print("}  // namespace mg")


if __name__ == "__main__":
    main()
