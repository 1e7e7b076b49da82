"""Writes mg_log_table.h, the tables of the binary64 logarithm that the
binary64 mode applies to its uniforms u = (2w + 1) 2^-33 (mg_em_step.cuh,
ln_u01):

* c_j = 64 / (64 + j), j = 0..64, rounded to binary64;
* for k = 0..33 and j = 0..63, -k ln 2 - ln(c_j) of that rounded c_j to 50
  significant digits, as a pair of binary64 numbers (hi = the nearest
  binary64, lo = the nearest to the rest), so that
  ln(2^-k f) = (hi + lo) + ln(f c_j) holds exactly for the stored c_j and
  one 16-byte load gives both parts.

Run from this directory:  python gen_log_table.py > mg_log_table.h
"""
import mpmath

mpmath.mp.dps = 50

K, J = 34, 64


def pair(v):
    hi = float(v)
    return hi, float(v - mpmath.mpf(hi))


def main():
    c = [float(mpmath.mpf(64) / (64 + j)) for j in range(65)]  # correctly rounded
    kj = [pair(-k * mpmath.log(2) - mpmath.log(mpmath.mpf(c[j])))
          for k in range(K) for j in range(J)]

    def arr(vals):
        body = ",\n".join("    " + ", ".join(v.hex() for v in vals[i:i + 3])
                          for i in range(0, len(vals), 3))
        return f"__device__ const double kLogC[{len(vals)}] = {{\n{body}}};\n"

    def arr2(name, vals):
        body = ",\n".join("    " + ", ".join(f"{{{h.hex()}, {l.hex()}}}" for h, l in vals[i:i + 2])
                          for i in range(0, len(vals), 2))
        return f"__device__ const double2 {name}[{len(vals)}] = {{\n{body}}};\n"

    print("// mg_log_table.h -- written by gen_log_table.py (do not edit): the tables")
    print("// of the binary64 logarithm of the binary64 mode's uniforms.")
    print("#pragma once\n\nnamespace mg {\n")
    print("// c_j = 64 / (64 + j) rounded to binary64")
    print(arr(c))
    print(f"// -k ln 2 - ln(c_j) = kLogKJ[{J} k + j].x + kLogKJ[{J} k + j].y, "
          f"k = 0..{K - 1}, j = 0..{J - 1}")
    print(arr2("kLogKJ", kj))
    print("}  // namespace mg")


if __name__ == "__main__":
    main()
