"""Write hb_md5_table.h: the 64 MD5 additive constants of RFC 1321 Sec. 3.4.

T[i] is the integer part of 2^32 * |sin(i)| for i = 1..64 (radians).  They
are evaluated here with mpmath at 60 significant digits, far beyond what the
floor needs, and emitted as literals so every kernel step can use them as
immediates.  Run: python gen_md5_table.py > hb_md5_table.h
"""
import mpmath

mpmath.mp.dps = 60


def table():
    return [int(mpmath.floor(mpmath.mpf(2) ** 32 * abs(mpmath.sin(i)))) for i in range(1, 65)]


def main():
    t = table()
    print("/* Generated by gen_md5_table.py: T[i-1] = floor(2^32 |sin i|), RFC 1321 Sec. 3.4. */")
    print("#pragma once")
    print("#define HB_MD5_T_TABLE \\")
    rows = []
    for r in range(16):
        rows.append("    " + ", ".join("0x%08xu" % v for v in t[4 * r: 4 * r + 4]))
    print(", \\\n".join(rows))


if __name__ == "__main__":
    main()
