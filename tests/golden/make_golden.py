"""Write the stored expected values under tests/golden/ from the oracle only.

    python tests/golden/make_golden.py

irkgl16_coeffs_fp64.txt: the FP64 tables c, b, mu, eta, nu of the 8-stage
Gauss-Legendre method in the second-order floating-point form of
arXiv 2511.03655 Sec. 2.4 (Eq. Yi2 for mu, Eq. Qi2 / Eq. sympl_cond_2 for
eta, Eq. Pol0 for nu), as hex floats, one "name i j value" per line.
henon_heiles_ic.txt: the Henon-Heiles initial condition of Sec. 5.1
(q1 = 0, q2 = 0.3, p2 = 0.2, p1 > 0 from H = 1/12).
"""
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import coeffs  # noqa: E402


def main():
    hdr = ("# IRKGL16 FP64 coefficient tables (arXiv 2511.03655, Sec. 2.4: mu from Eq. Yi2,\n"
           "# eta from Eq. Qi2 with Eq. sympl_cond_2 exact, nu from Eq. Pol0 scaled by 1/b).\n"
           "# Written by tests/golden/make_golden.py from oracle/coeffs.py. name i j hexfloat\n")
    with open(os.path.join(HERE, "irkgl16_coeffs_fp64.txt"), "w") as f:
        f.write(hdr + coeffs.hexdump(coeffs.fp64_tables(8)))
    # Sec. 5.1: q1(0) = 0, q2(0) = 0.3, p2(0) = 0.2, p1 > 0 from H = 1/12
    q1, q2, p2 = 0.0, 0.3, 0.2
    rest = p2 * p2 / 2 + (q1 * q1 + q2 * q2) / 2 + (q1 * q1 * q2 - q2 ** 3 / 3)
    p1 = math.sqrt(2 * (1.0 / 12 - rest))
    with open(os.path.join(HERE, "henon_heiles_ic.txt"), "w") as f:
        f.write("# Henon-Heiles initial condition, arXiv 2511.03655 Sec. 5.1 (H = 1/12)\n")
        f.write("# q1 q2 p1 p2 (hex floats)\n")
        f.write(" ".join(float.hex(x) for x in (q1, q2, p1, p2)) + "\n")


if __name__ == "__main__":
    main()
