"""Write the oracle's Lebedev-Laikov quadrature tables (Sec. 2.2 uses them for
every sphere integral) from scipy.integrate.lebedev_rule.

Test infrastructure: the files written here are read only by the oracle.
Run once: python oracle/make_lebedev_data.py
"""
import os

import numpy as np
from scipy.integrate import lebedev_rule

DEGREES = [3, 5, 7, 9, 11, 13, 15, 17, 19, 21, 23, 25, 27, 29, 31, 35, 41, 47]

if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")
    os.makedirs(out, exist_ok=True)
    for d in DEGREES:
        x, w = lebedev_rule(d)
        n = x.shape[1]
        with open(os.path.join(out, "lebedev_%d.txt" % n), "w") as f:
            f.write("# Lebedev-Laikov rule, %d points, exact to degree %d; columns x y z w (sum w = 4 pi)\n" % (n, d))
            for k in range(n):
                f.write("%.17e %.17e %.17e %.17e\n" % (x[0, k], x[1, k], x[2, k], w[k]))
