"""Write lebedev_tables.h, the Lebedev-Laikov rules compiled into the library.

The rules come from scipy.integrate.lebedev_rule (weights normalised to sum to
4 pi).  Run once from the repository root:
    python paper_2203_00552_gb300/csrc/gen_lebedev_tables.py
"""
import os

from scipy.integrate import lebedev_rule

DEGREES = [3, 5, 7, 9, 11, 13, 15, 17, 19, 21, 23, 25, 27, 29, 31, 35, 41, 47]

if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    lines = ["// Generated by gen_lebedev_tables.py from scipy.integrate.lebedev_rule. Do not edit.",
             "// Each rule: n points, x y z w per point, exact to the stated degree; sum w = 4 pi.",
             "#pragma once", ""]
    entries = []
    for d in DEGREES:
        x, w = lebedev_rule(d)
        n = x.shape[1]
        name = "kLebedev%d" % n
        vals = []
        for k in range(n):
            vals += [x[0, k], x[1, k], x[2, k], w[k]]
        body = ",\n".join("  " + ", ".join("%.17e" % v for v in vals[i:i + 4]) for i in range(0, len(vals), 4))
        lines.append("static const double %s[%d] = {\n%s\n};" % (name, 4 * n, body))
        entries.append((n, d, name))
    lines.append("")
    lines.append("struct LebedevRule { int n; int degree; const double* xyzw; };")
    lines.append("static const LebedevRule kLebedevRules[] = {")
    for n, d, name in entries:
        lines.append("  {%d, %d, %s}," % (n, d, name))
    lines.append("};")
    lines.append("static const int kNumLebedevRules = %d;" % len(entries))
    with open(os.path.join(here, "lebedev_tables.h"), "w") as f:
        f.write("\n".join(lines) + "\n")
