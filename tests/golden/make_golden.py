"""Writes the stored expected values under tests/golden/ from the oracle alone.

analytic_line_ring_64.txt: the oracle's pierced faces of the 64^3 analytic
field (a straight vortex line along z through (31.37, 30.81) times a ring of
radius 12 h centred at (32, 32, 40), each factor r e^{i phi} / sqrt(r^2 + xi^2)
with xi = 2 h): face id, winding (Eq. 5 on every plaquette, Sec. 2.2.2) and the
sample of the face (the zero of its bilinear interpolant, the argmin of Eq. 6,
Sec. 3.3.3) in grid units, with its residual and flags.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402


def analytic_rows():
    psi = synth.analytic_line_ring()
    w, _ = oracle.identify(psi)
    ids, wn = oracle.face_list(w)
    loc = oracle.localize(psi, ids, wn)
    return psi.shape, ids, wn, loc


def main():
    shape, ids, wn, loc = analytic_rows()
    path = os.path.join(HERE, "analytic_line_ring_64.txt")
    with open(path, "w") as fh:
        fh.write("# pierced faces of the 64^3 analytic line and ring field, written by\n")
        fh.write("# tests/golden/make_golden.py from the FP64 oracle (Eq. 5, Sec. 2.2.2;\n")
        fh.write("# Eq. 6, Sec. 3.3.3).  Columns: face id = (linear node index << 2) | o\n")
        fh.write("# (o: 0 xy, 1 yz, 2 zx), winding, x y z of the sample (grid units),\n")
        fh.write("# residual |F|^2 at the sample, flags (1 anomalous, 2 ill-conditioned).\n")
        fh.write(f"# shape {shape[0]} {shape[1]} {shape[2]}\n")
        for k in range(len(ids)):
            x, y, z = loc["xyz"][k]
            fh.write(f"{int(ids[k])} {int(wn[k])} {x:.17g} {y:.17g} {z:.17g} "
                     f"{loc['resid'][k]:.17g} {int(loc['flags'][k])}\n")
    print(path, len(ids), "faces")


if __name__ == "__main__":
    main()
