"""Write the stored expected values under tests/golden/ from the FP64 oracle.

Only oracle/ and the seeded input generators are used.  The cases are tiny
(a few hundred grid points) so that every number can be re-derived by hand
or by any independent FP64 implementation of the definitions:

* Eq. 4 / Eq. VUP: output probabilities H[k, b] (sum of the normalised
  input probabilities of the grid points whose model value lies in bin b);
* Sec. 5.2 expectation fields: raw moments sum_i W y^j and central moments
  about the mean, j = 1..4;
* Sec. 5.2 / IPSA: derivatives of the raw moments with respect to each
  density's mu and sigma (uniform axes give 0).

Run:  python tests/golden/make_golden.py   (rewrites the .txt files)
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_1908_11246_gb300 import inputs as I  # noqa: E402


def cases():
    # 1-D: y = x^2 on 16 midpoints of [-1, 1], three Gaussians, 4 bins
    d1 = I.Densities(np.zeros((3, 1), np.uint8), np.array([[-0.3], [0.0], [0.45]]),
                     np.array([[0.2], [0.5], [0.15]]), np.zeros((3, 1)), np.zeros((3, 1)))
    yield I.Problem("tiny_1d_square", (16,), (-1.0,), (1.0,), I.MODEL_POLY, (0.0, 0.0, 1.0), d1, 4)
    # 2-D: y = sin x1 + 7 sin^2 x2 on a 6 x 5 grid, one density of each kind, 3 bins
    kind = np.array([[0, 0], [1, 1], [2, 0]], np.uint8)
    mu = np.array([[0.3, -0.5], [-1.0, 1.2], [0.8, 0.0]])
    sg = np.array([[0.9, 1.1], [2.5, 2.0], [1.0, 0.7]])
    lo = np.array([[0.0, 0.0], [0.0, 0.0], [-0.5, 0.0]])
    hi = np.array([[0.0, 0.0], [0.0, 0.0], [2.5, 0.0]])
    d2 = I.Densities(kind, mu, sg, lo, hi)
    yield I.Problem("tiny_2d_mixed", (6, 5), (-np.pi, -np.pi), (np.pi, np.pi), I.MODEL_SIN_SIN2_2D,
                    (1.0, 7.0), d2, 3)


def compute(p):
    res = O.solve(p)
    dmu, dsg = O.ipsa(p.n, p.lo, p.hi, res["y"], p.n_moments, p.dens)
    return {"hist": res["hist"], "raw": res["raw"], "central": res["central"], "dmu": dmu, "dsigma": dsg}


def path(name):
    return os.path.join(HERE, name + ".txt")


def write(p, vals):
    with open(path(p.name), "w") as f:
        f.write(f"# {p.name}: written by tests/golden/make_golden.py from the FP64 oracle\n")
        f.write("# Eq. 4 / Eq. VUP (hist), Sec. 5.2 moments (raw, central), IPSA derivatives (dmu, dsigma)\n")
        for key, a in vals.items():
            a = np.asarray(a, dtype=np.float64)
            f.write(f"{key} {' '.join(str(s) for s in a.shape)}\n")
            f.write(" ".join(repr(float(v)) for v in a.ravel()) + "\n")


def read(name):
    out = {}
    with open(path(name)) as f:
        lines = [ln for ln in f.read().splitlines() if ln and not ln.startswith("#")]
    for hdr, data in zip(lines[0::2], lines[1::2]):
        key, *shape = hdr.split()
        out[key] = np.array([float(v) for v in data.split()]).reshape([int(s) for s in shape])
    return out


if __name__ == "__main__":
    for p in cases():
        write(p, compute(p))
        print("wrote", path(p.name))
