"""The oracle's explicit-sample estimator against the hand-worked example of
Eq. 4 / Eq. 5 and the gradient in tests/golden (exact rationals)."""
import os
from fractions import Fraction

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "eq4_worked_example.txt")


def _load():
    vals = {}
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, val = (t.strip() for t in line.split("=", 1))
            rows = [[float(Fraction(x)) for x in r.split()] for r in val.split(";")]
            vals[key] = np.array(rows if len(rows) > 1 else rows[0])
    return vals


def test_worked_example():
    g = _load()
    R, w = g["R"], g["w"]
    assert R.shape == (int(g["N"][0]), int(g["d"][0]))
    out = oracle.saa_explicit(R, w[None], lam=float(g["lambda"][0]), grad=True)
    assert np.allclose(out["pbar"], g["pbar"], rtol=0, atol=1e-15)
    assert np.allclose(out["var"], g["var"], rtol=0, atol=1e-15)
    assert np.allclose(out["f"], g["f"], rtol=0, atol=1e-15)
    assert np.allclose(out["grad"][0], g["grad"], rtol=0, atol=1e-15)
