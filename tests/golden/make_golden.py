"""Write tests/golden/oracle_values.json from the FP64 oracle alone.

The paper prints no worked numerical example, so these stored values are not
the paper's: they freeze the oracle's own output at fixed points, so that a
change of platform (x86 vs Arm), compiler or oracle arithmetic shows up as a
failing test that has to be justified. Run from the repository root:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_values.json")


def GOLDEN_SPECS():
    """The models frozen here: pi pi pi (10, 30 knots), K pi pi (40), K K K (40)
    and the Re/Im S-wave form of the 10-knot pi pi pi model."""
    return (synth.pipipi(10), synth.pipipi(30), synth.kpipi(40), synth.kkk(40),
            synth.as_reim(synth.pipipi(10)))


def lattice(spec, n):
    t = spec.s_lo + (spec.s_hi - spec.s_lo) * (np.arange(n) + 0.5) / n
    a, b = np.meshgrid(t, t, indexing="ij")
    return np.stack([a.ravel(), b.ravel()], 1)


def main():
    cases = {}
    for spec in GOLDEN_SPECS():
        o = oracle.Oracle(spec)
        pts = lattice(spec, 9)
        pts = pts[o.inside(pts)]
        norm = lattice(spec, 40)
        norm = norm[o.inside(norm)]
        data = lattice(spec, 13)
        data = data[o.inside(data)]
        entry = {"events": pts.tolist(), "data": data.tolist(), "norm_side": 40}
        scale = 0.02 if spec.swave_form == "reim" else 0.05
        for label, p in (("true", synth.true_params(spec)),
                         ("perturbed", synth.perturbed_params(spec, 3, scale))):
            A = o.amp(p, pts)
            v, g = o.nll_grad(p, data, norm, threads=1)
            entry[label] = {"params": p.tolist(), "amp_re": A.real.tolist(),
                            "amp_im": A.imag.tolist(), "nll": v, "grad": g.tolist()}
        cases[spec.name] = entry
    with open(OUT, "w") as f:
        json.dump(cases, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
