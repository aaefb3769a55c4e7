"""Write tests/golden/cfg1_bruteforce.json from brute force (oracle/ only).

The paper prints no numbers for its worked example (App. A is diagrammatic), so the
stored values come from the dense definitions, Eqs. (ttns), (ttno), (abstr_application):
the norm of O|psi> for the 8-site chain (d=2, chi=8, D=4, float64, seed 0), its Schmidt
spectra on every cut (their tails give the Eckart-Young bound at each cap), and the
relative error of the oracle's CBC output at caps 8 and 16.

Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import brute, cbc  # noqa: E402
from synth import make_problem  # noqa: E402


def main():
    p = make_problem(1)
    par, ph = p.state.parent, p.state.phys
    ex = brute.apply_dense(par, p.state.tensors, p.op.tensors)
    out = {"citation": "Sec. III A (tensor-train CBC) and Eq. (abstr_application); "
                       "values from brute force, the paper prints none",
           "workload": "chain L=8 d=2 chi=8 D=4 float64 seed 0",
           "norm_O_psi": float(np.linalg.norm(ex)),
           "schmidt": {str(i): [float(x) for x in brute.schmidt_values(par, ph, ex, i)]
                       for i in range(1, len(par))},
           "cbc_rel_err": {}}
    for mb in (8, 16):
        r = cbc.cbc(par, p.state.tensors, p.op.tensors, mb)
        got = brute.dense_state(par, r.tensors)
        out["cbc_rel_err"][str(mb)] = float(np.linalg.norm(got - ex) / np.linalg.norm(ex))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cfg1_bruteforce.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
