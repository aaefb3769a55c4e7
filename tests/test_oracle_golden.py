"""The oracle and the generators against the stored brute-force fixture."""
import json
import os

import numpy as np

from oracle import brute, cbc
from synth import make_problem

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cfg1_bruteforce.json")


def test_cfg1_against_fixture():
    g = json.load(open(GOLD))
    p = make_problem(1)
    ex = brute.apply_dense(p.state.parent, p.state.tensors, p.op.tensors)
    assert abs(np.linalg.norm(ex) - g["norm_O_psi"]) <= 1e-13 * g["norm_O_psi"]
    for i, s in g["schmidt"].items():
        got = brute.schmidt_values(p.state.parent, p.state.phys, ex, int(i))
        np.testing.assert_allclose(got[: len(s)], s, rtol=1e-10, atol=1e-14 * s[0])
    for mb, e in g["cbc_rel_err"].items():
        r = cbc.cbc(p.state.parent, p.state.tensors, p.op.tensors, int(mb))
        got = brute.dense_state(p.state.parent, r.tensors)
        err = np.linalg.norm(got - ex) / np.linalg.norm(ex)
        assert abs(err - e) <= 1e-10 + 1e-8 * e, (mb, err, e)
    # the cap-16 run is untruncated: exact up to rounding
    assert g["cbc_rel_err"]["16"] < 1e-13
    # the cap-8 error is at least the Eckart-Young bound on the middle cut
    tail = np.sqrt(np.sum(np.array(g["schmidt"]["4"])[8:] ** 2)) / g["norm_O_psi"]
    assert g["cbc_rel_err"]["8"] >= tail
