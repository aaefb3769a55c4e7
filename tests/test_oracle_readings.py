"""Readings of the paper that the CUDA path relies on, checked on the oracle (CPU).

The backward sweep factors S = R Q on the bond toward the root (Eq. (tt_cbc_qr_decomp)).
When S has at least as many rows as columns, Q may be any unitary of the column space:
the output state does not depend on the choice.  The CUDA path takes Q = I there, which
also spares CholeskyQR an ill-conditioned square Gram; this pins that the choice leaves
the state unchanged (the bond is the column count either way).
"""
import numpy as np
import pytest

from oracle import cbc, metrics
from synth import make_problem


def _identity_for_square(monkeypatch):
    orig = cbc.lq_rows
    hits = []

    def lq(S):
        m, n = S.shape
        if m >= n:
            hits.append((m, n))
            return S.copy(), np.eye(n, dtype=S.dtype)
        return orig(S)

    monkeypatch.setattr(cbc, "lq_rows", lq)
    return hits


@pytest.mark.parametrize("case", [
    dict(L=8, chi=8, D=4, max_bond=8, dtype=np.float64, seed=0),
    dict(L=9, chi=12, D=3, max_bond=10, dtype=np.complex128, seed=1),
    dict(L=7, chi=6, D=2, d=3, max_bond=9, dtype=np.complex128, seed=2),
])
def test_square_or_tall_S_takes_identity(case, monkeypatch):
    p = make_problem(2, **case)
    ref = cbc.cbc(p.state.parent, p.state.tensors, p.op.tensors, p.max_bond)
    hits = _identity_for_square(monkeypatch)
    alt = cbc.cbc(p.state.parent, p.state.tensors, p.op.tensors, p.max_bond)
    assert hits, "the case has no square or tall S"
    assert alt.out_bonds == ref.out_bonds
    assert metrics.rel_err(p.state.parent, alt.tensors, ref.tensors) < 1e-12
