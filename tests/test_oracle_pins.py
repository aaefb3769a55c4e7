"""The oracle against brute force, the Eckart-Young bound and the paper's invariants."""
import numpy as np
import pytest

from oracle import brute, cbc, metrics
from synth import make_problem

from pins import ALL_CHECKS


@pytest.mark.parametrize("check", ALL_CHECKS, ids=lambda f: f.__name__)
def test_pin(check):
    check(cbc)


def test_choose_rank_rules():
    s = np.array([4.0, 2.0, 1.0, 0.5, 1e-14])
    assert cbc.choose_rank(s, 0, 0.0) == 4            # eps_rank drops the 1e-14
    assert cbc.choose_rank(s, 2, 0.0) == 2            # max_bond cap
    # tol: discarded weight of k=3 is 0.25 (+tiny) <= tol^2 * 21.25 iff tol >= 0.1085
    assert cbc.choose_rank(s, 0, 0.11) == 3
    assert cbc.choose_rank(s, 0, 0.10) == 4
    assert cbc.choose_rank(s, 2, 0.11) == 2            # both rules: the smaller k
    assert cbc.choose_rank(np.zeros(3), 5, 0.0) == 1   # zero matrix keeps one (zero) row


def test_dense_state_product_closed_form():
    """A bond-1 TTNS is the Kronecker product of its site vectors (node order)."""
    rng = np.random.default_rng(0)
    parent = [-1, 0, 1, 1]
    vecs = [rng.standard_normal(d) + 1j * rng.standard_normal(d) for d in (2, 3, 2, 2)]
    ts = [vecs[0].reshape(1, 2, 1), vecs[1].reshape(1, 3, 1, 1), vecs[2].reshape(1, 2),
          vecs[3].reshape(1, 2)]
    want = np.kron(np.kron(np.kron(vecs[0], vecs[1]), vecs[2]), vecs[3])
    np.testing.assert_allclose(brute.dense_state(parent, ts), want, rtol=1e-14, atol=1e-14)


def test_dense_operator_product_closed_form():
    """A bond-1 TTNO is the Kronecker product of its site matrices (node order)."""
    rng = np.random.default_rng(1)
    parent = [-1, 0, 0]
    mats = [rng.standard_normal((d, d)) for d in (2, 3, 2)]
    ws = [mats[0].reshape(1, 2, 2, 1, 1), mats[1].reshape(1, 3, 3), mats[2].reshape(1, 2, 2)]
    want = np.kron(np.kron(mats[0], mats[1]), mats[2])
    np.testing.assert_allclose(brute.dense_operator(parent, ws), want, rtol=1e-14, atol=1e-14)


def test_metric_against_dense_difference():
    p = make_problem(3, L=2, chi=6, D=3, max_bond=4, dtype=np.float64)
    a = cbc.cbc(p.state.parent, p.state.tensors, p.op.tensors, 4)
    b = cbc.cbc(p.state.parent, p.state.tensors, p.op.tensors, 3)
    va = brute.dense_state(p.state.parent, a.tensors)
    vb = brute.dense_state(p.state.parent, b.tensors)
    want = np.linalg.norm(va - vb) / np.linalg.norm(vb)
    got = metrics.rel_err(p.state.parent, a.tensors, b.tensors)
    assert abs(got - want) <= 1e-12 * max(want, 1.0)
    assert abs(metrics.tree_norm(p.state.parent, a.tensors) - np.linalg.norm(va)) <= 1e-14


def test_metric_resolves_tiny_differences():
    """A relative change of 1e-12 in one tensor is measured as 1e-12 (no sqrt(eps)
    cancellation floor), also with the change carried by the log scale."""
    p = make_problem(2, L=10, chi=8, D=4, max_bond=8, dtype=np.complex128)
    a = cbc.cbc(p.state.parent, p.state.tensors, p.op.tensors, 8).tensors
    d = 1e-12
    b = [t * (1 + d) if i == 4 else t for i, t in enumerate(a)]
    assert abs(metrics.rel_err(p.state.parent, b, a) - d) < 1e-3 * d
    assert abs(metrics.rel_err(p.state.parent, a, a, np.log1p(d), 0.0) - d) < 1e-3 * d


def test_oracle_output_bonds_clamped():
    """Forward ranks never exceed d * previous rank nor the cap; backward bonds never
    exceed d * next bond (Hilbert-space limits of the projection)."""
    p = make_problem(2, L=12, chi=16, D=4, max_bond=12, dtype=np.complex128)
    r = cbc.cbc(p.state.parent, p.state.tensors, p.op.tensors, 12)
    for i in range(1, len(r.env_ranks)):
        assert r.env_ranks[i] <= min(12, 2 * r.env_ranks[i - 1])
    L = len(r.out_bonds)
    for i in range(1, L - 1):
        assert r.out_bonds[i] <= 2 * r.out_bonds[i + 1]
    assert r.out_bonds[L - 1] <= 2


def test_metric_single_node():
    """A one-site network has no bond: the distance is that of the two tensors."""
    a = [np.array([[1.0, 2.0]])]
    b = [np.array([[1.0, 2.5]])]
    assert abs(metrics.rel_err([-1], a, b) - 0.5 / np.linalg.norm([1.0, 2.5])) < 1e-15


def test_chain_applied_norm_matches_brute_force():
    """The sandwich <psi|O^H O|psi> equals ||O psi||^2 of the dense vector (Eqs. (ttns),
    (ttno)), real and complex, d = 2 and 3."""
    from oracle import brute, metrics
    for kw in [dict(L=6, chi=6, D=3, dtype=np.complex128), dict(L=7, chi=8, D=4, d=3,
                                                              dtype=np.float64, seed=2)]:
        p = make_problem(2, max_bond=0, **kw)
        ex = brute.apply_dense(p.state.parent, p.state.tensors, p.op.tensors)
        got = metrics.chain_applied_norm2(p.state.tensors, p.op.tensors)
        assert abs(got - np.linalg.norm(ex) ** 2) <= 1e-13 * np.linalg.norm(ex) ** 2


def test_chain_applied_overlap_matches_brute_force():
    """<phi|O|psi> of two chains equals the dense inner product (the CBC output of the
    oracle as phi, so the value is also ||psi'||^2 by the projection identity)."""
    from oracle import brute, metrics
    from oracle import cbc as ocbc
    p = make_problem(2, L=7, chi=8, D=3, max_bond=5, dtype=np.complex128, seed=3)
    r = ocbc.cbc(p.state.parent, p.state.tensors, p.op.tensors, p.max_bond)
    ex = brute.apply_dense(p.state.parent, p.state.tensors, p.op.tensors)
    phi = brute.dense_state(p.state.parent, r.tensors)
    got = metrics.chain_applied_overlap(p.state.tensors, p.op.tensors, r.tensors)
    want = np.vdot(phi, ex)
    assert abs(got - want) <= 1e-13 * abs(want)
    assert abs(got.real - np.linalg.norm(phi) ** 2) <= 1e-12 * abs(want)
