"""GPU parity of the comparison methods of Sec. III C (Zip-Up, SRC, direct) against their oracle.

They run through the C ABI (zipup_apply, src_apply, direct_apply) on the same seeded inputs as the
oracle; SRC gets the same random matrices.  Bars: FP64 path <= 1e-10, mixed <= 1e-6
(relative 2-norm distance of the output states, oracle.metrics.rel_err); bonds equal.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import comparators, metrics  # noqa: E402
from synth import make_problem, sketch_matrices  # noqa: E402

FP64_BAR, MIXED_BAR = 1e-10, 1e-6


def _run(method, p, precision, arg):
    from paper_2601_19650_gb300 import _cbc

    st, op = p.state, p.op
    hs = _cbc.create_from_host(st.parent, st.phys, st.bond, st.tensors, "state")
    ho = _cbc.create_from_host(op.parent, op.phys, op.bond, op.tensors, "op")
    try:
        opt = _cbc.make_options(precision)
        if method == "zipup":
            out = _cbc.zipup_apply(hs, ho, arg[0], arg[1], opt)
        elif method == "direct":
            out = _cbc.direct_apply(hs, ho, arg[0], arg[1], opt)
        else:
            out = _cbc.src_apply(hs, ho, arg[0], arg[1], opt)
        try:
            cplx = np.iscomplexobj(st.tensors[0])
            res = _cbc.fetch_network(out, _cbc.output_shape_fn(st.parent, st.phys), cplx)
            disc = _cbc.ttn_get_discarded(out)
        finally:
            _cbc.ttn_destroy(out)
    finally:
        _cbc.ttn_destroy(hs)
        _cbc.ttno_destroy(ho)
    return res, disc


def _omega(p, s, seed=11):
    return sketch_matrices(p.state.phys, s, seed=seed, cplx=np.iscomplexobj(p.state.tensors[0]))


ZIP_CASES = [
    dict(config=1, max_bond=16), dict(config=1, max_bond=3),
    dict(config=2, L=7, chi=8, D=3, max_bond=5, dtype=np.complex128, seed=3),
    dict(config=2, L=5, chi=5, D=2, d=3, max_bond=4, dtype=np.complex128, seed=2),
    dict(config=2, L=12, chi=32, D=4, max_bond=24, seed=1),
    dict(config=2, L=16, chi=64, D=8, max_bond=64, seed=4),
    dict(config=2, L=1, chi=4, D=2, max_bond=4, dtype=np.complex128),
]


@pytest.mark.parametrize("precision,bar", [(0, FP64_BAR), (1, MIXED_BAR)])
@pytest.mark.parametrize("case", ZIP_CASES, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()
                                                                   if k != "dtype"))
def test_zipup_matches_oracle(case, precision, bar):
    case = dict(case)
    cfg = case.pop("config")
    p = make_problem(cfg, **case)
    (got, bonds, log_norm), disc = _run("zipup", p, precision, (p.max_bond, 0.0))
    ref = comparators.zipup_tt(p.state.tensors, p.op.tensors, p.max_bond)
    assert list(bonds) == list(ref.out_bonds), (bonds, ref.out_bonds)
    e = metrics.rel_err(p.state.parent, got, ref.tensors, log_norm, 0.0)
    assert e <= bar, e
    # discarded weight per edge: the oracle's relative weight beyond the kept rank
    L = len(p.state.tensors)
    rel = 1e-8 if precision == 0 else 1e-4
    for cut, i in zip(ref.forward_cuts, range(L - 1, 0, -1)):
        w = cut.s ** 2
        ref_d = float(np.sum(w[cut.k:]) / np.sum(w))
        assert abs(disc[i] - ref_d) <= rel * max(ref_d, 1e-6) + 1e-12, (i, disc[i], ref_d)


@pytest.mark.parametrize("precision,bar", [(0, FP64_BAR), (1, MIXED_BAR)])
def test_zipup_tolerance(precision, bar):
    p = make_problem(2, L=10, chi=16, D=4, max_bond=0, dtype=np.complex128, seed=9)
    tol = 1e-2
    (got, bonds, log_norm), _ = _run("zipup", p, precision, (0, tol))
    ref = comparators.zipup_tt(p.state.tensors, p.op.tensors, 0, tol)
    assert list(bonds) == list(ref.out_bonds), (bonds, ref.out_bonds)
    e = metrics.rel_err(p.state.parent, got, ref.tensors, log_norm, 0.0)
    assert e <= bar, e


SRC_CASES = [
    dict(config=1, max_bond=16, s=16), dict(config=1, max_bond=3, s=3),
    dict(config=2, L=7, chi=8, D=3, max_bond=5, dtype=np.complex128, seed=3, s=5),
    dict(config=2, L=5, chi=5, D=2, d=3, max_bond=4, dtype=np.complex128, seed=2, s=9),
    dict(config=2, L=12, chi=32, D=4, max_bond=24, seed=1, s=24),
    dict(config=2, L=16, chi=64, D=8, max_bond=64, seed=4, s=64),
    dict(config=2, L=2, chi=4, D=2, max_bond=4, dtype=np.complex128, s=7),
]


@pytest.mark.parametrize("precision,bar", [(0, FP64_BAR), (1, MIXED_BAR)])
@pytest.mark.parametrize("case", SRC_CASES, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()
                                                                   if k != "dtype"))
def test_src_matches_oracle(case, precision, bar):
    case = dict(case)
    cfg, s = case.pop("config"), case.pop("s")
    p = make_problem(cfg, **case)
    om = _omega(p, s)
    (got, bonds, log_norm), _ = _run("src", p, precision, (s, om))
    ref = comparators.src_tt(p.state.tensors, p.op.tensors, om)
    assert list(bonds) == list(ref.out_bonds), (bonds, ref.out_bonds)
    e = metrics.rel_err(p.state.parent, got, ref.tensors, log_norm, 0.0)
    assert e <= bar, e


DIRECT_CASES = [
    dict(config=1, max_bond=16), dict(config=1, max_bond=3),
    dict(config=2, L=7, chi=8, D=3, max_bond=5, dtype=np.complex128, seed=3),
    dict(config=2, L=5, chi=5, D=2, d=3, max_bond=4, dtype=np.complex128, seed=2),
    dict(config=2, L=12, chi=32, D=4, max_bond=24, seed=1),
    dict(config=2, L=10, chi=32, D=8, max_bond=32, seed=4),
    dict(config=2, L=1, chi=4, D=2, max_bond=4, dtype=np.complex128),
]


@pytest.mark.parametrize("precision,bar", [(0, FP64_BAR), (1, MIXED_BAR)])
@pytest.mark.parametrize("case", DIRECT_CASES, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()
                                                                      if k != "dtype"))
def test_direct_matches_oracle(case, precision, bar):
    case = dict(case)
    cfg = case.pop("config")
    p = make_problem(cfg, **case)
    (got, bonds, log_norm), disc = _run("direct", p, precision, (p.max_bond, 0.0))
    ref = comparators.direct_tt(p.state.tensors, p.op.tensors, p.max_bond)
    assert list(bonds) == list(ref.out_bonds), (bonds, ref.out_bonds)
    e = metrics.rel_err(p.state.parent, got, ref.tensors, log_norm, 0.0)
    assert e <= bar, e


@pytest.mark.parametrize("precision,bar", [(0, FP64_BAR), (1, MIXED_BAR)])
def test_direct_tolerance(precision, bar):
    p = make_problem(2, L=10, chi=16, D=4, max_bond=0, dtype=np.complex128, seed=9)
    (got, bonds, log_norm), _ = _run("direct", p, precision, (0, 1e-2))
    ref = comparators.direct_tt(p.state.tensors, p.op.tensors, 0, 1e-2)
    assert list(bonds) == list(ref.out_bonds), (bonds, ref.out_bonds)
    e = metrics.rel_err(p.state.parent, got, ref.tensors, log_norm, 0.0)
    assert e <= bar, e


def test_comparators_reject_trees():
    from paper_2601_19650_gb300 import _cbc

    p = make_problem(3, L=2, chi=4, D=2, max_bond=4, dtype=np.float64)
    st, op = p.state, p.op
    hs = _cbc.create_from_host(st.parent, st.phys, st.bond, st.tensors, "state")
    ho = _cbc.create_from_host(op.parent, op.phys, op.bond, op.tensors, "op")
    try:
        with pytest.raises(_cbc.CBCError, match="tensor trains"):
            _cbc.zipup_apply(hs, ho, 4, 0.0)
        with pytest.raises(_cbc.CBCError, match="tensor trains"):
            _cbc.src_apply(hs, ho, 4, sketch_matrices(st.phys, 4))
        with pytest.raises(_cbc.CBCError, match="tensor trains"):
            _cbc.direct_apply(hs, ho, 4, 0.0)
    finally:
        _cbc.ttn_destroy(hs)
        _cbc.ttno_destroy(ho)
