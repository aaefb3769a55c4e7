"""CUDA path (through the C ABI) against the FP64 oracle and brute force.

Bar (FP64 path): relative 2-norm distance between the output states <= 1e-10.  The
distance is measured without densifying (oracle.metrics: direct-sum network + QR
sweep), so it resolves differences far below the bar.
"""
import numpy as np
import pytest

from oracle import brute, cbc, metrics
from synth import make_problem

from gpu_helpers import run_gpu

pytestmark = pytest.mark.gpu

FP64_BAR = 1e-10


def _compare(prob, bar=FP64_BAR, **kw):
    got, bonds, log_norm = run_gpu(prob, **kw)
    mb = kw.get("max_bond", prob.max_bond)
    tol = kw.get("tol", prob.tol)
    ref = cbc.cbc(prob.state.parent, prob.state.tensors, prob.op.tensors, mb, tol)
    e = metrics.rel_err(prob.state.parent, got, ref.tensors, log_norm, 0.0)
    assert list(bonds) == list(ref.out_bonds), (bonds, ref.out_bonds)
    assert e <= bar, (prob.name, e)
    # output non-root tensors are isometries
    for i, t in enumerate(got):
        if prob.state.parent[i] < 0:
            continue
        q = t.reshape(t.shape[0], -1)
        assert np.abs(q @ q.conj().T - np.eye(q.shape[0])).max() < 1e-11
    return e


def test_cfg1_exact_against_brute_force():
    p = make_problem(1, max_bond=16)
    got, bonds, log_norm = run_gpu(p)
    ex = brute.apply_dense(p.state.parent, p.state.tensors, p.op.tensors)
    v = brute.dense_state(p.state.parent, got) * np.exp(log_norm)
    assert np.linalg.norm(v - ex) <= 1e-12 * np.linalg.norm(ex)


def test_cfg1_truncated():
    _compare(make_problem(1))


@pytest.mark.parametrize("L,chi,D,mb,seed", [
    (2, 4, 2, 4, 0), (1, 1, 3, 4, 1), (3, 4, 3, 3, 2), (12, 16, 4, 16, 0), (12, 16, 4, 5, 3),
    (20, 33, 5, 40, 4), (9, 8, 3, 0, 5)])
def test_complex_chain_small(L, chi, D, mb, seed):
    p = make_problem(2, L=L, chi=chi, D=D, max_bond=mb, seed=seed)
    _compare(p)


def test_real_chain_d3():
    p = make_problem(2, L=10, chi=12, D=4, d=3, max_bond=9, dtype=np.float64, seed=6)
    _compare(p)


def test_tolerance_mode():
    p = make_problem(2, L=10, chi=16, D=4, max_bond=0, seed=7)
    _compare(p, max_bond=0, tol=3e-2)
    _compare(p, max_bond=12, tol=1e-3)


def test_cfg2_full_fp64():
    """L=64, d=2, chi=128, D=16, max_bond=128, complex64 inputs: the bench workload."""
    _compare(make_problem(2))


def test_topology_mismatch_is_reported():
    from paper_2601_19650_gb300 import _cbc
    a = make_problem(2, L=4, chi=4, D=2, max_bond=4)
    b = make_problem(2, L=5, chi=4, D=2, max_bond=4)
    hs = _cbc.create_from_host(a.state.parent, a.state.phys, a.state.bond, a.state.tensors, "state")
    ho = _cbc.create_from_host(b.op.parent, b.op.phys, b.op.bond, b.op.tensors, "op")
    with pytest.raises(_cbc.CBCError) as ei:
        _cbc.cbc_apply(hs, ho, 4, 0.0)
    assert ei.value.code == 2
    _cbc.ttn_destroy(hs)
    _cbc.ttno_destroy(ho)


# ---------------------------------------------------------------------------------------
# mixed path: tensor-core slices for contractions and Gram products, FP64 eigensolver,
# Cholesky and triangular solves.  Bar: relative state error <= 1e-6.
# ---------------------------------------------------------------------------------------
MIXED_BAR = 1e-6


def _compare_mixed(prob, **kw):
    from paper_2601_19650_gb300 import _cbc
    got, bonds, log_norm = run_gpu(prob, precision=_cbc.CBC_PREC_MIXED, **kw)
    ref = cbc.cbc(prob.state.parent, prob.state.tensors, prob.op.tensors,
                  kw.get("max_bond", prob.max_bond), kw.get("tol", prob.tol))
    e = metrics.rel_err(prob.state.parent, got, ref.tensors, log_norm, 0.0)
    assert list(bonds) == list(ref.out_bonds), (bonds, ref.out_bonds)
    assert e <= MIXED_BAR, (prob.name, e)
    return e


def test_mixed_cfg1():
    _compare_mixed(make_problem(1))


@pytest.mark.parametrize("L,chi,D,mb,seed", [(2, 4, 2, 4, 0), (12, 16, 4, 16, 0),
                                             (12, 16, 4, 5, 3), (20, 33, 5, 40, 4)])
def test_mixed_complex_chain_small(L, chi, D, mb, seed):
    _compare_mixed(make_problem(2, L=L, chi=chi, D=D, max_bond=mb, seed=seed))


def test_mixed_cfg2_full():
    """The bench workload: L=64, d=2, chi=128, D=16, max_bond=128, complex64."""
    _compare_mixed(make_problem(2))


# ---------------------------------------------------------------------------------------
# batched serving set: independent instances of different sizes, one stream each,
# applied concurrently by cbc_apply_batched
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("precision,bar", [(0, FP64_BAR), (1, MIXED_BAR)])
def test_batched_heterogeneous(precision, bar):
    import torch

    from paper_2601_19650_gb300 import _cbc
    from synth.networks import make_batch

    probs = make_batch(n=6, scale=4)   # L 4..16, chi 8..64, D 1..8, float32, seed j
    streams = [torch.cuda.Stream() for _ in probs]
    hs, ho = [], []
    for p, s in zip(probs, streams):
        hs.append(_cbc.create_from_host(p.state.parent, p.state.phys, p.state.bond,
                                        p.state.tensors, "state", s.cuda_stream))
        ho.append(_cbc.create_from_host(p.op.parent, p.op.phys, p.op.bond, p.op.tensors,
                                        "op", s.cuda_stream))
    outs = _cbc.cbc_apply_batched(hs, ho, [p.max_bond for p in probs], [0.0] * len(probs),
                                  _cbc.make_options(precision), workers=3)
    for p, o in zip(probs, outs):
        got, bonds, log_norm = _cbc.fetch_network(
            o, _cbc.output_shape_fn(p.state.parent, p.state.phys), False)
        ref = cbc.cbc(p.state.parent, p.state.tensors, p.op.tensors, p.max_bond)
        assert list(bonds) == list(ref.out_bonds)
        e = metrics.rel_err(p.state.parent, got, ref.tensors, log_norm, 0.0)
        assert e <= bar, (p.name, e)
    for h in outs + hs:
        _cbc.ttn_destroy(h)
    for h in ho:
        _cbc.ttno_destroy(h)


# ---------------------------------------------------------------------------------------
# the paper's own benchmark shape (Sec. IV A): MPS L=50, d=3, D_S=D_O=40, complex entries
# with Re, Im ~ U[-0.5, 1], swept over the target bond
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("max_bond", [4, 16, 40])
@pytest.mark.parametrize("precision", [0, 1])
def test_paper_benchmark_shape(max_bond, precision):
    p = make_problem("P", max_bond=max_bond)
    if precision == 0:
        _compare(p)
    else:
        _compare_mixed(p)


# ---------------------------------------------------------------------------------------
# large bonds: the paths for matrices too large for shared memory
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("precision", [0, 1])
def test_large_bonds(precision):
    # bond 480 in the middle of a d = 4 chain: the CholeskyQR Gram is 480 x 480 (blocked
    # Cholesky with its panel read from global memory, triangular solve with the factor in
    # global memory) and a truncation Gram is 960 x 960 (tridiagonal reduction with the
    # rows in global memory, one-vector-per-CTA back transformation)
    p = make_problem(2, seed=3, L=10, d=4, chi=480, D=2, max_bond=480)
    if precision == 0:
        _compare(p)
    else:
        _compare_mixed(p)


# ---------------------------------------------------------------------------------------
# lockstep groups: cbc_apply_batched runs instances of one shape as one launch per step
# ---------------------------------------------------------------------------------------
def _apply_batched(probs, precision, workers=1, max_group=0):
    """All instances through cbc_apply_batched (one stream each); host outputs and the
    launch statistics of the call."""
    import torch

    from paper_2601_19650_gb300 import _cbc

    streams = [torch.cuda.Stream() for _ in probs]
    hs, ho = [], []
    for p, s in zip(probs, streams):
        hs.append(_cbc.create_from_host(p.state.parent, p.state.phys, p.state.bond,
                                        p.state.tensors, "state", s.cuda_stream))
        ho.append(_cbc.create_from_host(p.op.parent, p.op.phys, p.op.bond, p.op.tensors,
                                        "op", s.cuda_stream))
    torch.cuda.synchronize()
    _cbc.cbc_stats_reset()
    _cbc.cbc_stats_enable(True)
    try:
        outs = _cbc.cbc_apply_batched(hs, ho, [p.max_bond for p in probs],
                                      [p.tol for p in probs],
                                      _cbc.make_options(precision, max_group=max_group),
                                      workers=workers)
    finally:
        stats = _cbc.cbc_stats_read()
        _cbc.cbc_stats_enable(False)
    res = []
    for p, o in zip(probs, outs):
        cplx = np.iscomplexobj(p.state.tensors[0])
        res.append(_cbc.fetch_network(o, _cbc.output_shape_fn(p.state.parent, p.state.phys),
                                      cplx))
    for h in outs + hs:
        _cbc.ttn_destroy(h)
    for h in ho:
        _cbc.ttno_destroy(h)
    return res, stats


def _check_against_oracle(probs, res, bar):
    refs = []
    for p, (got, bonds, log_norm) in zip(probs, res):
        ref = cbc.cbc(p.state.parent, p.state.tensors, p.op.tensors, p.max_bond, p.tol)
        assert list(bonds) == list(ref.out_bonds), (p.name, bonds, ref.out_bonds)
        e = metrics.rel_err(p.state.parent, got, ref.tensors, log_norm, 0.0)
        assert e <= bar, (p.name, p.seed, e)
        refs.append(ref)
    return refs


@pytest.mark.parametrize("precision,bar,count", [(0, FP64_BAR, 4), (1, MIXED_BAR, 4),
                                                 (0, FP64_BAR, 9), (1, MIXED_BAR, 9)])
def test_group_lockstep(precision, bar, count):
    # 4 instances: one cluster per matrix; 9: one CTA per matrix for the Cholesky
    L = 9
    probs = [make_problem(2, seed=20 + j, L=L, chi=16, D=4, max_bond=12) for j in range(count)]
    res, stats = _apply_batched(probs, precision)
    _check_against_oracle(probs, res, bar)
    # one eigensolver launch group per cut for the whole group, not one per instance
    assert stats["eig"]["groups"] == L - 1, stats["eig"]


@pytest.mark.parametrize("precision,bar", [(0, FP64_BAR), (1, MIXED_BAR)])
def test_group_wide_batch(precision, bar):
    # 20 instances keeping 128 eigenvectors at the middle cuts: enough CTAs for the
    # 32-vectors-per-CTA back transformation (double-float in the mixed path), one CTA
    # per matrix for the Cholesky, clusters for the tridiagonal reduction
    probs = [make_problem(2, seed=60 + j, L=16, chi=64, D=4, max_bond=128) for j in range(20)]
    res, stats = _apply_batched(probs, precision)
    _check_against_oracle(probs, res, bar)
    # one eigensolver launch group per cut for the whole group; a cut whose truncation one
    # instance refines (second level, on that instance alone) adds one group of its own
    assert 16 - 1 <= stats["eig"]["groups"] <= 16 - 1 + 2 * len(probs), stats["eig"]
    assert stats["tridiag"]["launches"] >= 16 - 1


@pytest.mark.parametrize("precision,bar", [(0, FP64_BAR), (1, MIXED_BAR)])
def test_group_larger_than_32(precision, bar):
    # max_group 64: 40 instances in one lockstep group (grids and workspaces scale with the
    # group; every launch covers all 40)
    L = 8
    probs = [make_problem(2, seed=200 + j, L=L, chi=16, D=4, max_bond=12) for j in range(40)]
    res, stats = _apply_batched(probs, precision, max_group=64)
    _check_against_oracle(probs, res, bar)
    assert stats["eig"]["groups"] == L - 1, stats["eig"]


def test_group_mixed_shapes_and_real():
    # two shapes interleaved (two groups) plus a real-valued group
    probs = [make_problem(2, seed=30 + j, L=7 + (j % 2), chi=12, D=3, max_bond=10)
             for j in range(4)]
    probs += [make_problem(2, seed=40 + j, L=6, chi=10, D=3, d=3, max_bond=8,
                           dtype=np.float64) for j in range(3)]
    res, _ = _apply_batched(probs, 0, workers=2)
    _check_against_oracle(probs, res, FP64_BAR)


def test_group_rank_disagreement_reruns_members():
    # tolerance truncation: ranks depend on each instance's spectrum; when they differ
    # the group is rerun member by member, with the same results as single calls
    L = 8
    probs = [make_problem(2, seed=50 + j, tol=3e-2, L=L, chi=12, D=3, max_bond=0)
             for j in range(3)]
    res, stats = _apply_batched(probs, 0)
    refs = _check_against_oracle(probs, res, FP64_BAR)
    if len({tuple(r.out_bonds) for r in refs}) > 1:
        assert stats["eig"]["groups"] > L - 1, stats["eig"]


# ---------------------------------------------------------------------------------------
# trees (Sec. III B): binary trees with leaf-only physical legs, T-trees, fork trees
# ---------------------------------------------------------------------------------------
TREE_CASES = [
    dict(L=2, chi=6, D=3, max_bond=64, dtype=np.float64),                  # exact
    dict(L=3, chi=8, D=4, max_bond=3, dtype=np.float64, seed=1),
    dict(L=2, chi=5, D=2, max_bond=4, d=3, dtype=np.complex128, seed=2),
    dict(topo="ttree", L=3, d=2, chi=6, D=3, max_bond=5, dtype=np.complex128, seed=4),
    dict(topo="ftps", L=3, d=2, chi=6, D=2, max_bond=5, dtype=np.float64, seed=5),
    dict(L=4, chi=16, D=4, max_bond=16, dtype=np.float32, seed=0),        # config-3 family
]


@pytest.mark.parametrize("case", TREE_CASES, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()
                                                                      if k != "dtype"))
def test_tree_fp64(case):
    _compare(make_problem(3, **case))


@pytest.mark.parametrize("case", TREE_CASES[1:4] + TREE_CASES[5:], ids=lambda c: str(c.get("seed", 0)))
def test_tree_mixed(case):
    _compare_mixed(make_problem(3, **case))


def test_tree_exact_against_brute_force():
    p = make_problem(3, L=2, chi=6, D=3, max_bond=10 ** 6, dtype=np.float64)
    got, bonds, log_norm = run_gpu(p)
    ex = brute.apply_dense(p.state.parent, p.state.tensors, p.op.tensors)
    v = brute.dense_state(p.state.parent, got) * np.exp(log_norm)
    assert np.linalg.norm(v - ex) <= 1e-12 * np.linalg.norm(ex)


def test_cfg3_full_fp64():
    """Perfect binary tree of depth 6 (64 leaves, d=2), chi=64, D=8, cap 64, float32."""
    _compare(make_problem(3))


def test_cfg3_full_mixed():
    _compare_mixed(make_problem(3))
