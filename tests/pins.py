"""Checks that pin the CBC oracle to facts outside itself.

Each check takes the oracle module (so the mutation test can hand in a deliberately
broken copy) and raises AssertionError when the fact does not hold.  None of them
re-types the oracle's formulas: they compare with brute force (dense state vectors
and operator matrices built from the TTNS/TTNO definitions, Eqs. (ttns), (ttno)),
with the Eckart-Young bound, and with identities the paper's construction implies.
"""
from __future__ import annotations

import numpy as np

from oracle import brute, metrics
from synth import make_problem
from synth.networks import random_network


def _run(cbc_mod, p, max_bond=None, tol=0.0, tree=False):
    mb = p.max_bond if max_bond is None else max_bond
    if tree:
        return cbc_mod.cbc_tree(p.state.parent, p.state.tensors, p.op.tensors, mb, tol)
    return cbc_mod.cbc(p.state.parent, p.state.tensors, p.op.tensors, mb, tol)


def small_cases():
    """Tiny chains and trees on which brute force is cheap."""
    out = [make_problem(1, max_bond=16), make_problem(1, max_bond=8)]
    out.append(make_problem(2, L=6, chi=6, D=3, max_bond=64, dtype=np.complex128))
    out.append(make_problem(2, L=7, chi=8, D=3, max_bond=5, dtype=np.complex128, seed=3))
    out.append(make_problem(3, L=2, chi=6, D=3, max_bond=64, dtype=np.float64))
    out.append(make_problem(3, L=3, chi=8, D=4, max_bond=3, dtype=np.float64, seed=1))
    out.append(make_problem(3, L=2, chi=5, D=2, max_bond=4, d=3, dtype=np.complex128, seed=2))
    out.append(make_problem(3, topo="ttree", L=2, d=2, chi=4, D=2, max_bond=3,
                            dtype=np.complex128, seed=4))
    return out


def check_exact_without_truncation(cbc_mod):
    """With a bond cap above every exact rank, CBC returns O|psi> itself (Sec. III: the
    output is O|psi> projected onto the compressed form; with nothing compressed the
    projection is the identity)."""
    cases = [make_problem(1, max_bond=16),
             make_problem(2, L=6, chi=6, D=3, max_bond=10 ** 6, dtype=np.complex128),
             make_problem(3, L=2, chi=6, D=3, max_bond=10 ** 6, dtype=np.float64),
             make_problem(3, topo="ttree", L=2, d=2, chi=4, D=2, max_bond=10 ** 6,
                          dtype=np.complex128, seed=4)]
    for p in cases:
        r = _run(cbc_mod, p)
        ex = brute.apply_dense(p.state.parent, p.state.tensors, p.op.tensors)
        got = brute.dense_state(p.state.parent, r.tensors)
        e = np.linalg.norm(got - ex) / np.linalg.norm(ex)
        assert e < 1e-11, (p.name, e)


def check_eckart_young(cbc_mod):
    """No state with bond <= D on some edge is closer to O|psi> than the weight that the
    SVD of O|psi> across that edge discards beyond D."""
    for p in small_cases():
        r = _run(cbc_mod, p)
        ex = brute.apply_dense(p.state.parent, p.state.tensors, p.op.tensors)
        got = brute.dense_state(p.state.parent, r.tensors)
        assert max(r.out_bonds) <= max(p.max_bond, 1), (p.name, r.out_bonds)
        bound = brute.eckart_young_bound(p.state.parent, p.state.phys, ex, p.max_bond)
        err = np.linalg.norm(got - ex)
        assert err >= bound * (1 - 1e-10) - 1e-14, (p.name, err, bound)


def check_projection(cbc_mod):
    """The output is the orthogonal projection of O|psi> onto the span of the new
    isometries (Eqs. (tt_cbc_final_contraction), (cbc_final_contraction) project the
    original network; the root keeps S): psi' = V V^H O psi, and therefore
    ||O psi||^2 = ||psi'||^2 + ||O psi - psi'||^2."""
    for p in small_cases():
        r = _run(cbc_mod, p)
        ex = brute.apply_dense(p.state.parent, p.state.tensors, p.op.tensors)
        got = brute.dense_state(p.state.parent, r.tensors)
        V = brute.isometry_map(p.state.parent, r.tensors)
        proj = V @ (V.conj().T @ ex)
        e = np.linalg.norm(proj - got) / np.linalg.norm(ex)
        assert e < 1e-11, (p.name, "projection", e)
        lhs = np.linalg.norm(ex) ** 2
        rhs = np.linalg.norm(got) ** 2 + np.linalg.norm(ex - got) ** 2
        assert abs(lhs - rhs) <= 1e-11 * lhs, (p.name, "pythagoras", lhs, rhs)


def check_isometries(cbc_mod):
    """Every non-root output tensor is an isometry toward its parent (QR factor)."""
    for p in small_cases():
        r = _run(cbc_mod, p)
        for i, t in enumerate(r.tensors):
            if p.state.parent[i] < 0:
                continue
            q = t.reshape(t.shape[0], -1)
            e = np.abs(q @ q.conj().T - np.eye(q.shape[0])).max()
            assert e < 1e-12, (p.name, i, e)


def check_chain_as_tree(cbc_mod):
    """On a chain, the tree algorithm (Sec. III B) and the tensor-train algorithm
    (Sec. III A) produce the same state."""
    for p in [make_problem(1, max_bond=8), make_problem(1, max_bond=3),
              make_problem(2, L=9, chi=10, D=4, max_bond=7, dtype=np.complex128, seed=5)]:
        a = cbc_mod.cbc_tt(p.state.tensors, p.op.tensors, p.max_bond)
        b = cbc_mod.cbc_tree(p.state.parent, p.state.tensors, p.op.tensors, p.max_bond)
        e = metrics.rel_err(p.state.parent, b.tensors, a.tensors)
        assert e < 1e-11, (p.name, e)


def _random_unitary(rng, n, cplx):
    if cplx:
        z = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    else:
        z = rng.standard_normal((n, n))
    q, r = np.linalg.qr(z)
    return q


def _gauge(net, rng):
    """Insert U U^H on every bond (U random unitary): same network, new tensors."""
    cplx = np.iscomplexobj(net.tensors[0])
    ts = [t.astype(np.complex128 if cplx else np.float64) for t in net.tensors]
    ch = net.children
    for i in range(net.n):
        if net.parent[i] < 0:
            continue
        U = _random_unitary(rng, int(net.bond[i]), cplx)
        # child i: T_i <- U^H T_i on its parent leg; parent p: T_p <- T_p U on the leg to i
        ts[i] = np.tensordot(U.conj().T, ts[i], axes=([1], [0]))
        p = int(net.parent[i])
        ax = (2 if net.kind == "state" else 3) + ch[p].index(i)
        t = np.tensordot(ts[p], U, axes=([ax], [0]))
        ts[p] = np.moveaxis(t, -1, ax)
    return ts


def check_unitary_gauge_invariance(cbc_mod):
    """Changing the gauge of the input networks by unitaries on every bond leaves the
    output state unchanged (only Gram matrices and QR row spaces enter, Sec. III)."""
    rng = np.random.default_rng(11)
    for p in [make_problem(1, max_bond=5),
              make_problem(3, L=3, chi=8, D=4, max_bond=3, dtype=np.float64, seed=1),
              make_problem(2, L=7, chi=8, D=3, max_bond=5, dtype=np.complex128, seed=3)]:
        a = _run(cbc_mod, p)
        ts = _gauge(p.state, rng)
        ws = _gauge(p.op, rng)
        b = cbc_mod.cbc(p.state.parent, ts, ws, p.max_bond)
        e = metrics.rel_err(p.state.parent, b.tensors, a.tensors)
        assert e < 1e-9, (p.name, e)


def check_scale_equivariance(cbc_mod):
    """CBC(lam psi, mu O) = lam mu CBC(psi, O)."""
    p = make_problem(2, L=7, chi=8, D=3, max_bond=5, dtype=np.complex128, seed=3)
    a = _run(cbc_mod, p)
    lam, mu = 3.5 - 0.25j, -0.125 + 2j
    ts = [t * lam if i == 0 else t for i, t in enumerate(p.state.tensors)]
    ws = [w * mu if i == 3 else w for i, w in enumerate(p.op.tensors)]
    b = cbc_mod.cbc(p.state.parent, ts, ws, p.max_bond)
    ta = [t * (lam * mu) if i == 0 else t for i, t in enumerate(a.tensors)]
    e = metrics.rel_err(p.state.parent, b.tensors, ta)
    assert e < 1e-11, e


def check_product_operator_exact(cbc_mod):
    """A product operator (operator bond 1) keeps the state's bond dimensions, so a cap
    at the state's bond is exact."""
    p = make_problem(2, L=8, chi=6, D=1, max_bond=6, dtype=np.complex128, seed=7)
    r = _run(cbc_mod, p)
    ex = brute.apply_dense(p.state.parent, p.state.tensors, p.op.tensors)
    got = brute.dense_state(p.state.parent, r.tensors)
    assert np.linalg.norm(got - ex) < 1e-11 * np.linalg.norm(ex)


def check_tolerance_rule(cbc_mod):
    """With a tolerance, every forward compression discards a relative weight below
    tol^2 and keeps the smallest such rank."""
    p = make_problem(2, L=8, chi=8, D=4, max_bond=0, dtype=np.complex128, seed=8)
    tol = 1e-2
    r = _run(cbc_mod, p, max_bond=0, tol=tol)
    for c in r.forward_cuts:
        w = c.s ** 2
        assert np.sum(w[c.k:]) <= tol * tol * np.sum(w) * (1 + 1e-12)
        if c.k > 1:
            assert np.sum(w[c.k - 1:]) > tol * tol * np.sum(w)


def check_first_cut_keeps_dominant_gram(cbc_mod):
    """At the first bond that is truncated, nothing was truncated before it, so the
    environment L^[i] must reproduce the best rank-k approximation of the exact left
    Gram B^H B (B = dense left block of O|psi>, brute force): the compression keeps the
    dominant part of the reduced-density-like matrix (Sec. III, DMC idea; Sec. III A)."""
    for p in [make_problem(1, max_bond=8), make_problem(1, max_bond=3),
              make_problem(2, L=7, chi=8, D=3, max_bond=5, dtype=np.complex128, seed=3)]:
        r = cbc_mod.cbc_tt(p.state.tensors, p.op.tensors, p.max_bond)
        L = len(p.state.tensors)
        done = False
        for i in range(1, L):
            B = brute.chain_left_block(p.state.tensors, p.op.tensors, i)
            G = B.conj().T @ B
            lam, V = np.linalg.eigh(G)
            lam, V = lam[::-1], V[:, ::-1]
            k = int(r.env_ranks[i])
            rank = int(np.count_nonzero(lam > 1e-12 * lam[0]))
            assert k == min(p.max_bond, rank), (p.name, i, k, rank)
            Gk = (V[:, :k] * lam[:k]) @ V[:, :k].conj().T
            env = np.asarray(r.envs[i]).reshape(k, -1)
            e = np.abs(env.conj().T @ env - Gk).max() / lam[0]
            assert e < 1e-11, (p.name, i, e)
            if k < rank:
                done = True
                break
        assert done, p.name


def _best_rank_k_gram(B, max_bond):
    """Numerical rank of B, the rank k = min(max_bond, rank), and the best rank-k part
    of B^H B from the SVD of B (Eckart-Young), scaled by the largest singular value."""
    _, s, Vh = np.linalg.svd(B, full_matrices=False)
    rank = int(np.count_nonzero(s > 1e-10 * s[0]))
    k = min(int(max_bond), rank) if max_bond > 0 else rank
    Gk = (Vh[:k].conj().T * s[:k] ** 2) @ Vh[:k]
    return rank, k, Gk, s[0] ** 2


def check_tree_cuts_keep_dominant_gram(cbc_mod):
    """On a branching tree, every compression whose inputs are all exact (nothing was
    truncated in the environments it contracts) keeps the best rank-k part of the exact
    Gram of its block of O|psi>, built by brute force: step 1 (Eq.
    (cbc_tree_first_contraction)) sees the subtree of the edge, step 2 (Eq.
    (cbc_tree_second_contraction)) everything else (Sec. III B).  At least one truncated
    step-1 cut and one truncated step-2 cut must be checked."""
    cases = [make_problem(3, L=2, chi=6, D=3, max_bond=1, dtype=np.complex128, seed=5),
             make_problem(3, L=2, chi=6, D=3, max_bond=4, dtype=np.complex128, seed=6),
             make_problem(3, topo="ttree", L=2, d=2, chi=4, D=2, max_bond=3,
                          dtype=np.complex128, seed=4)]
    trunc = {"sub": 0, "rest": 0}
    for p in cases:
        par = [int(x) for x in p.state.parent]
        ch = p.state.children
        r = cbc_mod.cbc_tree(par, p.state.tensors, p.op.tensors, p.max_bond)
        envs = r.envs

        def check(env, k_node, side):
            B = brute.edge_block(par, p.state.tensors, p.op.tensors, k_node, side)
            rank, k, Gk, s0 = _best_rank_k_gram(B, p.max_bond)
            e = np.asarray(env).reshape(np.asarray(env).shape[0], -1)
            assert e.shape[0] == k, (p.name, side, k_node, e.shape, k, rank)
            err = np.abs(e.conj().T @ e - Gk).max() / s0
            assert err < 1e-11, (p.name, side, k_node, err)
            if k < rank:
                trunc[side] += 1
            return k == rank

        exact_sub = {}
        post = [v for v in cbc_mod._postorder(par)]
        root = post[-1]
        for i in post:
            if i == root:
                continue
            if all(exact_sub[c] for c in ch[i]):
                exact_sub[i] = check(envs["sub"][i], i, "sub")
            else:
                exact_sub[i] = False
        exact_down = {root: True}
        for i in reversed(post):
            for k in ch[i]:
                ok_in = exact_down[i] and all(exact_sub[c] for c in ch[i] if c != k)
                exact_down[k] = check(envs["down"][k], k, "rest") if ok_in else False
    assert trunc["sub"] > 0 and trunc["rest"] > 0, trunc


ALL_CHECKS = [
    check_first_cut_keeps_dominant_gram,
    check_tree_cuts_keep_dominant_gram,
    check_exact_without_truncation,
    check_eckart_young,
    check_projection,
    check_isometries,
    check_chain_as_tree,
    check_unitary_gauge_invariance,
    check_scale_equivariance,
    check_product_operator_exact,
    check_tolerance_rule,
]
