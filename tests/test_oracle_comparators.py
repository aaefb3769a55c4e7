"""Pins of the comparison-method oracle (Zip-Up and SRC on chains, Sec. III C).

Every check takes the module (so that a deliberately broken copy can be handed in) and
compares it with facts outside it: the dense state vector and operator matrix built from
the TTNS/TTNO definitions (``oracle.brute``), dense SVDs of dense blocks of O|psi>, the
dense Khatri-Rao product of the random matrices, and the projection identity.
"""
import importlib.util
import os
import sys
import types

import numpy as np
import pytest

from oracle import brute
from synth import make_problem, sketch_matrices

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SOURCE = os.path.join(ROOT, "oracle", "comparators.py")


def _cases():
    return [make_problem(1, max_bond=16), make_problem(1, max_bond=3),
            make_problem(2, L=6, chi=6, D=3, max_bond=4, dtype=np.complex128),
            make_problem(2, L=7, chi=8, D=3, max_bond=5, dtype=np.complex128, seed=3),
            make_problem(2, L=5, chi=5, D=2, d=3, max_bond=4, dtype=np.complex128, seed=2)]


def _suffix_isometry(tensors, i):
    """Rows: the bond between sites i-1 and i; columns: (sigma'_i .. sigma'_{L-1})."""
    L = len(tensors)
    V = np.asarray(tensors[L - 1])                      # (k, d)
    for j in range(L - 2, i - 1, -1):
        t = np.asarray(tensors[j])                      # (k_j, d, k_{j+1})
        V = np.tensordot(t, V, axes=([2], [0])).reshape(t.shape[0], -1)
    return V


def _row_projector(A):
    """Projector onto the row space of A, acting from the right on row vectors."""
    u, s, vh = np.linalg.svd(A, full_matrices=False)
    r = int(np.count_nonzero(s > s[0] * 1e-10)) if s.size and s[0] > 0 else 0
    return vh[:r].conj().T @ vh[:r]


def _hpsi_unfolded(p, i):
    ex = brute.apply_dense(p.state.parent, p.state.tensors, p.op.tensors)
    left = int(np.prod(p.state.phys[:i]))
    return ex.reshape(left, -1)


def _run_zipup(mod, p, max_bond=None):
    return mod.zipup_tt(p.state.tensors, p.op.tensors,
                        p.max_bond if max_bond is None else max_bond)


def _omega(p, s):
    return sketch_matrices(p.state.phys, s, seed=7, cplx=np.iscomplexobj(p.state.tensors[0]))


def _run_src(mod, p, s=None):
    s = p.max_bond if s is None else s
    return mod.src_tt(p.state.tensors, p.op.tensors, _omega(p, s))


# ---- checks shared by both methods ------------------------------------------------------
def _exact(run):
    for p in [make_problem(1, max_bond=16),
              make_problem(2, L=6, chi=6, D=3, max_bond=10 ** 3, dtype=np.complex128),
              make_problem(2, L=5, chi=5, D=2, d=3, max_bond=300, dtype=np.complex128)]:
        r = run(p)
        ex = brute.apply_dense(p.state.parent, p.state.tensors, p.op.tensors)
        got = brute.dense_state(p.state.parent, r.tensors)
        e = np.linalg.norm(got - ex) / np.linalg.norm(ex)
        assert e < 1e-11, (p.name, e)


def _projection_and_isometries(run):
    for p in _cases():
        r = run(p)
        for i in range(1, len(r.tensors)):
            q = r.tensors[i].reshape(r.tensors[i].shape[0], -1)
            e = np.abs(q @ q.conj().T - np.eye(q.shape[0])).max()
            assert e < 1e-12, (p.name, i, e)
        ex = brute.apply_dense(p.state.parent, p.state.tensors, p.op.tensors)
        got = brute.dense_state(p.state.parent, r.tensors)
        V = brute.isometry_map(p.state.parent, r.tensors)
        e = np.linalg.norm(V @ (V.conj().T @ ex) - got) / np.linalg.norm(ex)
        assert e < 1e-11, (p.name, "projection", e)
        lhs = np.linalg.norm(ex) ** 2
        rhs = np.linalg.norm(got) ** 2 + np.linalg.norm(ex - got) ** 2
        assert abs(lhs - rhs) <= 1e-11 * lhs, (p.name, lhs, rhs)


# ---- Zip-Up -----------------------------------------------------------------------------
def check_zipup_exact(mod):
    """No truncation: Zip-Up returns O|psi> itself."""
    _exact(lambda p: _run_zipup(mod, p, 10 ** 6))


def check_zipup_projection(mod):
    """Isometries toward site 0, and the output is O|psi> projected onto their span."""
    _projection_and_isometries(lambda p: _run_zipup(mod, p))


def check_zipup_keeps_best_local_subspace(mod):
    """At every site i >= 1 the kept subspace is the dominant right singular subspace of
    the dense block of O|psi> on sites i.. (its bond to site i-1 open) projected onto what
    the earlier steps kept: the block Zip-Up compresses, built here by brute force."""
    for p in _cases():
        r = _run_zipup(mod, p)
        L = len(r.tensors)
        P_right = None
        for i in range(L - 1, 0, -1):
            B = brute.edge_block(p.state.parent, p.state.tensors, p.op.tensors, i, "sub")
            Z = B.T                                     # rows (alpha beta), cols sigma'_i..
            if P_right is not None:
                Z = Z @ np.kron(np.eye(int(p.state.phys[i])), P_right)
            k = r.tensors[i].shape[0]
            u, s, vh = np.linalg.svd(Z, full_matrices=False)
            if k < s.size and (s[k - 1] - s[k]) < 1e-8 * s[0]:
                continue                                # no unique subspace at this cut
            V = _suffix_isometry(r.tensors, i)
            P = V.conj().T @ V
            ref = vh[:k].conj().T @ vh[:k]
            e = np.abs(P - ref).max()
            assert e < 1e-9, (p.name, i, e)
            P_right = P


# ---- SRC --------------------------------------------------------------------------------
def check_src_exact(mod):
    """A sketch at least as wide as every exact rank: SRC returns O|psi> itself."""
    _exact(lambda p: _run_src(mod, p, 64))


def check_src_projection(mod):
    _projection_and_isometries(lambda p: _run_src(mod, p))


def check_src_sketch_is_khatri_rao(mod):
    """The sketch environment on the edge (i-1, i) equals Omega^T B, with B the dense left
    block of O|psi> on sites 0..i-1 (bonds to site i open) and Omega the dense Khatri-Rao
    product of the sites' random matrices: column j is the Kronecker product of column j
    of each site's matrix."""
    for p in _cases()[2:]:
        s = p.max_bond
        om = _omega(p, s)
        r = _run_src(mod, p, s)
        C = r.envs
        for i in range(1, len(p.state.tensors)):
            B = brute.chain_left_block(p.state.tensors, p.op.tensors, i)
            KR = np.ones((1, s), dtype=np.result_type(om[0], B))
            for k in range(i):
                KR = np.stack([np.kron(KR[:, j], om[k][:, j]) for j in range(s)], axis=1)
            ref = KR.T @ B
            got = C[i].reshape(C[i].shape[0], -1)
            assert got.shape == ref.shape, (p.name, i, got.shape, ref.shape)
            e = np.abs(got - ref).max() / np.abs(ref).max()
            assert e < 1e-12, (p.name, i, e)


def check_src_keeps_sketched_row_space(mod):
    """At every site i >= 1 the kept subspace is the row space of the first r rows of the
    dense sketch Omega^T (O|psi> unfolded at the edge (i-1, i)) projected onto what the
    earlier steps kept (r the generic rank of the sketched block)."""
    for p in _cases():
        s = p.max_bond
        om = _omega(p, s)
        r = _run_src(mod, p, s)
        L = len(r.tensors)
        P_right = None
        for i in range(L - 1, 0, -1):
            H = _hpsi_unfolded(p, i)
            KR = np.ones((1, s), dtype=np.result_type(om[0], H))
            for k in range(i):
                KR = np.stack([np.kron(KR[:, j], om[k][:, j]) for j in range(s)], axis=1)
            Y = KR.T @ H
            if P_right is not None:
                Y = Y @ np.kron(np.eye(int(p.state.phys[i])), P_right)
            a, b = p.state.tensors[i].shape[0], p.op.tensors[i].shape[0]
            rk = max(1, min(s, int(np.prod(p.state.phys[:i])), a * b))
            ref = _row_projector(Y[:rk])
            V = _suffix_isometry(r.tensors, i)
            P = V.conj().T @ V
            e = np.abs(P - ref).max()
            assert e < 1e-8, (p.name, i, e)
            P_right = P


# ---- direct (contract, then QR and SVD sweeps) -------------------------------------------
def _run_direct(mod, p, max_bond=None):
    return mod.direct_tt(p.state.tensors, p.op.tensors,
                         p.max_bond if max_bond is None else max_bond)


def check_direct_exact(mod):
    _exact(lambda p: _run_direct(mod, p, 10 ** 6))


def check_direct_projection(mod):
    _projection_and_isometries(lambda p: _run_direct(mod, p))


def check_direct_first_cut_is_optimal(mod):
    """The first truncation (the last edge) sees O|psi> with an orthonormal left part: it
    keeps the dominant right Schmidt vectors of the brute-force O|psi> across that edge."""
    for p in _cases():
        r = _run_direct(mod, p)
        L = len(r.tensors)
        H = _hpsi_unfolded(p, L - 1)
        k = r.tensors[L - 1].shape[0]
        u, s, vh = np.linalg.svd(H, full_matrices=False)
        if k < s.size and (s[k - 1] - s[k]) < 1e-8 * s[0]:
            continue
        q = r.tensors[L - 1].reshape(k, -1)
        e = np.abs(q.conj().T @ q - vh[:k].conj().T @ vh[:k]).max()
        assert e < 1e-9, (p.name, e)


def check_direct_sequential_bound(mod):
    """Sequential SVD truncation with orthonormal left parts: ||O psi - psi'||^2 is at most
    the sum over the edges of the weight that the best approximation of the same bond
    discards on that edge (each step's discarded weight is at most that edge's
    Eckart-Young tail of O|psi>)."""
    for p in _cases():
        r = _run_direct(mod, p)
        ex = brute.apply_dense(p.state.parent, p.state.tensors, p.op.tensors)
        got = brute.dense_state(p.state.parent, r.tensors)
        L = len(r.tensors)
        bound2 = 0.0
        for i in range(1, L):
            s = np.linalg.svd(_hpsi_unfolded(p, i), compute_uv=False)
            bound2 += float(np.sum(s[r.out_bonds[i]:] ** 2))
        err2 = float(np.linalg.norm(ex - got) ** 2)
        assert err2 <= bound2 * (1 + 1e-9) + 1e-24, (p.name, err2, bound2)


CHECKS = [check_zipup_exact, check_zipup_projection, check_zipup_keeps_best_local_subspace,
          check_src_exact, check_src_projection, check_src_sketch_is_khatri_rao,
          check_src_keeps_sketched_row_space, check_direct_exact, check_direct_projection,
          check_direct_first_cut_is_optimal, check_direct_sequential_bound]


@pytest.mark.parametrize("check", CHECKS, ids=lambda c: c.__name__)
def test_comparator_oracle_pin(check):
    from oracle import comparators
    check(comparators)


MUTATIONS = {
    "zipup-R-update-drops-conj": ('R = np.einsum("yPx,abPx->yab", Q.conj(), Z, optimize=True)      # = (U_k s_k)^T',
                                  'R = np.einsum("yPx,abPx->yab", Q, Z, optimize=True)      # = (U_k s_k)^T'),
    "zipup-keeps-smallest": ("Q = Vh[:k].reshape(k, d, c)                     # (chi'",
                             "Q = Vh[-k:].reshape(k, d, c)                     # (chi'"),
    "zipup-operator-in-out-swapped": ('Z = np.einsum("asyB,bPsB->abPy", Y, W[i], optimize=True)        # sum over sigma, beta_i',
                                      'Z = np.einsum("asyB,bsPB->abPy", Y, W[i], optimize=True)        # sum over sigma, beta_i'),
    "src-omega-conjugated": ('Om = np.asarray(omega[i])', 'Om = np.asarray(omega[i]).conj()'),
    "src-sketch-not-khatri-rao": ('C.append(np.einsum("jPAB,Pj->jAB", Lp, Om, optimize=True))',
                                  'C.append(np.einsum("jPAB,Pk->kAB", Lp, Om, optimize=True))'),
    "src-rank-ignores-left-dimension": ("return max(1, min(s, p_left, a * b))",
                                        "return max(1, min(s, a * b))"),
    "direct-remainder-not-pushed": ('        N[i + 1] = np.einsum("xr,rPy->xPy", R, N[i + 1], optimize=True)\n',
                                    '        pass\n'),
    "direct-carry-without-singular-values": ('N[i - 1] = np.einsum("xPl,lk->xPk", N[i - 1], U[:, :k] * s[:k], optimize=True)',
                                             'N[i - 1] = np.einsum("xPl,lk->xPk", N[i - 1], U[:, :k], optimize=True)'),
    "direct-keeps-smallest": ('out[i] = Vh[:k].reshape(k, d, r)', 'out[i] = Vh[-k:].reshape(k, d, r)'),
    "direct-operator-in-out-swapped": ('t = np.einsum("asA,bPsB->abPAB", T[i], W[i], optimize=True)',
                                       't = np.einsum("asA,bsPB->abPAB", T[i], W[i], optimize=True)'),
    "src-R-update-drops-conj": ('R = np.einsum("yPx,abPx->yab", Q.conj(), Z, optimize=True)\n    out[L - 1] = out[L - 1][..., 0]\n    bonds = [1] + [int(out[i].shape[0]) for i in range(1, L)]\n    return CBCResult(out, [], ',
                                'R = np.einsum("yPx,abPx->yab", Q, Z, optimize=True)\n    out[L - 1] = out[L - 1][..., 0]\n    bonds = [1] + [int(out[i].shape[0]) for i in range(1, L)]\n    return CBCResult(out, [], '),
}


def _mutant(name, old, new):
    src = open(SOURCE).read()
    assert src.count(old) == 1, f"mutation {name}: pattern found {src.count(old)} times"
    src = src.replace(old, new).replace("from .cbc import", "from oracle.cbc import")
    modname = f"comparators_mutant_{name.replace('-', '_')}"
    mod = types.ModuleType(modname)
    sys.modules[modname] = mod
    exec(compile(src, f"<mutant {name}>", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_comparator_mutation_is_caught(name):
    old, new = MUTATIONS[name]
    mod = _mutant(name, old, new)
    caught = []
    for check in CHECKS:
        try:
            check(mod)
        except Exception as e:
            caught.append((check.__name__, type(e).__name__))
    assert caught, f"no pin caught mutation {name}"
