"""Relative 2-norm distance between two TTNS on the same tree, without densifying.

TEST INFRASTRUCTURE ONLY (see ``oracle/cbc.py``).

``|| e^{la} psi_a - e^{lb} psi_b || / || e^{lb} psi_b ||`` is computed from the
direct-sum network: on every bond the two index ranges are stacked, each node tensor
is block diagonal (the A block, the B block, zeros elsewhere) and the B block of the
root carries the minus sign, so the network contracts to ``psi_a - psi_b``.  Its norm
comes from a leaves-to-root sweep of reduced QR factorisations, which is backward
stable; unlike ``<a|a> + <b|b> - 2 Re <a|b>`` it does not lose half the digits to
cancellation, so differences down to ~1e-14 relative are resolved.
"""
from __future__ import annotations

from typing import List

import numpy as np


def _children(parent) -> List[List[int]]:
    ch: List[List[int]] = [[] for _ in range(len(parent))]
    for j, p in enumerate(parent):
        if p >= 0:
            ch[int(p)].append(j)
    return ch


def _postorder(parent) -> List[int]:
    ch = _children(parent)
    root = [j for j, p in enumerate(parent) if p < 0][0]
    order, stack = [], [(root, False)]
    while stack:
        v, done = stack.pop()
        if done:
            order.append(v)
        else:
            stack.append((v, True))
            stack.extend((c, False) for c in reversed(ch[v]))
    return order


def tree_norm(parent, tensors) -> float:
    """2-norm of a TTNS by a leaves-to-root QR sweep (layout ``[parent, phys, children...]``)."""
    parent = [int(p) for p in parent]
    ch = _children(parent)
    post = _postorder(parent)
    work = [np.asarray(t, dtype=np.complex128) for t in tensors]
    for i in post:
        t = work[i]
        if parent[i] < 0:
            return float(np.linalg.norm(t.reshape(-1)))
        # rows: (phys, children...), cols: parent leg
        mat = np.moveaxis(t, 0, -1).reshape(-1, t.shape[0])
        _, r = np.linalg.qr(mat, mode="reduced")        # mat = Q r, r: (k, parent)
        p = parent[i]
        j = ch[p].index(i)
        axis = 2 + j                                     # child leg j of the parent tensor
        tp = work[p]
        tp = np.moveaxis(np.tensordot(tp, r, axes=([axis], [1])), -1, axis)
        work[p] = tp
    raise AssertionError("no root")


def direct_sum_difference(parent, ta, tb, scale_a: float = 1.0, scale_b: float = 1.0):
    """Node tensors of the network representing ``scale_a psi_a - scale_b psi_b``."""
    parent = [int(p) for p in parent]
    out = []
    if len(parent) == 1:                 # one node: no bond to stack along
        a = np.asarray(ta[0], dtype=np.complex128)
        b = np.asarray(tb[0], dtype=np.complex128)
        return [a * scale_a - b * scale_b]
    for i in range(len(parent)):
        a = np.asarray(ta[i], dtype=np.complex128)
        b = np.asarray(tb[i], dtype=np.complex128)
        if parent[i] < 0:
            a = a * scale_a
            b = -b * scale_b
        shape = [a.shape[0] + b.shape[0] if parent[i] >= 0 else 1, a.shape[1]]
        shape += [x + y for x, y in zip(a.shape[2:], b.shape[2:])]
        c = np.zeros(shape, dtype=np.complex128)
        if parent[i] >= 0:
            sa = (slice(0, a.shape[0]), slice(None)) + tuple(slice(0, x) for x in a.shape[2:])
            sb = (slice(a.shape[0], None), slice(None)) + tuple(slice(x, None) for x in a.shape[2:])
        else:
            sa = (slice(None), slice(None)) + tuple(slice(0, x) for x in a.shape[2:])
            sb = (slice(None), slice(None)) + tuple(slice(x, None) for x in a.shape[2:])
        c[sa] = a
        c[sb] = b
        out.append(c)
    return out


def rel_err(parent, ta, tb, log_a: float = 0.0, log_b: float = 0.0) -> float:
    """``|| e^{log_a} psi_a - e^{log_b} psi_b || / || e^{log_b} psi_b ||``."""
    nb = tree_norm(parent, tb)
    diff = direct_sum_difference(parent, ta, tb, float(np.exp(log_a - log_b)), 1.0)
    return tree_norm(parent, diff) / nb


def chain_applied_norm2(state, op) -> float:
    """||O |psi>||^2 for an MPO applied to an MPS (chain rooted at site 0, canonical
    layouts), by contracting the sandwich <psi| O^H O |psi> site by site from the left in
    FP64: the environment E[a, b, b', a'] carries the open bonds of psi, O, conj(O) and
    conj(psi) (Eqs. (ttns), (ttno); no truncation).  Together with the projection identity
    ||O psi - psi'||^2 = ||O psi||^2 - ||psi'||^2 it gives the error of a CBC result
    without densifying O |psi>."""
    L = len(state)
    E = np.ones((1, 1, 1, 1), dtype=np.complex128)
    for i in range(L):
        t = np.asarray(state[i], dtype=np.complex128)
        w = np.asarray(op[i], dtype=np.complex128)
        if i == L - 1:
            t = t[..., None]
            w = w[..., None]
        # E[a, b, c, e] with a: psi, b: O, c: conj(O), e: conj(psi)
        X = np.einsum("abce,asA->bcesA", E, t, optimize=True)          # sum a
        Y = np.einsum("bcesA,bPsB->cePAB", X, w, optimize=True)         # sum b, s
        Z = np.einsum("cePAB,cPtC->etABC", Y, w.conj(), optimize=True)  # sum c, P
        E = np.einsum("etABC,etD->ABCD", Z, t.conj(), optimize=True)    # sum e, t
    return float(E.reshape(-1)[0].real)


def chain_applied_overlap(state, op, out) -> complex:
    """<phi| O |psi> for a chain: phi the network ``out`` (canonical layout, as a CBC result
    without its scalar), contracted from the left with an environment E[x, b, a] over the
    open bonds of conj(phi), O and psi (Eqs. (ttns), (ttno))."""
    L = len(state)
    E = np.ones((1, 1, 1), dtype=np.complex128)
    for i in range(L):
        t = np.asarray(state[i], dtype=np.complex128)
        w = np.asarray(op[i], dtype=np.complex128)
        q = np.asarray(out[i], dtype=np.complex128)
        if i == L - 1:
            t, w, q = t[..., None], w[..., None], q[..., None]
        X = np.einsum("xba,asA->xbsA", E, t, optimize=True)      # sum a
        Y = np.einsum("xbsA,bPsB->xPAB", X, w, optimize=True)     # sum b, s
        E = np.einsum("xPAB,xPX->XBA", Y, q.conj(), optimize=True)  # sum x, P
    return complex(E.reshape(-1)[0])
