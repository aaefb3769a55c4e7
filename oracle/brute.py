"""Brute-force references for tiny networks (dense state vector, dense operator matrix).

TEST INFRASTRUCTURE ONLY (see ``oracle/cbc.py``).  These follow the definitions of a
TTNS, Eq. (ttns), and of a TTNO, Eq. (ttno), directly: contract every node tensor into
one dense tensor with the physical legs in ascending node id.  ``O |psi>`` of
Eq. (abstr_application) is then a matrix-vector product, and the singular values of
that vector across each edge give the Eckart-Young lower bound on the error of any
state whose bond on that edge is at most ``D``.
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np


def _children(parent) -> List[List[int]]:
    ch: List[List[int]] = [[] for _ in range(len(parent))]
    for j, p in enumerate(parent):
        if p >= 0:
            ch[int(p)].append(j)
    return ch


def _subtree(parent, i) -> List[int]:
    ch = _children(parent)
    out, stack = [], [i]
    while stack:
        v = stack.pop()
        out.append(v)
        stack.extend(ch[v])
    return out


def _contract_subtree(parent, tensors, i, nphys_legs):
    """Dense tensor of the subtree of ``i``: legs ``[parent_bond, phys legs...]`` and the
    list of node ids (each node contributes ``nphys_legs`` consecutive legs)."""
    ch = _children(parent)
    t = np.asarray(tensors[i])
    order = [i]
    # t legs: [parent, phys * nphys_legs, children...]
    for c in ch[i]:
        sub, sub_order = _contract_subtree(parent, tensors, c, nphys_legs)
        # contract the first child leg still open (it sits right after the phys legs
        # collected so far) with the parent leg of the child subtree
        pos = 1 + nphys_legs * len(order)
        t = np.tensordot(t, sub, axes=([pos], [0]))
        # tensordot appends the child's phys legs at the end; move them before the
        # remaining child legs
        n_new = sub.ndim - 1
        nd = t.ndim
        keep_front = list(range(pos))
        remaining_children = list(range(pos, nd - n_new))
        new_legs = list(range(nd - n_new, nd))
        t = t.transpose(keep_front + new_legs + remaining_children)
        order += sub_order
    return t, order


def dense_state(parent, tensors) -> np.ndarray:
    """State vector of a TTNS with physical legs in ascending node id (Eq. (ttns))."""
    parent = [int(p) for p in parent]
    root = parent.index(-1)
    t, order = _contract_subtree(parent, tensors, root, 1)
    t = t[0]                                   # root's parent leg has dimension 1
    perm = np.argsort(order)
    return np.ascontiguousarray(t.transpose(perm)).reshape(-1)


def dense_operator(parent, tensors) -> np.ndarray:
    """Operator matrix of a TTNO, rows = out legs, cols = in legs, node order (Eq. (ttno))."""
    parent = [int(p) for p in parent]
    root = parent.index(-1)
    t, order = _contract_subtree(parent, tensors, root, 2)
    t = t[0]
    n = len(order)
    # legs are (out_j, in_j) pairs in `order`
    pos = {node: k for k, node in enumerate(order)}
    outs = [2 * pos[j] for j in range(n)]
    ins = [2 * pos[j] + 1 for j in range(n)]
    t = t.transpose(outs + ins)
    dim = int(np.prod(t.shape[:n]))
    return np.ascontiguousarray(t).reshape(dim, dim)


def apply_dense(parent, state, op) -> np.ndarray:
    """Exact ``O |psi>`` (Eq. (abstr_application))."""
    return dense_operator(parent, op) @ dense_state(parent, state)


def schmidt_values(parent, phys: Sequence[int], vec: np.ndarray, i: int) -> np.ndarray:
    """Singular values of ``vec`` across the edge between node ``i`` and its parent."""
    parent = [int(p) for p in parent]
    n = len(parent)
    sub = sorted(_subtree(parent, i))
    rest = [j for j in range(n) if j not in sub]
    t = vec.reshape([int(d) for d in phys])
    dsub = int(np.prod([int(phys[j]) for j in sub]))
    m = t.transpose(sub + rest).reshape(dsub, -1)
    return np.linalg.svd(m, compute_uv=False)


def eckart_young_bound(parent, phys, vec: np.ndarray, max_bond: int) -> float:
    """max over edges of the weight a bond of ``max_bond`` must discard (absolute norm)."""
    best = 0.0
    for i, p in enumerate(parent):
        if p < 0:
            continue
        s = schmidt_values(parent, phys, vec, i)
        best = max(best, float(np.sqrt(np.sum(s[max_bond:] ** 2))))
    return best


def isometry_map(parent, tensors) -> np.ndarray:
    """Dense map from the root tensor's entries to the full state: the network with the
    root tensor replaced by the identity.  Columns index the root tensor (row-major)."""
    parent = [int(p) for p in parent]
    root = parent.index(-1)
    rt = np.asarray(tensors[root])
    size = rt.size
    cols = []
    for e in range(size):
        unit = np.zeros(size, dtype=rt.dtype)
        unit[e] = 1.0
        ts = list(tensors)
        ts[root] = unit.reshape(rt.shape)
        cols.append(dense_state(parent, ts))
    return np.stack(cols, axis=1)


def chain_left_block(state, op, i: int) -> np.ndarray:
    """Dense left block of ``O |psi>`` for the first ``i`` sites of a chain, as a matrix
    ``B[(sigma'_1..sigma'_i), (alpha_i, beta_i)]`` (the open bonds to site i+1).

    ``B^H B`` is the exact left Gram on the bond after site ``i``: the object whose
    dominant eigenspace a compression of that bond keeps (Sec. III)."""
    psi = np.asarray(state[0])[0]                       # (sigma, alpha_1)
    O = np.asarray(op[0])[0]                            # (sigma', sigma, beta_1)
    for j in range(1, i):
        t = np.asarray(state[j])                        # (alpha, sigma, alpha')
        w = np.asarray(op[j])                           # (beta, sigma', sigma, beta')
        psi = np.tensordot(psi, t, axes=([psi.ndim - 1], [0]))
        psi = psi.reshape(-1, t.shape[-1])
        O = np.tensordot(O, w, axes=([O.ndim - 1], [0]))    # (..out.., ..in.., s', s, b')
        # O legs: (outs, ins, sigma', sigma, beta'): regroup to (outs sigma', ins sigma, beta')
        nout = O.shape[0]
        nin = O.shape[1]
        O = O.transpose(0, 2, 1, 3, 4).reshape(nout * w.shape[1], nin * w.shape[2], w.shape[3])
    B = np.einsum("Psb,sa->Pab", O, psi)
    return B.reshape(B.shape[0], -1)


def edge_block(parent, state, op, k: int, side: str) -> np.ndarray:
    """Dense block of ``O |psi>`` on one side of the edge between node ``k`` and its parent.

    ``side="sub"`` takes the nodes of the subtree of ``k``, ``side="rest"`` all the other
    nodes.  The result is the matrix ``B[(sigma'_j, j in the block, ascending), (alpha, beta)]``
    with ``(alpha, beta)`` the state and operator bonds of that edge left open, i.e. the
    block of the exact network (Eqs. (ttns), (ttno)) that a compression of that edge sees:
    ``B^H B`` is the exact Gram on the edge from that side (Sec. III B, steps 1 and 2)."""
    parent = [int(p) for p in parent]
    n = len(parent)
    ch = _children(parent)
    sub = set(_subtree(parent, k))
    nodes = sorted(sub) if side == "sub" else [j for j in range(n) if j not in sub]
    if side not in ("sub", "rest") or parent[k] < 0:
        raise ValueError("edge_block: need a non-root node and side 'sub' or 'rest'")
    inset = set(nodes)
    nxt = [0]

    def lab():
        nxt[0] += 1
        return nxt[0] - 1

    ls = {j: lab() for j in nodes}            # sigma_j
    lso = {j: lab() for j in nodes}           # sigma'_j
    la = {j: lab() for j in range(n) if parent[j] >= 0}   # alpha on edge (j, parent j)
    lb = {j: lab() for j in range(n) if parent[j] >= 0}   # beta on edge (j, parent j)
    st_ops, op_ops = [], []
    for j in nodes:
        pa = la[j] if parent[j] >= 0 else lab()   # the root's parent leg has dimension 1
        pb = lb[j] if parent[j] >= 0 else lab()
        st_ops += [np.asarray(state[j]), [pa, ls[j]] + [la[c] for c in ch[j]]]
        op_ops += [np.asarray(op[j]), [pb, lso[j], ls[j]] + [lb[c] for c in ch[j]]]
        for c in ch[j]:
            assert (c in inset) or c == k
    psi = np.einsum(*st_ops, [ls[j] for j in nodes] + [la[k]], optimize=True)
    B = np.einsum(*op_ops, psi, [ls[j] for j in nodes] + [la[k]],
                  [lso[j] for j in nodes] + [la[k], lb[k]], optimize=True)
    return B.reshape(-1, B.shape[-2] * B.shape[-1])
