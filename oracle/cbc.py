"""FP64 CPU oracle of the Cholesky-based compression (CBC), Sec. III of arXiv 2601.19650.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or execute
this module: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it, to check and to time the CUDA path.

It is a plain, slow transcription of the method in float64 / complex128 NumPy:
contractions are ``numpy.einsum`` on named legs, the compression is a truncated
``numpy.linalg.svd`` (an SVD is the compression the paper names, Sec. III A) and the
new node tensors come from ``numpy.linalg.qr`` (Eqs. (tt_cbc_qr_decomp),
(cbc_tree_qr)).  It shares no code with the GPU path, which reaches the same result
through Gram matrices, a Hermitian eigensolver and CholeskyQR.

Readings of the paper taken here (every one is listed with its reason in the design
notes of the repository):

* legs are identified by name, not by their position in the printed subscripts
  (the order of ``alpha``/``beta`` legs varies between Eqs. (tt_cbc_first_contraction),
  (right_sweep_init_contr) and (tt_cbc_final_contraction));
* the output case "if i = 0" of Sec. III A means the leftmost site;
* the tree R-update Eq. (cbc_final_contraction) uses the complex conjugate ``Q*`` as in
  the tensor-train Eq. (tt_cbc_final_contraction);
* rank rule (Sec. III A compresses to a target bond dimension; Sec. V mentions an SVD
  tolerance as the adaptive alternative): keep the singular values ``s_j > eps_rank * s_0``, then the
  smallest ``k`` whose discarded weight ``sum_{j>=k} s_j^2 <= tol^2 sum_j s_j^2`` (if
  ``tol > 0``), then at most ``max_bond`` (if ``max_bond > 0``);
* when the QR of Eq. (tt_cbc_qr_decomp) / (cbc_tree_qr) has more rows than columns on
  the decomposed leg, the reduced QR keeps ``min(rows, cols)`` and the bond shrinks.

Layouts are the canonical ones of ``synth.networks``: state ``[parent, phys,
children...]``, operator ``[parent, phys_out, phys_in, children...]``.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Tuple

import numpy as np

EPS_RANK = 1e-12


# --------------------------------------------------------------------------------------
# compression of a fused leg (Sec. III A, text after Eq. (tt_cbc_first_contraction))
# --------------------------------------------------------------------------------------

def choose_rank(s: np.ndarray, max_bond: int, tol: float, eps_rank: float = EPS_RANK) -> int:
    """Number of singular values kept by the rank rule described in the module doc."""
    s = np.asarray(s, dtype=np.float64)
    if s.size == 0 or s[0] <= 0.0:
        return 1
    k = int(np.count_nonzero(s > eps_rank * s[0]))
    if tol > 0.0:
        w = s ** 2
        tail = np.concatenate([np.cumsum(w[::-1])[::-1], [0.0]])  # tail[k] = sum_{j>=k} w_j
        k_tol = int(np.nonzero(tail <= tol * tol * tail[0])[0][0])
        k = min(k, max(k_tol, 1))
    if max_bond > 0:
        k = min(k, int(max_bond))
    return max(k, 1)


@dataclasses.dataclass
class CutInfo:
    """What one compression did: full spectrum, kept rank, discarded weight, gap."""
    s: np.ndarray
    k: int

    @property
    def discarded(self) -> float:
        return float(np.sum(self.s[self.k:] ** 2))

    @property
    def gap(self) -> float:
        """Relative gap (s_{k-1} - s_k) / s_0 at the truncation point (inf if nothing cut)."""
        if self.k >= self.s.size or self.s[0] == 0:
            return float("inf")
        return float((self.s[self.k - 1] - self.s[self.k]) / self.s[0])


def compress_rows(M: np.ndarray, max_bond: int, tol: float, eps_rank: float):
    """Compress the row leg of ``M`` (rows = the fused leg) with a truncated SVD.

    Returns ``diag(s_k) V_k^H`` (the factor that keeps the Gram ``M^H M`` up to the
    truncation; any isometry on the large leg is dropped, Sec. III A) and the cut info.
    """
    U, s, Vh = np.linalg.svd(M, full_matrices=False)
    k = choose_rank(s, max_bond, tol, eps_rank)
    return s[:k, None] * Vh[:k, :], CutInfo(s, k)


def lq_rows(S: np.ndarray):
    """``S = R Q`` with ``Q`` row-orthonormal (QR of ``S^H``), Eq. (tt_cbc_qr_decomp)."""
    Qh, Rh = np.linalg.qr(S.conj().T, mode="reduced")
    return Rh.conj().T, Qh.conj().T


# --------------------------------------------------------------------------------------
# tensor train, Sec. III A
# --------------------------------------------------------------------------------------

@dataclasses.dataclass
class CBCResult:
    tensors: List[np.ndarray]          # canonical layout, the new TTNS / MPS
    forward_cuts: List[CutInfo]        # compressions of the first sweep(s)
    env_ranks: List[int]               # chi_i of the environments
    out_bonds: List[int]               # bond of each node to its parent in the output
    envs: Optional[object] = None      # environments kept for checking (TT: list of L^[i];
                                       # trees: {"sub": L^[i], "down": L^[(p_k, k)]} by node)


def _as_tt(state, op):
    """Give every site an explicit right leg (dim 1 at the last site)."""
    T, W = [], []
    L = len(state)
    for i in range(L):
        t = np.asarray(state[i], dtype=np.complex128 if np.iscomplexobj(state[i]) else np.float64)
        w = np.asarray(op[i], dtype=np.complex128 if np.iscomplexobj(op[i]) else np.float64)
        if i == L - 1:
            t = t[..., None]
            w = w[..., None]
        T.append(t)
        W.append(w)
    if any(np.iscomplexobj(x) for x in T + W):
        T = [t.astype(np.complex128) for t in T]
        W = [w.astype(np.complex128) for w in W]
    return T, W


def cbc_tt(state: List[np.ndarray], op: List[np.ndarray], max_bond: int = 0,
           tol: float = 0.0, eps_rank: float = EPS_RANK) -> CBCResult:
    """CBC of an MPO applied to an MPS (Sec. III A).

    ``state[i]`` has legs (alpha_{i-1}, sigma_i, alpha_i) and ``op[i]`` has legs
    (beta_{i-1}, sigma'_i, sigma_i, beta_i); the last site has no right leg.
    Sites are 0-based here; the paper's site ``i`` is index ``i-1``.
    """
    T, W = _as_tt(state, op)
    L = len(T)
    dt = T[0].dtype
    # forward sweep: L^[0] = 1, then Eq. (tt_cbc_first_contraction) + truncation
    env = [np.ones((1, 1, 1), dtype=dt)]              # env[i] = L^[i] (chi_i, alpha_i, beta_i)
    cuts: List[CutInfo] = []
    for i in range(L - 1):                              # paper's sites 1 .. L-1
        # sum over alpha_{i-1}, then over (sigma_i, beta_{i-1})
        X = np.einsum("xab,asA->xbsA", env[i], T[i], optimize=True)
        Lp = np.einsum("xbsA,bPsB->xPAB", X, W[i], optimize=True)
        chi, d, A, B = Lp.shape
        M = Lp.reshape(chi * d, A * B)                  # rows: fused (chi_{i-1}, sigma')
        Lnew, info = compress_rows(M, max_bond, tol, eps_rank)
        env.append(Lnew.reshape(-1, A, B))
        cuts.append(info)
    # backward sweep: R^[L] = 1, Eqs. (right_sweep_init_contr), (tt_cbc_qr_decomp),
    # (tt_cbc_final_contraction)
    R = np.ones((1, 1, 1), dtype=dt)                    # R^[i] (chi_i, alpha_i, beta_i)
    out: List[Optional[np.ndarray]] = [None] * L
    for i in range(L - 1, -1, -1):
        # the partial contraction Z = T calT R is shared by S and by the R update
        # (App. A: "reuse a partial contraction result from the previous site")
        Y = np.einsum("asA,yAB->asyB", T[i], R, optimize=True)          # sum over alpha_i
        Z = np.einsum("asyB,bPsB->abPy", Y, W[i], optimize=True)        # sum over sigma, beta_i
        S = np.einsum("xab,abPy->Pxy", env[i], Z, optimize=True)        # (sigma', chi_{i-1}, chi_i)
        d, m, c = S.shape
        if i == 0:
            out[0] = S.transpose(1, 0, 2)               # T'^[1] = S^[1], legs (1, sigma', chi_1)
            break
        Smat = S.transpose(1, 0, 2).reshape(m, d * c)   # rows chi_{i-1}, cols (sigma', chi_i)
        _, Q = lq_rows(Smat)
        Q = Q.reshape(-1, d, c)                         # (chi'_{i-1}, sigma', chi_i)
        out[i] = Q
        # Eq. (tt_cbc_final_contraction): sum over sigma', chi_i of Q* with Z
        R = np.einsum("yPx,abPx->yab", Q.conj(), Z, optimize=True)
    # drop the dummy right leg of the last site to return the canonical layout
    out[L - 1] = out[L - 1][..., 0]
    bonds = [1] + [int(out[i].shape[0]) for i in range(1, L)]
    return CBCResult(out, cuts, [int(e.shape[0]) for e in env], bonds, env)


# --------------------------------------------------------------------------------------
# general trees, Sec. III B
# --------------------------------------------------------------------------------------

def _children(parent) -> List[List[int]]:
    n = len(parent)
    ch: List[List[int]] = [[] for _ in range(n)]
    for j in range(n):
        if parent[j] >= 0:
            ch[int(parent[j])].append(j)
    return ch


def _postorder(parent) -> List[int]:
    ch = _children(parent)
    root = int(np.nonzero(np.asarray(parent) < 0)[0][0])
    order, stack = [], [(root, False)]
    while stack:
        v, done = stack.pop()
        if done:
            order.append(v)
        else:
            stack.append((v, True))
            stack.extend((c, False) for c in reversed(ch[v]))
    return order


# integer leg labels used in the einsum calls of one node contraction
_S_IN, _S_OUT, _A_P, _B_P, _X_P, _X_NEW = 0, 1, 2, 3, 4, 5


def _a(j):  # alpha leg to child j
    return 10 + 3 * j


def _b(j):  # beta leg to child j
    return 11 + 3 * j


def _x(j):  # chi leg of the environment on child j
    return 12 + 3 * j


def _node_operands(T, W, nch):
    t_legs = [_A_P, _S_IN] + [_a(j) for j in range(nch)]
    w_legs = [_B_P, _S_OUT, _S_IN] + [_b(j) for j in range(nch)]
    return [T, t_legs, W, w_legs]


def _contract(ops, out_legs):
    """Contract ``[T, legs, W, legs, env, legs, ...]`` one pair at a time.

    Every leg label occurs at most twice; a label shared by the running result and the
    next operand is summed, every other label stays open.  The order is the node
    tensor T, the first environment (if any), the operator tensor W, then the remaining
    operands, which keeps the intermediates no larger than the result of one node.
    """
    pairs = [(ops[k], list(ops[k + 1])) for k in range(0, len(ops), 2)]
    t, w, rest = pairs[0], pairs[1], pairs[2:]
    order = [t] + rest[:1] + [w] + rest[1:]
    cur, cl = order[0]
    for x, xl in order[1:]:
        shared = set(cl) & set(xl)
        res = [a for a in cl if a not in shared] + [a for a in xl if a not in shared]
        cur = np.einsum(cur, cl, x, xl, res, optimize=True)
        cl = res
    return np.einsum(cur, cl, list(out_legs))


def cbc_tree(parent, state: List[np.ndarray], op: List[np.ndarray], max_bond: int = 0,
             tol: float = 0.0, eps_rank: float = EPS_RANK) -> CBCResult:
    """CBC of a TTNO applied to a TTNS on the same tree (Sec. III B).

    Step 1 (leaves to root), Eq. (cbc_tree_first_contraction): subtree tensors L^[i].
    Step 2 (root to leaves), Eq. (cbc_tree_second_contraction): complement tensors
    L^[(i,k)] for every child k of every non-leaf i.
    Step 3 (leaves to root), Eqs. (cbc_tree_third_contraction), (cbc_tree_qr),
    (cbc_final_contraction): site tensors, QR toward the parent, projected R^[i].
    """
    parent = [int(p) for p in parent]
    n = len(parent)
    ch = _children(parent)
    post = _postorder(parent)
    root = post[-1]
    cplx = any(np.iscomplexobj(x) for x in list(state) + list(op))
    dt = np.complex128 if cplx else np.float64
    T = [np.asarray(t, dtype=dt) for t in state]
    W = [np.asarray(w, dtype=dt) for w in op]
    one = np.ones((1, 1, 1), dtype=dt)
    cuts: List[CutInfo] = []

    # ---- step 1: L^[i] for every non-root node, children first
    Lsub: Dict[int, np.ndarray] = {}
    for i in post:
        if i == root:
            continue
        ops = _node_operands(T[i], W[i], len(ch[i]))
        for j, c in enumerate(ch[i]):
            ops += [Lsub[c], [_x(j), _a(j), _b(j)]]
        out_legs = [_S_OUT] + [_x(j) for j in range(len(ch[i]))] + [_A_P, _B_P]
        Lp = _contract(ops, out_legs)
        A, B = Lp.shape[-2:]
        Lnew, info = compress_rows(Lp.reshape(-1, A * B), max_bond, tol, eps_rank)
        Lsub[i] = Lnew.reshape(-1, A, B)
        cuts.append(info)

    # ---- step 2: L^[(i,k)] top-down; the root's parent environment is the scalar 1
    Ldown: Dict[int, np.ndarray] = {root: one}          # Ldown[k] = L^[(p_k, k)]
    for i in reversed(post):
        if not ch[i]:
            continue
        for jk, k in enumerate(ch[i]):
            ops = _node_operands(T[i], W[i], len(ch[i]))
            ops += [Ldown[i], [_X_P, _A_P, _B_P]]
            for j, c in enumerate(ch[i]):
                if c != k:
                    ops += [Lsub[c], [_x(j), _a(j), _b(j)]]
            out_legs = ([_S_OUT, _X_P] + [_x(j) for j, c in enumerate(ch[i]) if c != k]
                        + [_a(jk), _b(jk)])
            Lp = _contract(ops, out_legs)
            A, B = Lp.shape[-2:]
            Lnew, info = compress_rows(Lp.reshape(-1, A * B), max_bond, tol, eps_rank)
            Ldown[k] = Lnew.reshape(-1, A, B)
            cuts.append(info)

    # ---- step 3: S^[i], QR toward the parent, R^[i]; leaves first
    R: Dict[int, np.ndarray] = {}
    out: List[Optional[np.ndarray]] = [None] * n
    for i in post:
        nc = len(ch[i])
        base = _node_operands(T[i], W[i], nc)
        env_ops = [Ldown[i], [_X_P, _A_P, _B_P]]
        for j, c in enumerate(ch[i]):
            env_ops += [R[c], [_x(j), _a(j), _b(j)]]
        out_legs = [_X_P, _S_OUT] + [_x(j) for j in range(nc)]
        S = _contract(base + env_ops, out_legs)   # [chi_p, sigma', chi_c...]
        if i == root:
            out[i] = S
            continue
        shp = S.shape
        Smat = S.reshape(shp[0], -1)                    # rows chi_p, cols (sigma', chi_c...)
        _, Q = lq_rows(Smat)                            # S = R Q: Q isometric toward the parent
        Q = Q.reshape((-1,) + shp[1:])
        out[i] = Q
        ops = list(base)
        for j, c in enumerate(ch[i]):
            ops += [R[c], [_x(j), _a(j), _b(j)]]
        ops += [Q.conj(), [_X_NEW, _S_OUT] + [_x(j) for j in range(nc)]]
        R[i] = _contract(ops, [_X_NEW, _A_P, _B_P])
    bonds = [int(out[i].shape[0]) for i in range(n)]
    ranks = [int(Lsub[i].shape[0]) for i in sorted(Lsub)]
    return CBCResult(out, cuts, ranks, bonds, {"sub": Lsub, "down": Ldown})


def cbc(parent, state, op, max_bond: int = 0, tol: float = 0.0,
        eps_rank: float = EPS_RANK) -> CBCResult:
    """Dispatch on the topology: the chain rooted at node 0 uses Sec. III A."""
    parent = [int(p) for p in parent]
    if parent == list(range(-1, len(parent) - 1)):
        return cbc_tt(state, op, max_bond, tol, eps_rank)
    return cbc_tree(parent, state, op, max_bond, tol, eps_rank)
