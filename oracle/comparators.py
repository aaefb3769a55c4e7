"""FP64 CPU oracle of three comparison methods of Sec. III C of arXiv 2601.19650, on chains.

TEST INFRASTRUCTURE ONLY (see ``oracle/cbc.py``): only ``tests/`` and the CPU legs of
``bench.py`` import it.  Plain einsum / ``numpy.linalg`` transcriptions, shared with
nothing on the GPU path.

* ``zipup_tt`` -- the Zip-Up method: a single sweep over the sites that contracts each
  operator and state tensor with the already compressed part and truncates that bond
  at once by an SVD, using only what has been compressed so far (Sec. III C).  The
  sweep runs from the last site to the first, so the output has the layout of CBC's:
  every non-root tensor an isometry toward site 0, the scalar part at site 0.
* ``src_tt`` -- successive randomised compression (SRC): one Gaussian matrix of shape
  ``d x s`` per site, joined across the sites by the Khatri-Rao product (the sketch
  index ``j`` is shared by every site), contracted with the network into sketch
  environments (a first sweep, like CBC's environments but with the random matrices
  in place of the truncated SVD), then a second sweep in which each new tensor is the
  orthonormal row basis (LQ) of the sketched block (Sec. III C).  The random matrices
  are inputs, so the GPU path and this oracle see the same ones.
* ``direct_tt`` -- the direct method: contract operator and state into one MPS (bond
  ``alpha beta`` on every edge), then compress it as a separate step: a QR sweep from the
  first site makes every site but the last left-orthonormal, and a sweep of truncated SVDs
  from the last site back to the first keeps the dominant right singular vectors of each
  site (the Schmidt vectors of the current state, since the part to the left is
  orthonormal) and passes the rest to the left.

Readings (listed with their reasons in the design notes):

* Zip-Up runs on the state as given (the paper mentions an optional canonical form
  first; it is not applied);
* Zip-Up's truncation uses CBC's rank rule (floor, tolerance, cap) on the singular
  values of the block it compresses;
* SRC's bond on the edge between sites ``i-1`` and ``i`` is the generic rank of the
  sketched block, ``r = min(s, prod_{k<i} d_k, alpha_{i-1} beta_{i-1})``: only the
  first ``r`` sketch rows enter the LQ (beyond that the block is rank deficient);
  when ``r`` is at least the column count ``d_i chi_i`` the new tensor is the identity
  (any unitary gives the same state), as for CBC;
* SRC's new tensor is the Q of the LQ of the sketched block's first ``r`` rows (the
  paper's QR; Householder QR here, so any condition number of the block is handled).
"""
from __future__ import annotations

from typing import List, Optional

import numpy as np

from .cbc import EPS_RANK, CBCResult, CutInfo, _as_tt, choose_rank, lq_rows


def zipup_tt(state: List[np.ndarray], op: List[np.ndarray], max_bond: int = 0,
             tol: float = 0.0, eps_rank: float = EPS_RANK) -> CBCResult:
    """Zip-Up of an MPO applied to an MPS (Sec. III C), last site to first.

    At site ``i`` the carried tensor ``R`` (bond to site ``i+1`` already compressed)
    is contracted with ``T^[i]`` and ``W^[i]`` into ``Z[(alpha_{i-1} beta_{i-1}),
    (sigma'_i chi_i)]``; its truncated SVD ``Z ~ U_k s_k V_k^H`` gives the new tensor
    ``V_k^H`` and the carry ``U_k s_k = Z V_k`` for the next site.
    """
    T, W = _as_tt(state, op)
    L = len(T)
    dt = T[0].dtype
    R = np.ones((1, 1, 1), dtype=dt)                    # (chi_i, alpha_i, beta_i)
    out: List[Optional[np.ndarray]] = [None] * L
    cuts: List[CutInfo] = []
    for i in range(L - 1, -1, -1):
        Y = np.einsum("asA,yAB->asyB", T[i], R, optimize=True)          # sum over alpha_i
        Z = np.einsum("asyB,bPsB->abPy", Y, W[i], optimize=True)        # sum over sigma, beta_i
        a, b, d, c = Z.shape
        if i == 0:
            out[0] = Z.reshape(1, d, c)                 # a = b = 1 at the first site
            break
        U, s, Vh = np.linalg.svd(Z.reshape(a * b, d * c), full_matrices=False)
        k = choose_rank(s, max_bond, tol, eps_rank)
        cuts.append(CutInfo(s, k))
        Q = Vh[:k].reshape(k, d, c)                     # (chi'_{i-1}, sigma', chi_i)
        out[i] = Q
        R = np.einsum("yPx,abPx->yab", Q.conj(), Z, optimize=True)      # = (U_k s_k)^T
    out[L - 1] = out[L - 1][..., 0]
    bonds = [1] + [int(out[i].shape[0]) for i in range(1, L)]
    return CBCResult(out, cuts, bonds[1:], bonds)


def src_sketch_envs(T: List[np.ndarray], W: List[np.ndarray],
                    omega: List[np.ndarray]) -> List[np.ndarray]:
    """Sketch environments of SRC: ``C[i][j, alpha_{i-1}, beta_{i-1}]`` is the block of
    ``O|psi>`` on sites ``0 .. i-1`` contracted on its physical legs with column ``j`` of
    every site's random matrix (the Khatri-Rao product).  ``C[0]`` is the scalar 1."""
    L = len(T)
    dt = T[0].dtype
    C = [np.ones((1, 1, 1), dtype=dt)]
    for i in range(L - 1):
        X = np.einsum("jab,asA->jbsA", C[i], T[i], optimize=True)      # sum over alpha_{i-1}
        Lp = np.einsum("jbsA,bPsB->jPAB", X, W[i], optimize=True)      # sum over beta, sigma
        Om = np.asarray(omega[i])                                        # (sigma', j)
        if Lp.shape[0] == 1:                          # the first site: no sketch index yet
            C.append(np.einsum("PAB,Pj->jAB", Lp[0], Om, optimize=True))
        else:                                         # same j on every site (Khatri-Rao)
            C.append(np.einsum("jPAB,Pj->jAB", Lp, Om, optimize=True))
    return C


def src_rank(phys, C_i: np.ndarray, i: int) -> int:
    """Rows of the sketch environment on the edge (i-1, i) that enter the LQ."""
    s, a, b = C_i.shape
    p_left = int(np.prod([int(x) for x in phys[:i]])) if i > 0 else 1
    return max(1, min(s, p_left, a * b))


def src_tt(state: List[np.ndarray], op: List[np.ndarray], omega: List[np.ndarray]) -> CBCResult:
    """SRC of an MPO applied to an MPS (Sec. III C) with the given random matrices
    ``omega[i]`` (``d_i x s``; the last site's is not used)."""
    T, W = _as_tt(state, op)
    L = len(T)
    dt = np.result_type(T[0].dtype, *[np.asarray(o).dtype for o in omega[:max(L - 1, 0)]])
    T = [t.astype(dt) for t in T]
    W = [w.astype(dt) for w in W]
    C = src_sketch_envs(T, W, [np.asarray(o, dtype=dt) for o in omega])
    phys = [t.shape[1] for t in T]
    R = np.ones((1, 1, 1), dtype=dt)
    out: List[Optional[np.ndarray]] = [None] * L
    for i in range(L - 1, -1, -1):
        Y = np.einsum("asA,yAB->asyB", T[i], R, optimize=True)
        Z = np.einsum("asyB,bPsB->abPy", Y, W[i], optimize=True)
        r = src_rank(phys, C[i], i) if i > 0 else 1
        S = np.einsum("xab,abPy->Pxy", C[i][:r], Z, optimize=True)      # (sigma', r, chi_i)
        d, m, c = S.shape
        if i == 0:
            out[0] = S.transpose(1, 0, 2)
            break
        if m >= d * c:
            Q = np.eye(d * c, dtype=dt).reshape(d * c, d, c)
        else:
            _, Qm = lq_rows(S.transpose(1, 0, 2).reshape(m, d * c))   # the paper's QR
            Q = Qm.reshape(-1, d, c)
        out[i] = Q
        R = np.einsum("yPx,abPx->yab", Q.conj(), Z, optimize=True)
    out[L - 1] = out[L - 1][..., 0]
    bonds = [1] + [int(out[i].shape[0]) for i in range(1, L)]
    return CBCResult(out, [], [int(c.shape[0]) for c in C], bonds, C)


def direct_tt(state: List[np.ndarray], op: List[np.ndarray], max_bond: int = 0,
              tol: float = 0.0, eps_rank: float = EPS_RANK) -> CBCResult:
    """The direct method on a chain (Sec. III C): contract, then compress by a QR sweep
    (first site to last) and a truncating SVD sweep (last site to first), CBC's rank rule
    on each Schmidt spectrum."""
    T, W = _as_tt(state, op)
    L = len(T)
    dt = T[0].dtype
    # 1. the product MPS: N_i[(alpha beta), sigma', (alpha' beta')]
    N = []
    for i in range(L):
        t = np.einsum("asA,bPsB->abPAB", T[i], W[i], optimize=True)
        a, b, d, A, B = t.shape
        N.append(t.reshape(a * b, d, A * B))
    # 2. left-orthonormal sites 0 .. L-2 (QR), the remainder pushed to the right
    for i in range(L - 1):
        l, d, r = N[i].shape
        Q, R = np.linalg.qr(N[i].reshape(l * d, r), mode="reduced")
        N[i] = Q.reshape(l, d, -1)
        N[i + 1] = np.einsum("xr,rPy->xPy", R, N[i + 1], optimize=True)
    # 3. truncating SVDs from the last site to the first
    out: List[Optional[np.ndarray]] = [None] * L
    cuts: List[CutInfo] = []
    for i in range(L - 1, 0, -1):
        l, d, r = N[i].shape
        U, s, Vh = np.linalg.svd(N[i].reshape(l, d * r), full_matrices=False)
        k = choose_rank(s, max_bond, tol, eps_rank)
        cuts.append(CutInfo(s, k))
        out[i] = Vh[:k].reshape(k, d, r)
        N[i - 1] = np.einsum("xPl,lk->xPk", N[i - 1], U[:, :k] * s[:k], optimize=True)
    out[0] = N[0]                                       # (1, sigma', chi_1)
    out[L - 1] = out[L - 1][..., 0]
    bonds = [1] + [int(out[i].shape[0]) for i in range(1, L)]
    return CBCResult(out, cuts, bonds[1:], bonds)

