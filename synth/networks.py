"""Topologies, bond-dimension clamps and seeded random TTNS/TTNO tensors.

Layout convention (shared by every consumer; it fixes *where* each leg sits, not
how anything is computed):

* A network on ``n`` nodes is given by ``parent[i]`` (``-1`` for the root), the
  physical dimension ``phys[i]`` (1 for a purely virtual node) and ``bond[i]``, the
  dimension of the edge from ``i`` to its parent (1 at the root).
* State node tensor ``T[i]`` has legs ``[parent, phys, children...]`` with the
  children in ascending node id (Sec. II A, Eq. (ttns): ``T^[i]_{sigma_i, alpha_vec_i}``).
* Operator node tensor ``W[i]`` has legs ``[parent, phys_out, phys_in, children...]``
  (Sec. II C, Eq. (ttno): ``calT^[i]_{sigma'_i sigma_i beta_vec_i}``).
* A tensor train (MPS/MPO) is the chain ``parent[i] = i-1`` rooted at the first
  site, which is the imaginary-site-0 convention of Sec. II B with site 1 as the
  effective root.  The last site is a leaf and has no child leg.

Random entries follow the synthetic workloads: real Gaussian, complex Gaussian
``(x+iy)/sqrt(2)``, or the uniform ``[-0.5, 1]`` real/imaginary parts of the
paper's random benchmark (Sec. IV A).  Each tensor is scaled to unit Frobenius
norm before the cast to its storage dtype, so every consumer sees bit-identical
values.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np


# --------------------------------------------------------------------------------------
# topologies
# --------------------------------------------------------------------------------------

def chain_topology(L: int, d: int):
    """Tensor train with ``L`` sites of physical dimension ``d`` rooted at site 0."""
    parent = np.arange(-1, L - 1, dtype=np.int32)
    phys = np.full(L, d, dtype=np.int64)
    return parent, phys


def binary_tree_topology(depth: int, d: int):
    """Perfect binary tree of the given depth (Sec. IV A, binary TTNS).

    Nodes are numbered breadth first (root 0, children of ``n`` are ``2n+1, 2n+2``).
    Only the ``2**depth`` leaves carry a physical leg of dimension ``d``; the
    ``2**depth - 1`` internal nodes are virtual (physical dimension 1).
    """
    n = 2 ** (depth + 1) - 1
    parent = np.array([-1] + [(j - 1) // 2 for j in range(1, n)], dtype=np.int32)
    phys = np.ones(n, dtype=np.int64)
    phys[2 ** depth - 1:] = d
    return parent, phys


def t_tree_topology(L: int, d: int):
    """T-tree (Sec. IV A): a virtual centre node with three chains of ``L`` physical sites."""
    parent = [-1]
    phys = [1]
    for _ in range(3):
        prev = 0
        for _ in range(L):
            parent.append(prev)
            phys.append(d)
            prev = len(parent) - 1
    return np.array(parent, dtype=np.int32), np.array(phys, dtype=np.int64)


def ftps_topology(L: int, d: int):
    """Fork tensor product structure (Sec. IV A): a virtual backbone of ``L`` nodes,
    each carrying a physical chain of ``L`` sites."""
    parent = []
    phys = []
    backbone_prev = -1
    for _ in range(L):
        parent.append(backbone_prev)
        phys.append(1)
        b = len(parent) - 1
        prev = b
        for _ in range(L):
            parent.append(prev)
            phys.append(d)
            prev = len(parent) - 1
        backbone_prev = b
    return np.array(parent, dtype=np.int32), np.array(phys, dtype=np.int64)


def children_of(parent: Sequence[int]) -> List[List[int]]:
    """Children of every node in ascending node id."""
    n = len(parent)
    ch: List[List[int]] = [[] for _ in range(n)]
    for j in range(n):
        p = int(parent[j])
        if p >= 0:
            ch[p].append(j)
    return ch


def _postorder(parent: Sequence[int]) -> List[int]:
    ch = children_of(parent)
    root = [j for j in range(len(parent)) if parent[j] < 0]
    assert len(root) == 1, "exactly one root expected"
    order: List[int] = []
    stack = [(root[0], False)]
    while stack:
        v, done = stack.pop()
        if done:
            order.append(v)
        else:
            stack.append((v, True))
            for c in reversed(ch[v]):
                stack.append((c, False))
    return order


def clamp_bonds(parent, phys, cap: int, power: int = 1) -> np.ndarray:
    """Bond dimension of every edge, clamped to what the Hilbert space allows.

    The edge from ``i`` to its parent gets ``min(cap, P_sub**power, P_rest**power)``
    where ``P_sub`` is the product of physical dimensions in the subtree of ``i`` and
    ``P_rest`` the product over the remaining sites (``power`` = 1 for a state,
    2 for an operator).  A second pass keeps every edge no larger than the product of
    the other legs at either end, so no node tensor is forced to be rank deficient.
    """
    n = len(parent)
    ch = children_of(parent)
    post = _postorder(parent)
    sub = [1] * n
    for v in post:
        s = int(phys[v]) ** power
        for c in ch[v]:
            s *= sub[c]
        sub[v] = s
    root = post[-1]
    total = sub[root]
    bond = [1] * n
    for v in range(n):
        if v == root:
            continue
        bond[v] = int(min(cap, sub[v], total // sub[v]))
    # local consistency (only bites for unusual topologies)
    changed = True
    while changed:
        changed = False
        for v in post:
            if v == root:
                continue
            lim = int(phys[v]) ** power
            for c in ch[v]:
                lim *= bond[c]
            if bond[v] > lim:
                bond[v] = lim
                changed = True
        for v in reversed(post):
            for c in ch[v]:
                lim = int(phys[v]) ** power * bond[v]
                for c2 in ch[v]:
                    if c2 != c:
                        lim *= bond[c2]
                if bond[c] > lim:
                    bond[c] = lim
                    changed = True
    return np.array(bond, dtype=np.int64)


# --------------------------------------------------------------------------------------
# random tensors
# --------------------------------------------------------------------------------------

@dataclasses.dataclass
class Network:
    """A TTNS (``kind='state'``) or TTNO (``kind='op'``) in the canonical leg layout."""

    parent: np.ndarray
    phys: np.ndarray
    bond: np.ndarray
    tensors: List[np.ndarray]
    kind: str = "state"

    @property
    def n(self) -> int:
        return len(self.parent)

    @property
    def children(self) -> List[List[int]]:
        return children_of(self.parent)

    @property
    def root(self) -> int:
        return int(np.nonzero(np.asarray(self.parent) < 0)[0][0])

    @property
    def dtype(self):
        return self.tensors[0].dtype

    def shape_of(self, i: int):
        ch = self.children[i]
        cb = [int(self.bond[c]) for c in ch]
        if self.kind == "state":
            return (int(self.bond[i]), int(self.phys[i]), *cb)
        return (int(self.bond[i]), int(self.phys[i]), int(self.phys[i]), *cb)


def _draw(rng: np.random.Generator, shape, dist: str) -> np.ndarray:
    if dist == "gauss_real":
        x = rng.standard_normal(shape)
    elif dist == "gauss_complex":
        x = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)
    elif dist == "uniform_complex":
        # Sec. IV A: real and imaginary parts iid uniform on [-0.5, 1]
        x = rng.uniform(-0.5, 1.0, shape) + 1j * rng.uniform(-0.5, 1.0, shape)
    elif dist == "uniform_real":
        x = rng.uniform(-0.5, 1.0, shape)
    else:
        raise ValueError(f"unknown distribution {dist!r}")
    nrm = np.sqrt(np.sum(np.abs(x) ** 2))
    return x / nrm


def random_network(parent, phys, bond, kind: str, dtype, dist: str,
                   rng: np.random.Generator) -> Network:
    """Draw every node tensor (in node order) with unit Frobenius norm."""
    net = Network(np.asarray(parent, dtype=np.int32), np.asarray(phys, dtype=np.int64),
                  np.asarray(bond, dtype=np.int64), [], kind)
    for i in range(net.n):
        t = _draw(rng, net.shape_of(i), dist)
        net.tensors.append(np.ascontiguousarray(t.astype(dtype)))
    return net


# --------------------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------------------

@dataclasses.dataclass
class Problem:
    name: str
    state: Network
    op: Network
    max_bond: int
    tol: float
    seed: int


_DIST_OF = {
    np.dtype(np.float64): "gauss_real",
    np.dtype(np.float32): "gauss_real",
    np.dtype(np.complex64): "gauss_complex",
    np.dtype(np.complex128): "gauss_complex",
}

# (topology, sizes, dtype) of each workload; sizes can be overridden to make smaller
# cases of the same shape family for parity tests.
CONFIGS = {
    # MPO on MPS, L=8, d=2, chi=8, D=4, target 8; float64 N(0,1), unit Frobenius
    1: dict(topo="chain", L=8, d=2, chi=8, D=4, max_bond=8, dtype=np.float64),
    # MPO on MPS, L=64, d=2, chi=128, D=16, target 128; complex64
    2: dict(topo="chain", L=64, d=2, chi=128, D=16, max_bond=128, dtype=np.complex64),
    # TTNO on TTNS, perfect binary tree of depth 6 (64 leaves, d=2), chi=64, D=8, target 64
    3: dict(topo="binary", L=6, d=2, chi=64, D=8, max_bond=64, dtype=np.float32),
    # one instance of the batched set; see make_batch()
    4: dict(topo="chain", L=32, d=2, chi=64, D=8, max_bond=64, dtype=np.float32),
    # large tensor train: L=100, d=4, chi=1024, D=32, target 1024; complex64
    5: dict(topo="chain", L=100, d=4, chi=1024, D=32, max_bond=1024, dtype=np.complex64),
    # the paper's own random benchmark shape (Sec. IV A), MPS part
    "P": dict(topo="chain", L=50, d=3, chi=40, D=40, max_bond=40, dtype=np.complex128,
              dist="uniform_complex"),
}


def _topology(topo: str, L: int, d: int):
    if topo == "chain":
        return chain_topology(L, d)
    if topo == "binary":
        return binary_tree_topology(L, d)
    if topo == "ttree":
        return t_tree_topology(L, d)
    if topo == "ftps":
        return ftps_topology(L, d)
    raise ValueError(topo)


def make_problem(config=2, seed: int = 0, tol: float = 0.0, **over) -> Problem:
    """Build one workload instance; keyword overrides shrink or reshape it."""
    spec = dict(CONFIGS[config])
    spec.update(over)
    dtype = np.dtype(spec["dtype"])
    dist = spec.get("dist", _DIST_OF[dtype])
    parent, phys = _topology(spec["topo"], spec["L"], spec["d"])
    sbond = clamp_bonds(parent, phys, spec["chi"], power=1)
    obond = clamp_bonds(parent, phys, spec["D"], power=2)
    rs = np.random.default_rng([seed, 0])
    ro = np.random.default_rng([seed, 1])
    st = random_network(parent, phys, sbond, "state", dtype, dist, rs)
    op = random_network(parent, phys, obond, "op", dtype, dist, ro)
    name = f"cfg{config}-" + "-".join(f"{k}{v}" for k, v in over.items()) if over else f"cfg{config}"
    return Problem(name, st, op, int(spec["max_bond"]), float(tol), seed)


def batch_shapes(n: int = 256, seed0: int = 0):
    """Per-instance (L, chi, D) of the batched serving set: L ~ U{16..64},
    chi in {32,64,128,256}, D in {4,8,16,32}; instance j draws from seed j."""
    out = []
    for j in range(seed0, seed0 + n):
        r = np.random.default_rng([j, 2])
        L = int(r.integers(16, 65))
        chi = int(r.choice([32, 64, 128, 256]))
        D = int(r.choice([4, 8, 16, 32]))
        out.append((L, chi, D))
    return out


def make_batch(n: int = 256, seed0: int = 0, scale: Optional[int] = None):
    """The batched set: instance j is a float32 MPO.MPS with its own seed and target = chi.

    ``scale`` divides chi and D (for small parity cases)."""
    probs = []
    for j, (L, chi, D) in zip(range(seed0, seed0 + n), batch_shapes(n, seed0)):
        if scale:
            chi = max(2, chi // scale)
            D = max(2, D // scale)
            L = max(4, L // scale)
        probs.append(make_problem(4, seed=j, L=L, chi=chi, D=D, max_bond=chi))
    return probs


def sketch_matrices(phys, s: int, seed: int = 0, cplx: bool = False) -> List[np.ndarray]:
    """The random matrices of the randomised comparator (SRC, Sec. III C): one ``d_i x s``
    Gaussian matrix per site, standard normal entries (complex ``(x+iy)/sqrt(2)`` when
    ``cplx``), float64 / complex128, drawn from ``default_rng([seed, 3])`` in site order."""
    rng = np.random.default_rng([seed, 3])
    out = []
    for d in phys:
        shape = (int(d), int(s))
        if cplx:
            x = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)
        else:
            x = rng.standard_normal(shape)
        out.append(np.ascontiguousarray(x))
    return out
