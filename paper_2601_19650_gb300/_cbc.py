"""ctypes binding of ``include/cbc.h`` (argument marshalling only).

Every function keeps the C name and forwards to ``libcbc.so``; all arithmetic runs in
the library's CUDA kernels.  The library must have been built (``build.build()``); if
it is missing the first call raises, there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcbc.so")

CBC_F32, CBC_F64, CBC_C64, CBC_C128 = 0, 1, 2, 3
CBC_PREC_FP64, CBC_PREC_MIXED = 0, 1
STATUS_NAMES = {
    0: "CBC_OK", 1: "CBC_ERR_INVALID_ARG", 2: "CBC_ERR_TOPOLOGY_MISMATCH", 3: "CBC_ERR_OOM",
    4: "CBC_ERR_NOT_POSITIVE_DEFINITE", 5: "CBC_ERR_NUMERICAL", 6: "CBC_ERR_TIMEOUT",
    7: "CBC_ERR_CUDA", 8: "CBC_ERR_UNSUPPORTED",
}

_DT_OF = {np.dtype(np.float32): CBC_F32, np.dtype(np.float64): CBC_F64,
          np.dtype(np.complex64): CBC_C64, np.dtype(np.complex128): CBC_C128}


class CBCError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class cbc_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("slices_fwd", ctypes.c_int),
                ("slices_bwd", ctypes.c_int), ("max_group", ctypes.c_int),
                ("eps_rank", ctypes.c_double), ("reserved_d", ctypes.c_double * 3)]


class cbc_stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 8), ("groups", ctypes.c_int64 * 8),
                ("ms", ctypes.c_double * 8), ("flops", ctypes.c_double * 8)]


KCLASS = {0: "gemm_f64", 1: "gemm_tc", 2: "eig", 3: "cholqr", 4: "aux", 5: "tc_issued",
          6: "tridiag"}

_lib = None


def lib():
    """Load libcbc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2601_19650_gb300.build` (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        P = ctypes.POINTER
        create_args = [ctypes.c_int, P(i32), P(i64), P(i64), ctypes.c_int, P(vp), ctypes.c_int,
                       vp, P(vp)]
        L.ttn_create.argtypes = create_args
        L.ttno_create.argtypes = create_args
        L.cbc_apply.argtypes = [vp, vp, i64, dbl, P(cbc_options), P(vp)]
        L.zipup_apply.argtypes = [vp, vp, i64, dbl, P(cbc_options), P(vp)]
        L.direct_apply.argtypes = [vp, vp, i64, dbl, P(cbc_options), P(vp)]
        L.cbc_rank_rule.argtypes = [ctypes.c_int, P(dbl), dbl, i64, dbl, dbl, P(ctypes.c_int),
                                    P(dbl)]
        L.cbc_rank_rule.restype = ctypes.c_int
        L.src_apply.argtypes = [vp, vp, i64, P(vp), ctypes.c_int, ctypes.c_int, P(cbc_options),
                                P(vp)]
        L.ttn_get_info.argtypes = [vp, P(i32), P(i64), P(dbl), P(dbl)]
        L.ttn_get_node.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int]
        L.ttn_get_network.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int]
        L.ttn_destroy.argtypes = [vp]
        L.ttno_destroy.argtypes = [vp]
        L.cbc_apply_tt_noalloc.argtypes = [ctypes.c_int, P(i64), P(i64), P(i64), ctypes.c_int,
                                           P(vp), P(vp), i64, dbl, vp, i64, P(i64), P(i64),
                                           P(dbl), vp]
        L.cbc_apply_tt_noalloc.restype = ctypes.c_int
        L.cbc_gemm.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.c_int, ctypes.c_int, vp, i64, ctypes.c_int, ctypes.c_int,
                               vp, i64, ctypes.c_int, ctypes.c_int, vp, i64, vp]
        L.cbc_gemm.restype = ctypes.c_int
        L.cbc_heev.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp,
                               vp, ctypes.c_int, vp]
        L.cbc_heev.restype = ctypes.c_int
        L.cbc_cholqr2.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp]
        L.cbc_cholqr2.restype = ctypes.c_int
        L.cbc_selftest_math.argtypes = [vp, vp, i64, vp]
        L.cbc_selftest_math.restype = ctypes.c_int
        L.cbc_selftest_wait.argtypes = [ctypes.c_longlong, P(ctypes.c_int), vp]
        L.cbc_selftest_wait.restype = ctypes.c_int
        L.cbc_apply_batched.argtypes = [ctypes.c_int, P(vp), P(vp), P(i64), P(dbl),
                                        P(cbc_options), ctypes.c_int, P(vp)]
        L.cbc_apply_batched.restype = ctypes.c_int
        L.cbc_stats_enable.argtypes = [ctypes.c_int]
        L.cbc_stats_reset.argtypes = []
        L.cbc_stats_read.argtypes = [P(cbc_stats)]
        for f in ("cbc_stats_enable", "cbc_stats_reset", "cbc_stats_read"):
            getattr(L, f).restype = ctypes.c_int
        L.cbc_last_error.restype = ctypes.c_char_p
        L.cbc_last_error.argtypes = []
        for f in ("ttn_create", "ttno_create", "cbc_apply", "ttn_get_info", "ttn_get_node",
                  "ttn_get_network", "ttn_destroy", "ttno_destroy", "zipup_apply", "src_apply",
                  "direct_apply"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def cbc_stats_enable(timing: bool):
    _check(lib().cbc_stats_enable(1 if timing else 0))


def cbc_stats_reset():
    _check(lib().cbc_stats_reset())


def cbc_stats_read() -> dict:
    st = cbc_stats()
    _check(lib().cbc_stats_read(ctypes.byref(st)))
    return {name: {"launches": int(st.launches[k]), "groups": int(st.groups[k]),
                   "ms": float(st.ms[k]), "flops": float(st.flops[k])}
            for k, name in KCLASS.items()}


def cbc_last_error() -> str:
    return lib().cbc_last_error().decode()


def _check(rc: int):
    if rc != 0:
        raise CBCError(rc, cbc_last_error())


def _create(fn, parent, phys, bond, dtype: int, ptrs: Sequence[int], on_device: bool,
            stream: Optional[int]):
    n = len(parent)
    par = (ctypes.c_int32 * n)(*[int(x) for x in parent])
    ph = (ctypes.c_int64 * n)(*[int(x) for x in phys])
    bd = (ctypes.c_int64 * n)(*[int(x) for x in bond])
    arr = (ctypes.c_void_p * n)(*[ctypes.c_void_p(int(p)) for p in ptrs])
    out = ctypes.c_void_p()
    _check(fn(n, par, ph, bd, dtype, arr, 1 if on_device else 0,
              ctypes.c_void_p(stream or 0), ctypes.byref(out)))
    return out


def ttn_create(parent, phys, bond, dtype: int, ptrs, on_device: bool, stream=None):
    return _create(lib().ttn_create, parent, phys, bond, dtype, ptrs, on_device, stream)


def ttno_create(parent, phys, bond, dtype: int, ptrs, on_device: bool, stream=None):
    return _create(lib().ttno_create, parent, phys, bond, dtype, ptrs, on_device, stream)


def make_options(precision: int = CBC_PREC_FP64, eps_rank: float = 0.0, slices_fwd: int = 0,
                 slices_bwd: int = 0, max_group: int = 0) -> cbc_options:
    o = cbc_options()
    o.precision = precision
    o.eps_rank = eps_rank
    o.slices_fwd = slices_fwd
    o.slices_bwd = slices_bwd
    o.max_group = max_group
    return o


def cbc_apply(state, op, max_bond: int, tol: float, opt: Optional[cbc_options] = None):
    out = ctypes.c_void_p()
    _check(lib().cbc_apply(state, op, int(max_bond), float(tol),
                           ctypes.byref(opt) if opt is not None else None, ctypes.byref(out)))
    return out


def zipup_apply(state, op, max_bond: int, tol: float, opt: Optional[cbc_options] = None):
    """Zip-Up comparison method (tensor trains); same arguments and output as cbc_apply."""
    out = ctypes.c_void_p()
    _check(lib().zipup_apply(state, op, int(max_bond), float(tol),
                             ctypes.byref(opt) if opt is not None else None, ctypes.byref(out)))
    return out


def cbc_rank_rule(w, beyond: float, max_bond: int, tol: float, floor_rel: float):
    """The library's truncation rank rule on host weights w (descending): (k, discarded)."""
    arr = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    k = ctypes.c_int()
    disc = ctypes.c_double()
    _check(lib().cbc_rank_rule(int(arr.size), arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                               float(beyond), int(max_bond), float(tol), float(floor_rel),
                               ctypes.byref(k), ctypes.byref(disc)))
    return k.value, disc.value


def direct_apply(state, op, max_bond: int, tol: float, opt: Optional[cbc_options] = None):
    """Direct method (contract, then QR and SVD sweeps; tensor trains); arguments and output
    as cbc_apply."""
    out = ctypes.c_void_p()
    _check(lib().direct_apply(state, op, int(max_bond), float(tol),
                              ctypes.byref(opt) if opt is not None else None, ctypes.byref(out)))
    return out


def src_apply(state, op, sketch_size: int, omega, opt: Optional[cbc_options] = None):
    """SRC comparison method (tensor trains) with host numpy random matrices omega[i]
    (d_i x sketch_size; real for real networks, complex for complex ones)."""
    arrs = [np.ascontiguousarray(o) for o in omega]
    ptrs = (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
    out = ctypes.c_void_p()
    _check(lib().src_apply(state, op, int(sketch_size), ptrs, _DT_OF[arrs[0].dtype], 0,
                           ctypes.byref(opt) if opt is not None else None, ctypes.byref(out)))
    return out


def cbc_apply_tt_noalloc(phys, state_bond, op_bond, dtype: int, state_ptrs, op_ptrs,
                         max_bond: int, tol: float, out_ptr: int, out_capacity: int, stream=None):
    """No-allocation tensor-train CBC: device input pointers, a caller-owned device output
    buffer; returns (out_offsets, out_bonds, log_norm)."""
    L = len(phys)
    ph = (ctypes.c_int64 * L)(*[int(x) for x in phys])
    sb = (ctypes.c_int64 * L)(*[int(x) for x in state_bond])
    obd = (ctypes.c_int64 * L)(*[int(x) for x in op_bond])
    sp = (ctypes.c_void_p * L)(*[ctypes.c_void_p(int(p)) for p in state_ptrs])
    op = (ctypes.c_void_p * L)(*[ctypes.c_void_p(int(p)) for p in op_ptrs])
    offs = (ctypes.c_int64 * L)()
    bonds = (ctypes.c_int64 * L)()
    ln = ctypes.c_double()
    _check(lib().cbc_apply_tt_noalloc(L, ph, sb, obd, int(dtype), sp, op, int(max_bond),
                                      float(tol), ctypes.c_void_p(int(out_ptr)),
                                      int(out_capacity), offs, bonds, ctypes.byref(ln),
                                      ctypes.c_void_p(stream or 0)))
    return np.array(offs[:], dtype=np.int64), np.array(bonds[:], dtype=np.int64), ln.value


def cbc_gemm(precision: int, slices: int, dtype: int, M: int, N: int, K: int, A_ptr: int,
             lda: int, transA: bool, conjA: bool, B_ptr: int, ldb: int, transB: bool,
             conjB: bool, C_ptr: int, ldc: int, stream=None):
    _check(lib().cbc_gemm(int(precision), int(slices), int(dtype), int(M), int(N), int(K),
                          ctypes.c_void_p(int(A_ptr)), int(lda), int(bool(transA)),
                          int(bool(conjA)), ctypes.c_void_p(int(B_ptr)), int(ldb),
                          int(bool(transB)), int(bool(conjB)), ctypes.c_void_p(int(C_ptr)),
                          int(ldc), ctypes.c_void_p(stream or 0)))


def cbc_heev(dtype: int, m: int, kmax: int, nb: int, A_ptr: int, lam_ptr: int, U_ptr: int,
             mixed: bool = False, stream=None):
    _check(lib().cbc_heev(int(dtype), int(m), int(kmax), int(nb), ctypes.c_void_p(int(A_ptr)),
                          ctypes.c_void_p(int(lam_ptr)), ctypes.c_void_p(int(U_ptr)),
                          1 if mixed else 0, ctypes.c_void_p(stream or 0)))


def cbc_cholqr2(dtype: int, m: int, n: int, nb: int, S_ptr: int, stream=None):
    _check(lib().cbc_cholqr2(int(dtype), int(m), int(n), int(nb), ctypes.c_void_p(int(S_ptr)),
                             ctypes.c_void_p(stream or 0)))


def cbc_selftest_math(x_ptr: int, out_ptr: int, n: int, stream=None):
    _check(lib().cbc_selftest_math(ctypes.c_void_p(int(x_ptr)), ctypes.c_void_p(int(out_ptr)),
                                   int(n), ctypes.c_void_p(stream or 0)))


def cbc_selftest_wait(limit_cycles: int, stream=None):
    """Returns (status code, returned flag) of the bounded-wait self-test."""
    ret = ctypes.c_int(0)
    rc = lib().cbc_selftest_wait(int(limit_cycles), ctypes.byref(ret), ctypes.c_void_p(stream or 0))
    return rc, ret.value


def cbc_apply_batched(states, ops, max_bond, tol, opt: Optional[cbc_options] = None,
                      workers: int = 0):
    """Run len(states) independent applications concurrently; returns the output handles."""
    n = len(states)
    st = (ctypes.c_void_p * n)(*[h.value for h in states])
    op = (ctypes.c_void_p * n)(*[h.value for h in ops])
    mb = (ctypes.c_int64 * n)(*[int(x) for x in max_bond])
    tl = (ctypes.c_double * n)(*[float(x) for x in tol])
    outs = (ctypes.c_void_p * n)()
    _check(lib().cbc_apply_batched(n, st, op, mb, tl,
                                   ctypes.byref(opt) if opt is not None else None,
                                   int(workers), outs))
    return [ctypes.c_void_p(outs[j]) for j in range(n)]


def ttn_get_info(t):
    n = ctypes.c_int32()
    _check(lib().ttn_get_info(t, ctypes.byref(n), None, None, None))
    bonds = (ctypes.c_int64 * n.value)()
    ln = ctypes.c_double()
    _check(lib().ttn_get_info(t, None, bonds, ctypes.byref(ln), None))
    return n.value, np.array(bonds[:], dtype=np.int64), ln.value


def ttn_get_discarded(t):
    """Relative discarded weight of the compression(s) of each node's parent edge."""
    n = ctypes.c_int32()
    _check(lib().ttn_get_info(t, ctypes.byref(n), None, None, None))
    d = (ctypes.c_double * n.value)()
    _check(lib().ttn_get_info(t, None, None, None, d))
    return np.array(d[:], dtype=np.float64)


def ttn_get_node(t, node: int, dst_ptr: int, dst_on_device: bool, dtype: int):
    _check(lib().ttn_get_node(t, int(node), ctypes.c_void_p(int(dst_ptr)),
                              1 if dst_on_device else 0, int(dtype)))


def ttn_destroy(t):
    _check(lib().ttn_destroy(t))


def ttno_destroy(t):
    _check(lib().ttno_destroy(t))


# ----------------------------------------------------------------------------------------
# convenience: whole networks in and out (still marshalling only)
# ----------------------------------------------------------------------------------------

def _host_ptrs(tensors):
    arrs = [np.ascontiguousarray(t) for t in tensors]
    return arrs, [a.ctypes.data for a in arrs]


def create_from_host(parent, phys, bond, tensors, kind: str = "state", stream=None):
    """Create a handle from host numpy tensors (canonical leg layout)."""
    arrs, ptrs = _host_ptrs(tensors)
    dt = _DT_OF[arrs[0].dtype]
    fn = ttn_create if kind == "state" else ttno_create
    return fn(parent, phys, bond, dt, ptrs, False, stream)


def create_from_device(parent, phys, bond, tensors, kind: str = "state", stream=None):
    """Create a handle from CUDA torch tensors (canonical leg layout, contiguous)."""
    import torch  # noqa: F401  (device memory comes from torch)
    dmap = {"torch.float32": CBC_F32, "torch.float64": CBC_F64,
            "torch.complex64": CBC_C64, "torch.complex128": CBC_C128}
    dt = dmap[str(tensors[0].dtype)]
    ptrs = [t.data_ptr() for t in tensors]
    fn = ttn_create if kind == "state" else ttno_create
    return fn(parent, phys, bond, dt, ptrs, True, stream)


def fetch_network(t, shapes_of_node, cplx: bool):
    """Copy every node of a TTNS handle to host (FP64 / complex128) -> (tensors, bonds, log_norm).

    One ttn_get_network call into one host buffer; the tensors are views of it."""
    n, bonds, log_norm = ttn_get_info(t)
    shapes = [shapes_of_node(i, bonds) for i in range(n)]
    sizes = [int(np.prod(sh)) for sh in shapes]
    buf = np.empty(sum(sizes), dtype=np.complex128 if cplx else np.float64)
    _check(lib().ttn_get_network(t, ctypes.c_void_p(buf.ctypes.data), 0,
                                 CBC_C128 if cplx else CBC_F64))
    out, off = [], 0
    for sh, sz in zip(shapes, sizes):
        out.append(buf[off:off + sz].reshape(sh))
        off += sz
    return out, bonds, log_norm


def output_shape_fn(parent, phys):
    """Shape of node i of an output TTNS given the output bonds (canonical layout)."""
    n = len(parent)
    ch = [[] for _ in range(n)]
    for j, p in enumerate(parent):
        if p >= 0:
            ch[int(p)].append(j)

    def shape(i, bonds):
        return (int(bonds[i]), int(phys[i])) + tuple(int(bonds[c]) for c in ch[i])
    return shape
