"""Helpers for tests that run the CUDA path through the C ABI and compare with the oracle."""
from __future__ import annotations

import numpy as np

from paper_2601_19650_gb300 import _cbc


def run_gpu(prob, max_bond=None, tol=None, precision=_cbc.CBC_PREC_FP64, eps_rank=0.0,
            slices_fwd=0, slices_bwd=0):
    """Apply prob.op to prob.state on the GPU through the C ABI; returns host tensors."""
    st, op = prob.state, prob.op
    hs = _cbc.create_from_host(st.parent, st.phys, st.bond, st.tensors, "state")
    ho = _cbc.create_from_host(op.parent, op.phys, op.bond, op.tensors, "op")
    try:
        opt = _cbc.make_options(precision, eps_rank, slices_fwd, slices_bwd)
        out = _cbc.cbc_apply(hs, ho, prob.max_bond if max_bond is None else max_bond,
                             prob.tol if tol is None else tol, opt)
        try:
            cplx = np.iscomplexobj(st.tensors[0]) or np.iscomplexobj(op.tensors[0])
            tens, bonds, log_norm = _cbc.fetch_network(
                out, _cbc.output_shape_fn(st.parent, st.phys), cplx)
        finally:
            _cbc.ttn_destroy(out)
    finally:
        _cbc.ttn_destroy(hs)
        _cbc.ttno_destroy(ho)
    return tens, bonds, log_norm
