"""GB300 (sm_103a) implementation of the Cholesky-based compression (CBC) that applies a
TTNO (MPO) to a TTNS (MPS) and compresses the result (arXiv 2601.19650, Sec. III).

The product is the CUDA library ``libcbc.so`` with the C ABI of ``include/cbc.h``;
``paper_2601_19650_gb300._cbc`` is its ctypes binding.  Build it in-tree with
``python -m paper_2601_19650_gb300.build``.
"""
from . import _cbc  # noqa: F401
from ._cbc import (  # noqa: F401
    CBCError,
    CBC_C64,
    CBC_C128,
    CBC_F32,
    CBC_F64,
    CBC_PREC_FP64,
    CBC_PREC_MIXED,
    cbc_apply,
    cbc_last_error,
    make_options,
    ttn_create,
    ttn_destroy,
    ttn_get_info,
    ttn_get_node,
    ttno_create,
    ttno_destroy,
)
