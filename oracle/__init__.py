"""FP64 CPU oracle of CBC (arXiv 2601.19650, Sec. III) and its checking helpers.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py``; never by the product path.

Parity status of each function (what pins it, in ``tests/test_oracle_*.py``):

* ``cbc.cbc_tt`` / ``cbc.cbc_tree``: pinned by brute force (exactness without
  truncation), the Eckart-Young lower bound, the projection identity, isometry,
  chain-as-tree agreement, gauge invariance and scale equivariance, and by a mutation
  test that plants typical mistakes and checks that a pin fails.
* ``brute.*``: pinned by closed forms (product states and operators) and by
  independent identities (the dense operator of a product TTNO is a Kronecker product).
* ``metrics.rel_err``: pinned against the dense difference on small cases and against
  exactly known differences.
"""
