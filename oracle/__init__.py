"""CPU oracle for the distance-bounded approximate point-in-polygon join.

TEST INFRASTRUCTURE ONLY: used by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``.  The product path never imports it.
"""
