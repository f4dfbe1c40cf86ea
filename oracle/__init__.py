"""FP64 CPU oracle of the elastic staggered-grid scheme.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import anything from this package.
It shares no code with the CUDA path in ``paper_2112_15071_gb300``.
"""
