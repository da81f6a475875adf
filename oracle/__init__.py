"""FP64 CPU oracle of the HPG-MxP solve path -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package.  The CUDA library never uses it.
"""
