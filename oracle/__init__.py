"""CPU float64 oracle for the RI-qsGW pass (arXiv 2210.17093, Sec. II).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline legs, never by the library.  It shares no code with
the CUDA path.
"""
