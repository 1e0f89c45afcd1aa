"""GB300-native block-tree construction (per-level Karp-Rabin pass) behind a C ABI.

The compute path is the CUDA library ``libbt.so`` (built from ``csrc/``);
``paper_2512_23314_gb300.bt`` is the thin ctypes binding with the same names
as the C entry points.  ``workloads`` generates the seeded synthetic texts.
"""
