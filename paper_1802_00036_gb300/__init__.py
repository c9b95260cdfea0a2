"""GB300-native depth completion (arXiv 1802.00036, Section IV) behind a C-ABI.

The compute path is the CUDA library ``libdc.so`` (sources in ``csrc/``),
reached through the thin ctypes binding in ``dc.py``; import it explicitly
(``from paper_1802_00036_gb300 import dc``).  ``synth`` makes seeded inputs.
"""
