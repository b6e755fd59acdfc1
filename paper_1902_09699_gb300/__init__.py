"""GB300-native PARSDMM: projections onto intersections of sets
(arXiv:1902.09699) as sm_103a CUDA kernels behind a C ABI.

``paper_1902_09699_gb300.sip`` is the thin ctypes binding of the C-ABI
library ``libsip.so`` (built by ``paper_1902_09699_gb300.build``);
``paper_1902_09699_gb300.workloads`` makes seeded synthetic inputs.
Importing the package loads nothing; the binding loads the library on first
use and raises if it is missing.
"""
