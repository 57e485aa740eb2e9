"""GB300-native H^2-matrix local low-rank updates (Boerm & Reimer, arXiv:1402.5056).

The compute path is ``libh2gb.so`` (hand-written sm_103a CUDA behind a C
ABI, ``include/h2gb.h``); ``paper_1402_5056_gb300.binding`` marshals Python
arguments to it and fails loudly at import when the library is missing.
``paper_1402_5056_gb300.build`` compiles the library in-tree.
"""
