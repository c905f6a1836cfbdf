"""GB300-native pTEBD layer (arXiv:2312.02667): CUDA kernels behind a C ABI.

``paper_2312_02667_gb300.ptebd`` is the Python binding of ``libptebd``.  Import
it explicitly; this package file stays empty of imports so that the seeded
input generators (``paper_2312_02667_gb300.inputs``) work on machines without
the built library.
"""
