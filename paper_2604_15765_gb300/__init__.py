"""Orkan on GB300: k-local conjugation of hermitian operators in the tiled
lower-triangle layout, as hand-written CUDA for sm_103a behind a C ABI.

``paper_2604_15765_gb300.orkan`` is the ctypes binding of include/orkan.h;
``paper_2604_15765_gb300.circuit`` issues a list of op dicts through it.
Importing either needs the compiled library (see ``build.build()``).
"""
__all__ = ["orkan", "circuit", "build"]
