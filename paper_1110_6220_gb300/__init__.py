"""GB300-native two-scale Eikonal solver (cell label-correcting, bucketed).

The compute path lives in the CUDA shared library ``libeik.so`` built from
``csrc/``; :mod:`paper_1110_6220_gb300.eik` is its thin ctypes binding.
:mod:`paper_1110_6220_gb300.workloads` holds the seeded synthetic inputs.

Importing the package itself loads nothing; ``from paper_1110_6220_gb300 import
eik`` loads the library and raises if it has not been built.
"""
__all__ = ["eik", "workloads"]
