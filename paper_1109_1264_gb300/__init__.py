"""SALT on GB300: fused vector-expression evaluation and BLAS-1 reductions.

The compute path lives in the CUDA shared library ``libsalt.so`` (built from
``csrc/``), whose C ABI is declared in ``include/salt.h``.  ``salt`` is the
thin ctypes binding of that ABI; ``inputs`` draws seeded synthetic data.
Submodules are imported lazily so that ``inputs`` can be used without the
CUDA library present.
"""
__all__ = ["salt", "inputs"]
