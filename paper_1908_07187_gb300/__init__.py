"""GB300-native dense state-vector engine for the gate-application hot path of
Quantum-Kit (arXiv:1908.07187).

The engine is the C-ABI library ``libqk.so`` (header ``include/qk.h``), built from
``csrc/`` by ``paper_1908_07187_gb300.build``.  ``paper_1908_07187_gb300.qk`` is its
thin ctypes binding.  Importing the binding raises if the library is not built:
there is no CPU fallback.
"""

__all__ = ["qk", "build"]
