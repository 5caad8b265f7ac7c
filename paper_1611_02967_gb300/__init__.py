"""GB300 (sm_103a) FAS multigrid solver for the second-order convex-splitting
Cahn-Hilliard-Hele-Shaw scheme (Chen, Feng, Liu, Wang, Wise, arXiv:1611.02967).

The solver lives in a CUDA shared library with a C ABI (``include/chhs.h``);
``paper_1611_02967_gb300.chhs`` is its thin ctypes binding.  Importing this
package loads nothing; the binding loads the library on first use and raises
if it is missing.
"""
__all__ = ["chhs", "inputs"]
