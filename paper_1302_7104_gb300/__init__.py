"""GB300 (sm_103a) implementation of the per-time-step hot path of the
polar-coordinate finite-difference lattice Boltzmann model for compressible
flow (Lin, Xu, Zhang, Li & Succi).

The compute lives in a CUDA shared library with a C ABI (``include/pclb.h``);
``paper_1302_7104_gb300.pclb`` is its thin Python binding.  Importing this
package loads nothing; the library is opened on first use of the binding.
"""
__all__ = ["inputs", "pclb"]
