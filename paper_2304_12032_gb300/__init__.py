"""lfx: one semi-implicit BDF step of P1-P1 VMS-LES incompressible Navier-Stokes on a GPU.

The compute path is liblfx.so (CUDA for sm_103a, C ABI in include/lfx.h); ``lfx`` is its
ctypes binding.  Build with ``python -m paper_2304_12032_gb300.build``.
"""
