"""GB300-native (sm_103a) EM-PIC timestep: spline gather, relativistic Boris
push, charge-conserving Esirkepov deposit and Yee FDTD update behind a C-ABI
shared library (``include/pic.h``).  The Python layer only marshals arguments;
the CUDA library is loaded on first use and its absence is an error."""

__all__ = ["inputs"]
