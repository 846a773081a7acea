"""GB300-native parallel tempering with isoenergetic cluster moves.

The compute path is the CUDA library ``_build/libicmpt.so`` (C ABI in
``include/icmpt.h``); ``icmpt`` is its thin ctypes binding, ``inputs`` the
seeded synthetic inputs and ``build`` the nvcc build for sm_103a.
Submodules are imported on demand so that ``inputs`` stays usable without
the compiled library.
"""
__all__ = ["build", "icmpt", "inputs"]
