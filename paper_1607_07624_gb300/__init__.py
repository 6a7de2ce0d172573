"""GB300-native modulated-pyramid single-conjugate AO loop (PASSATA's hot path).

Submodules:
  pas     ctypes binding of libpas.so (the C ABI in include/pas.h)
  calib   one-off host FP64 setup: phase screens, Zernike basis, pseudo-inverse
  system  the processing-object chain of one configuration on the GPU
  build   nvcc build of libpas.so for sm_103a

Importing ``pas`` (or ``system``) raises ImportError when libpas.so is not built:
there is no CPU fallback.
"""
__all__ = ["pas", "calib", "system", "build"]
