"""GB300-native explicit residual + SSP Runge-Kutta update of a high-order unstructured
finite-volume scheme for the compressible Navier-Stokes equations.

The compute path is libucns.so (CUDA kernels for sm_103a behind a C ABI,
``include/ucns.h``); ``ucns`` is its ctypes binding and ``inputs`` builds the
seeded synthetic meshes and states of the Taylor-Green workloads.
"""
from .ucns import Mesh, Net, Params, UcnsError, load  # noqa: F401
