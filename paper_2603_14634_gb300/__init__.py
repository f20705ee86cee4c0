"""GB300 (sm_103a) implementation of the PBD-R substep (arXiv 2603.14634).

- ``scenes``  seeded synthetic scene generators (inputs only)
- ``binding`` ctypes binding of the C ABI in ``include/pbdr.h``
- ``build``   nvcc build of ``lib/libpbdr.so``
"""
from . import scenes  # noqa: F401

__all__ = ["scenes", "binding", "build"]
