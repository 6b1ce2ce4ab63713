"""GB300 shift-and-invert eigensolver for IGA / refined-IGA discretizations.

The compute path is the CUDA library ``libriga.so`` (C ABI in
``include/riga.h``); ``riga.Riga`` is its ctypes binding and
``autograd.EigSum`` the torch.autograd wrapper of the eigenvalue adjoint.
``inputs`` holds the seeded synthetic mesh / coefficient generators.
"""
from .inputs import Mesh  # noqa: F401


def build():
    from .build import build as _b
    return _b()
