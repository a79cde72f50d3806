"""emrt: dynamic urban EM ray tracing on one GB300 (arXiv 2303.10521).

The compute path is libemrt.so (hand-written sm_103a CUDA kernels behind a
C-ABI, ``include/emrt.h``); this package holds its ctypes binding
(``_native``), a thin PyTorch front end (``engine``), the adjoint as a
``torch.autograd.Function`` (``autograd``), the build script (``build``) and
the seeded synthetic scene generator (``scenes``).  Importing the package
does not load the library; the first engine call does, and fails loudly if it
has not been built.
"""
__all__ = ["scenes", "engine", "build"]


def __getattr__(name):
    import importlib
    if name in ("engine", "scenes", "build", "autograd", "_native"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
