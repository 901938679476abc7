"""Plain FP64 CPU oracle of the LBE time step (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never does.
"""
from .oracle import Oracle, build, library_path, link_flux  # noqa: F401
