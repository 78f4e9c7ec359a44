"""CPU oracle for bulk AES — test infrastructure, never part of the product path.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.
"""
from .oracle import Oracle, build, load  # noqa: F401
