"""CPU oracle for sntrup key generation (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does: it
shares no code with it, and fails loudly when its CUDA extension is missing.

The arithmetic lives in ``sntrup_oracle.c`` (plain C, one key at a time,
schoolbook multiplication, extended-Euclid inversion).  This module compiles
it with gcc on first use and exposes it through ctypes with numpy arrays.
Section and equation references follow arXiv 2106.08759 ("OpenSSLNTRU").
"""
from .driver import *  # noqa: F401,F403
from .driver import PARAMS, build, lib  # noqa: F401
