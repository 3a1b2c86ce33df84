"""CPU FP64 oracle for the DA-based FMM (Coulomb kernel).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py`` may import this package.  The library it loads is the
plain C restatement of the paper's method in ``oracle/*.c`` and shares no code
with the CUDA path.  See ``oracle/oracle.h`` for what each function follows.
"""
from .oracle import *  # noqa: F401,F403
