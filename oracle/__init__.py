"""FP64 CPU oracle (test infrastructure only; see floquet_oracle.py).

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import this package.  The product path never does.
"""
from .floquet_oracle import *  # noqa: F401,F403
