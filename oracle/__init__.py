"""CPU oracle for the snapshot digest / dedup / census / restore / compare path.

Test infrastructure only: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only users.  The product library never
imports it.
"""
from .kc_oracle import *  # noqa: F401,F403
