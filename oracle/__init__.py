"""CPU oracle of the DECO MaxCut hot path.

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product library.
"""
from . import deco_oracle  # noqa: F401
from . import mpnn_oracle  # noqa: F401
