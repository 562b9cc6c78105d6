"""CPU FP64 oracle of the ChASE hot path: test infrastructure only.

Imported only by tests/, __graft_entry__.smoke() and bench.py's cpu_baseline and
reference legs. The product path never imports it.
"""
from . import chase_oracle  # noqa: F401
from . import grad_oracle  # noqa: F401
