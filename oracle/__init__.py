"""Plain, slow FP64 CPU oracle for the localized sparsifying preconditioner's stencil setup.

TEST INFRASTRUCTURE ONLY. Only `tests/`, `__graft_entry__.smoke()` and `bench.py`'s CPU
baseline may import this package. The library under `paper_1607_02560_gb300/` never imports
it and shares no code with it.
"""

from .lsp_oracle import *  # noqa: F401,F403
from .lsp_oracle import __all__  # noqa: F401
