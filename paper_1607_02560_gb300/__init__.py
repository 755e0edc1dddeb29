"""GB300 (sm_103a) stencil setup of the localized sparsifying preconditioner.

The compute path is liblsp.so (CUDA kernels behind the C ABI of include/lsp.h); `lsp` is its
thin Python binding. Build the library with `paper_1607_02560_gb300.build.build()`.
"""

from .lsp import (  # noqa: F401
    EIG, FLAG_DEGENERATE, FLAG_NONSYMMETRIC, FLAG_NOT_CONVERGED, MODE, POLICY, Context,
    LspError, Mlp, declared_symbols, default_opts, lib,
)
