"""Plain, slow FP64 CPU oracle for TT sums, dots, TT-rounding and the six TT
orthogonalization schemes of Coulaud, Giraud & Iannacito, "On some
orthogonalization schemes in Tensor Train format" (Sections 2-3).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The
product (the CUDA library and its Python binding) never imports, links or
executes anything from here, and nothing here imports the product.

Everything is NumPy float64.  Library primitives (LAPACK QR, SVD, Cholesky,
eigvalsh) serve as single steps; there is no blocking, fusion or reordering
beyond what the paper's definitions and algorithms state.

Pinned functions and their pins live in ``tests/test_oracle_*.py``.
"""
from .tt import (  # noqa: F401
    tt_full, tt_add, tt_scale, tt_dot, tt_norm, tt_orthogonalize_rl,
    tt_round, tt_diff_norm, bond_singular_values, tt_ranks, canonical_phi,
    canonical_e, compression_ratio, compression_gain,
)
from .schemes import (  # noqa: F401
    SCHEMES, tt_cgs, tt_mgs, tt_cgs2, tt_mgs2, tt_gram, tt_householder,
    tth_vec, apply_h_vec, loss_of_orthogonality, orthogonalize, gs_step,
)
from .operators import (  # noqa: F401
    laplace_1d, laplacian_ttm, ttm_full, tt_matvec, tt_round_rank, ones_tt, krylov_inputs, loo_curve,
)
from .variants import (  # noqa: F401
    right_sketch_contractions, tt_round_randomized, right_grams, tt_round_gram_svd, householder_apply,
    householder_q,
)
