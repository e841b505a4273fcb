"""GB300-native Lasso paths by coordinate descent with GAP SAFE screening.

Fercoq, Gramfort, Salmon, "Mind the duality gap: safer rules for the Lasso",
ICML 2015.  The solver is the C-ABI library ``liblassogs.so`` (hand-written
sm_103a kernels, see ``include/lassogs.h``); this package is its thin ctypes
binding.  Build the library with ``paper_1505_03410_gb300.build.build()``.
"""
from .lassogs import (EXPORTED, LASSO_BF16, LASSO_ERR_CUDA, LASSO_ERR_INVALID_ARG,  # noqa: F401
                      LASSO_ERR_NONFINITE, LASSO_ERR_NOT_CONVERGED, LASSO_ERR_TIMEOUT, LASSO_ERR_WORKSPACE,
                      LASSO_F32, LASSO_F64, LASSO_OK, STATS_DTYPE, LassoError, LassoOpts, LassoPathStats,
                      lasso_default_opts, lasso_lambda_grid, lasso_last_error, lasso_path, lasso_path_static,
                      lasso_path_workspace_size, load, solve_path, stats_to_numpy, lasso_batch,
                      lasso_batch_workspace_size, solve_batch, lasso_correlations_bf16,
                      lasso_correlations_f32, lasso_batch_tune, lasso_batch_tune_candidates,
                      lasso_batch_tune_workspace_size, tune_batch, lasso_path_phase_cycles, PHASES,
                      lasso_path_csc, lasso_path_csc_workspace_size, solve_path_csc)
from .shard import problem_range, solve_batch_sharded  # noqa: F401  (one process per GPU)
from . import lista  # noqa: F401  (learned warm start, include/lista.h)
from .lista import ListaNet  # noqa: F401
