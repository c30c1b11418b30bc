"""GB300-native filter stage of the seed-filter-extend pipeline.

Spaced-seed hits, the per-diagonal skip and the ungapped X-drop extension,
computed by hand-written CUDA kernels for sm_103a behind the C ABI of
include/sfe.h. `sfe` is the Python binding (argument marshalling only);
`build` compiles the library in-tree.
"""
from .sfe import (  # noqa: F401
    BATCH_HSP_DTYPE, EXT_DTYPE, GALIGN_DTYPE, YdropParams, ydrop_params, HIT_DTYPE, HSP_DTYPE, NO_CELL_PLANES, SCHED_LARGEST_FIRST,
    SCHED_NATURAL, SCHED_PREDICTED, SCHED_RANDOM, SKIP_PASSING_ONLY, STAGES, TIME_STAGES,
    WALK_PERSISTENT, WALK_SPECULATIVE, WALK_TWO_LAUNCHES,
    BatchPlan, Context, Index, MlpData, Params, SfeError, Stats, default_params, exported_symbols, lib,
    mlp_model_bytes, mlp_param_count,
)
