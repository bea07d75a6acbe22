"""GB300-native approximate multiplication of matrices with decay (SpAMM,
Truncmul and their combination) on quadtrees of dense leaf blocks.

The computation lives in libspamm.so (CUDA, sm_103a) behind the C ABI of
include/spamm.h; ``spamm`` is its Python binding."""
from . import spamm  # noqa: F401
from .spamm import (Context, Matrix, SpammError, spamm_error, spamm_from_blocks, spamm_from_coo,  # noqa: F401
                    spamm_from_dense, spamm_frob_norm, spamm_generate, spamm_kept_tasks, spamm_level_norms,
                    spamm_multiply, spamm_release, spamm_set_allocator, spamm_sync, spamm_to_blocks, spamm_to_dense,
                    spamm_truncate)
