"""FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package. The CUDA library never calls it.
"""
from .oracle import (  # noqa: F401
    build,
    verify,
    eval_point,
    forward,
    pair_coverage,
    pair_covers,
    pairs_coverage,
    layer_pair_fraction,
    ss_covered_fraction,
    space_size,
    threshold_literal,
    threshold_margin,
    digits,
    mask_words,
    TAU,
)
