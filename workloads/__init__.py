"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This package only *generates* relations, join trees and aggregate batches (the
problem statement of Sec. 1.1 and the application batches of Sec. 2).  It holds
none of the evaluation arithmetic: no join, no aggregation, no view.
"""
from .schemas import (  # noqa: F401
    Column, Relation, Schema, Agg,
    zipf_keys, sort_by_join_attributes, covar_batch, grouped_batch, pair_count_batch, cube_batch,
    config1, config2, config3, config3_classification, config4, config5_schema, tiny_schema, chain_schema,
    spread_keys, many_to_many,
    SEED_BASE,
)
from .tensors import to_device, to_pinned  # noqa: F401
