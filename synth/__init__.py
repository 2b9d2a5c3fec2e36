"""Seeded synthetic workloads shaped like the paper's indoor-localization data.

The paper's own data (video of a campus building, §4) is not available, so
every input here is generated: a serpentine corridor floor plan, a smooth
Gaussian random feature field over (x, y), scene aliasing, and noisy query
frames. This package holds no arithmetic of the retrieval or aggregation
method itself; both the oracle and the CUDA path consume its output bytes.
"""
from .floorplan import (  # noqa: F401
    CONFIGS,
    Database,
    FeatureField,
    Windows,
    make_database,
    make_point_queries,
    make_windows,
    db_seed,
    query_seed,
    path_length,
    path_positions,
)
