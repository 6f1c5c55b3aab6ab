"""Seeded synthetic inputs for the muon transport: histogram sets, geometries,
field maps and muon spectra.

This package only *makes inputs*. It holds none of the transport arithmetic
(no sampling from the tables, no rotation, no field interpolation, no RK4), so
both the FP64 oracle and the CUDA path can be fed from it without sharing any
of the method with each other.
"""
from .gen import (  # noqa: F401
    MATERIALS,
    Workload,
    histogram_set,
    muons_block,
    muons_shield,
    geometry_block1e4,
    geometry_shield1e6,
    geometry_tapered,
    solid,
    field_map_shield1e6,
    workload,
    batched_instances,
    batched_instance,
    batched_counts,
    magnet_field_map,
    batched_hist,
    BATCH_STEP_LEN,
    BATCH_MAX_STEPS,
    BATCH_SEED,
    SHIELD1E8_MUONS,
    SHIELD1E8_CHUNK,
    muons_shield1e8_chunk,
)
