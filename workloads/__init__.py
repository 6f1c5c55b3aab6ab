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
    muons_config0,
    muons_config1,
    geometry_config0,
    geometry_config1,
    geometry_tapered,
    solid,
    field_map_config1,
    workload,
    batched_instances,
    batched_instance,
    batched_counts,
    magnet_field_map,
    batched_hist,
    BATCH_STEP_LEN,
    BATCH_MAX_STEPS,
    BATCH_SEED,
    C4_MUONS,
    C4_CHUNK,
    muons_config4_chunk,
)
