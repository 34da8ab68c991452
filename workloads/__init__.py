"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This package only draws and evaluates input fields (desired states, bounds,
request mixes). It holds none of the interior point method's arithmetic, so
both the CUDA path and the oracle can be fed from it without sharing code.
"""
from .generators import (  # noqa: F401
    node_coords,
    yd_sin_product,
    yd_gaussian_sum,
    yd_cube_sin,
    yd_cd_bump,
    poisson_2d_sweep,
    serving_stream,
    heat_moving_target,
    Workload,
    workload_c1,
    workload_c2,
    workload_c3,
    workload_c4,
)
