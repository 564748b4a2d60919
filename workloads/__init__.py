"""Seeded synthetic inputs for the damped least-squares workloads.

This module holds no arithmetic of the method: it draws random numbers and lays them
out.  Both the CUDA path (through the tests and bench.py) and the CPU oracle receive
their inputs from here.  Values for single-precision workloads are drawn in float64
and rounded once to float32, so that both sides solve exactly the same problem.

Base seed of workload c is 20180209 + c; draws use numpy's Philox generator.
"""
from .gen import (  # noqa: F401
    SEED_BASE,
    block_angular_dense,
    batched_blocks,
    curvefit_problem,
    ellipse_system,
    ba_project,
    ba_system,
    banded_problem,
    banded_batch_shapes,
    mlp_init,
    rng_for,
)
