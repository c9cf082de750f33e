"""Seeded synthetic SDP instances shared by the oracle tests, the GPU tests and bench.py.

This module only draws random numbers and writes down problem data (A_0, A_1..A_m, b) in the
paper's notation (Sec. 1, problems (P)/(D)); it holds none of the method's arithmetic.
"""
from .rng import Xoshiro256ss
from .problems import (SDPInstance, lattice_maxcut, cycle_maxcut, complete_maxcut, graph_maxcut,
                       block_arrow, random_ring_maxcut, random_gnm_maxcut, small_random_sdp,
                       diagonal_lp_sdp, batch_mix, direct_sum, maxcut_direct_sum, workload)

__all__ = ["Xoshiro256ss", "SDPInstance", "lattice_maxcut", "cycle_maxcut", "complete_maxcut",
           "graph_maxcut", "block_arrow", "random_ring_maxcut", "random_gnm_maxcut",
           "small_random_sdp", "diagonal_lp_sdp", "batch_mix", "direct_sum",
           "maxcut_direct_sum", "workload"]
