"""Seeded synthetic inputs shared by the oracle tests, the CUDA tests and the
benchmark.

This package generates inputs only: cell-kind masks for the paper's geometries
(cylinder, Fig. 2; NACA0012, Appendix A; channel walls), macroscopic initial
fields (uniform flow, the convected vortex of Sec. 4.1, smooth random states)
and network weights.  It holds none of the lattice Boltzmann arithmetic, so
the oracle and the CUDA path stay independent.

Cell kinds: 0 fluid, 1 solid whose links count in the force, 2 solid that does
not count (channel walls).
"""
from .geometry import cylinder_mask, naca0012_mask, naca0012_half_thickness, add_walls
from .fields import (uniform_flow, random_smooth_state, convected_vortex,
                     vortex_batch_cases, glorot_mlp, batch_order)

__all__ = ["cylinder_mask", "naca0012_mask", "naca0012_half_thickness", "add_walls",
           "uniform_flow", "random_smooth_state", "convected_vortex", "vortex_batch_cases",
           "glorot_mlp", "batch_order"]
