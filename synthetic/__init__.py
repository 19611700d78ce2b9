"""Seeded synthetic inputs shared by the library's tests, the benchmark and the oracle.

Holds input generation only (systems, walker positions, imaginary times);
none of the Monte Carlo MP2 arithmetic lives here.
"""
from .systems import (CARTESIAN, SCANNED_WEIGHTS, SPEED_OF_LIGHT, TABLE1, TABLE1_ROW_FOR_Z, System,  # noqa: F401
                      make_system, nonrelativistic_variant, overlap_matrices,
                      time_reversed_coefficients, weight_row)
from .samples import imaginary_times, walker_positions  # noqa: F401
