"""GB300-native lattice Basic Scheme (Bergmann & Merkert, arXiv 1605.05712).

FFT-based elastic homogenization on arbitrary sampling lattices P(M): the
generalized Moulinec-Suquet fixed-point scheme (Sec. 3.2, Algorithm 1) with
the pattern FFT over the Smith-normal-form divisors (Sec. 2.2), as
hand-written CUDA for sm_103a behind the C ABI of ``include/lattice_ms.h``.

    from paper_1605_05712_gb300 import lattice_plan, basic_scheme_solve, lattice_fft
"""
from .api import (LAT_BOUNDARY_AVERAGE, LAT_BOUNDARY_ZERO, LAT_DIVERGED, LAT_FP64, LAT_MIXED,
                  LAT_NOT_CONVERGED, LAT_OK, LatticeError, LatticePlan, basic_scheme_solve,
                  basic_scheme_solve_async, basic_scheme_solve_batch, basic_scheme_solve_field, voigt_field, basic_scheme_solve_multi, lattice_fft, lattice_pass_times,
                  lattice_plan, lib, multi_workspace_bytes, gather, gather_map)

__all__ = ["lattice_plan", "lattice_pass_times", "basic_scheme_solve_async", "basic_scheme_solve_batch",
           "basic_scheme_solve_field", "voigt_field", "basic_scheme_solve_multi",
           "multi_workspace_bytes", "gather", "gather_map", "LatticePlan", "lattice_fft", "basic_scheme_solve", "lib", "LatticeError",
           "LAT_OK", "LAT_NOT_CONVERGED", "LAT_DIVERGED", "LAT_FP64", "LAT_MIXED",
           "LAT_BOUNDARY_AVERAGE", "LAT_BOUNDARY_ZERO"]
