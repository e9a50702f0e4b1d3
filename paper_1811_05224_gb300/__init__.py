"""GB300 (sm_103a) space-time BEM for the 2D heat equation.

The hot path of the preconditioned space-time Galerkin BEM (arXiv:1811.05224):
assembly of V_h, K_h, D_h and block-Toeplitz products inside preconditioned
GMRES, in hand-written CUDA behind the C ABI of include/stbem.h.
"""
from .api import (Context, Domain, GradedMesh, Mesh, Ragged, apply, pipe_peaks, nu_apply, nu_assemble, nu_lumped_mass,
                  nu_rhs, nu_solve, evaluate, m0_apply, m0_assemble, planewave_data, rhs_initial, apply_tc, assemble, assemble_ops, assemble_lags, lumped_mass, mixed_mass_inverse, rhs,  # noqa: F401
                  apply_tc3, bf16_split3, ExactOperand, exact_slices, apply_exact, tc_tune, tune_cache,
                  tune_cache_get, tune_cache_put, tune_cache_clear, grad, rhs_batched, round_f32, solve, solve_adjoint, solve_batched,
                  solve_mixed, to_bf16, FFTOperator, fft_operator, apply_fft, solve_fft)
from .autograd import neumann_solve  # noqa: F401
from . import shard  # noqa: F401

__all__ = ["Context", "Mesh", "pipe_peaks", "assemble", "assemble_ops", "assemble_lags", "apply", "rhs", "lumped_mass", "solve", "solve_mixed", "round_f32", "to_bf16", "apply_tc", "bf16_split3", "apply_tc3", "ExactOperand", "exact_slices", "apply_exact", "tc_tune", "tune_cache", "tune_cache_get", "tune_cache_put", "tune_cache_clear", "rhs_batched", "solve_batched", "solve_adjoint", "grad",
           "neumann_solve", "Ragged", "mixed_mass_inverse", "Domain", "m0_assemble", "m0_apply", "planewave_data",
           "rhs_initial", "evaluate", "FFTOperator", "fft_operator", "apply_fft", "solve_fft"]
