"""GB300-native PolyDG monodomain solver: two-level additive Schwarz PCG (arXiv 2512.19536).

The compute lives in ``libpolydg.so`` (hand-written sm_103a CUDA behind the C
ABI of ``include/polydg.h``); this package is its ctypes binding.  Importing
the package does not load the library; the first call does, and fails loudly
if it has not been built.
"""
from ._native import (PolyDG, ASM, Simulation, PolyDGError, load, polydg_setup, polydg_setup3d,
                      setup_mesh, asm_setup,
                      asm_apply, asm_autotune, pcg_solve_trace, lanczos_extremes, pcg_solve, sim_create, monodomain_step, sim_get_state,
                      sim_set_potential, sim_set_history, spd_inverse_static, Batch, batch_create, batch_step,
                      GuessModel, guess_n_params, guess_create, guess_propose, guess_train_step,
                      sim_set_guess, SharedLocal, shared_local_setup, shared_local_apply,
                      sim_set_shared_local, sim_set_ionic_form, sim_set_state, sim_get_ionic_coeffs,
                      sim_get_ionic_aux, sim_set_ionic_aux, set_wait_limit,
                      EXPORTS, LIB_PATH, POLYDG_OK, POLYDG_EINVAL, POLYDG_ENOMEM, POLYDG_ECUDA, POLYDG_ENOTSPD, POLYDG_ENOTCONV,
                      POLYDG_EBREAKDOWN, POLYDG_ENONFINITE)

__all__ = ["PolyDG", "ASM", "Simulation", "PolyDGError", "load", "polydg_setup", "polydg_setup3d",
           "setup_mesh", "asm_setup",
           "asm_apply", "asm_autotune", "pcg_solve_trace", "lanczos_extremes", "pcg_solve", "sim_create", "monodomain_step", "sim_get_state",
           "sim_set_potential", "sim_set_history", "spd_inverse_static", "Batch", "batch_create", "batch_step",
           "GuessModel", "guess_n_params", "guess_create", "guess_propose", "guess_train_step",
           "sim_set_guess", "SharedLocal", "shared_local_setup", "shared_local_apply",
           "sim_set_shared_local", "sim_set_ionic_form", "sim_set_state", "sim_get_ionic_coeffs",
           "sim_get_ionic_aux", "sim_set_ionic_aux", "set_wait_limit", "EXPORTS", "LIB_PATH"]
