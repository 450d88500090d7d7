"""GB300-native second-moment-method (SMM) transport: C-ABI library
(libsmm.so, hand-written CUDA for sm_103a) and its thin Python binding."""
from .smm import (SMM_INFLOW_NODAL, SMM_INFLOW_VACUUM, SMM_SOURCE_ANGULAR, SMM_SOURCE_ISOTROPIC, SMM_SWEEP_FP32_REFINED,
                  SMM_SWEEP_FP64, Handle, SMMError, load_library, smm_create, smm_default_options, smm_destroy, smm_get_psi,
                  smm_get_state, smm_iterate, smm_moment_solve, smm_moments, smm_quadrature, smm_set_moments,
                  smm_set_spin_timeout, smm_set_state, smm_state_size, smm_sweep)

__all__ = ["SMM_INFLOW_NODAL", "SMM_INFLOW_VACUUM", "SMM_SOURCE_ANGULAR", "SMM_SOURCE_ISOTROPIC",
           "SMM_SWEEP_FP32_REFINED", "SMM_SWEEP_FP64", "Handle", "SMMError", "load_library", "smm_create",
           "smm_default_options", "smm_destroy", "smm_get_psi", "smm_get_state", "smm_iterate", "smm_moment_solve",
           "smm_moments", "smm_quadrature", "smm_set_moments", "smm_set_spin_timeout", "smm_set_state", "smm_state_size", "smm_sweep"]
