"""GB300 coherent-fitness engine for the PSO-based fully-coherent all-sky CBC search
(Normandin & Mohanty, arXiv:2002.02150): a C-ABI CUDA library (libfcas.so) and its binding."""

from .fcas import (FcasError, Context, fcas_create, fcas_fitness, fcas_fitness_noalloc, fcas_destroy, fcas_last_error, fcas_get_info,
                   fcas_profile_enable, fcas_profile_read, load_library, LIB_PATH, pso_config, fcas_pso_init,
                   fcas_pso_update, fcas_search, fcas_gradient, coherent_fitness, fcas_polish, fcas_autotune,
                   fcas_set_shape, fcas_group_create, Group, segment_seed, FCAS_SETUP_LAZY_SCRATCH, pso_theta,
                   fcas_tau_tiles, time_slide_background, fcas_condition_number, pso_save, pso_load, pso_run)

__all__ = ["FcasError", "Context", "fcas_create", "fcas_fitness", "fcas_fitness_noalloc", "fcas_destroy", "fcas_last_error",
           "fcas_get_info", "fcas_profile_enable", "fcas_profile_read", "load_library", "LIB_PATH", "pso_config",
           "fcas_pso_init", "fcas_pso_update", "fcas_search", "fcas_gradient", "coherent_fitness", "fcas_polish",
           "fcas_autotune", "fcas_set_shape", "fcas_group_create", "Group", "segment_seed", "FCAS_SETUP_LAZY_SCRATCH",
           "pso_theta", "fcas_tau_tiles", "time_slide_background", "fcas_condition_number", "pso_save", "pso_load",
           "pso_run"]
