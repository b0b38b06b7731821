"""GB300 (sm_103a) implementation of the LB-SMRT collide-and-stream step (Yan & Shan,
arXiv 2401.11086): libsmrt (C ABI, include/smrt.h) and its thin Python binding."""
from .api import (LB_F32, LB_F32_CONS64, LB_F64, LB_MOM_D, LB_MOM_Q, LB_MOM_RHO,  # noqa: F401
                  LB_MOM_SIGMA, LB_MOM_THETA, LB_MOM_U, Context, LatticeDesc, SmrtError,
                  lb_destroy, lb_error_string, lb_fill_equilibrium, lb_init_lattice,
                  lb_lattice_named, lb_moments, lb_moments_adjoint, lb_num_moment_rows,
                  lb_poll_status, lb_step_adjoint,
                  lb_rankine_hugoniot, lb_set_frame_shift, lb_shock_frame, lb_shock_shift,
                  lb_autotune, lb_get_schedule, lb_set_schedule, lb_step_graph,
                  lb_test_barrier_timeout, lb_set_relaxation, lb_step,
                  LB_MODEL_ES_BGK, LB_MODEL_SMRT, lb_set_collision_model, lb_hermite_convergence)
