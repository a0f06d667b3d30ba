"""GB300-native (sm_103a) time step of the quadrature-based finite-difference relativistic lattice Boltzmann
model for massless particles (Blaga & Ambrus, arXiv:1608.03004).

The compute path is the CUDA library ``librlb.so`` (sources in ``csrc/``, C ABI in ``include/rlb.h``);
``binding`` exposes its entry points under the same names; ``adjoint.run_moments`` wraps the library's adjoint
entry points in a torch.autograd.Function. ``workloads`` holds the seeded synthetic inputs.
Importing this package loads nothing; the library is loaded on the first call and a missing library is an
error, never a fallback.
"""
from .binding import (  # noqa: F401
    BC_OPEN,
    BC_PERIODIC,
    FIELDS,
    NFIELDS,
    STORAGE,
    STORAGE_BF16,
    STORAGE_F32,
    STORAGE_F64,
    Handle,
    Launch,
    ORDER_COST,
    ORDER_INTERLEAVE,
    SCHED_COUNTER,
    SCHED_STRIDE,
    SCHED_TILE,
    RlbError,
    Tube,
    library_path,
    load,
    rlb_destroy,
    rlb_autotune,
    rlb_backward,
    rlb_error_string,
    rlb_get_launch,
    rlb_get_state,
    rlb_halo_pack,
    rlb_halo_size,
    rlb_halo_unpack,
    rlb_init,
    rlb_init_riemann,
    rlb_init_vjp,
    rlb_moments,
    rlb_fields_vjp,
    rlb_moments_vjp,
    rlb_quadrature,
    rlb_record,
    rlb_set_launch,
    rlb_set_state,
    rlb_stage,
    rlb_state_size,
    rlb_step,
    rlb_step_static,
    rlb_stiffness_limit,
    rlb_suggest_dt,
    rlb_sync,
    rlb_warnings,
)
