"""GB300 (sm_103a) implementation of the ALI hot path of non-LTE line radiative transfer
(De Ceuster et al. 2019, "Magritte I"): ray tracing, Feautrier formal solve with the
diagonal or band-diagonal approximate Lambda operator, statistical equilibrium and Ng
acceleration, as
hand-written CUDA kernels behind the C ABI in include/magritte_gb300.h."""
from .binding import (  # noqa: F401
    Context, Batch, MLP, MagritteError, load, default_options, declared_symbols, lib_path, measure_pipe_rates,
    MG_FP64, MG_MIXED, MG_GEOM_3D, MG_GEOM_SPHERICAL_1D, MG_INIT_LTE, MG_INIT_GIVEN, MG_INIT_MLP,
    MG_OK, MG_ERR_NOT_CONVERGED, MG_WARN_DEAD_END_RAYS, MG_WARN_NEG_POP_FALLBACK, MG_WARN_NEG_OPACITY,
)
