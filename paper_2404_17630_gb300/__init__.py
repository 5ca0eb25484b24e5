"""GB300-native M1 radiative-transfer subcycle (arXiv:2404.17630).

The compute path is the CUDA library ``libm1rt.so`` (C ABI in include/rt.h);
``rt`` is its Python binding.
"""
from .rt import (RT, RTError, make_config, rt_create, rt_destroy, rt_get_fields, rt_init_mesh, rt_max_dt,  # noqa: F401
                 rt_mesh_info, rt_set_gas, rt_set_radiation, rt_set_sources, rt_stage_chemistry,
                 rt_stage_fluxes, rt_stage_gradients, rt_stage_transport, rt_step, rt_sync, rt_adjoint, RT_FP64,
                 RT_MIXED)
from .autograd import RTStepFunction, rt_step_autograd  # noqa: F401
