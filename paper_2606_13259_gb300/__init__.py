"""GB300-native volumetric delay-and-sum beamforming (paper Sec. 2, Eq. 1-2).

    from paper_2606_13259_gb300 import Plan, das
    plan = Plan.from_scene(scene, storage="f32", max_batch=20)
    image = plan.forward(y)            # y: (B, Q, M, K) on the GPU
    image = das(y, c, plan)            # differentiable in y and c

The compute path is the CUDA library libdas_gb300.so (include/das.h); this
package only marshals arguments.  Build it with `build.build()`.
"""
from ._lib import (DAS_STORE_BF16, DAS_STORE_F16, DAS_STORE_F32, DAS_TX_DIVERGING, DAS_TX_NONE, DAS_TX_PLANE,
                   DASError)
from .plan import Batch, DASFunction, Plan, das, host_empty

__all__ = ["Plan", "Batch", "DASFunction", "das", "host_empty", "DASError", "DAS_TX_DIVERGING", "DAS_TX_PLANE", "DAS_TX_NONE",
           "DAS_STORE_F32", "DAS_STORE_F16", "DAS_STORE_BF16"]
