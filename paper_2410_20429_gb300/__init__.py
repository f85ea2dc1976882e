"""GB300 (sm_103a) implementation of the MARS path tracer (Meyer et al.,
SIGGRAPH Asia 2024): a wavefront path tracer with per-technique Russian
roulette and splitting counts learned by a fixed-point scheme.

The compute lives in ``libmars.so`` (hand-written CUDA, C ABI in
``include/mars.h``); this package only marshals arguments.  Loading fails
loudly when the library has not been built."""
from ._abi import (  # noqa: F401
    MARS_BVH_LBVH,
    MARS_BVH_SAH,
    MARS_CACHE_NO_GRAPHS,
    MARS_INJECT_ALLOC,
    MARS_INJECT_LAUNCH,
    MARS_ERR_BUSY,
    MARS_ERR_CUDA,
    MARS_ERR_INVALID_ARG,
    MARS_ERR_NOT_FOUND,
    MARS_ERR_OOM,
    MARS_ERR_TIMEOUT,
    MARS_JOB_DONE,
    MARS_JOB_FAILED,
    MARS_JOB_QUEUED,
    MARS_JOB_RUNNING,
    MARS_MODE_FIXED,
    MARS_MODE_MARS,
    MARS_MODE_WARMUP,
    MARS_TECH_BSDF,
    MARS_TECH_GUIDED,
    MARS_TECH_LIGHT,
    MARS_TECH_NEE,
    MARS_WEIGHTS_AWARE,
    MARS_WEIGHTS_UNAWARE,
    MarsError,
    load,
)
from .renderer import (  # noqa: F401
    Cache,
    Scene,
    Server,
    inject_failure,
    scene_desc,
    training_schedule,
    training_step_ends,
)
