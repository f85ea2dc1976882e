"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module only builds scene *descriptions* (plain numpy arrays) and the
per-configuration run parameters.  It contains none of the rendering or
sample-allocation arithmetic; both implementations read the same arrays.
"""
from .scenes import (  # noqa: F401
    Scene,
    WorkloadConfig,
    box_scene,
    furnace_scene,
    guided_room_scene,
    area_light_plane_scene,
    light_step_scene,
    occluded_light_plane_scene,
    config_box,
    config_guided,
    config_heightfield,
    config_large,
    config_bdpt_heightfield,
    config_bdpt_large,
    heightfield_scene,
    random_count_fields,
    random_guide_cdf,
    random_pixel_estimate,
    serving_requests,
    TECH_BSDF,
    TECH_NEE,
    TECH_GUIDED,
    TECH_LIGHT,
    MAT_LAMBERT,
    MAT_GGX,
)
