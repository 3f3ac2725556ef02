"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This package only draws numbers: Gaussian parameters, cameras, stable/unstable
flags, pixel masks and jittered copies of a scene.  It holds none of the
rasterizer's arithmetic (no projection, compositing, depth rule or gradient), so
both the CPU oracle and the CUDA path can consume its output without sharing
any of the method's code.
"""

from .scenes import (  # noqa: F401
    Camera,
    Layout,
    Scene,
    concat_scenes,
    disc_gaussian,
    flag_blobs,
    identity_camera,
    jitter_scene,
    look_at_camera,
    multiroom_scene,
    random_masks,
    room_camera_candidates,
    room_scene,
    scatter_scene,
    stack_scene,
    sh_coefficients,
)
