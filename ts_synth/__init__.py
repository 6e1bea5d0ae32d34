"""Seeded synthetic inputs for the triangle-splatting rasterizer.

This package only draws random numbers and lays out arrays (vertex buffers,
face lists, pinhole cameras, world-to-camera poses, target images).  It holds
none of the rasterizer's arithmetic: no projection, no window function, no
compositing.  Both the CPU oracle tests and the CUDA path consume these arrays,
so it imports neither of them.
"""
from .scenes import (  # noqa: F401
    Scene,
    random_triangles_scene,
    room_map,
    room_scene,
    trajectory_poses,
    look_at,
    noise_targets,
    tiny_scene,
    mixed_keyframe_cameras,
    perturb_pose,
    request_stream,
)
