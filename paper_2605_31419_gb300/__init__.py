"""GB300-native differentiable triangle-splatting rasterizer (Triangle Splatting SLAM, Sec. 3.1-3.3).

The compute path is libts (hand-written CUDA for sm_103a, C ABI in include/ts_api.h); this package
is its Python binding.  Importing it loads the in-tree libts.so and raises ImportError when the
library has not been built: there is no CPU fallback.
"""
from . import binding  # noqa: F401
from .binding import (  # noqa: F401
    TsError, ts_default_params, ts_plan_init, ts_workspace_size, ts_workspace_init, ts_project, ts_bin,
    ts_render_fwd, ts_render_bwd, ts_render_fwd_n, ts_render_bwd_n, ts_render_step_l1, ts_pose_grad,
    ts_l1_loss, ts_l1_loss_noalloc, ts_pho_loss, ts_normal_loss, ts_equilateral, ts_pose_apply, ts_pose_adam,
    ts_sync_status, ts_face_stats, ts_covisibility, TS_FLAG_PERSISTENT, TS_FLAG_NORMALS, TS_FLAG_STATS,
    TS_FLAG_MIN_OPACITY, TS_FLAG_FACE_SIGMA, TS_FLAG_FORWARD_ONLY,
    ts_plan_layout,
    ts_debug_copy, ts_debug_timeout_probe, ts_set_stage_events, ts_status_string,
)

binding.lib()  # fail loudly here if libts.so is missing

from .rasterizer import Map, Rasterizer, poses_tensor  # noqa: E402,F401
from .autograd import RenderFunction, render  # noqa: E402,F401
from .tracking import Tracker, pose_error  # noqa: E402,F401
from .batch import MultiViewStep, autotune, params_of  # noqa: E402,F401
from .serve import Request, Server, latency_stats, serve_plain  # noqa: E402,F401
