"""GB300-native (sm_103a) MeshSplats hot path: fan conversion, tile-binned exact-order
rendering, its adjoint and the fine-tune update, behind the C ABI of
include/meshsplats.h (libmeshsplats.so) with a thin torch front end."""
from . import _lib  # noqa: F401
from .api import (BatchRenderer, FanAdam, FanMLP, MeshRenderer, RayTracer, Renderer, SplatRenderer, RenderFn,  # noqa: F401
                  camera_struct, fine_tune_loss, gather_rows, l1_loss, mesh_build, mesh_build_3d,
                  mesh_prior_backward, mesh_prior_build, prune_faces, prune_fans, render, render_params,
                  spatial_order, spatially_ordered, three_fan_copies, three_fan_sum_copies, tris_to_fans)
