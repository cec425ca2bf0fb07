"""B300-native differentiable 2D Gaussian ray tracing of secondary rays (2DGRT).

Hot path of the transport-aware optimisation of IRGS++ (arXiv 2607.22780): MIS sampling of
secondary directions, LBVH traversal, ray-surfel intersection, k-buffer ordering,
front-to-back compositing and the rendering-equation estimate, plus its adjoint -- all
in the CUDA library ``libgrt.so`` (C ABI in ``include/grt.h``).  This package is the
thin Python binding; ``workloads`` draws seeded synthetic inputs.
"""
from .api import (DEFAULT_PARAMS, Environment, GBuffer, Scene, ShadeRequest, SurfelGrads, gbuffer_primary,
                  sampling, shade_backward, shade_batch, shade_count, shade_pixels, trace_backward, trace_count,
                  trace_forward, trace_params, version)

__all__ = ["DEFAULT_PARAMS", "Environment", "GBuffer", "Scene", "ShadeRequest", "SurfelGrads", "gbuffer_primary",
           "sampling", "shade_backward", "shade_batch", "shade_count", "shade_pixels", "trace_backward",
           "trace_count", "trace_forward", "trace_params", "version"]
