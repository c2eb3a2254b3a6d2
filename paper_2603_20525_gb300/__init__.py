"""GB300 (sm_103a) rollout planner for the sampling MPC hot path of
arxiv 2603.20525: batched single-rigid-body rollouts on a heightmap with the
energy-stability-margin constraint, cost and a fused empirical argmin, behind
the C-ABI of include/atp.h.  ``atp`` is the ctypes binding."""
from . import atp  # noqa: F401
from .atp import Context, AtpError, decode_out  # noqa: F401
