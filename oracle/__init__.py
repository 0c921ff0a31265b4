"""FP64 CPU oracle of the per-frame non-rigid deformation solve (Zhou & Jagadeesan,
"Real-time Surface Deformation Recovery from Stereo Videos").

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check of the entry module and the CPU
baseline leg of the benchmark may import this package. The product path (the CUDA library and
its Python binding) never imports, links or runs anything here, and this package imports nothing
from the product path.

It is a plain, slow, step-by-step restatement of the method in float64 numpy:

* quat.py    quaternion algebra (product matrices, rotation, exponential map)
* frame.py   back-projection of a depth map and finite-difference normals (Section 2,
             point-to-plane ICP needs the normal directions)
* ransac.py  1-point RANSAC with reweighting, Eq. 2-4 and Section 2.1 (30 references,
             10 reweighting iterations)
* dqb.py     dual-quaternion warp of template points by their neighbouring control points
             (Section 2: a point follows a blend of nearby control points) and its Jacobian
* terms.py   the three cost terms of Eq. 1: ICP (Tukey, point-to-plane, projective
             association), ORB matches (Section 2.1 weights) and dense ARAP (Eq. 5-6)
* solver.py  template set-up, normal-equation assembly, damped Gauss-Newton with a Cholesky
             solve (Section 2, Levenberg-Marquardt + Cholesky), state update

Every reading of a point the paper leaves open is a named parameter in solver.Params and is the
same reading the CUDA path implements. Parity pins live in tests/test_oracle_*.py.
"""
from .solver import Params, Template, FrameResult, setup_template, solve_frame  # noqa: F401
