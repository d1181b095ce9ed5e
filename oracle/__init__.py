"""FP64 CPU oracle for smooth contact-manifold generation (arXiv 2602.20304).

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
CUDA library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the product path (the
C-ABI library and its Python binding) never does, and shares no code with it.

Everything here is plain PyTorch on the CPU in float64, written step by step
from the paper's text: the smooth operators of Sec. III, the SDF primitives
of Sec. IV-B, vertex-SDF contacts of Sec. IV-C, the edge-edge routine of
Sec. IV-D (regularised box-QP, smoothed active set, witness points, sign,
penetration, nearest-neighbour, clashing and activity indicators) and the
SoftSort top-K reduction of Sec. III to K contact points.  Gradients come from
PyTorch autograd through this same float64 code.

Parity status per function is listed in each module's header; the final
K-point reduction is a reading of the paper (it defines the SoftSort operator
but not this use of it) and is "parity unpinned" by the paper's own numbers.
"""

from .smooth import (sigmoid, relu_s, clip_s, greater_s, smaller_s, within_s,  # noqa: F401
                     argmin_s, lse, sign_s, softplus)
from .sdf import local_vertices, sdf_local, sdf_world, quat_to_rot  # noqa: F401
from .edge_edge import solve_box_qp, solve_box_qp_hard, ee_witness, ee_candidates  # noqa: F401
from .vertex_face import vf_witness  # noqa: F401
from .manifold import (Params, pair_candidates, soft_topk_reduce, pair_manifold,  # noqa: F401
                       batch_manifold, batch_manifold_grad)
