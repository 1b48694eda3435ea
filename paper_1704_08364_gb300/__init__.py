"""GB300-native BST filtered backprojection of parallel-beam sinograms.

The hot path (Sec. 2 of "Low-complexity Distributed Tomographic
Backprojection for large datasets", Theorem 2.1 / Eq. 3) runs in hand-written
sm_103a CUDA kernels behind the C ABI of include/bst.h (libbst.so); this
package is the thin Python binding over it.  There is no CPU fallback: the
calls fail loudly when libbst.so is missing.
"""
from .api import (BACKPROJECT, FILTER, BstError, BstFbpFn, Plan, RaggedBatch, backproject,  # noqa: F401
                  brute_backproject, clear_plans, fbp, fbp_autograd, fbp_ragged, plan_for, radon_adjoint)
