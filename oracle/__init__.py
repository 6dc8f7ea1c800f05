"""FP64 CPU oracle for the dashSVD hot path.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import anything from this
package. The GPU library never imports, links or calls it, and it shares no
code with the GPU library: the only thing both sides read is the seeded matrix
from ``datagen``.

Contents
* ``philox``       -- Philox4x32-10 + Box-Muller Gaussian block (Alg. 5 step 1)
* ``dashsvd_ref``  -- eigSVD (Alg. 3) and dashSVD with PVE control (Alg. 5),
                      fixed-p (Alg. 4) and unshifted (Alg. 1) modes
* ``metrics``      -- eps_PVE, eps_sigma, eps_res (Sec. 4), Theorem 1 and
                      Lemma 6 bounds
* ``mlp_ref``      -- the learned form's shift/stop network: features,
                      forward, loss gradient, Adam

Every function is pinned by ``tests/test_oracle_*.py`` against something other
than itself (published test vectors, closed forms, brute force, invariants).
"""
from .dashsvd_ref import EPS64, PassRecord, Result, dashsvd, eigsvd, pve_ratio  # noqa: F401
from .philox import box_muller, gaussian_block, philox4x32_10  # noqa: F401
from . import metrics, mlp_ref  # noqa: F401
