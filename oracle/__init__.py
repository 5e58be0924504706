"""Oracle: plain, slow, FP64 CPU implementation of the SPDHG+ PET hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` import it.  The CUDA library (``paper_1808_07150_gb300``) never
imports, links or executes anything here, and this package imports nothing from it; the two
share only the seeded input generators of ``synth``, which hold none of the method.

What it computes (Ehrhardt, Markiewicz, Schoenlieb, "Faster PET reconstruction with non-smooth
priors by randomization and preconditioning"):

* ``siddon.c`` / ``_native``: the projector's line integrals (Sec. 1.2 "P performs the
  projection"), by Siddon's parametric method and, independently, by per-voxel slab clipping;
* ``algorithms``: the data term and its conjugate (Sec. 2.1, Eqs. EQU:LOCALDISTANCE, EQU:PET:CVX),
  the KL dual prox (Example in Sec. 2.2), TV / dTV / aTV / TGV operators and their dual
  projections (Sec. 2.1, Sec. 4.3), step sizes (Theorem "Step Size Parameters"), balanced and
  uniform sampling (Sec. 4.2), SPDHG (Algorithm 2), PDHG (Algorithm 1), MLEM (Eq. EQU:MLEM),
  the objective Psi and the relative objective / PSNR metrics (Sec. 4);
* ``unet``: the learned warm start (no counterpart in the paper; it only replaces x0 of
  Algorithm 2): 3x3x3 convolution, 2x2x2 transposed convolution, max-pooling, ReLU, the 3-D
  U-Net forward pass and its exact backward pass, the MSE loss.

Pins (tests/test_oracle_*.py, run with ``-m "not gpu"``): dense slab-clipping matrix vs the
Siddon traversal; exact line integrals through voxel boxes; chord through the image box;
analytic disk chords; the KL conjugate against a numeric supremum; the KL prox against brute-force
1-D minimisation and its b = 0 special case; Fenchel-Young equality; the gradient on ramps and
its adjointness; ||grad|| closed form against power iteration; dTV special cases; the
symmetrised gradient on linear fields; the step-size condition (Eq. EQU:STEPSIZE) on dense
blocks; PDHG == SPDHG for one block with p = 1; ML optimality (KKT) of long SPDHG runs and
agreement with MLEM; sampler frequencies; U-Net: convolution against scipy.ndimage.correlate and
the definition, adjoint identities of every backward, finite differences of the network loss.
No function here is "parity unpinned".
"""
from ._native import build, threads  # noqa: F401
from . import algorithms  # noqa: F401
from . import unet  # noqa: F401
from .algorithms import *  # noqa: F401,F403
