"""FlexProofs (arXiv 2601.03031) all-proofs pass on one GB300 (sm_103a).

The hot path -- VC.Setup, VC.Commit and VC.OpenAll over BLS12-381 -- runs in hand-written CUDA
kernels behind the C ABI of include/flexproofs.h (libflexproofs.so, built in-tree by build.py).
This package holds the ctypes binding (_lib), the build script and the seeded input generators.
"""
from . import inputs  # noqa: F401
from ._lib import (PP, Commitment, FlexProofsError, Proofs, load, vc_commit, vc_proof_get,  # noqa: F401
                   vc_prove_all, vc_setup)
