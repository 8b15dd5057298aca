"""CPU oracle for alternating cross interpolation (ACI).

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, FP64/complex128 restatement
of the paper's method (Algorithms 1-5, Appendix B) and of the O(chi^4) Kronecker-delta
Hadamard product it is compared with (Sec. 2.9, Appendix A). Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import it. The
CUDA library never calls it, and it shares no code with the CUDA library; both
read their inputs from the ``synthetic`` package.

Parity status per function (what pins each one independently of itself) is listed
in each module's header.
"""

from .algorithms import (
    aci, ldu, ldu_rook, factorise, crossinterpolate, localupdate, leftframe, rightframe, apply_op,
    magnitude, pivot_key, init_guess, assemble_output, pi_tensor,
)
from .hadamard import hadamard_kron, tt_round_svd
from .rng import splitmix64_uniform, random_tt_counter

__all__ = [
    "aci", "ldu", "ldu_rook", "factorise", "crossinterpolate", "localupdate", "leftframe", "rightframe",
    "apply_op", "magnitude", "pivot_key", "init_guess", "assemble_output", "pi_tensor",
    "hadamard_kron", "tt_round_svd", "splitmix64_uniform", "random_tt_counter",
]
