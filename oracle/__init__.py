"""FP64 CPU oracle for lattice spline evaluation (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path in
``paper_2102_08518_b300``; neither imports the other.

It evaluates the convolution sum of Eq. 1 naively (every stored site whose
support contains x contributes c_n phi(x - n)), with phi the centred,
lattice-normalised box spline; see ``orc.c`` for the definitions and the
recurrence.  ``specs`` holds the oracle's own copy of the spline and lattice
definitions of the benchmarked splines (Sec. 5.1) and of the ZP element of
Fig. 1.
"""
from .lib import (OrcSpec, box, phi, phi_grad, phi_hess, eval_sum, eval_sum_grad, eval_sum_hess, adjoint,
                  design_triplets, morton3, build_library, library_path)
from . import specs

__all__ = ["OrcSpec", "box", "phi", "phi_grad", "phi_hess", "eval_sum", "eval_sum_grad", "eval_sum_hess", "adjoint",
           "design_triplets", "morton3", "build_library", "library_path", "specs"]
