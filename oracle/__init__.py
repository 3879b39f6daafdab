"""FP64 CPU oracle for the PolyDG monodomain step with two-level additive Schwarz PCG.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, deliberately
unoptimised restatement of the method, written to be checked against the
paper by eye: interior-penalty PolyDG assembly on polygonal meshes (Sec. 3,
Eq. eta and Eq. coer), the Crank-Nicolson step with explicit extrapolation of
the ion term (Eq. fully-discrete-1), the two-level additive Schwarz
preconditioner (Sec. 4, Eq. prec) and preconditioned conjugate gradients.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the GPU library never does, and it never imports
the GPU library.  Everything here is float64 numpy/scipy on the host.

Parity status per part is listed in each module's docstring.  The ionic model
(``oracle.ionic``) is "parity unpinned" as physics: its constants are restated
from the cited Barreto-Cressman publications, which are not available to check.
"""
