"""Plain FP64 CPU oracle for environment-recycled iPEPS imaginary-time evolution.

This package is TEST INFRASTRUCTURE, not product code. Only the test suite,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import or run it. It shares no code with the CUDA
path (``paper_1411_0391_gb300``) and imports nothing from it.

It follows Phien, McCulloch and Vidal, "Faster convergence of imaginary time
evolution tensor network algorithms by recycling the environment"
(arXiv:1411.0391), step by step, in numpy float64 with LAPACK SVD/EVD as
library primitives:

    model        Sec. V.A / VI.A   TFIM, Trotter gates, iMPO and iPEPO
    ctmrg        Sec. VI.B item 1  double layer, CTM environment (Fig. 21a)
    fullupdate   Sec. VI.B item 2  pre-truncation, bond environment (Fig. 21b),
                                   cost function Eq. (var), ALS Eq. (var1)
    canonical    Sec. IV           iPEPS canonical form Eqs. (17)-(20) and
                                   gauge fixing by local fidelity Eq. (25)
    recycle      Sec. VI.C         renormalised gate and recycled steps (fixed
                                   windows and the threshold trigger), the
                                   simple-update step of the Sec. VI.D comparison
    observables  Sec. VI.D         m_z, energy per site/link
    gradient     (beyond the paper) energy gradient of the 1-site iPEPS by
                                   central differences, the reference for a
                                   CTMRG fixed-point adjoint
    imps         Sec. III, V       1D canonical form, gauge fix, recycling
    classical    (pin only)        2D classical Ising network for CTMRG pins
    ed           (pin only)        exact diagonalisation on small tori

Where the paper leaves a step unspecified (the CTMRG moves are only cited,
the figures that define E1..E6 are missing), the function that takes the step
states the reading it follows in its docstring.
"""
