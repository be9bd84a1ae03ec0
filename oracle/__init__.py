"""CPU oracle for PSWF-LR (test infrastructure only).

This package is the slow, plain FP64 reference that the CUDA path is checked
against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
/ ``--impl reference`` legs of ``bench.py`` may import it; the product path
(``paper_2606_06617_b300``) never does, and this package never imports the
product.  It shares no code, tables or constants with the CUDA library.

Levels (each GPU output is compared with the level it targets):

* O1, :mod:`oracle.grid` -- the discrete PSWF-LR algorithm of Methods,
  "Accelerating atom-grid spreading with PSWFs", steps (i)-(iv) plus the
  inverse transform and gather, written in plain PyTorch FP64 ops (so that
  autograd gives the exact gradient of the discrete operator).
* O2, :mod:`oracle.direct` -- the continuous reciprocal sum of Eq. (Fourier)
  by direct structure factors, no grid.
* O3, :mod:`oracle.ewald` -- classical Ewald sums with the incomplete-gamma
  screening of Eq. (screening), plus explicit image sums for absolutely
  convergent exponents; :mod:`oracle.realspace` gives the PSWF real-space
  complement and self terms needed to compare totals with O3.

Building blocks: :mod:`oracle.pswf` (psi_0^c by a Nystrom discretisation of
Eq. (psidefinit)) and :mod:`oracle.mollifiers` (G_p, Phi-hat_p, W-hat,
self-energy and zero-frequency terms).
"""
