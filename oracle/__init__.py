"""FP64 CPU oracle of the Faceted HyperSARA PDFB hot path (arXiv 2003.07358).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The GPU library never calls it, and it shares no code, tables,
constants or helpers with the GPU library (``paper_2003_07358_gb300``).  Its
only shared dependency is the input generator ``fhs_synth``, which holds none
of the method's arithmetic.

Plain, slow, obviously correct numpy in float64: every function follows one
passage of the paper (cited in its docstring) with no blocking, fusion or
reordering beyond what that passage states.  Library primitives used as
steps: ``numpy.fft`` (the DFT F of Eq. 1), ``numpy.i0`` (the modified Bessel
function in the Kaiser-Bessel kernel), ``numpy.roots`` (Daubechies spectral
factorisation), ``scipy.special.gammaln`` (chi-distribution moments).

Modules
-------
nufft     Measurement operator Phi = G F Z (Eq. 1), direct DFT, Kaiser-Bessel kernel.
wavelets  Daubechies db1..db8 filters, zero-padded multilevel 2-D DWT, SARA Psi^dagger / Psi.
facets    Spatial tiling, faceted SARA operators Psi_q^dagger S_q, nuclear facets and D_q windows.
prox      Table 2 proximal operators, one-sided Jacobi SVD, dual updates of Algorithm 2.
pdfb      Parameters (Section 2.3-2.4 heuristics, Eq. 3 radii), Algorithm 2 iteration,
          Algorithm 1 weights, SNR metrics (Section 4.2).

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` except the synthetic input recipe itself (a
convention, not a result of the method).
"""
