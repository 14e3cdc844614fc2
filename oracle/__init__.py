"""FP64 CPU oracle for the particle-mesh force step of PySCo (arXiv 2410.20501).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link or
execute anything in this package; only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, table or constant with the CUDA library: every function here is written
directly from the paper (section / equation cited in each docstring) in plain
numpy float64, slow and literal, so that a reader can check it against the paper
by eye.

Modules
-------
cosmology  background expansion E(a), supercomoving time, growth factors (§2.2,
           §3.1, Appendix A)
mesh       TSC mass assignment and its inverse, finite-difference gradients, the
           7-point Laplacian, cell keys (§3.2, §3.4, Table 1)
poisson    exact discrete inverse of the 7-point Laplacian (FFT_7pt, §3.7) and
           the paper's linear multigrid (§3.5, §3.6.1)
fr         Hu-Sawicki f(R) scalaron: background, depressed cubic and its
           closed-form root, non-linear (FAS) multigrid (§2.x, §3.6.2, §3.10)
step       force evaluation and the kick-drift-kick leapfrog (§3.4 Integrator)
power      the simple power-spectrum estimator (§4)

Every function that has no independent pin in ``tests/test_oracle_*.py`` says
"parity unpinned" in its docstring.
"""
