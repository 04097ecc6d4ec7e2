"""CPU FP64 oracle for RA-FEAST (arXiv 2512.01257).

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports, links or runs
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it. It
shares no code with the CUDA library; both sides read their inputs from the
seeded generators in ``workloads/``.

Contents (each function cites the paper passage it restates):

* ``quadrature``  - contour nodes z_j and weights w_j (Section 2.1, Eq. 2).
* ``philox``      - Philox-4x64-10 counter generator and Box-Muller normals,
                    used to draw the Gaussian test matrix Omega (Algorithm 2).
* ``cocg``        - conjugate orthogonal CG for the complex symmetric shifted
                    systems (z_j I - A) X_j = Q (Algorithm 1, Algorithm 2).
* ``feast``       - filter application, QR, Rayleigh-Ritz, residuals and the
                    FEAST / RA-FEAST outer loops (Algorithms 1 and 2).
* ``exact``       - the exact answer the iteration converges to: closed-form
                    grid spectra, dense eigh, ARPACK shift-invert (Eq. 1).
* ``metrics``     - sin-theta subspace distance, eigenvalue errors.

Parity pins live in ``tests/test_oracle_*.py``; a function without one is
marked "parity unpinned" in its docstring.
"""
