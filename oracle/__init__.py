"""FP64 CPU oracle for the S-fraction multiscale finite-volume method.

TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library imports, links or runs
this package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code with the CUDA path: the two
sides meet only in ``sfm_inputs`` (seeded velocity models, cuts, positions and
the Ricker wavelet), which holds none of the method's arithmetic.

The oracle restates the paper (Druskin, Mamonov, Zaslavsky, "S-fraction
multiscale finite-volume method for spectrally accurate wave propagation")
step by step, in plain NumPy/SciPy float64:

* ``fine``     - fine-grid operator of Eq. (1) (vertex-centred finite volume,
                 per-cell assembly), global/slit assembly, fine FDTD.
* ``faces``    - face basis F^alpha (section "Stage 1", m functions per face).
* ``rom``      - Algorithm 1 step (1.1): block rational Krylov subspace with a
                 single repeated shift (Eqs. 6-7), Galerkin ROM (Eq. 5).
* ``sfrac``    - Algorithm 1 steps (1.2)-(1.3): block Lanczos (Eq. 8) and the
                 S-fraction transform (Eq. 13); transfer functions Eqs. 4, 9,
                 15.
* ``project``  - Algorithm 1 step (1.4): source and receiver rows via Eq. 16.
* ``coupled``  - Algorithm 1 stage 2: face coupling Eqs. 17-18, interior
                 update Eq. 19, leapfrog; assembled mass/stiffness, energy and
                 CFL limit.
* ``pipeline`` - the whole offline stage for a problem from ``sfm_inputs``.
* ``fidelity`` - trace errors of the coupled ROM against the global and the
                 slit fine grids (section "Numerical experiments").
* ``surrogate``- CPU reference of a learned map from a velocity block to its
                 S-fraction coefficients (an extension of the offline stage).

Every reading of a passage the paper leaves open is stated where it is used.
"""
