"""FP64 CPU oracle for randomized tensor-ring decomposition (rTRD).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
link this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, table or constant generator with the CUDA library; the two meet only
at the seeded input generators in ``paper_1901_01652_gb300.workloads``.

Everything here is plain NumPy/SciPy in float64, written from the paper
(Yuan, Li, Cao, Zhao, "Randomized Tensor Ring Decomposition and Its
Application to Large-scale Data Reconstruction", arXiv:1901.01652):

* ``philox``  - Philox4x64-10 counter-based generator (Salmon et al., SC'11),
                the source of the Gaussian test matrices (Algorithm 1, step 4).
* ``omega``   - the Gaussian quantile table and the test matrices Omega_n.
* ``mxfp8``   - block-scaled float8 (e4m3, one power-of-two scale per 32
                values) copy of X read by the FP8 form of the sketch.
* ``tensor``  - unfoldings, mode-n products, TR format (Eq. 1, Eq. 2).
* ``rtrd``    - Algorithm 1 (sketch, QR, projection, back-projection), the
                TR-ALS and TR-SVD decomposers it calls, RSE (Section 4).
* ``proposer`` - the learned proposer of K_n and R_n (this build's own
                definition; the paper fixes them by hand in Section 4):
                spectrum features, MLP forward/backward, Adam, decoding.

Pins: every function is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` against closed forms, brute force on tiny inputs,
invariants and independent library routines.  Free-rank TR-SVD is pinned only
through its published error bound (parity of its rank choice is partly
unpinned, see the TR-SVD docstring).
"""
