"""FP64 CPU oracle for the TTNO / TTNS hot path of the tree-tensor-network vibrational solver.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously-correct restatement of the
paper's definitions (Sec. II) in NumPy float64. It is imported only by ``tests/``, by
``__graft_entry__.smoke()`` and by the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py``. The product path (the CUDA library and its Python binding) never imports, links or
executes anything in here, and nothing in here imports the product path.

Modules
-------
network   TTNS/TTNO contraction to dense (Eqs. ttns, ttno), the state-diagram TTNO
          construction (Sec. II.A.3), environments, Gram entries, H_eff and the exact
          TTNO x TTNS product (Sec. II.C).
solvers   MINRES (Paige & Saunders 1975), QR gauge moves, ALS (Sec. II.C.3), variational
          fitting (Sec. II.C.2), block LOBPCG (Alg. 2), block inverse iteration (Alg. 3).
closed    closed-form spectra used as pins (uncoupled limit, normal modes of the bilinear model).
"""
