"""CPU oracle of dSMC (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline / reference
legs import this package.  The CUDA library and its binding never import it, and it never
imports them.

Contents:
  * ``core``    -- ctypes binding of the FP64 C oracle (Algorithms 1, 2, 5, 6, 8 of the paper)
                   and of the device-precision pair samplers used for the index contract.
  * ``kalman``  -- Kalman filter, Rauch-Tung-Striebel smoother and exact log-likelihood of a
                   linear-Gaussian model (the closed form that pins dSMC on such models).
  * ``grid``    -- forward-backward smoothing of a one-dimensional model on a fine grid
                   (the numerical reference for the stochastic-volatility model).
"""
