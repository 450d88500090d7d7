"""CPU oracle for the SMM transport hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 NumPy implementation of what the GPU path computes,
written from the paper (Olivier & Haut, "High-Order Finite Element Second
Moment Methods for Linear Transport"):

* ``quadrature``   -- Gauss-Legendre / Gauss-Lobatto rules, level-symmetric S_N
* ``fem``          -- mapped Q_p nodal basis on curved quads (Sec. "Finite
                      Element Preliminaries": mesh map, Jacobian, F^{-T} grad)
* ``transport``    -- upwind DG S_N discretization and the sweep (Sec.
                      "Transport Discretization")
* ``closures``     -- discrete SMM closures T, beta, E_b0, J_in (Eqs.
                      correction_tensor_disc, bdr_correction_factor_disc,
                      eb0_disc, broken_Tdiv)
* ``ipsmm``        -- interior penalty SMM moment system (Eq. ipsmm)
* ``smm``          -- the fixed-point map G and its iteration (Eqs. moment:G,
                      moment:smm_fp, fixed-point), plus plain source iteration

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product (``paper_2304_07386_gb300``) never
imports it, and it never imports the product; the two share only the seeded
input generators in ``smm_workloads``.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, exact polynomial reproduction, brute-force
global solves or the paper's printed iteration counts.
"""
