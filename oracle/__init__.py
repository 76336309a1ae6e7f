"""CPU oracle for the SiPO projection LP (test infrastructure only).

A plain, slow, FP64 restatement of what the solver computes, written from the
paper (Eqs. 2-3 forward model, Eqs. 19-24 / 32-37 / 40-45 linear programs,
Sec. 6.1 KKT conditions, Eqs. 6-8, 27 and 46 metrics).  It exists to check the
CUDA path and shares no code, tables or helpers with it.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import anything from this package.  The product path
(the ``paper_2604_08997_gb300`` package and its C library) never does.

Modules:
  operators  -- projector P, backprojector P^T, attenuation, PSF K, A, A^T
  lp         -- domain partition, normalisation, LP data, residuals, metrics
  pdhg       -- restarted primal-dual hybrid gradient solve of the LP
  simplex    -- dense two-phase simplex (Bland's rule) for tiny LPs
  sample     -- single-output evaluation of the operators at full size
"""
