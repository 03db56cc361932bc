"""FP64 CPU oracle for the open-rectangular-pipe Poisson solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path (the only common dependency is the input generator
package ``inputs``, which holds none of the method's arithmetic).

Modules
-------
green   -- the Green functions: pipe sine series (Eq. 7), the R function
           (Eq. 9), the longitudinal IGF g_z (Eq. 15) and R_int (Eq. 16),
           the free-space 1/r (Eq. 3).
pipe    -- the three solvers of the discretised problem (Eq. 4 with the pipe
           Green function): O1 brute-force sum, O2 naive-DFT version of the
           four-term formula Eq. 10, O3 the same with scipy.fft; their
           adjoints; the free-space Hockney solve (Eq. 5); the doubled-grid
           tables of Fig. 1 / Eq. A.3.
conv1d  -- the 1-D convolution / correlation identities of Appendix A.

Every function cites the passage it follows.  All arithmetic is FP64.
"""
