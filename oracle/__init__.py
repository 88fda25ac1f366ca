"""CPU oracle for the real-time population-dynamics QMC step (arXiv:2502.18929).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  It
shares no code with the CUDA library (``paper_2502_18929_gb300``).

* ``qmc_oracle.c`` -- the plain single-threaded method (C, -ffp-contract=off).
* ``oracle.py``    -- ctypes wrapper around it.
* ``dense.py``     -- dense FP64 Liouvillian of Eq. (2) and the deterministic
  Euler / AB2 recursions, for tiny n.
* ``learn.py``     -- FP64 training events, loss and gradient of the learned
  proposal's network (the library's extension; not in the paper).
"""
