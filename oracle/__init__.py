"""CPU oracle of the stabilised DQMC Green's-function path.

TEST INFRASTRUCTURE, not part of the library.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its ``cpu_baseline`` leg and its
``--impl reference`` arm) may import it.  It shares no code with the CUDA path
in ``paper_2003_05286_gb300``; the two meet only in the seeded input
generators of ``dqmc_inputs``, which hold none of the method's arithmetic.

* ``oracle.dqmc``  -- FP64 NumPy/SciPy restatement of the paper's pipeline:
  pivoted-QR UDT chain (Sec. 4), Loh inversions (Sec. 5, 6), log det, and the
  log-det gradient 1 - G_l(i,i).
* ``oracle.exact`` -- exact references that pin it: non-interacting closed
  forms and mpmath brute force.
"""
from . import dqmc, exact  # noqa: F401
