"""CPU oracle of the D-iteration hot path.

TEST INFRASTRUCTURE ONLY: plain, slow, obviously correct FP64 code that
restates the paper (X = P X + B, Eqs. 1-3; the fluid/history recursions
Eqs. defF/defH; the cyclic threshold sweep of Sec. 2.4).  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  It shares no code with the CUDA library and never calls it.
"""
