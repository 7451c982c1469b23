"""FP64 CPU oracle for BSGD -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct code written from the paper (Gao, Biguri and
Blumensath, "Block stochastic gradient descent for large-scale tomographic
reconstruction in a parallel network", arXiv:1903.11874). Only tests/,
__graft_entry__.smoke() and bench.py's CPU-baseline leg may import it; the
CUDA library neither imports nor links anything here, and nothing here comes
from the CUDA library.

Contents and the passages they follow:
  projector.py  Siddon FP / BP of any row set and column block (Sec. 1, Eq. 1;
                Sec. 2, Eq. 3)
  bsgd.py       Algorithm 1 literally, its snapshot form, BSGD-IM cells
                (Algorithm 2), residual-weighted pairs, power-iteration step
  tv.py         TV prox of BSGD-TV (Algorithm 4, Eqs. 9-10) by FGP
  rng.py        SplitMix64 sampling spec
Every function is pinned by a "not gpu" test in tests/test_oracle_*.py.
"""
from . import projector, rng, tv, bsgd  # noqa: F401
from .projector import Geometry  # noqa: F401
