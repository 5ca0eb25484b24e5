"""FP64 CPU oracle of the M1 RT subcycle -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It loads ``rt_oracle.c`` (plain C,
single thread, no FMA contraction), compiled with gcc on first use; the same
source built with -fopenmp runs its independent per-cell and per-face loops on
all host cores with bitwise the same results (``Oracle(..., threads=0)``).  It shares
no code with the CUDA path.
"""
from .oracle import (COOLING_TERMS, Oracle, OracleConfig, build_oracle_lib, cooling_coeffs,  # noqa: F401
                     default_config, oracle_threads_available, rate_probe, rates)
