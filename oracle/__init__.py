"""FP64 CPU oracle of the M1 RT subcycle -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It loads ``rt_oracle.c`` (plain C,
single thread, no FMA contraction), compiled with gcc on first use.  It shares
no code with the CUDA path.
"""
from .oracle import Oracle, OracleConfig, build_oracle_lib, default_config, rate_probe  # noqa: F401
