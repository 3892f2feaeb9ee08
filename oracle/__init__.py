"""CPU oracle for PTSBE -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package. The CUDA library never imports, links or calls it.
"""
from .oracle import Oracle, build_oracle, oracle_lib_path  # noqa: F401
