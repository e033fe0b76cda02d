"""FP64 CPU oracle for the ERF compressible dycore step (arXiv 2412.04395).

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the product path never does.  It shares no code with the CUDA
library in ``paper_2412_04395_gb300``.
"""
from .erf_oracle import (Oracle, OracleConfig, build_oracle, lib_path, interp, weno5,
                         thomas, eos, hse_column, ustar, psi_m, set_threads, qvs, rain_speed,
                         rain_evap, config_from, from_workload)

__all__ = ["Oracle", "OracleConfig", "build_oracle", "lib_path", "interp", "weno5", "thomas",
           "eos", "hse_column", "ustar", "psi_m", "set_threads", "qvs", "rain_speed", "rain_evap",
           "config_from", "from_workload"]
