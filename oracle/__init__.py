"""CPU oracle for randomized approximate Cholesky + PCG (test infrastructure).

Only the test-suite, the package smoke check and the benchmark's CPU-baseline
leg may import this package.  It wraps ``rchol_oracle.c`` (plain C, FP64,
compiled with ``-ffp-contract=off``) through ctypes; see that file's header for
what each function computes and which passage of the ParAC paper it follows.
"""
from .oracle import (  # noqa: F401
    build, lib, philox4x64_10, slot_uniform, suffix_scan, pick_bruteforce, pick_search,
    eliminate_one, eliminate_one_ac, ingest, factor, factor_tracked, dp_update, precond_apply, pcg,
    OracleError, KIND_AUTO, KIND_LAPLACIAN, KIND_SDDM,
)
