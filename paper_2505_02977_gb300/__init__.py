"""GB300-native randomized approximate Cholesky (rchol elimination scheduled by
ParAC's dynamic dependency counters) with a PCG solver, behind a C ABI.

The compute path is ``libparac.so`` (hand-written sm_103a CUDA, see ``csrc/``);
``parac`` is the thin ctypes binding with the C entry points' names, and
``workloads`` builds the seeded synthetic inputs.  Importing this package loads
nothing; importing ``parac`` loads the library and fails loudly if it is absent.
"""
import os

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG_DIR, "libparac.so")
