"""B300-native Monte Carlo integrator for the lepton-loop-free QED vertex graphs
of arXiv:1905.08007 (Volkov): per-graph subtracted Feynman-parametric
integrands, Deg-based Hepp-sector densities (Eq. (1)), Philox sampling, FP64
evaluation with double-double re-evaluation, compensated reductions.

The compute path is the native library ``libqedmc.so`` (CUDA, sm_103a); this
package is a thin ctypes binding with the C ABI's names.  Importing it does
not need a GPU; every call that computes does, and fails loudly without one.
"""
from ._lib import (  # noqa: F401
    QedError,
    Graph,
    Result,
    Context,
    Diagram,
    enumerate_graphs,
    gauge_class,
    lib_path,
    load_library,
    merge_results,
    fp64_peak,
)
from .classes import class_table  # noqa: F401
