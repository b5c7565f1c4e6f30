"""GB300 (sm_103a) solver for the mapped adjoint Lindblad equation of arXiv 2203.05526.

The numerical work runs in ``libbq.so`` (CUDA kernels + C ABI, include/bq.h); this package
is the thin ctypes binding.  ``build.build()`` compiles the library in-tree.
"""

from .binding import (BQError, ProblemHandle, State, check, exported_symbols, fma_peak, fma_peak_count, grad_record_bytes,  # noqa: F401
                      launch_count, lib,
                      map_opts, plan, problem_from_spec)
