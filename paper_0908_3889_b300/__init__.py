"""B300-native batched post-Newtonian inspiral integrator (arXiv:0908.3889).

The compute path is the CUDA library ``libpn_b300.so`` (sources in ``csrc/``,
C ABI in ``include/pn_batch.h``); this package is its thin Python binding.
"""
from .api import (Batch, PNAdjointFn, PNError, adjoint, alloc_inputs, alloc_outputs, dist, inputs_struct, integrate, outputs_struct,
                  params, pn_abi_version, pn_batch_adjoint, pn_batch_autotune, pn_batch_destroy, pn_batch_eval_rhs, pn_batch_histogram, pn_batch_init, pn_batch_kde,
                  pn_batch_integrate, pn_batch_integrate_budget, pn_batch_host_wait, pn_batch_integrate_host, pn_batch_integrate_host_async, pn_batch_resume,
                  pn_batch_masses, pn_batch_sample, pn_batch_timing, pn_batch_set_params, pn_batch_stats, pn_batch_stats_segments,
                  pn_integrate_noalloc, sweep,
                  pn_ks_uniform,
                  pn_last_error, segment, to_device, to_numpy)
from . import _native as native

__all__ = ["Batch", "PNAdjointFn", "PNError", "adjoint", "alloc_inputs", "alloc_outputs", "dist", "inputs_struct", "integrate",
           "outputs_struct", "params", "pn_abi_version", "pn_batch_adjoint", "pn_batch_autotune",
           "pn_batch_destroy", "pn_batch_eval_rhs", "pn_batch_histogram", "pn_batch_init", "pn_batch_kde", "pn_batch_integrate",
           "pn_batch_integrate_budget", "pn_batch_host_wait", "pn_batch_integrate_host",
           "pn_batch_integrate_host_async", "pn_batch_masses", "pn_batch_timing", "pn_batch_resume", "pn_batch_sample",
           "pn_batch_set_params", "pn_batch_stats", "pn_batch_stats_segments", "pn_integrate_noalloc", "sweep", "pn_ks_uniform", "pn_last_error",
           "segment", "to_device", "to_numpy",
           "native"]
