"""Batched accurate normalization of vectors and quaternions on GB300 (sm_103a),
after W. F. Mascarenhas, "Fast and accurate normalization of vectors and
quaternions" (arXiv 1606.06508).

The work is done by libnormgb.so (C ABI in include/normgb.h, CUDA kernels in
csrc/).  ``_lib`` is its ctypes binding (same names as the C entry points);
``api`` adds torch-tensor helpers and the autograd Function.  Importing this
package loads nothing; the library is loaded on first use and an ImportError
is raised if it has not been built.
"""

__all__ = ["normalize", "normalize_backward", "NormalizeFn", "Plan", "normalize_to_rotation",
           "naive_normalize", "copy_", "plan_for"]


def __getattr__(name):
    if name in __all__:
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
