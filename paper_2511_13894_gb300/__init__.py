"""GB300 (sm_103a) restarted PDHG with the corner-push phase of Rothberg,
"Backing PDHG into a Corner" (arXiv 2511.13894).

The compute path is the CUDA library libpdhgc.so (C-ABI in include/pdhgc.h);
`paper_2511_13894_gb300.pdhgc` is its Python binding.  The binding's names
are re-exported here lazily so that `paper_2511_13894_gb300.build` can run
before the library exists.
"""

_EXPORTS = {"lp_create", "lp_from_dict", "LP", "Batch", "Guide", "uniform", "probe_gather",
            "default_params", "default_corner_params", "Params", "CornerParams", "Report", "PdhgcError",
            "FP64", "FP32_BULK", "AVERAGED", "HALPERN", "PHASE1", "CORNER", "DUAL_CORNER", "STATUS_NAMES", "lib"}


def __getattr__(name):
    if name in _EXPORTS:
        from . import pdhgc
        return getattr(pdhgc, name)
    raise AttributeError(name)
