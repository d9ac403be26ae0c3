"""GB300-native GCMe nonbonded force/energy library (arXiv 2403.08148).

The compute path is libgcme.so (CUDA, sm_103a), reached through its C ABI
(include/gcme.h); ``binding`` marshals torch tensors and numpy arrays into
those calls.  There is no CPU fallback: without the built library every
entry point raises.
"""
from .binding import (Batch, Context, GcmeError, Params, Server, System, load,  # noqa: F401
                      build_cells_noalloc, cells_noalloc_size,
                      params_from, validate, FORCE_SCALE, NTERMS, TERM_NAMES,
                      GCME_BULK, GCME_SLAB_NONMETAL, GCME_SLAB_IMAGE, GCME_FP32, GCME_FP64,
                      GCME_PAIR_AUTO, GCME_PAIR_LIST, GCME_PAIR_CELLS)
from .builder import build, LIB  # noqa: F401
