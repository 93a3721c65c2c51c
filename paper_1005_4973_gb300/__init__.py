"""MTGP generation on one GB300 GPU: a C-ABI library of hand-written sm_103a
kernels (include/mtgp.h) with a thin Python binding.

The first use of any name from this package loads
paper_1005_4973_gb300/_build/libmtgp.so and raises ImportError if it is not
built (python -m paper_1005_4973_gb300.build): there is no fallback path.
"""
import importlib


def __getattr__(name):
    mod = importlib.import_module(".mtgp", __name__)
    try:
        return getattr(mod, name)
    except AttributeError:
        raise AttributeError(f"module {__name__!r} has no attribute {name!r}") from None
