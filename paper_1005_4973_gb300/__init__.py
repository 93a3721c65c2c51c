"""MTGP generation on one GB300 GPU: a C-ABI library of hand-written sm_103a
kernels (include/mtgp.h) with a thin Python binding.

The first use of an API name from this package loads
paper_1005_4973_gb300/_build/libmtgp.so and raises ImportError if it is not
built (python -m paper_1005_4973_gb300.build): there is no fallback path.
Submodules (build, workloads) import without the library.
"""
import importlib
import importlib.util


def __getattr__(name):
    if not name.startswith("__") and importlib.util.find_spec(f"{__name__}.{name}") is not None:
        return importlib.import_module(f".{name}", __name__)
    mod = importlib.import_module(".mtgp", __name__)
    try:
        return getattr(mod, name)
    except AttributeError:
        raise AttributeError(f"module {__name__!r} has no attribute {name!r}") from None
