"""GB300-native share-domain iris uniqueness check (arXiv 2405.04463, Alg. 3 hot path).

The C ABI of ``libipcheck.so`` (include/ipcheck.h) is bound in ``binding.py``; its names are
re-exported here on first use, so that ``paper_2405_04463_gb300.build`` stays importable
before the library exists. Using any binding name without a built library raises
ImportError: there is no CPU fallback.
"""
import importlib


def __getattr__(name):
    if name.startswith("__") or name in ("binding", "build", "workload"):
        raise AttributeError(name)
    return getattr(importlib.import_module(__name__ + ".binding"), name)
