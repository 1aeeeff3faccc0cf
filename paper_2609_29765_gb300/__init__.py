"""GB300-native structure-adaptive tile Cholesky (numeric phase), arxiv 2609.29765.

Host analysis + CUDA (sm_103a) numeric replay behind the C ABI in include/stc.h;
``api.Plan`` / ``api.Factor`` are the Python face.  Importing the package does not load
the native library; the first call that needs it does, and fails loudly if it is absent.
"""
__all__ = ["Plan", "Factor"]


def __getattr__(name):
    if name in ("Plan", "Factor"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
