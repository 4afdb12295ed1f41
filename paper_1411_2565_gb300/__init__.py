"""GB300-native LLG hot path of Zhu, "Grace" (arXiv:1411.2565).

The compute lives in the in-tree CUDA library ``libgrace.so`` (C ABI in
``include/grace.h``); this package only marshals arguments.  Import the binding
lazily so that ``paper_1411_2565_gb300.build`` works without torch or a GPU.
"""


def __getattr__(name):
    if name in ("Grace", "GraceBatch"):
        from . import grace
        return getattr(grace, name)
    raise AttributeError(name)
