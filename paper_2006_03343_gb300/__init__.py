"""GB300-native wall-modeled immersed boundary stress stage (Liu & Stevens,
arXiv:2006.03343, Sec. 3).

The compute path is the sm_103a CUDA library ``libwmibm.so`` behind the C ABI
declared in ``include/wmibm.h``; ``wmibm`` is its thin ctypes binding.  The
binding is imported lazily so that input generation works on machines without
the library; calling into it without a built library raises.
"""

__all__ = ["inputs", "wmibm", "autotune"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
