"""GB300-native two-phase SpGEMM (C = A*B on CSR, int32 indices, float64 values).

The compute path is the CUDA library ``libkk_spgemm.so`` (hand-written kernels
for sm_103a) behind the C ABI declared in ``include/kk_spgemm.h``; the
``spgemm`` module is its Python binding.  ``inputs`` builds seeded synthetic
matrices.  Submodules are imported lazily so that ``inputs`` works on machines
without a GPU.
"""
__all__ = ["inputs", "spgemm", "build"]


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)


def __getattr__(name):
    import importlib
    if name in ("inputs", "spgemm", "_build"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
