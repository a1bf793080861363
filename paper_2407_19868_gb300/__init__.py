"""GB300-native POREMAPS permeability solver (pseudo-unsteady Stokes on voxel images).

The compute path is the CUDA library ``libpm_gb300.so`` behind the C ABI declared in
``include/poremaps_gb.h``; :mod:`paper_2407_19868_gb300.api` is its thin Python
binding.  Importing the package loads nothing: the library is opened on first use
and raises if it has not been built.
"""

__all__ = ["api", "geometry"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
