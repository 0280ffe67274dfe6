"""GB300-native Potential Difference Reduction (PDR) for multicommodity-flow feasibility.

The compute path lives in ``libpdr.so`` (CUDA C++ for sm_103a behind a C ABI,
declared in ``include/pdr.h``); ``pdr`` is its thin ctypes binding and
``instances`` builds seeded synthetic inputs.  Importing the package loads
nothing: the native library is opened on first use of ``pdr``.
"""

__all__ = ["instances", "pdr"]
