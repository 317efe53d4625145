"""GB300 (sm_103a) phase-averaged rotating shallow water on the sphere.

The compute path is the CUDA library ``libpavg.so`` (C-ABI, ``include/pavg.h``);
``paper_2103_07706_gb300.pavg`` is its thin ctypes binding and ``inputs``
builds seeded synthetic states.  Importing the package loads nothing;
``load()`` / ``pavg`` load the library and fail loudly when it is missing.
"""

__all__ = ["inputs", "pavg"]
