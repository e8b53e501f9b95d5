"""GB300-native SU(N) unfolding and RK4 propagation of GKSL master equations (arXiv:1812.11626).

The compute path is the CUDA library ``libgksl`` (``csrc/``), reached through the
thin ctypes binding in ``gksl.py``. ``workloads.py`` builds seeded synthetic
inputs. Importing this package loads nothing native; import ``.gksl`` for that.
"""
