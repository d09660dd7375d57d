"""GB300-native geometric multigrid for H(div)-DG Darcy/Brinkman flow.

The compute path lives in the CUDA library ``libmgdarcy.so`` (sources in
``csrc/``, C interface in ``include/mgdarcy.h``); ``mgdarcy`` is the thin
ctypes binding.  Importing this package does not load the library.
"""
