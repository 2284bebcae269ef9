"""GB300-native EDP / RMS energy minimisation (arXiv 1410.7922).

The compute path is the CUDA library ``libedp.so`` (``csrc/``) behind the
C-ABI declared in ``include/edp.h``; ``edp`` is its thin Python binding.
Importing this package loads nothing; ``paper_1410_7922_gb300.edp`` loads the
library on first use and raises if it is missing.
"""
