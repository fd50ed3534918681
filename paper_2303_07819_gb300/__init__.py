"""GB300-native msDEM hot path (Deng, Stechmann & Chen, arXiv 2303.07819).

The compute path lives in the CUDA library ``libmsdem.so`` (sources in
``csrc/``); ``paper_2303_07819_gb300.msdem`` is its thin ctypes binding.
Importing the package loads nothing; the library is loaded on first use and
importing the binding fails loudly when the library is missing.
"""
