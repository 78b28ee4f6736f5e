"""GB300-native conservative cut-cell MAC projection step (arXiv 2211.10698).

The computation lives in ``libccm.so`` (CUDA, sm_103a) behind the C ABI of
``include/ccm.h``; ``paper_2211_10698_gb300.ccm`` is its ctypes binding and
``paper_2211_10698_gb300.inputs`` describes the seeded synthetic problems.
"""
__all__ = ["ccm", "inputs", "build"]
