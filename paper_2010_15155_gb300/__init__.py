"""GB300-native (sm_103a) evaluator of the Kernel Aggregated Fast Multipole Method
(Yan & Blackwell, arXiv:2010.15155).

The compute path is the CUDA library ``libkafmm.so`` (C ABI: include/kafmm.h); ``kafmm`` is
its Python binding.  Build with ``python -m paper_2010_15155_gb300.build``.
"""
from . import kafmm  # noqa: F401
from .kafmm import Plan, KafmmError  # noqa: F401
