"""CPU ORACLE for the KAFMM evaluator -- test infrastructure, not product code.

Plain, slow, FP64 statements of what the method computes (Yan & Blackwell,
arXiv:2010.15155): ``direct`` holds the direct kernel sums (the definition of the result,
Eq. kernelsumlinear), ``tree`` the adaptive octree and U/V/W/X lists, ``kafmm`` the plain
KAFMM traversal, ``periodic`` the lattice sums behind the triply periodic operator.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
this package.  It shares no code with the CUDA evaluator.
"""
