"""GB300-native (sm_103a) evaluator of the Kernel Aggregated Fast Multipole Method
(Yan & Blackwell, arXiv:2010.15155).

The compute path is the CUDA library ``libkafmm.so`` (C ABI: include/kafmm.h); ``kafmm`` is
its Python binding.  Build with ``python -m paper_2010_15155_gb300.build``.

Example (Stokeslet, sources = targets, forces f, mixed precision on the tensor cores)::

    import torch
    from paper_2010_15155_gb300 import kafmm as K
    y = torch.rand(262144, 3, device="cuda")            # points in [0, 1)^3
    f = torch.randn(262144, 3, device="cuda")           # forces
    plan = K.Plan(K.STOKESLET, p=10, q=128)             # order p, <= q points per leaf
    plan.set_points(y)                                  # tree, lists, work lists
    u = plan.eval(f)                                    # velocities [N, 3]
    plan.close()

Other problems: ``K.LAPLACE`` (q -> phi), ``K.RPY`` ([f, b] -> [u, lap u], then
``K.kafmm_rpy_velocity`` for sphere velocities), ``K.STOKES_DL`` (D -> [p, u]),
``K.STOKES_REG`` ([f, eps] -> u), ``K.LAPLACE_QD`` ([q, d] -> [phi, grad, Hessian]),
``K.STOKES_PVEL`` ([f, q] -> [p, u]).  ``bc=K.BC_PX``, ``K.BC_PXY`` or ``K.BC_PXYZ`` for
singly, doubly or triply periodic sums, ``K.BC_WALL`` (``K.BC_WALL_PX``, ``K.BC_WALL_PXY``) for
a no-slip wall (with periodicity along it),
``precision=K.PREC_FP64`` for the plain FP64 form, ``set_points_batched`` for many independent
problems in one forest, ``K.kafmm_autotune`` to time the tensor-core configurations.
"""
from . import kafmm  # noqa: F401
from .kafmm import Plan, KafmmError  # noqa: F401
