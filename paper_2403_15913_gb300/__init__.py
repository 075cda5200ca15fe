"""GB300-native KKT step of a filter line-search interior-point method on
dynamic NLPs, with the Lifted-KKT and HyKKT hybrid solvers of Pacaud & Shin
(arXiv 2403.15913).  All numerics run in the in-tree CUDA library
``libkkt_gb300.so`` (C ABI in include/kkt.h); this package only marshals
arguments."""
from .solver import KKTBatchSolver, KKTSolver, KKTError, autotune_batch, default_options  # noqa: F401
from .tray import TrayModel  # noqa: F401
from .ipm import IPMBatch, IPMSolver  # noqa: F401
from .serve import NMPCServer  # noqa: F401
