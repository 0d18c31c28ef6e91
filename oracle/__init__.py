"""Serial FP64 oracle for ADMM on a factor graph (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The product library never does.
"""
from .oracle import (  # noqa: F401
    OracleGraph, build_oracle, from_problem, oracle_prox, T_PACK_PAIR, T_PACK_WALL,
    T_PACK_RADIUS_LIN, T_PACK_RADIUS_QUAD, T_SVM_HINGE, T_SVM_L2, T_MPC_DYN,
    T_MPC_QUAD, T_MPC_BOX, T_FIX, T_SVM_MARGIN, T_SVM_SLACK, T_EQUAL,
)
