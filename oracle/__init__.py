"""FP64 CPU oracle of the conservative Allen-Cahn phase-field LBM.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product library never imports,
links or executes anything in this package.  It shares no code with the CUDA
path; both sides only take the same seeded inputs.

``Oracle`` wraps ``pflbm_oracle.cpp`` (plain loops, two-array streaming, full
moment matrices) through ctypes.  See that file's header for the equations and
the readings it follows.  ``tangent`` runs the same arithmetic in dual numbers
for the exact derivative of a phi functional with respect to M, xi or sigma.
"""
from .oracle import (Oracle, from_params, tables, mrt_collide, build_oracle, tangent, COLL_MRT, COLL_BGK,
                     COLL_MRT_ALL_EQUAL, SCHED_CONCURRENT, SCHED_SEQUENTIAL)

__all__ = ["Oracle", "from_params", "tables", "mrt_collide", "build_oracle", "tangent", "COLL_MRT", "COLL_BGK",
           "COLL_MRT_ALL_EQUAL", "SCHED_CONCURRENT", "SCHED_SEQUENTIAL"]
