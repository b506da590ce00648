"""GB300-native conservative Allen-Cahn phase-field LBM (PFLBM) hot path.

libpflbm.so (CUDA, sm_103a) behind the C interface include/pflbm.h;
``pflbm.Simulation`` is the Python front end, ``workloads`` builds seeded inputs.
"""
