"""GB300-native rank-profile-revealing PLUQ decomposition over Z/pZ.

The compute path is the C-ABI library ``libpluq.so`` (CUDA kernels for sm_103a
plus a native recursion driver); ``paper_1301_4438_gb300.pluq`` is its thin
Python binding and ``paper_1301_4438_gb300.workloads`` draws seeded inputs.
Importing the package loads nothing: the binding loads the library on first
use and raises if it is missing.
"""
