"""Exact Ball Mapper construction on GB300 (sm_103a).

The compute path lives in the CUDA library built from ``csrc/``; ``binding``
marshals arguments to its C-ABI.  ``workloads`` holds the seeded synthetic
input generators only.
"""
