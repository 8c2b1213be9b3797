"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This package holds no arithmetic of the contraction method itself: it only
draws PEPS site tensors, boundary-MPS operands and Hamiltonian terms with the
shapes and value distributions of the workloads, rounds them to the storage
precision the GPU path uses, and hands the same values to both sides.
"""
from .peps_inputs import *  # noqa: F401,F403
