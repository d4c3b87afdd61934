"""Seeded synthetic inputs shared by the CUDA path, the CPU oracle, the tests and the bench.

This package draws random numbers and lays them out in the input formats of the C-ABI
(species per atom, strain per bond slot, tight-binding parameter tables, Lanczos start
blocks, doping profiles).  It holds none of the method's arithmetic: no Hamiltonian
element, no eigen-solve, no charge or potential is computed here.
"""
from .workloads import *  # noqa: F401,F403
