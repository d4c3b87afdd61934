"""CPU oracle for the OMEN 3-D tight-binding / Schrödinger–Poisson hot path (test infrastructure).

Plain, slow, obviously correct FP64 (complex128 where the Hamiltonian is complex) reference
implementations, written from the paper's statement of the method (Section III-A: eigenstates
of an empirical sp3s*/sp3d5s* tight-binding Hamiltonian by an iterative eigensolver, charge
from filled states, finite-difference Poisson, self-consistency) and from the textbook
definitions that the paper relies on but does not print (Slater–Koster two-centre integrals,
Harrison bond-length scaling, Lanczos, conjugate gradients).

This package is test infrastructure.  Only the tests, the smoke check and the CPU-baseline
leg of the benchmark may import it; the library's own code path never does, and it shares
no code with the CUDA implementation (only the seeded input generators in `synth`).

Modules
-------
sk           Slater–Koster bond blocks built by rotating the bond-frame block (definition of
             sigma/pi/delta bonds), Harrison scaling.
lattice      zincblende sites and a brute-force neighbour search (k-d tree).
hamiltonian  explicit CSR assembly (onsite, spin–orbit, bonds, Bloch phases, potential).
bulk         two-atom bulk H(k) and its eigenvalues folded onto a periodic supercell.
eigs         dense eigensolve, plain Lanczos and folded-spectrum Lanczos with full
             reorthogonalisation.
poisson      3-D finite-difference Poisson (periodic x,y; Dirichlet z) by direct solve and CG.
charge       Fermi–Dirac filling, Fermi level by bisection, cloud-in-cell deposit and gather.
effmass      single-band effective-mass Hamiltonian on a uniform grid (explicit CSR).
vff          Keating valence force field: strain energy, forces, relaxation, bond strains.
spmv         the plain CSR product of csr_matvec.c over all host cores (timing the oracle's
             repeated H·X; same sums as scipy's product).
"""
