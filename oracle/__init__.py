"""Plain, slow FP64 CPU oracle for the TTNS real-time sweep.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code with the CUDA library; the only
module both sides read is the seeded input generator
(``paper_1710_01362_gb300.workloads``), which holds none of the method's
arithmetic.

Every function follows a passage of the paper (arXiv:1710.01362, "Multi-
dimensional Tensor Network Simulation of Open Quantum Dynamics in Singlet
Fission"), cited by equation or section, and the readings of the passages the
paper leaves open (its Supplement, which holds the TDVP algorithm, is not part
of the paper text).

Modules
  chain        orthogonal-polynomial chain maps (Methods, "Tensor Network States"; Eq. 2)
  model        star Hamiltonian terms, tree topology, bond clamp, initial state (Eq. 2)
  linalg       Householder QR with the fixed completion rule; Lanczos exponential
  ttns         environment blocks, H_eff, one-site TDVP step, observables
  statevector  dense reference for tiny trees (exact propagation)

Parity status per function (what pins it, in tests/test_oracle_*.py):
  chain_ohmic            pinned (Laguerre closed form vs quadrature + Lanczos)
  chain_from_modes       pinned (inverse spectral problem: chain spectrum = modes)
  householder_qr         pinned (numpy QR up to column phases; reconstruction)
  expm_lanczos           pinned (scipy expm on dense matrices)
  tdvp step              pinned at full bond dimension (exact vs state vector),
                         zero coupling (Rabi formula), pure dephasing (closed form),
                         norm / energy conservation, time reversibility
  tdvp at truncated D    parity unpinned beyond invariants (no closed form exists)
"""
