"""Plain FP64 CPU oracle for the two-site QC-DMRG hot path.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py, never by the product path.  It shares no code,
header, table or helper with the CUDA library.

  fock    determinant / Fock-space machinery and full CI (exact energies)
  blocks  explicit block bases, V^T H V, exact renormalized operators, RDM
"""
