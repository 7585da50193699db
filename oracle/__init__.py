"""CPU FP64 oracle for the two-site DMRG sweep (TEST INFRASTRUCTURE ONLY).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import anything from this package.  The product path (the CUDA library and
its Python binding) never imports, links or executes it, and this package
imports nothing from the product path.

Modules
  fock  -- Jordan-Wigner Fock-space operators; brute-force H and RDMs for
           small active spaces (the plain definitions).
  fci   -- determinant-space FCI with colex string addressing (Sec.
           "Computational details", CI addressing) and Davidson; RDMs.
  mpo   -- MPO of the active-space Hamiltonian (Sec. "Cholesky decomposition
           for the wavefunction", item (i)) built term by term.
  dmrg  -- symmetry-blocked two-site DMRG with Davidson and SVD decimation
           (Fig. 2 and its section).
  states -- excited states of the sector: the eigenpairs that deflated
           sweeps converge to, with <S^2> from the 2-RDM (Sec. "Excited
           states: dual-penalty deflation and NACMEs").
  entropy -- one- and two-orbital reduced density matrices (fermionic
           partial traces), entropies and the mutual information.
  ordering -- Fiedler ordering of orbitals from a coupling matrix.
  precond -- Davidson correction vectors: Jacobi, Olsen, shift-and-invert
           inner PCG (Sec. "Computational details", preconditioner family).

Every function cites the passage it follows.  Parity status of each
function is stated in its docstring; all are pinned by tests under
tests/test_oracle_*.py except where "parity unpinned" is written.
"""
