"""Excited states of the active space: CPU reference (TEST INFRASTRUCTURE ONLY).

The paper reaches excited states by penalty deflation: the lower converged
states stay resident and are projected into every two-site optimisation
through overlap environments.  Roots are selected, and every reported root
is checked, by <S^2> (Sec. "Excited states: dual-penalty deflation and
NACMEs").  Its dual penalty lambda S_z^2 + mu (N - N_el)^2 (Eq. dualpen)
only lifts states outside the (N_el, S_z) sector.  It is zero inside the
sector, and a solver that is blocked by (N_alpha, N_beta), as this one is,
never leaves it.

At full bond dimension the deflated sweep converges to the eigenpairs of H
in the sector.  So the reference for it is the definition: the eigenpairs
of the sector Hamiltonian (dense FCI), ordered by energy, each carrying
<S^2>.  Root selection keeps those whose <S^2> is within `tol` of the
target.

<S^2> comes from the spin-summed 2-RDM Gamma_pqrs =
sum_st <a+_ps a+_rt a_st a_qs> through the identity
    S^2 = -1/2 sum_pq e_pqqp - N^2/4 + N,   e_pqrs = E_pq E_rs - delta_qr E_ps,
so <S^2> = -1/2 sum_pq Gamma_pqqp - N^2/4 + N in a state of fixed N.
Pinned in tests/test_oracle_states.py against the operator
S_z^2 + (S_+ S_- + S_- S_+)/2 built from Jordan-Wigner strings (fock.py),
against closed forms (one electron 3/4, a closed shell 0, a high-spin pair
2), and against the Hubbard dimer's closed-form spectrum.
"""
from __future__ import annotations

import numpy as np

from . import fci


def spin_square_from_rdm(g2: np.ndarray, n_elec: int) -> float:
    """<S^2> = -1/2 sum_pq Gamma_pqqp - N^2/4 + N."""
    n = g2.shape[0]
    s = sum(g2[p, q, q, p] for p in range(n) for q in range(n))
    return float(-0.5 * s - n_elec * n_elec / 4.0 + n_elec)


def sector_spectrum(h, eri, n_alpha, n_beta, nroots, dense_limit=2000):
    """Lowest nroots eigenpairs of H in the (N_alpha, N_beta) sector (dense
    FCI up to dense_limit determinants, block Davidson to |r| < 1e-10 above)
    with <S^2> of each.  Returns (energies, S^2 values, CI vectors)."""
    F = fci.FCI(h, eri, n_alpha, n_beta)
    w, v = F.ground_state(tol=1e-10, nroots=nroots, max_iter=400, max_space=max(24, 4 * nroots),
                          dense_limit=dense_limit)
    w, v = np.asarray(w)[:nroots], np.asarray(v)[:, :nroots]
    s2 = np.array([spin_square_from_rdm(F.rdms(v[:, i])[1], n_alpha + n_beta) for i in range(v.shape[1])])
    return w, s2, v


def select_roots(energies, s2, target_s2, nroots, tol=0.1):
    """Indices of the lowest nroots states with |<S^2> - target| < tol
    (the <S^2>-based root selection)."""
    keep = [i for i in range(len(energies)) if abs(s2[i] - target_s2) < tol]
    return keep[:nroots]
