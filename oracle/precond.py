"""Davidson correction vectors: CPU FP64 reference (TEST INFRASTRUCTURE ONLY).

The two-site Davidson of the paper carries a run-time-selectable
preconditioner family: Jacobi, deflation-aware diagonal, Olsen, and a
shift-and-invert inner-PCG mode with an indefiniteness guard.  None of them
may change the converged energies (Sec. "Computational details", the
paragraph on the device-native perturbative correction and state-averaged
orbital optimisation).  The paper does not write the formulas out.  This
module states the textbook forms that both this reference and the CUDA
library use, for a Ritz pair (theta, x) with |x| = 1 and residual
r = H x - theta x, where d is the diagonal of H:

  guarded denominator  den_i = d_i - theta, replaced by +-1e-8 (the sign of
                       den_i, + for 0) where |den_i| < 1e-8
  Jacobi               t = -r / den
  Olsen                t = -(r - eps x) / den,  eps = (x . r/den) / (x . x/den)
                       (Olsen, Jorgensen and Simons, Chem. Phys. Lett. 169,
                       463 (1990)): the diagonal step corrected so that
                       x . t = 0
  shift-and-invert     Jacobi-Davidson correction equation
  inner PCG            (I - x x^T)(H - theta)(I - x x^T) t = -r,  t orthogonal to x,
                       solved by preconditioned conjugate gradients from
                       t = 0 with the projected diagonal preconditioner
                       z = K^-1 v - (x . K^-1 v)/(x . K^-1 x) K^-1 x,  K = den.
                       At most `steps` iterations, stopping when the
                       residual norm falls below rel_tol |r|.  Indefiniteness
                       guard: a search direction p with p . A p <= 0 (A is
                       indefinite on the complement of x when theta lies
                       above the lowest eigenvalue) ends the iteration, and
                       the iterate reached so far is returned.  With that
                       guard on the first direction, the result is the
                       preconditioned residual, which is the Olsen
                       correction.

The deflation-aware diagonal belongs to deflated excited-state solves: the
diagonal of H_eff + w sum_j phi_j phi_j^T is d + w sum_j phi_j^2, and the
members above take it as their d (oracle/states.py holds the excited-state
reference).

Pinned in tests/test_oracle_precond.py:
  * x . t = 0 for Olsen and for the inner-PCG result;
  * with a constant diagonal and a Ritz pair, Olsen equals Jacobi;
  * zero inner steps give Olsen;
  * many inner steps solve the projected correction equation;
  * Davidson converges to the lowest eigenvalue of numpy.linalg.eigh with
    every correction, and to the FCI energy of a small active space.
"""
from __future__ import annotations

import numpy as np


def guarded_den(d, theta):
    """d - theta with |.| >= 1e-8 (sign kept, + for exact zero)."""
    den = np.asarray(d, dtype=np.float64) - theta
    return np.where(np.abs(den) < 1e-8, np.where(den >= 0, 1e-8, -1e-8), den)


def jacobi_correction(r, d, theta):
    return -np.asarray(r, dtype=np.float64) / guarded_den(d, theta)


def olsen_correction(x, r, d, theta):
    den = guarded_den(d, theta)
    a = float(np.dot(x, r / den))
    b = float(np.dot(x, x / den))
    eps = a / b if b != 0.0 else 0.0
    return -(np.asarray(r, dtype=np.float64) - eps * np.asarray(x, dtype=np.float64)) / den


def projected_precond(v, x, den):
    """K^-1 v made orthogonal to x in the K^-1 metric (result . x = 0)."""
    kv = v / den
    kx = x / den
    b = float(np.dot(x, kx))
    return kv - (float(np.dot(x, kv)) / b) * kx if b != 0.0 else kv


def pcg_correction(matvec, x, r, d, theta, steps=4, rel_tol=0.1):
    """Inner PCG on the projected correction equation (see module text).
    Returns (t, number of matvecs)."""
    x = np.asarray(x, dtype=np.float64)
    den = guarded_den(d, theta)

    def A(p):
        w = matvec(p) - theta * p
        return w - float(np.dot(x, w)) * x

    rhs = -np.asarray(r, dtype=np.float64)
    rhs = rhs - float(np.dot(x, rhs)) * x
    t = np.zeros_like(rhs)
    res = rhs.copy()
    z = projected_precond(res, x, den)
    p = z.copy()
    rz = float(np.dot(res, z))
    nrhs = float(np.linalg.norm(rhs))
    nmv = 0
    for j in range(steps):
        ap = A(p)
        nmv += 1
        pap = float(np.dot(p, ap))
        if pap <= 0.0:
            if j == 0:
                t = z.copy()
            break
        alpha = rz / pap
        t = t + alpha * p
        res = res - alpha * ap
        if float(np.linalg.norm(res)) < rel_tol * nrhs:
            break
        z = projected_precond(res, x, den)
        rz_new = float(np.dot(res, z))
        p = z + (rz_new / rz) * p
        rz = rz_new
    if steps == 0:
        t = z.copy()
    return t, nmv
