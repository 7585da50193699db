"""Learned Davidson preconditioner: CPU FP64 reference (TEST INFRASTRUCTURE
ONLY).

The paper carries a run-time-selectable Davidson preconditioner family and
requires that the preconditioner never changes the converged energies (Sec.
"Computational details", device-native perturbative correction paragraph).
The learned member is not in the paper; its reading (stated once, used by
both the CUDA kernels and this reference):

  correction  t_i = -r_i / (d_i - theta) * (1 + clip(g_i, -0.9, 4))   (d = H_eff diagonal;
              the clip is the range of the targets, so an input unlike the
              training data cannot blow a component up)
  network     g_i = w2 . relu(W1 f_i + b1) + b2, W1: 128 x F, one hidden
              layer of width 128 ("2-layer": two weight layers)
  features    f_i = [ (d_i - theta) / s,  r_i / |r|,  |r_i| / |r|,
                      log(|d_i - theta| + 1e-12),  log |r|,  it / 32,
                      sign(d_i - theta),  1 ]            (F = 8)
              with s = the RMS of (d - theta) over the vector
  loss        L = sum_i w_i (g_i - y_i)^2 / sum_i w_i + lam * mean_i g_i^2
              (the second term is a prior towards g = 0, the Jacobi step,
              for elements the weighted data say little about), with the target
              y_i = clip(a e_i / tj_i - 1, -0.9, 4) and weight
              w_i = tj_i^2 / (1 + (a e_i / tj_i - 1)^2) where tj = -r/(d-theta)
              is the Jacobi step, e the component of (converged vector -
              current vector) orthogonal to the current vector, and
              a = (tj . e) / (e . e) the best single scale.
Pinned in tests/test_oracle_mlp.py: analytic gradients against central
finite differences, g = 0 reduces to the Jacobi step.
"""
from __future__ import annotations

import numpy as np

F = 8
H = 128


def features(r, d, theta, it):
    r = np.asarray(r, dtype=np.float64)
    den = np.asarray(d, dtype=np.float64) - theta
    rn = np.linalg.norm(r) + 1e-300
    s = np.sqrt(np.mean(den * den)) + 1e-300
    f = np.empty((r.size, F))
    f[:, 0] = den / s
    f[:, 1] = r / rn
    f[:, 2] = np.abs(r) / rn
    f[:, 3] = np.log(np.abs(den) + 1e-12)
    f[:, 4] = np.log(rn)
    f[:, 5] = it / 32.0
    f[:, 6] = np.sign(den)
    f[:, 7] = 1.0
    return f


def jacobi_step(r, d, theta):
    den = np.asarray(d, dtype=np.float64) - theta
    den = np.where(np.abs(den) < 1e-8, np.where(den >= 0, 1e-8, -1e-8), den)
    return -np.asarray(r) / den


def targets(tj, e):
    """Per-element target y and weight w (module docstring)."""
    a = float(tj @ e) / float(e @ e + 1e-300)
    ratio = a * e / np.where(np.abs(tj) > 1e-300, tj, 1e-300)
    y = np.clip(ratio - 1.0, -0.9, 4.0)
    w = tj * tj / (1.0 + (ratio - 1.0) ** 2)
    return y, w


class MLP:
    def __init__(self, W1, b1, w2, b2):
        self.W1 = np.asarray(W1, dtype=np.float64)   # (H, F)
        self.b1 = np.asarray(b1, dtype=np.float64)   # (H,)
        self.w2 = np.asarray(w2, dtype=np.float64)   # (H,)
        self.b2 = float(b2)

    def params(self):
        return np.concatenate([self.W1.ravel(), self.b1, self.w2, [self.b2]])

    @staticmethod
    def from_params(p):
        W1 = p[:H * F].reshape(H, F)
        b1 = p[H * F:H * F + H]
        w2 = p[H * F + H:H * F + 2 * H]
        return MLP(W1, b1, w2, p[-1])

    def forward(self, f):
        z = f @ self.W1.T + self.b1
        h = np.maximum(z, 0.0)
        return h @ self.w2 + self.b2, z, h

    def loss_and_grad(self, f, y, w, lam=0.0):
        g, z, h = self.forward(f)
        W = float(np.sum(w))
        n = g.size
        dg = 2.0 * w * (g - y) / W + 2.0 * lam * g / n
        loss = float(np.sum(w * (g - y) ** 2) / W + lam * np.sum(g * g) / n)
        gw2 = h.T @ dg
        gb2 = float(np.sum(dg))
        dh = np.outer(dg, self.w2) * (z > 0)
        gW1 = dh.T @ f
        gb1 = dh.sum(axis=0)
        grad = np.concatenate([gW1.ravel(), gb1, gw2, [gb2]])
        return loss, grad


def precondition(r, d, theta, it, net: MLP):
    """t = jacobi step * (1 + clip(g, -0.9, 4))."""
    tj = jacobi_step(r, d, theta)
    g, _, _ = net.forward(features(r, d, theta, it))
    return tj * (1.0 + np.clip(g, -0.9, 4.0))
