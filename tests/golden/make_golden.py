"""Writes the stored FCI reference values under tests/golden/.

Calls only the CPU oracle (oracle/fock.py, oracle/fci.py) on inputs from
gbd_synth; run from the repository root:
    python tests/golden/make_golden.py [--cas12]
The CAS(12,12) reference (853,776 determinants, Davidson to ||r|| < 1e-9)
takes a few minutes and about 3 GB of memory.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from gbd_synth import make_integrals  # noqa: E402
from oracle import fci, fock  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def cas6():
    h, chol = make_integrals(6, 18, 1)
    eri = fock.eri_from_chol(chol)
    w, v, st = fock.ground_state(h, eri, 3, 3, nroots=2)
    g1, g2 = fock.rdms(v[:, 0], st, 6)
    out = dict(source="oracle/fock.py dense diagonalisation of the (3,3) sector "
                      "of the Jordan-Wigner H; integrals gbd_synth.make_integrals(6, 18, seed=1)",
               n_orb=6, n_elec=6, two_sz=0, n_chol=18, seed=1,
               E0=float(w[0]), E1=float(w[1]), gap=float(w[1] - w[0]),
               rdm1=g1.tolist(), rdm2_trace=float(np.einsum("pprr->", g2)),
               rdm2_fro=float(np.linalg.norm(g2)))
    with open(os.path.join(HERE, "fci_cas6_m64_seed1.json"), "w") as f:
        json.dump(out, f, indent=1)


def cas12():
    h, chol = make_integrals(12, 36, 2)
    eri = fock.eri_from_chol(chol)
    f = fci.FCI(h, eri, 6, 6)
    e, x = fci.davidson(lambda v: f.sigma(v).ravel(), f.diagonal().ravel(), tol=1e-9,
                        max_iter=300, nroots=2)
    g1, g2 = f.rdms(x[:, 0])
    out = dict(source="oracle/fci.py Knowles-Handy Davidson (tol 1e-9, two roots) in the "
                      "(6,6) sector; integrals gbd_synth.make_integrals(12, 36, seed=2)",
               n_orb=12, n_elec=12, two_sz=0, n_chol=36, seed=2, n_det=f.Na * f.Nb,
               E0=float(e[0]), E1=float(e[1]), gap=float(e[1] - e[0]),
               rdm1=g1.tolist(), rdm2_trace=float(np.einsum("pprr->", g2)),
               rdm2_fro=float(np.linalg.norm(g2)))
    with open(os.path.join(HERE, "fci_cas12_m256_seed2.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    cas6()
    if "--cas12" in sys.argv:
        cas12()
