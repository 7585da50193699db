"""Writes the stored reference values under tests/golden/.

Calls only the CPU oracle (oracle/fock.py, oracle/fci.py, oracle/dmrg.py) on
inputs from gbd_synth; run from the repository root:
    python tests/golden/make_golden.py [--cas12] [--dmrg]
The CAS(12,12) reference (853,776 determinants, Davidson to ||r|| < 1e-9)
takes a few minutes and about 3 GB of memory.  --dmrg writes the oracle
DMRG sweeps that the GPU parity tests compare with (adaptive bond dimension
at CAS(8,8); CAS(10,10) at M = 96); the oracle is slow, so these take tens of
minutes.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from gbd_synth import make_integrals  # noqa: E402
from oracle import dmrg, fci, fock  # noqa: E402

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


def dmrg_run(name, n, ne, nq, seed, M, sweeps, tol, max_discarded=0.0, m_min=1, two_sz=0):
    h, chol = make_integrals(n, nq, seed)
    d, sw = dmrg.run(h, chol, ne, two_sz, [M] * sweeps, [tol] * sweeps, seed=seed, max_discarded=max_discarded,
                     m_min=m_min)
    out = dict(source="oracle/dmrg.py run(): seeded initial MPS, two-site sweeps, SVD decimation; integrals "
                      f"gbd_synth.make_integrals({n}, {nq}, seed={seed})",
               n_orb=n, n_elec=ne, two_sz=two_sz, n_chol=nq, seed=seed, M=M, sweeps=sweeps, tol=tol,
               max_discarded=max_discarded, m_min=m_min, sweep_energies=[float(e) for e in sw],
               energy=float(d.energy()),
               bonds=[[[q[0], q[1], d.dims[b][q]] for q in sorted(d.dims[b])] for b in range(n + 1)])
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(out, f, indent=1)


DMRG_RUNS = {
    "dmrg_cas8_m48_adaptive1e-6.json": dict(n=8, ne=8, nq=10, seed=3, M=48, sweeps=3, tol=1e-10,
                                            max_discarded=1e-6, m_min=4),
    "dmrg_cas8_m48_adaptive1e-4.json": dict(n=8, ne=8, nq=10, seed=3, M=48, sweeps=3, tol=1e-10,
                                            max_discarded=1e-4, m_min=2),
    "dmrg_cas10_m96_seed7.json": dict(n=10, ne=10, nq=20, seed=7, M=96, sweeps=2, tol=1e-9),
    # problems of the batched-solve test (half filling, S_z = 1/2 when odd)
    "dmrg_batch_n6_seed11.json": dict(n=6, ne=6, nq=8, seed=11, M=32, sweeps=2, tol=1e-8),
    "dmrg_batch_n8_seed13.json": dict(n=8, ne=8, nq=10, seed=13, M=48, sweeps=2, tol=1e-8),
    "dmrg_batch_n7_seed15.json": dict(n=7, ne=7, nq=9, seed=15, M=40, sweeps=2, tol=1e-8, two_sz=1),
}


if __name__ == "__main__":
    cas6()
    if "--cas12" in sys.argv:
        cas12()
    if "--dmrg" in sys.argv:
        only = [a for a in sys.argv[1:] if a.endswith(".json")]
        for name, kw in DMRG_RUNS.items():
            if not only or name in only:
                dmrg_run(name, **kw)
