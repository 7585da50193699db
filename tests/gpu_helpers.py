"""Shared helpers of the GPU parity tests: moving an oracle MPS into the
library's canonical block format and matching channel labels."""
import numpy as np

from oracle import mpo as ompo
from oracle.mpo import QN


def export_mps(d):
    """(n_sectors, triples, data) of an oracle DMRG state in canonical blocks."""
    ns, tr, data = [], [], []
    for k in range(d.n + 1):
        secs = sorted(d.dims[k])
        ns.append(len(secs))
        for q in secs:
            tr += [q[0], q[1], d.dims[k][q]]
    for i in range(d.n):
        for ql in sorted(d.dims[i]):
            for s in range(4):
                qr = (ql[0] + QN[s][0], ql[1] + QN[s][1])
                if qr not in d.dims[i + 1]:
                    continue
                b = d.sites[i].get((ql, s))
                if b is None:
                    b = np.zeros((d.dims[i][ql], d.dims[i + 1][qr]))
                data.append(b.reshape(-1))
    return np.array(ns), np.array(tr), np.concatenate(data)


def label_keys(m, bond):
    """Library channel keys (kind<<40 | nops<<32 | c0<<16 | c1) of the oracle MPO."""
    out = []
    for lab in m.labels[bond]:
        kind, n, codes = ompo.label_key(lab)
        c0 = codes[0] if n > 0 else 0
        c1 = codes[1] if n > 1 else 0
        out.append((kind << 40) | (n << 32) | (c0 << 16) | c1)
    return out
