"""Shared helpers of the GPU parity tests: moving an oracle MPS into the
library's canonical block format and matching channel labels."""
import numpy as np

from oracle import dmrg
from oracle import mpo as ompo
from oracle.mpo import QN


def export_mps(d):
    """(n_sectors, triples, data) of an oracle DMRG state in canonical blocks."""
    return dmrg.canonical_blocks(d)


def label_keys(m, bond):
    """Library channel keys (kind<<40 | nops<<32 | c0<<16 | c1) of the oracle MPO."""
    out = []
    for lab in m.labels[bond]:
        kind, n, codes = ompo.label_key(lab)
        c0 = codes[0] if n > 0 else 0
        c1 = codes[1] if n > 1 else 0
        out.append((kind << 40) | (n << 32) | (c0 << 16) | c1)
    return out
