"""Shared helpers for the parity tests: scheme dicts, layouts, error metrics."""
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "schemes.json")) as fh:
    SCHEMES = json.load(fh)

OPS = ("dx", "dy", "dz", "dxx", "dyy", "dzz", "dxy", "dxz", "dyz")


def desc(name, with_closure=True):
    e = SCHEMES[name]
    d = {"deriv": e["d"], "order": e["order"], "a": e["a"], "rhs": e["rhs"]}
    if with_closure:
        d["closure"] = e["closure"]
    return d


def oracle_sch(name):
    from oracle import cfd as C
    e = SCHEMES[name]
    return C.Sch(e["d"], e["a"], tuple(e["rhs"]), tuple(e["closure"]))


def rel_max(got, want):
    """max |got - want| / max |want| (the error metric of the parity tests)."""
    den = np.abs(want).max()
    return float(np.abs(np.asarray(got, np.float64) - want).max() / (den if den > 0 else 1.0))


def uniform_blocks_from_oracle(ext):
    """(nbz, nby, nbx, E, E, E) -> list of per-block (E,E,E) arrays in block index order."""
    nbz, nby, nbx = ext.shape[:3]
    return [ext[bz, by, bx] for bz in range(nbz) for by in range(nby) for bx in range(nbx)]


def pack_fields(per_field_ext):
    """list over fields of (nbz, nby, nbx, E,E,E) -> flat buffer [block][field][E^3]."""
    nf = len(per_field_ext)
    nbz, nby, nbx = per_field_ext[0].shape[:3]
    E = per_field_ext[0].shape[-1]
    arr = np.stack(per_field_ext, axis=3)          # (nbz, nby, nbx, nf, E, E, E)
    return np.ascontiguousarray(arr.reshape(nbz * nby * nbx, nf, E, E, E)).reshape(-1)


def unpack_out(flat, nblocks, nf, nops, N):
    return flat.reshape(nblocks, nf, nops, N, N, N)


def oracle_out_to_blocks(res_op, N):
    """(nbz, nby, nbx, N,N,N) -> (nblocks, N,N,N)."""
    nbz, nby, nbx = res_op.shape[:3]
    return res_op.reshape(nbz * nby * nbx, N, N, N)


def wavenumber(name, eta):
    """eta~^d of a centred scheme (Eq. fdpwerrdef written out for alpha^(d) = (a, 1, a))."""
    e = SCHEMES[name]
    M = (len(e["rhs"]) - 1) // 2
    num = sum(e["rhs"][i] * np.exp(1j * (i - M) * eta) for i in range(2 * M + 1))
    den = 1 + 2 * e["a"] * np.cos(eta)
    return (num / den / (1j ** e["d"])).real
