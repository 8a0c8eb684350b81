"""CPU-side checks of the C-ABI library: it builds, loads, exports every
declared symbol, and rejects bad host arguments before touching a GPU."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cfd():
    from paper_2302_14858_gb300 import build
    build.build()
    from paper_2302_14858_gb300 import cfd as c
    return c


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", fn)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:cfd_status|void|const char \*|unsigned long long)\s*\**\s*(cfd_\w+)\s*\(", txt, re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol(cfd):
    names = declared_symbols()
    assert len(names) >= 12
    for n in names:
        assert hasattr(cfd._lib, n), n
    assert set(cfd.EXPORTS) <= names


def test_scheme_create_rejects_bad_input(cfd):
    from tests.helpers import desc
    good = desc("Q13_1_d1")
    bad = dict(good, deriv=2)
    with pytest.raises(cfd.CfdError) as e:
        cfd.cfd_scheme_create(bad, None)
    assert e.value.status == cfd.CFD_ERR_ARG
    bad = dict(good, a=0.5)
    with pytest.raises(cfd.CfdError):
        cfd.cfd_scheme_create(bad, None)
    bad = dict(good, rhs=[0.1, -0.05, -0.78, 0.0, 0.78, 0.05, -0.002])   # not antisymmetric
    with pytest.raises(cfd.CfdError):
        cfd.cfd_scheme_create(bad, None)
    with pytest.raises(cfd.CfdError):
        cfd.cfd_scheme_create(None, None)


@pytest.mark.parametrize("name", ["P1_d1", "P2_d1", "P3_d1", "P1_d2", "P2_d2", "P3_d2", "Q13_1_d1", "Q13_1_d2",
                                  "Q13_4pi5_d1", "Q13_4pi5_d2"])
def test_library_closure_matches_oracle(cfd, name):
    """cfd_scheme_create with closure=NULL builds the C_0-matched closure; the oracle derived it independently."""
    from tests.helpers import SCHEMES, desc
    d = desc(name, with_closure=False)
    first, second = (d, None) if d["deriv"] == 1 else (None, d)
    s = cfd.cfd_scheme_create(first, second)
    got = cfd.cfd_scheme_closure(s, d["deriv"])
    want = SCHEMES[name]["closure"]
    assert len(got) == len(want)
    for g_, w in zip(got, want):
        assert abs(g_ - w) <= 4e-16 * max(1.0, abs(w)) + 1e-18


def test_bind_rejects_bad_layout(cfd):
    from tests.helpers import desc
    from paper_2302_14858_gb300 import workloads as W
    s = cfd.cfd_scheme_create(desc("Q13_1_d1"), desc("Q13_1_d2"))
    m = W.uniform_mesh(32, 16, 4)
    with pytest.raises(cfd.CfdError) as e:
        cfd.cfd_blocks_bind(s, [12] * m.nblocks, m.dx, m.neighbors, 4, cfd.CFD_F64)
    assert e.value.status == cfd.CFD_ERR_UNSUPPORTED
    with pytest.raises(cfd.CfdError):
        cfd.cfd_blocks_bind(s, m.n, m.dx, m.neighbors, 3, cfd.CFD_F64)      # ghosts too narrow
    bad = m.neighbors.copy()
    bad[0, 0] = m.nblocks + 5
    with pytest.raises(cfd.CfdError):
        cfd.cfd_blocks_bind(s, m.n, m.dx, bad, 4, cfd.CFD_F64)
    n = list(m.n)
    n[1] = 32                                     # neighbour of a different size
    with pytest.raises(cfd.CfdError):
        cfd.cfd_blocks_bind(s, n, m.dx, m.neighbors, 4, cfd.CFD_F64)


def test_workspace_size_of_a_raw_address_must_be_given(cfd):
    """A workspace passed as a raw device address carries no size: the binding asks for it
    instead of reporting an unchecked one to the library."""
    assert cfd._nbytes(None) == 0
    assert cfd._nbytes(0x7F0000000000, 4096) == 4096
    with pytest.raises(ValueError):
        cfd._nbytes(0x7F0000000000)
