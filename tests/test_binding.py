"""CPU checks of the ctypes binding's marshalling: with the library replaced by a recorder, every
wrapper passes the handle, the tensors' device addresses, the workspace size, the 2S coefficient
descriptor and the stream through unchanged (no GPU and no arithmetic involved)."""
import pytest


@pytest.fixture()
def rec(monkeypatch):
    from paper_2302_14858_gb300 import build
    build.build()
    from paper_2302_14858_gb300 import cfd
    calls = []

    class Recorder:
        def __getattr__(self, name):
            def f(*args):
                calls.append((name, args))
                return 0
            return f

    monkeypatch.setattr(cfd, "_lib", Recorder())
    B = cfd.Blocks.__new__(cfd.Blocks)
    B.handle = 0            # falsy: the wrapper's destructor releases nothing
    return cfd, calls, B


def _tensors():
    import torch
    return torch.zeros(16, dtype=torch.float64), torch.zeros(4, dtype=torch.float64), \
        torch.zeros(64, dtype=torch.uint8)


def test_apply_and_advect_pass_addresses_sizes_and_stream(rec):
    cfd, calls, B = rec
    f, o, w = _tensors()
    cfd.cfd_apply(B, f, 2, cfd.CFD_OP_ALL, cfd.CFD_TC_BF16_EXACT, 1, o, w, 7)
    cfd.cfd_apply(B, f, 2, cfd.CFD_OP_DX, 0, 0, o, 0xABC0, 7, work_bytes=4096)
    cfd.cfd_advect(B, f, 1, o, 0, 1, o, None, 9)
    cfd.cfd_apply_biased(B, f, 1, cfd.CFD_OP_DY, -1, 0, 2, o, w, 5)
    assert calls[0] == ("cfd_apply", (0, f.data_ptr(), 2, 0x1FF, cfd.CFD_TC_BF16_EXACT, 1, o.data_ptr(),
                                      w.data_ptr(), 64, 7))
    assert calls[1][1][7:] == (0xABC0, 4096, 7)
    assert calls[2] == ("cfd_advect", (0, f.data_ptr(), 1, o.data_ptr(), 0, 1, o.data_ptr(), None, 0, 9))
    assert calls[3][1][3:] == (cfd.CFD_OP_DY, -1, 0, 2, o.data_ptr(), w.data_ptr(), 64, 5)


def test_lsrk_descriptor_reaches_the_library(rec):
    cfd, calls, B = rec
    f, o, w = _tensors()
    coef = ([0.0, -0.5], [1.0, 0.25], [0.5, 0.75], [1.0, 2.0])
    seen = []

    def grab(name, args):
        d = next(a._obj for a in args if hasattr(a, "_obj") and isinstance(a._obj, cfd.LsrkDesc))
        seen.append((name, d.stages, [[p[i] for i in range(d.stages)] for p in (d.gamma1, d.gamma2, d.beta,
                                                                                  d.delta)]))

    cfd.cfd_wave_lsrk_step(B, f, f, 0.1, coef, 0.04, 4, 0, 0, w, 3)
    grab(*calls[-1])
    cfd.cfd_shifted_wave_lsrk_step(B, f, f, o, 0.1, coef, 0.04, 4, 0, 1, w, 3)
    grab(*calls[-1])
    cfd.cfd_advect_lsrk_step(B, f, 1, o, 0.1, coef, 0.0, 4, 0, 1, w, 3)
    grab(*calls[-1])
    assert [s[0] for s in seen] == ["cfd_wave_lsrk_step", "cfd_shifted_wave_lsrk_step", "cfd_advect_lsrk_step"]
    for _, m, arrays in seen:
        assert m == 2 and arrays == [list(c) for c in coef]
    with pytest.raises(ValueError):
        cfd.cfd_advect_lsrk_step(B, f, 1, o, 0.1, ([0.0], [1.0, 0.5], [0.5], [1.0]), 0.0, 4, 0, 1, w, 3)


def test_raw_workspace_address_without_size_is_refused(rec):
    cfd, calls, B = rec
    f, o, _ = _tensors()
    with pytest.raises(ValueError):
        cfd.cfd_apply(B, f, 1, cfd.CFD_OP_DX, 0, 0, o, 0xABC0, 7)
    assert calls == []
