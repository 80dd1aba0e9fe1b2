"""The C ABI library loads, exports every symbol include/ppl.h declares, and
rejects bad arguments on the host (no GPU needed: nothing here launches work)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ppl_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def ppl():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2010_08454_gb300 as ppl
    return ppl


def test_exports_every_declared_symbol(ppl):
    names = _declared("ppl.h")
    assert "ppl_infer_is" in names and "ppl_resample" in names
    lib = ctypes.CDLL(ppl.binding.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(ppl.exported_symbols()) == names


def test_status_strings(ppl):
    assert ppl.ppl_status_string(0) == "ok"
    assert ppl.ppl_status_string(4) == "NaN log-weight"
    assert ppl.ppl_status_string(6) == "bounded device wait expired"
    assert ppl.ppl_status_string(99) == "unknown status"


def test_workspace_size(ppl):
    m = ppl.poly_model()
    a = ppl.ppl_workspace_size(m, 1000, 32)
    b = ppl.ppl_workspace_size(m, 1 << 24, 256)
    assert 0 < a < b
    assert b >= (1 << 24) * (8 + 4)  # prefix sums + log-weights
    assert ppl.ppl_workspace_size(m, 0, 32) == 0
    assert ppl.ppl_workspace_size(m, 1 << 31, 32) == 0


def test_host_side_argument_checks(ppl):
    lib = ppl.lib()
    m = ppl.poly_model()
    bad = ppl.poly_model(min_deg=2, max_deg=7)  # five degrees: more than four
    data = ppl.PplData(None, None, 0)
    # invalid model, null result, null workspace: rejected before any CUDA call
    assert lib.ppl_infer_is(ctypes.byref(bad), ctypes.byref(data), 10, 0, ctypes.c_void_p(256),
                            None, None, ctypes.c_void_p(256), 1 << 30, None) == ppl.PPL_EINVAL
    assert lib.ppl_infer_is(ctypes.byref(m), ctypes.byref(data), 10, 0, None, None, None,
                            ctypes.c_void_p(256), 1 << 30, None) == ppl.PPL_EINVAL
    assert lib.ppl_infer_is(ctypes.byref(m), ctypes.byref(data), 10, 0, ctypes.c_void_p(256),
                            None, None, None, 1 << 30, None) == ppl.PPL_EINVAL
    # misaligned or too-small workspace
    assert lib.ppl_infer_is(ctypes.byref(m), ctypes.byref(data), 10, 0, ctypes.c_void_p(256),
                            None, None, ctypes.c_void_p(264), 1 << 30, None) == ppl.PPL_EINVAL
    assert lib.ppl_infer_is(ctypes.byref(m), ctypes.byref(data), 10, 0, ctypes.c_void_p(256),
                            None, None, ctypes.c_void_p(256), 100, None) == ppl.PPL_EINVAL
    # discrete benchmarks: unknown model, limit out of range, null result
    for model, limit in [(7, 3), (1, 64), (1, -1), (2, 0), (2, 64)]:
        assert lib.ppl_infer_discrete(model, None, 0, limit, 10, 0, ctypes.c_void_p(256), None,
                                      None, ctypes.c_void_p(256), 1 << 30,
                                      None) == ppl.PPL_EINVAL
    assert lib.ppl_infer_discrete(1, None, 0, 3, 10, 0, None, None, None, ctypes.c_void_p(256),
                                  1 << 30, None) == ppl.PPL_EINVAL
    # customdist: invalid weight or scale
    for kw in [dict(w1=1.5), dict(sigma1=0.0), dict(obs_sigma=-1.0)]:
        cm = ppl.customdist_model(**kw)
        assert lib.ppl_infer_customdist(ctypes.byref(cm), None, 0, 10, 0, ctypes.c_void_p(256),
                                        None, None, ctypes.c_void_p(256), 1 << 30,
                                        None) == ppl.PPL_EINVAL
    # resample needs exactly one of lw / q_fixed
    assert lib.ppl_resample(None, None, 10, 10, 0, 0, 0, ctypes.c_void_p(256),
                            ctypes.c_void_p(256), 1 << 30, None) == ppl.PPL_EINVAL
    assert lib.ppl_resample(ctypes.c_void_p(256), ctypes.c_void_p(512), 10, 10, 0, 0, 0,
                            ctypes.c_void_p(256), ctypes.c_void_p(256), 1 << 30,
                            None) == ppl.PPL_EINVAL
    # smc step wants the state-space model and t >= 1
    lg = ppl.lgssm_model()
    args = [ctypes.c_void_p(256)] * 5
    assert lib.ppl_smc_step(ctypes.byref(m), 0.0, 1, 0, args[0], args[1], 10, args[2], args[3],
                            args[4], ctypes.c_void_p(256), 1 << 30, None) == ppl.PPL_EINVAL
    assert lib.ppl_smc_step(ctypes.byref(lg), 0.0, 0, 0, args[0], args[1], 10, args[2], args[3],
                            args[4], ctypes.c_void_p(256), 1 << 30, None) == ppl.PPL_EINVAL
    assert lib.ppl_gather(None, 10, 4, None, 10, None, None) == ppl.PPL_EINVAL
    # resample + gather: lw, both record buffers and a positive stride required
    v = ctypes.c_void_p(256)
    for lw_, si, so, st in [(None, v, v, 32), (v, None, v, 32), (v, v, None, 32), (v, v, v, 0)]:
        assert lib.ppl_resample_gather(lw_, None, 10, 10, 0, 0, 0, si, st, so, v, v, 1 << 30,
                                       None) == ppl.PPL_EINVAL
    assert lib.ppl_rng_words(0, 0, 0, 1, 10, 2, ctypes.c_void_p(8), None) == ppl.PPL_EINVAL
