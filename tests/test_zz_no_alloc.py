"""The workspace-free resampler, for callers that cannot allocate device memory
(a plugin whose host owns every device allocation, a real-time loop that must
not stall on cudaMalloc).  It is called through the C ABI and must return the
same ancestors as ppl_resample, bit for bit, on two calls in a row (the second
call reuses the static scratch the first one left behind)."""
import ctypes

import numpy as np
import pytest

import synth
from gpu_util import load_ppl

pytestmark = pytest.mark.gpu


def test_noalloc_resample_matches_workspace_resample_twice():
    import torch
    ppl = load_ppl()
    lib = ppl.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [("lw", 262147, 262147, synth.log_weights(262147, 5, "normal", scale=4.0)),
             ("lw", 262147, 100003, synth.log_weights(262147, 7, "sparse", scale=4.0)),
             ("q", 1 << 20, 777777, synth.fixed_weights(1 << 20, 6))]
    for call in range(2):
        for kind, n, m, data in cases:
            t = torch.from_numpy(np.ascontiguousarray(
                data if kind == "lw" else data.view(np.int64))).cuda()
            lw = t if kind == "lw" else None
            q = t if kind == "q" else None
            ref = ppl.ppl_resample(m, 9, instance=1, t=call, lw=lw, q_fixed=q)
            anc = torch.full((m,), -7, dtype=torch.int32, device="cuda")
            st = lib.ppl_resample_noalloc(
                ctypes.c_void_p(lw.data_ptr()) if lw is not None else None,
                ctypes.c_void_p(q.data_ptr()) if q is not None else None, n, m,
                ctypes.c_uint64(9), 1, call, ctypes.c_void_p(anc.data_ptr()), stream)
            assert st == ppl.PPL_OK
            assert lib.ppl_resample_noalloc_status(stream) == ppl.PPL_OK
            assert torch.equal(anc, ref), (call, kind)
    # every weight zero: the device reports PPL_EEMPTY through the status call,
    # and the next call, which clears the status word, reports PPL_OK again
    dead = torch.full((5000,), float("-inf"), dtype=torch.float32, device="cuda")
    anc = torch.empty(5000, dtype=torch.int32, device="cuda")
    assert lib.ppl_resample_noalloc(ctypes.c_void_p(dead.data_ptr()), None, 5000, 5000,
                                    ctypes.c_uint64(1), 0, 0, ctypes.c_void_p(anc.data_ptr()),
                                    stream) == ppl.PPL_OK
    assert lib.ppl_resample_noalloc_status(stream) == ppl.PPL_EEMPTY
    live = torch.zeros(5000, dtype=torch.float32, device="cuda")
    assert lib.ppl_resample_noalloc(ctypes.c_void_p(live.data_ptr()), None, 5000, 5000,
                                    ctypes.c_uint64(1), 0, 0, ctypes.c_void_p(anc.data_ptr()),
                                    stream) == ppl.PPL_OK
    assert lib.ppl_resample_noalloc_status(stream) == ppl.PPL_OK
    assert torch.equal(anc, ppl.ppl_resample(5000, 1, lw=live))
    # beyond the static scratch: rejected before any work
    big = torch.zeros((1 << 20) + 1, dtype=torch.float32, device="cuda")
    out = torch.empty(16, dtype=torch.int32, device="cuda")
    assert lib.ppl_resample_noalloc(ctypes.c_void_p(big.data_ptr()), None, big.numel(), 16,
                                    ctypes.c_uint64(0), 0, 0, ctypes.c_void_p(out.data_ptr()),
                                    stream) == ppl.PPL_EINVAL
