"""Helpers shared by the GPU parity tests (marshalling only, no arithmetic)."""
import numpy as np
import pytest


def load_ppl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2010_08454_gb300 as ppl
    ppl.lib()
    return ppl


def gpu_is(ppl, x, y, N, seed, **model_kw):
    import torch
    model = ppl.poly_model(**model_kw)
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    yd = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float32)).cuda()
    lw = torch.empty(N, dtype=torch.float32, device="cuda")
    parts = ppl.poly_particles(N)
    ws = ppl.workspace(model, N, len(x))
    res = ppl.read_result(ppl.ppl_infer_is(model, xd, yd, N, seed, lw_out=lw,
                                           particles_out=parts, ws=ws))
    c, n, origin = ppl.decode_particles(parts)
    return res, lw.cpu().numpy(), n.cpu().numpy(), c.cpu().numpy(), origin.cpu().numpy()
