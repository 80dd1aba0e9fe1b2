"""Python binding of libppl.so (include/ppl.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: PyTorch provides device memory and the current CUDA
stream, the library does the work.  If libppl.so has not been built the
binding raises; there is no CPU fallback.
"""
import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libppl.so")
_LIB = None

PPL_OK, PPL_EINVAL, PPL_ENOMEM, PPL_ECUDA, PPL_ENAN, PPL_EEMPTY, PPL_ETIMEOUT = range(7)
PPL_MODEL_POLY, PPL_MODEL_LGSSM = 1, 2
POLY_RECORD_FLOATS = 8  # ppl_poly_particle: c[6], n (int32 bits), origin (uint32 bits)


class PplError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {ppl_status_string(status)} ({status})")


class PplModel(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int32), ("min_deg", ctypes.c_int32),
                ("max_deg", ctypes.c_int32), ("coef_offset", ctypes.c_int32),
                ("obs_sigma", ctypes.c_float), ("prior_sigma", ctypes.c_float),
                ("phi", ctypes.c_float), ("q_sigma", ctypes.c_float)]


class PplData(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("len", ctypes.c_int64)]


class PplIsResult(ctypes.Structure):
    _fields_ = [("log_z", ctypes.c_double), ("lse", ctypes.c_double), ("ess", ctypes.c_double),
                ("max_lw", ctypes.c_double), ("argmax", ctypes.c_int64),
                ("n_particles", ctypes.c_int64), ("map_deg", ctypes.c_int32),
                ("n_deg", ctypes.c_int32), ("p_n", ctypes.c_double * 4),
                ("mean_c", ctypes.c_double * 6), ("deg_mean", (ctypes.c_double * 6) * 4),
                ("deg_var", (ctypes.c_double * 6) * 4), ("deg_max_lw", ctypes.c_double * 4),
                ("deg_argmax", ctypes.c_int64 * 4), ("status", ctypes.c_int32),
                ("pad", ctypes.c_int32)]

    def as_dict(self):
        return {
            "log_z": self.log_z, "lse": self.lse, "ess": self.ess, "max_lw": self.max_lw,
            "argmax": self.argmax, "n_particles": self.n_particles, "map_deg": self.map_deg,
            "n_deg": self.n_deg, "p_n": np.array(self.p_n[:]),
            "mean_c": np.array(self.mean_c[:]),
            "deg_mean": np.array([r[:] for r in self.deg_mean]),
            "deg_var": np.array([r[:] for r in self.deg_var]),
            "deg_max_lw": np.array(self.deg_max_lw[:]),
            "deg_argmax": np.array(self.deg_argmax[:]), "status": self.status,
        }


RESULT_BYTES = ctypes.sizeof(PplIsResult)
PARTIAL_BYTES = 384  # ppl_is_partial

class PplCustomdistModel(ctypes.Structure):
    _fields_ = [("w1", ctypes.c_float), ("mu1", ctypes.c_float), ("sigma1", ctypes.c_float),
                ("mu2", ctypes.c_float), ("sigma2", ctypes.c_float), ("obs_sigma", ctypes.c_float)]


class PplCustomdistResult(ctypes.Structure):
    _fields_ = [("log_z", ctypes.c_double), ("lse", ctypes.c_double), ("ess", ctypes.c_double),
                ("max_lw", ctypes.c_double), ("mean_x", ctypes.c_double),
                ("var_x", ctypes.c_double), ("n_particles", ctypes.c_int64),
                ("status", ctypes.c_int32), ("pad", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


def customdist_model(w1=0.3, mu1=-2.0, sigma1=0.5, mu2=1.5, sigma2=1.0, obs_sigma=1.0):
    return PplCustomdistModel(w1, mu1, sigma1, mu2, sigma2, obs_sigma)


PPL_DISCRETE_MAX_VALUES = 64
DISCRETE_MODELS = {"biasedcoin": 0, "binomial": 1, "geometric": 2}


class PplDiscreteResult(ctypes.Structure):
    _fields_ = [("log_z", ctypes.c_double), ("ess", ctypes.c_double),
                ("max_lw", ctypes.c_double), ("mean", ctypes.c_double),
                ("n_particles", ctypes.c_int64), ("n_values", ctypes.c_int32),
                ("status", ctypes.c_int32), ("value", ctypes.c_double * PPL_DISCRETE_MAX_VALUES),
                ("prob", ctypes.c_double * PPL_DISCRETE_MAX_VALUES),
                ("count", ctypes.c_int64 * PPL_DISCRETE_MAX_VALUES)]

    def as_dict(self):
        n = self.n_values
        return {"log_z": self.log_z, "ess": self.ess, "max_lw": self.max_lw, "mean": self.mean,
                "n_particles": self.n_particles, "n_values": n, "status": self.status,
                "value": np.array(self.value[:n]), "prob": np.array(self.prob[:n]),
                "count": np.array(self.count[:n])}


class PplResamplePlan(ctypes.Structure):
    _fields_ = [("total", ctypes.c_uint64), ("stride", ctypes.c_uint64),
                ("offset", ctypes.c_uint64), ("c_base", ctypes.c_uint64),
                ("k_first", ctypes.c_int64), ("k_end", ctypes.c_int64),
                ("m", ctypes.c_int64), ("n_total", ctypes.c_int64)]


class PplBatchPlan(ctypes.Structure):
    _fields_ = [("ppt", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("n_inst", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("n_items", ctypes.c_int64), ("max_len", ctypes.c_int64),
                ("total_particles", ctypes.c_int64), ("work", ctypes.c_double)]

_SIGS = {
    "ppl_status_string": (ctypes.c_char_p, [ctypes.c_int32]),
    "ppl_workspace_size": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64]),
    "ppl_workspace_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "ppl_infer_is": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                    ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                    ctypes.c_void_p]),
    "ppl_infer_is_instance": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                             ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_size_t, ctypes.c_void_p]),
    "ppl_infer_is_suffstat": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                             ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_size_t, ctypes.c_void_p]),
    "ppl_gemm_bf16": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                     ctypes.c_void_p]),
    "ppl_infer_customdist": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                            ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_size_t, ctypes.c_void_p]),
    "ppl_infer_discrete": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "ppl_infer_is_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                         ctypes.c_void_p]),
    "ppl_logsumexp": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "ppl_resample": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                    ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                                    ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_size_t, ctypes.c_void_p]),
    "ppl_resample_known_max": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                              ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                                              ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_size_t, ctypes.c_void_p]),
    "ppl_selftest_scan_timeout": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                                 ctypes.c_void_p, ctypes.c_size_t,
                                                 ctypes.c_void_p]),
    "ppl_resample_gather": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                                           ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_size_t, ctypes.c_void_p]),
    "ppl_gather": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                  ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                  ctypes.c_void_p]),
    "ppl_smc_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_float, ctypes.c_int32,
                                    ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                    ctypes.c_void_p]),
    "ppl_smc_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                   ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                   ctypes.c_void_p]),
    "ppl_grid_barrier_probe": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                              ctypes.c_size_t, ctypes.c_void_p]),
    "ppl_rng_words": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                     ctypes.c_uint32, ctypes.c_int64, ctypes.c_int32,
                                     ctypes.c_void_p, ctypes.c_void_p]),
    "ppl_resample_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                            ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                                            ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]),
    "ppl_resample_noalloc_status": (ctypes.c_int, [ctypes.c_void_p]),
    "ppl_batched_workspace_size": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_void_p,
                                                     ctypes.c_int32, ctypes.c_int32]),
    "ppl_batched_prepare": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                           ctypes.c_void_p]),
    "ppl_infer_is_batched": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                            ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "ppl_batched_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                            ctypes.c_char_p, ctypes.c_void_p, ctypes.c_void_p]),
    "ppl_batched_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "ppl_proposal_num_params": (ctypes.c_int64, []),
    "ppl_proposal_workspace_size": (ctypes.c_size_t, [ctypes.c_int32]),
    "ppl_proposal_features": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                             ctypes.c_void_p, ctypes.c_void_p]),
    "ppl_proposal_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "ppl_proposal_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                         ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                         ctypes.c_void_p]),
    "ppl_proposal_train": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_uint64, ctypes.c_float,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                          ctypes.c_void_p]),
    "ppl_proposal_train_init": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                               ctypes.c_size_t, ctypes.c_void_p]),
    "ppl_proposal_train_steps": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                                ctypes.c_int32, ctypes.c_uint64, ctypes.c_float,
                                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                                ctypes.c_void_p]),
    "ppl_infer_is_learned": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                            ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                            ctypes.c_void_p]),
    "ppl_posterior_reduce": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_size_t, ctypes.c_void_p]),
    "ppl_infer_is_partial": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                            ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "ppl_is_merge": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                    ctypes.c_void_p]),
    "ppl_resample_shard_total": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                                ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_size_t, ctypes.c_void_p]),
    "ppl_resample_shard_plan": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                               ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                                               ctypes.c_uint32, ctypes.c_void_p]),
    "ppl_resample_shard": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
}


def exported_symbols():
    """Names the binding expects libppl.so to export."""
    return list(_SIGS)


def lib():
    """Load libppl.so; raises if it has not been built (no fallback)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libppl.so is not built ({LIB_PATH}); run "
                               "paper_2010_08454_gb300/build.py or __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _check(status, where):
    if status != PPL_OK:
        raise PplError(status, where)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_f32(t, name):
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    return t


def ppl_status_string(status):
    return lib().ppl_status_string(int(status)).decode()


def poly_model(min_deg=2, max_deg=5, coef_offset=1, obs_sigma=0.5, prior_sigma=10.0):
    return PplModel(PPL_MODEL_POLY, min_deg, max_deg, coef_offset, obs_sigma, prior_sigma, 0.0,
                    0.0)


def lgssm_model(phi=0.9, q_sigma=1.0, obs_sigma=0.5):
    return PplModel(PPL_MODEL_LGSSM, 0, 0, 0, obs_sigma, 0.0, phi, q_sigma)


def ppl_workspace_size(model, n_particles, data_len=0):
    return int(lib().ppl_workspace_size(ctypes.byref(model), int(n_particles), int(data_len)))


def workspace(model, n_particles, data_len=0, device="cuda"):
    """A device workspace big enough for every call on this many particles."""
    n = ppl_workspace_size(model, n_particles, data_len)
    if n == 0:
        raise ValueError("invalid workspace request")
    return torch.empty(n, dtype=torch.uint8, device=device)


def ppl_workspace_status(ws, stream=None):
    return int(lib().ppl_workspace_status(_ptr(ws), _stream(stream)))


def result_tensor(device="cuda"):
    return torch.zeros(RESULT_BYTES, dtype=torch.uint8, device=device)


def read_result(res_dev):
    """Copy a device ppl_is_result to the host (synchronises) and decode it."""
    raw = res_dev.detach().cpu().numpy().tobytes()
    return PplIsResult.from_buffer_copy(raw).as_dict()


def ppl_infer_is(model, x, y, n_particles, seed, out=None, lw_out=None, particles_out=None,
                 ws=None, stream=None):
    """Likelihood weighting on the line-fitting model; returns the device result buffer."""
    _dev_f32(x, "x")
    _dev_f32(y, "y")
    if ws is None:
        ws = workspace(model, n_particles, x.numel(), x.device)
    if out is None:
        out = result_tensor(x.device)
    data = PplData(x.data_ptr(), y.data_ptr(), x.numel())
    st = lib().ppl_infer_is(ctypes.byref(model), ctypes.byref(data), int(n_particles),
                            ctypes.c_uint64(seed), _ptr(out), _ptr(lw_out), _ptr(particles_out),
                            _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "ppl_infer_is")
    return out


def ppl_infer_is_instance(model, x, y, n_particles, seed, instance, out=None, lw_out=None,
                          particles_out=None, ws=None, stream=None):
    """ppl_infer_is with the counter field `instance` set (independent instances)."""
    _dev_f32(x, "x")
    _dev_f32(y, "y")
    if ws is None:
        ws = workspace(model, n_particles, x.numel(), x.device)
    if out is None:
        out = result_tensor(x.device)
    data = PplData(x.data_ptr(), y.data_ptr(), x.numel())
    st = lib().ppl_infer_is_instance(ctypes.byref(model), ctypes.byref(data), int(n_particles),
                                     ctypes.c_uint64(seed), int(instance), _ptr(out),
                                     _ptr(lw_out), _ptr(particles_out), _ptr(ws), ws.numel(),
                                     _stream(stream))
    _check(st, "ppl_infer_is_instance")
    return out


def ppl_infer_is_suffstat(model, x, y, n_particles, seed, instance=0, out=None, lw_out=None,
                          particles_out=None, ws=None, stream=None):
    """ppl_infer_is_instance with the factor from the data's sufficient statistics."""
    _dev_f32(x, "x")
    _dev_f32(y, "y")
    if ws is None:
        ws = workspace(model, n_particles, x.numel(), x.device)
    if out is None:
        out = result_tensor(x.device)
    data = PplData(x.data_ptr(), y.data_ptr(), x.numel())
    st = lib().ppl_infer_is_suffstat(ctypes.byref(model), ctypes.byref(data), int(n_particles),
                                     ctypes.c_uint64(seed), int(instance), _ptr(out),
                                     _ptr(lw_out), _ptr(particles_out), _ptr(ws), ws.numel(),
                                     _stream(stream))
    _check(st, "ppl_infer_is_suffstat")
    return out


def ppl_gemm_bf16(A, B, M, N, K, sam, sak, sbn, sbk, C=None, ws=None, stream=None):
    """C[m, n] = sum_k A[m sam + k sak] B[n sbn + k sbk] on the tensor cores (BF16 in, FP32 out)."""
    if A.dtype != torch.bfloat16 or B.dtype != torch.bfloat16:
        raise TypeError("A and B must be bfloat16")
    if ws is None:
        ws = workspace(poly_model(), 1, 0)
    if C is None:
        C = torch.empty((M, N), dtype=torch.float32, device=A.device)
    st = lib().ppl_gemm_bf16(_ptr(A), sam, sak, _ptr(B), sbn, sbk, M, N, K, _ptr(C), _ptr(ws),
                             ws.numel(), _stream(stream))
    _check(st, "ppl_gemm_bf16")
    return C, ws


def ppl_infer_customdist(model, y, n_particles, seed, x_out=None, lw_out=None, ws=None,
                         stream=None):
    """Likelihood weighting on customdist; returns the decoded result."""
    if y is not None and y.numel() > 0:
        _dev_f32(y, "y")
    if ws is None:
        ws = workspace(poly_model(), n_particles, 0)
    out = torch.zeros(ctypes.sizeof(PplCustomdistResult), dtype=torch.uint8, device=ws.device)
    n = 0 if y is None else y.numel()
    st = lib().ppl_infer_customdist(ctypes.byref(model), _ptr(y) if n else None, n,
                                    int(n_particles), ctypes.c_uint64(seed), _ptr(out),
                                    _ptr(x_out), _ptr(lw_out), _ptr(ws), ws.numel(),
                                    _stream(stream))
    _check(st, "ppl_infer_customdist")
    return PplCustomdistResult.from_buffer_copy(out.cpu().numpy().tobytes()).as_dict()


def ppl_infer_discrete(model, n_particles, seed, flips=None, limit=0, codes_out=None,
                       lw_out=None, ws=None, stream=None):
    """Likelihood weighting on a tiny discrete benchmark; returns the decoded result."""
    m = DISCRETE_MODELS[model] if isinstance(model, str) else int(model)
    if ws is None:
        ws = workspace(poly_model(), 1, 0)
    out = torch.zeros(ctypes.sizeof(PplDiscreteResult), dtype=torch.uint8, device=ws.device)
    n_flips = 0 if flips is None else flips.numel()
    st = lib().ppl_infer_discrete(m, _ptr(flips), n_flips, int(limit), int(n_particles),
                                  ctypes.c_uint64(seed), _ptr(out), _ptr(codes_out), _ptr(lw_out),
                                  _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "ppl_infer_discrete")
    raw = out.cpu().numpy().tobytes()
    return PplDiscreteResult.from_buffer_copy(raw).as_dict()


def ppl_infer_is_host(model, x_host, y_host, n_particles, seed, ws, stream=None):
    """The same with host (preferably pinned) inputs and a host result; synchronises."""
    res = PplIsResult()
    st = lib().ppl_infer_is_host(ctypes.byref(model), ctypes.c_void_p(x_host.data_ptr()),
                                 ctypes.c_void_p(y_host.data_ptr()), x_host.numel(),
                                 int(n_particles), ctypes.c_uint64(seed), ctypes.byref(res),
                                 _ptr(ws), ws.numel(), _stream(stream))
    if st not in (PPL_OK, PPL_ENAN, PPL_EEMPTY, PPL_ETIMEOUT):
        _check(st, "ppl_infer_is_host")
    return res.as_dict()


def ppl_logsumexp(lw, out=None, ws=None, stream=None):
    """[LSE, ESS, max, argmax] in a float64 device tensor."""
    _dev_f32(lw, "lw")
    if ws is None:
        ws = workspace(poly_model(), lw.numel(), 0, lw.device)
    if out is None:
        out = torch.empty(4, dtype=torch.float64, device=lw.device)
    st = lib().ppl_logsumexp(_ptr(lw), lw.numel(), _ptr(out), _ptr(ws), ws.numel(),
                             _stream(stream))
    _check(st, "ppl_logsumexp")
    return out


def ppl_resample(m, seed, instance=0, t=0, lw=None, q_fixed=None, ancestors=None, ws=None,
                 stream=None):
    """Systematic resampling; returns int32 ancestors[m] on the device."""
    src = lw if lw is not None else q_fixed
    n = src.numel()
    if lw is not None:
        _dev_f32(lw, "lw")
    elif not (q_fixed.is_cuda and q_fixed.dtype in (torch.int64, torch.uint64)):
        raise ValueError("q_fixed must be a 64-bit integer CUDA tensor")
    if ws is None:
        ws = workspace(poly_model(), max(n, m), 0, src.device)
    if ancestors is None:
        ancestors = torch.empty(m, dtype=torch.int32, device=src.device)
    st = lib().ppl_resample(_ptr(lw), _ptr(q_fixed), n, int(m), ctypes.c_uint64(seed),
                            int(instance), int(t), _ptr(ancestors), _ptr(ws), ws.numel(),
                            _stream(stream))
    _check(st, "ppl_resample")
    return ancestors


def ppl_resample_known_max(m, seed, lw, max_lw_dev, instance=0, t=0, ancestors=None, ws=None,
                           stream=None):
    """ppl_resample from lw with its maximum already on the device (float64 scalar)."""
    _dev_f32(lw, "lw")
    n = lw.numel()
    if ws is None:
        ws = workspace(poly_model(), max(n, m), 0, lw.device)
    if ancestors is None:
        ancestors = torch.empty(m, dtype=torch.int32, device=lw.device)
    st = lib().ppl_resample_known_max(_ptr(lw), ctypes.c_void_p(max_lw_dev.data_ptr()), n,
                                      int(m), ctypes.c_uint64(seed), int(instance), int(t),
                                      _ptr(ancestors), _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "ppl_resample_known_max")
    return ancestors


def ppl_selftest_scan_timeout(q_fixed, max_spin, ws=None, stream=None):
    """Run the scan with a silent first tile; returns the device status (PPL_ETIMEOUT)."""
    n = q_fixed.numel()
    if ws is None:
        ws = workspace(poly_model(), n, 0, q_fixed.device)
    return int(lib().ppl_selftest_scan_timeout(_ptr(q_fixed), n, int(max_spin), _ptr(ws),
                                               ws.numel(), _stream(stream)))


def result_max_lw(res_dev):
    """The device float64 max_lw field of a ppl_is_result buffer (no copy)."""
    return res_dev[24:32].view(torch.float64)


def ppl_resample_gather(m, seed, lw, state_in, max_lw_dev=None, instance=0, t=0,
                        state_out=None, ancestors=None, ws=None, stream=None):
    """Resampling (as ppl_resample / ppl_resample_known_max) and the gather of
    the resampled records in one call; returns (ancestors, state_out)."""
    _dev_f32(lw, "lw")
    if not state_in.is_contiguous():
        raise ValueError("state_in must be contiguous")
    n = lw.numel()
    if state_in.shape[0] != n:
        raise ValueError("state_in must hold one record per particle")
    stride = state_in[0].numel() * state_in.element_size() if state_in.dim() > 1 else \
        state_in.element_size()
    if ws is None:
        ws = workspace(poly_model(), max(n, m), 0, lw.device)
    if ancestors is None:
        ancestors = torch.empty(m, dtype=torch.int32, device=lw.device)
    if state_out is None:
        state_out = torch.empty((m,) + tuple(state_in.shape[1:]), dtype=state_in.dtype,
                                device=state_in.device)
    mx = ctypes.c_void_p(max_lw_dev.data_ptr()) if max_lw_dev is not None else None
    st = lib().ppl_resample_gather(_ptr(lw), mx, n, int(m), ctypes.c_uint64(seed), int(instance),
                                   int(t), _ptr(state_in), stride, _ptr(state_out),
                                   _ptr(ancestors), _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "ppl_resample_gather")
    return ancestors, state_out


def ppl_gather(state_in, ancestors, state_out=None, stream=None):
    """state_out[k] = state_in[ancestors[k]] over the leading dimension."""
    if not state_in.is_contiguous():
        raise ValueError("state_in must be contiguous")
    m = ancestors.numel()
    stride = state_in[0].numel() * state_in.element_size() if state_in.dim() > 1 else \
        state_in.element_size()
    if state_out is None:
        state_out = torch.empty((m,) + tuple(state_in.shape[1:]), dtype=state_in.dtype,
                                device=state_in.device)
    st = lib().ppl_gather(_ptr(state_in), state_in.shape[0], stride, _ptr(ancestors), m,
                          _ptr(state_out), _stream(stream))
    _check(st, "ppl_gather")
    return state_out


def ppl_smc_step(model, y_t, t, seed, x, lw, logz_acc, resampled, logz_est, ws, stream=None):
    """One bootstrap-filter step on the device state (x, lw, logz_acc, resampled, logz_est)."""
    st = lib().ppl_smc_step(ctypes.byref(model), float(y_t), int(t), ctypes.c_uint64(seed),
                            _ptr(x), _ptr(lw), x.numel(), _ptr(logz_acc), _ptr(resampled),
                            _ptr(logz_est), _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "ppl_smc_step")


def ppl_smc_run(model, y, n, seed, ws=None, out=None, stream=None):
    """All T steps of the filter in one kernel; returns a dict of device tensors."""
    T = y.numel()
    dev = y.device
    if ws is None:
        ws = workspace(model, n, T, dev)
    if out is None:
        out = {"x": torch.empty(n, dtype=torch.float32, device=dev),
               "lw": torch.empty(n, dtype=torch.float32, device=dev),
               "log_z": torch.empty(1, dtype=torch.float64, device=dev),
               "resampled": torch.empty(T, dtype=torch.int32, device=dev),
               "ess": torch.empty(T, dtype=torch.float64, device=dev)}
    st = lib().ppl_smc_run(ctypes.byref(model), _ptr(y), T, ctypes.c_uint64(seed), int(n),
                           _ptr(out["x"]), _ptr(out["lw"]), _ptr(out["log_z"]),
                           _ptr(out["resampled"]), _ptr(out["ess"]), _ptr(ws), ws.numel(),
                           _stream(stream))
    _check(st, "ppl_smc_run")
    out["ws"] = ws
    return out


def ppl_grid_barrier_probe(blocks, n_barriers, ws=None, stream=None):
    """n_barriers grid barriers of the filter's kind, nothing else; returns ws."""
    if ws is None:
        ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    st = lib().ppl_grid_barrier_probe(int(blocks), int(n_barriers), _ptr(ws), ws.numel(),
                                      _stream(stream))
    _check(st, "ppl_grid_barrier_probe")
    return ws


def ppl_rng_words(seed, instance, step, purpose, n_particles, n_blocks, out=None, stream=None):
    """uint32 words [n_particles, n_blocks, 4] on the device (as int32 storage)."""
    if out is None:
        out = torch.empty((n_particles, n_blocks, 4), dtype=torch.int32, device="cuda")
    st = lib().ppl_rng_words(ctypes.c_uint64(seed), int(instance), int(step), int(purpose),
                             int(n_particles), int(n_blocks), _ptr(out), _stream(stream))
    _check(st, "ppl_rng_words")
    return out


def ppl_posterior_reduce(model, particles, lw=None, out=None, ws=None, stream=None):
    n = particles.shape[0]
    if ws is None:
        ws = workspace(model, n, 0, particles.device)
    if out is None:
        out = result_tensor(particles.device)
    st = lib().ppl_posterior_reduce(ctypes.byref(model), _ptr(particles), _ptr(lw), n,
                                    _ptr(out), _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "ppl_posterior_reduce")
    return out


def partial_tensor(n_partials=1, device="cuda"):
    """Device storage for n_partials ppl_is_partial records (16-byte aligned)."""
    return torch.zeros((n_partials, PARTIAL_BYTES), dtype=torch.uint8, device=device)


def ppl_infer_is_partial(model, x, y, first_particle, n_particles, seed, instance=0,
                         partial=None, lw_out=None, particles_out=None, ws=None, stream=None):
    """One shard's partial of likelihood weighting over particles
    [first_particle, first_particle + n_particles); returns the partial buffer."""
    _dev_f32(x, "x")
    _dev_f32(y, "y")
    if ws is None:
        ws = workspace(model, n_particles, x.numel(), x.device)
    if partial is None:
        partial = partial_tensor(1, x.device)
    data = PplData(x.data_ptr(), y.data_ptr(), x.numel())
    st = lib().ppl_infer_is_partial(ctypes.byref(model), ctypes.byref(data), int(first_particle),
                                    int(n_particles), ctypes.c_uint64(seed), int(instance),
                                    _ptr(partial), _ptr(lw_out), _ptr(particles_out), _ptr(ws),
                                    ws.numel(), _stream(stream))
    _check(st, "ppl_infer_is_partial")
    return partial


def ppl_is_merge(partials, out=None, stream=None):
    """The population's summary from its shards' partials [P, PARTIAL_BYTES] (device)."""
    if partials.dim() != 2 or partials.shape[1] != PARTIAL_BYTES or not partials.is_contiguous():
        raise ValueError("partials must be a contiguous [P, 384] uint8 device tensor")
    if out is None:
        out = result_tensor(partials.device)
    st = lib().ppl_is_merge(_ptr(partials), partials.shape[0], _ptr(out), _stream(stream))
    _check(st, "ppl_is_merge")
    return out


def ppl_resample_shard_total(lw, max_lw_dev, n_total, total=None, ws=None, stream=None):
    """This shard's sum of fixed-point weights (a uint64 device scalar, as int64 storage)."""
    _dev_f32(lw, "lw")
    if ws is None:
        ws = workspace(poly_model(), 1, 0, lw.device)
    if total is None:
        total = torch.zeros(1, dtype=torch.int64, device=lw.device)
    st = lib().ppl_resample_shard_total(_ptr(lw), lw.numel(), _ptr(max_lw_dev), int(n_total),
                                        _ptr(total), _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "ppl_resample_shard_total")
    return total


def ppl_resample_shard_plan(totals, n_total, m, seed, instance=0, t=0):
    """Host: every shard's plan from the shards' sums (uint64, shard order)."""
    tot = np.ascontiguousarray(np.asarray(totals, dtype=np.uint64))
    plans = (PplResamplePlan * len(tot))()
    st = lib().ppl_resample_shard_plan(tot.ctypes.data_as(ctypes.c_void_p), len(tot), int(n_total),
                                       int(m), ctypes.c_uint64(seed), int(instance), int(t), plans)
    _check(st, "ppl_resample_shard_plan")
    return list(plans)


def ppl_resample_shard(lw, first_particle, max_lw_dev, plan, ancestors=None, state_in=None,
                       state_out=None, ws=None, stream=None):
    """This shard's outputs [plan.k_first, plan.k_end): (ancestors, state_out)."""
    _dev_f32(lw, "lw")
    n_out = plan.k_end - plan.k_first
    if ws is None:
        ws = workspace(poly_model(), lw.numel(), 0, lw.device)
    if ancestors is None:
        ancestors = torch.empty(max(n_out, 1), dtype=torch.int32, device=lw.device)
    stride = 0
    if state_in is not None:
        if not state_in.is_contiguous():
            raise ValueError("state_in must be contiguous")
        stride = state_in[0].numel() * state_in.element_size() if state_in.dim() > 1 else \
            state_in.element_size()
        if state_out is None:
            state_out = torch.empty((max(n_out, 1),) + tuple(state_in.shape[1:]),
                                    dtype=state_in.dtype, device=state_in.device)
    st = lib().ppl_resample_shard(_ptr(lw), lw.numel(), int(first_particle), _ptr(max_lw_dev),
                                  ctypes.byref(plan), _ptr(ancestors), _ptr(state_in), stride,
                                  _ptr(state_out), _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "ppl_resample_shard")
    return ancestors[:n_out], (state_out[:n_out] if state_out is not None else None)


def poly_particles(n, device="cuda"):
    """An uninitialised [n, 8] float32 buffer of ppl_poly_particle records."""
    return torch.empty((n, POLY_RECORD_FLOATS), dtype=torch.float32, device=device)


def decode_particles(p):
    """(c[n, 6] float32, degree[n] int32, origin[n] int64) of a record buffer."""
    c = p[:, :6]
    deg = p[:, 6].contiguous().view(torch.int32)
    origin = p[:, 7].contiguous().view(torch.int32).to(torch.int64) & 0xFFFFFFFF
    return c, deg, origin


# ---- batched likelihood weighting ---------------------------------------
def _host_i64(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def ppl_batched_workspace_size(data_off, part_off, ppt=1):
    d, dp = _host_i64(data_off)
    p, pp = _host_i64(part_off)
    return int(lib().ppl_batched_workspace_size(dp, pp, len(d) - 1, int(ppt)))


def batched_workspace(data_off, part_off, device="cuda"):
    n = ppl_batched_workspace_size(data_off, part_off, 1)
    if n == 0:
        raise ValueError("invalid batch offsets")
    return torch.empty(n, dtype=torch.uint8, device=device)


def ppl_batched_prepare(model, data_off, part_off, ppt, blocks_per_sm, ws, stream=None):
    d, dp = _host_i64(data_off)
    p, pp = _host_i64(part_off)
    plan = PplBatchPlan()
    st = lib().ppl_batched_prepare(ctypes.byref(model), dp, pp, len(d) - 1, int(ppt),
                                   int(blocks_per_sm), ctypes.byref(plan), _ptr(ws), ws.numel(),
                                   _stream(stream))
    _check(st, "ppl_batched_prepare")
    return plan


def ppl_infer_is_batched(model, x, y, data_off, part_off, seed, plan, out, ws, stream=None):
    """Launch on device tensors x, y (float32) and data_off, part_off (int64)."""
    st = lib().ppl_infer_is_batched(ctypes.byref(model), _ptr(x), _ptr(y), _ptr(data_off),
                                    _ptr(part_off), plan.n_inst, ctypes.c_uint64(seed),
                                    ctypes.byref(plan), _ptr(out), _ptr(ws), ws.numel(),
                                    _stream(stream))
    _check(st, "ppl_infer_is_batched")
    return out


def ppl_batched_autotune(model, x, y, data_off, part_off, data_off_host, part_off_host, seed,
                         out, ws, cache_path=None, stream=None):
    d, dp = _host_i64(data_off_host)
    p, pp = _host_i64(part_off_host)
    plan = PplBatchPlan()
    st = lib().ppl_batched_autotune(ctypes.byref(model), _ptr(x), _ptr(y), _ptr(data_off),
                                    _ptr(part_off), dp, pp, len(d) - 1, ctypes.c_uint64(seed),
                                    _ptr(out), _ptr(ws), ws.numel(),
                                    cache_path.encode() if cache_path else None,
                                    ctypes.byref(plan), _stream(stream))
    _check(st, "ppl_batched_autotune")
    return plan


def ppl_batched_status(ws, stream=None):
    return int(lib().ppl_batched_status(_ptr(ws), _stream(stream)))


def batch_results_tensor(n_inst, device="cuda"):
    return torch.zeros(n_inst * RESULT_BYTES, dtype=torch.uint8, device=device)


def read_batch_results(out, n_inst):
    raw = out.detach().cpu().numpy().tobytes()
    return [PplIsResult.from_buffer_copy(raw, i * RESULT_BYTES).as_dict() for i in range(n_inst)]


# ---- learned proposal ---------------------------------------------------
def ppl_proposal_num_params():
    return int(lib().ppl_proposal_num_params())


def proposal_workspace(batch, device="cuda"):
    return torch.empty(int(lib().ppl_proposal_workspace_size(int(batch))), dtype=torch.uint8,
                       device=device)


def pack_params(weights, device="cuda"):
    """[W1, b1, W2, b2, W3, b3] (numpy or torch) -> one FP32 device buffer."""
    flat = [torch.as_tensor(np.asarray(w, dtype=np.float32)).reshape(-1) for w in weights]
    return torch.cat(flat).to(device)


def ppl_proposal_features(x, y, stream=None):
    n_sets = x.shape[0]
    feat = torch.empty((n_sets, 64), dtype=torch.bfloat16, device=x.device)
    _check(lib().ppl_proposal_features(_ptr(x), _ptr(y), n_sets, _ptr(feat), _stream(stream)),
           "ppl_proposal_features")
    return feat


def ppl_proposal_forward(model, params, x, y, out=None, ws=None, stream=None):
    n_sets = x.shape[0]
    if ws is None:
        ws = proposal_workspace(n_sets, x.device)
    if out is None:
        out = torch.empty((n_sets, 48), dtype=torch.float32, device=x.device)
    _check(lib().ppl_proposal_forward(ctypes.byref(model), _ptr(params), _ptr(x), _ptr(y),
                                      n_sets, _ptr(out), _ptr(ws), ws.numel(), _stream(stream)),
           "ppl_proposal_forward")
    return out


def ppl_proposal_grad(model, params, pair0, batch, seed, ws=None, stream=None):
    if ws is None:
        ws = proposal_workspace(batch, params.device)
    grad = torch.empty_like(params)
    loss = torch.zeros(1, dtype=torch.float64, device=params.device)
    _check(lib().ppl_proposal_grad(ctypes.byref(model), _ptr(params), int(pair0), int(batch),
                                   ctypes.c_uint64(seed), _ptr(grad), _ptr(loss), _ptr(ws),
                                   ws.numel(), _stream(stream)), "ppl_proposal_grad")
    return grad, loss


def ppl_proposal_train(model, params, adam_m, adam_v, n_pairs, batch, epochs, seed, lr=1e-3,
                       loss_per_step=None, ws=None, stream=None):
    if ws is None:
        ws = proposal_workspace(batch, params.device)
    _check(lib().ppl_proposal_train(ctypes.byref(model), _ptr(params), _ptr(adam_m),
                                    _ptr(adam_v), int(n_pairs), int(batch), int(epochs),
                                    ctypes.c_uint64(seed), float(lr), _ptr(loss_per_step),
                                    _ptr(ws), ws.numel(), _stream(stream)), "ppl_proposal_train")


def ppl_proposal_train_init(params, batch, ws, stream=None):
    _check(lib().ppl_proposal_train_init(_ptr(params), int(batch), _ptr(ws), ws.numel(),
                                         _stream(stream)), "ppl_proposal_train_init")


def ppl_proposal_train_steps(model, params, adam_m, adam_v, n_pairs, batch, n_steps, seed,
                             lr=1e-3, loss_per_step=None, ws=None, stream=None):
    _check(lib().ppl_proposal_train_steps(ctypes.byref(model), _ptr(params), _ptr(adam_m),
                                          _ptr(adam_v), int(n_pairs), int(batch), int(n_steps),
                                          ctypes.c_uint64(seed), float(lr), _ptr(loss_per_step),
                                          _ptr(ws), ws.numel(), _stream(stream)),
           "ppl_proposal_train_steps")


def ppl_infer_is_learned(model, x, y, data_off, part_off, seed, plan, proposal, out, ws,
                         stream=None):
    _check(lib().ppl_infer_is_learned(ctypes.byref(model), _ptr(x), _ptr(y), _ptr(data_off),
                                      _ptr(part_off), plan.n_inst, ctypes.c_uint64(seed),
                                      ctypes.byref(plan), _ptr(proposal), _ptr(out), _ptr(ws),
                                      ws.numel(), _stream(stream)), "ppl_infer_is_learned")
    return out
