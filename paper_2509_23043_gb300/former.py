"""ctypes binding of libptformer.so (include/pt_former.h): IsingFormer inference on the GPU.

Argument marshalling only: the model, its scoring pass and its sampler run in the library.
Device arrays are torch CUDA tensors (device memory and streams only). The library must be
built (paper_2509_23043_gb300.build); there is no fallback.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

from . import PTError

LIB_PATH = Path(__file__).resolve().parent / "_build" / "libptformer.so"
_lib = None


class _Cfg(C.Structure):
    _fields_ = [("n_spins", C.c_int32), ("d_model", C.c_int32), ("n_heads", C.c_int32),
                ("n_layers", C.c_int32), ("d_ff", C.c_int32), ("attn_mode", C.c_int32),
                ("proj_mode", C.c_int32)]


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2509_23043_gb300.build`")
    L = C.CDLL(str(LIB_PATH))
    vp = C.c_void_p
    L.pt_former_param_count.argtypes = [C.POINTER(_Cfg)]
    L.pt_former_param_count.restype = C.c_size_t
    L.pt_former_create.argtypes = [C.POINTER(vp), C.POINTER(_Cfg), vp, C.c_size_t, vp]
    L.pt_former_score.argtypes = [vp, C.c_int32, vp, vp, vp, vp]
    L.pt_former_sample.argtypes = [vp, C.c_int32, vp, vp, C.c_int32, C.c_uint64, C.c_uint32, vp, vp]
    L.pt_former_score_gemm_flops.argtypes = [vp, C.c_int32]
    L.pt_former_score_gemm_flops.restype = C.c_double
    L.pt_former_destroy.argtypes = [vp]
    L.pt_former_check.argtypes = [vp]
    L.pt_former_last_error.restype = C.c_char_p
    for f in ("pt_former_create", "pt_former_score", "pt_former_sample", "pt_former_destroy", "pt_former_check"):
        getattr(L, f).restype = C.c_int
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        raise PTError(status, lib().pt_former_last_error().decode())


def _dp(t):
    return None if t is None else C.c_void_p(t.data_ptr())


class Former:
    """One IsingFormer on the current CUDA device and stream."""

    def __init__(self, shape, packed_params: np.ndarray, stream=None, attn_mode: int = 0, proj_mode: int = 0):
        """attn_mode 0: scoring attention on the tensor cores (for N <= 256, N a multiple of 8,
        scores, causal softmax and P V in one tcgen05 kernel; else as mode 2 where its scores
        fit, else the streaming kernel); 1: always the streaming kernel; 2: tensor-core
        attention with the scores, the softmax and P V as separate cuBLASLt products and kernel. proj_mode 0: the first FFN map by
        this library's tcgen05 kernel (bias and GELU fused) from 16384 rows, cuBLASLt for the
        rest; 1: cuBLASLt products and a GELU kernel; 2: the tcgen05 kernels for every
        projection whose shape suits them (bias, GELU, residual fused), at any size."""
        import torch
        self.shape = shape
        self.cfg = _Cfg(shape.n_spins, shape.d_model, shape.n_heads, shape.n_layers, shape.d_ff, attn_mode, proj_mode)
        p = np.ascontiguousarray(packed_params, dtype=np.uint16)
        s = torch.cuda.current_stream().cuda_stream if stream is None else stream
        h = C.c_void_p()
        _check(lib().pt_former_create(C.byref(h), C.byref(self.cfg), p.ctypes.data, p.size, C.c_void_p(s)))
        self.handle = h

    def __del__(self):
        if getattr(self, "handle", None):
            lib().pt_former_destroy(self.handle)
            self.handle = None

    def score(self, spins, beta, logits: bool = False):
        """log q(x | beta) [B] (and logits [B][N][2]) of device spins int8 [B][N], beta [B]."""
        import torch
        B = spins.shape[0]
        lq = torch.empty(B, dtype=torch.float32, device=spins.device)
        lg = torch.empty((B, self.shape.n_spins, 2), dtype=torch.float32, device=spins.device) if logits else None
        _check(lib().pt_former_score(self.handle, B, _dp(spins), _dp(beta), _dp(lq), _dp(lg)))
        return (lq, lg) if logits else lq

    def sample(self, beta, seed: int, stream_id: int = 0, prefix=None, out=None, logq=None):
        """B configurations int8 [B][N] and their log q, drawn at device inverse temperatures
        beta [B]; prefix int8 [B][n_prefix] (device) fixes the first spins."""
        import torch
        B = beta.shape[0]
        out = torch.empty((B, self.shape.n_spins), dtype=torch.int8, device=beta.device) if out is None else out
        logq = torch.empty(B, dtype=torch.float32, device=beta.device) if logq is None else logq
        npre = 0 if prefix is None else prefix.shape[1]
        _check(lib().pt_former_sample(self.handle, B, _dp(beta), _dp(prefix), npre, seed & 0xFFFFFFFFFFFFFFFF,
                                      stream_id & 0xFFFFFFFF, _dp(out), _dp(logq)))
        return out, logq

    def check(self):
        """Raise if a bounded wait of a tcgen05 product kernel ran out (synchronises)."""
        _check(lib().pt_former_check(self.handle))

    def score_gemm_flops(self, B: int) -> float:
        return float(lib().pt_former_score_gemm_flops(self.handle, B))
