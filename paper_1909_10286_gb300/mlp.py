"""Binding of the learned move ranker's C ABI (bl_mlp_*, bl_gemm_bf16):
argument marshalling only, every computation runs in the library's kernels.
Device buffers come from torch; the binding passes their raw pointers."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import biolog


def _lib():
    L = biolog.load()
    if not getattr(L, "_mlp_bound", False):
        vp = C.c_void_p
        L.bl_mlp_create.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_uint64, vp, C.POINTER(vp)]
        L.bl_mlp_forward.argtypes = [vp, vp, C.c_int32, vp]
        L.bl_mlp_grads.argtypes = [vp, vp, vp, C.c_int32, vp]
        L.bl_mlp_train_step.argtypes = [vp, vp, vp, C.c_int32, C.c_float, vp]
        L.bl_mlp_train_step_sampled.argtypes = [vp, vp, vp, C.c_int64, C.c_int32, C.c_uint64, C.c_float, vp]
        L.bl_mlp_get.argtypes = [vp, C.c_int32, vp, vp, vp, vp, vp, vp, vp, vp]
        L.bl_mlp_set.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.bl_mlp_free.argtypes = [vp]
        L.bl_mlp_last_error.argtypes = [vp]
        L.bl_mlp_last_error.restype = C.c_char_p
        L.bl_gemm_bf16.argtypes = [vp, vp, vp, vp, vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, vp, vp]
        L._mlp_bound = True
    return L


def _check(rc, h=None):
    if rc != biolog.BL_OK:
        msg = _lib().bl_mlp_last_error(h) or b""
        raise biolog.BiologError(rc, msg.decode())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _np(a):
    return C.c_void_p(a.ctypes.data)


def gemm_bf16(a, b, bias=None, relu=False, out_f32=True, out_bf16=False, stream=None):
    """C = a @ b.T (+bias, ReLU) on the tensor cores; a [M x K], b [N x K] torch bf16 CUDA tensors."""
    import torch

    M, K = a.shape
    N = b.shape[0]
    cf = torch.empty((M, N), dtype=torch.float32, device=a.device) if out_f32 else None
    cb = torch.empty((M, N), dtype=torch.bfloat16, device=a.device) if out_bf16 else None
    err = torch.zeros(1, dtype=torch.int32, device=a.device)
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(_lib().bl_gemm_bf16(_ptr(a), _ptr(b), _ptr(bias), _ptr(cf), _ptr(cb), M, N, K, int(relu), _ptr(err),
                               C.c_void_p(s.cuda_stream)))
    torch.cuda.synchronize()
    if int(err.item()):
        raise biolog.BiologError(biolog.BL_ETIMEOUT, "tensor-core GEMM wait gave up")
    return cf if out_f32 else cb


class MLP:
    """in -> H -> H -> H -> 1 ranker; parameters live on the GPU."""

    def __init__(self, in_dim: int = 64, hidden: int = 256, max_batch: int = 1 << 16, seed: int = 0, stream=None):
        import torch

        self.in_dim, self.hidden, self.max_batch = in_dim, hidden, max_batch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        _check(_lib().bl_mlp_create(in_dim, hidden, max_batch, seed, C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.h = h

    def _shapes(self):
        H, I = self.hidden, self.in_dim
        return [(H, I), (H,), (H, H), (H,), (H, H), (H,), (H,), (1,)]

    def get(self, grads: bool = False):
        arrs = [np.zeros(s, np.float32) for s in self._shapes()]
        _check(_lib().bl_mlp_get(self.h, int(grads), *[_np(a) for a in arrs]), self.h)
        return arrs

    def set(self, arrs):
        arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in arrs]
        _check(_lib().bl_mlp_set(self.h, *[_np(a) for a in arrs]), self.h)

    def copy(self, stream=None, max_batch: int | None = None) -> "MLP":
        """A network with the same weights (Adam state reset), e.g. on a search handle's stream."""
        net = MLP(self.in_dim, self.hidden, max_batch or self.max_batch, stream=stream)
        net.set(self.get())
        return net

    def forward(self, x, y=None):
        import torch

        M = x.shape[0]
        y = y if y is not None else torch.empty(M, dtype=torch.float32, device=x.device)
        _check(_lib().bl_mlp_forward(self.h, _ptr(x), M, _ptr(y)), self.h)
        return y

    def grads(self, x, target) -> float:
        loss = C.c_float(0.0)
        _check(_lib().bl_mlp_grads(self.h, _ptr(x), _ptr(target), x.shape[0], C.byref(loss)), self.h)
        return loss.value

    def train_step(self, x, target, lr: float) -> float:
        loss = C.c_float(0.0)
        _check(_lib().bl_mlp_train_step(self.h, _ptr(x), _ptr(target), x.shape[0], float(lr), C.byref(loss)), self.h)
        return loss.value

    def train_step_sampled(self, X, T, batch: int, seed: int, lr: float) -> float:
        """One Adam step on `batch` rows the library draws from the dataset (X [n x in] bf16, T [n] float32)."""
        loss = C.c_float(0.0)
        _check(_lib().bl_mlp_train_step_sampled(self.h, _ptr(X), _ptr(T), int(X.shape[0]), int(batch), int(seed),
                                                float(lr), C.byref(loss)), self.h)
        return loss.value

    def close(self):
        if getattr(self, "h", None):
            _lib().bl_mlp_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
