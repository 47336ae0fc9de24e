"""Python front end of the surrogate network (axpic_mlp_* in libaxpic): device
tensors in and out through torch, parameters as a flat FP32 vector in the
library's layout. All arithmetic runs in the library's kernels."""
import numpy as np
import torch

from . import _lib

LAYOUT = (("W1", (4, 64)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (64, 96)), ("b3", (96,)))


def flatten(P):
    """dict of arrays -> flat FP32 vector in the library's order."""
    return np.concatenate([np.asarray(P[k], dtype=np.float32).reshape(-1) for k, _ in LAYOUT])


def unflatten(v):
    out, o = {}, 0
    for k, shp in LAYOUT:
        n = int(np.prod(shp))
        out[k] = np.asarray(v[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


class SurrogateNet:
    def __init__(self, device="cuda:0", stream=None):
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.h = _lib.axpic_mlp_create(self.stream.cuda_stream)

    def set_params(self, P):
        _lib.axpic_mlp_set_params(self.h, flatten(P) if isinstance(P, dict) else P)

    def get_params(self):
        return unflatten(_lib.axpic_mlp_get_params(self.h))

    def forward(self, X):
        X = X.contiguous()
        Z = torch.empty((X.shape[0], 96), dtype=torch.float32, device=self.device)
        _lib.axpic_mlp_forward(self.h, X.data_ptr(), X.shape[0], Z.data_ptr())
        return Z

    def gradients(self, X, Zt):
        X, Zt = X.contiguous(), Zt.contiguous()
        loss, g = _lib.axpic_mlp_gradients(self.h, X.data_ptr(), Zt.data_ptr(), X.shape[0])
        return loss, unflatten(g)

    def train_step(self, X, Zt, lr, want_loss=False):
        return _lib.axpic_mlp_train_step(self.h, X.data_ptr(), Zt.data_ptr(), X.shape[0], lr, want_loss)

    def close(self):
        if self.h is not None:
            h, self.h = self.h, None
            _lib.axpic_mlp_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
