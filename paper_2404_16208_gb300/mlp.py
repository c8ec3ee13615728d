"""Python binding of include/ranc_mlp.h (argument marshalling only)."""

import ctypes as C

import numpy as np

from . import ranc

_lib = ranc._lib
_vp, _i32 = C.c_void_p, C.c_int32
for _name, _args, _res in (
        ("ranc_mlp_create", [_i32, _vp, _i32, C.c_uint64, _vp, C.POINTER(_vp)], C.c_int),
        ("ranc_mlp_param_count", [_vp, C.POINTER(C.c_int64)], C.c_int),
        ("ranc_mlp_get_params", [_vp, _vp], C.c_int),
        ("ranc_mlp_set_params", [_vp, _vp], C.c_int),
        ("ranc_mlp_forward", [_vp, _vp, _i32, _vp], C.c_int),
        ("ranc_mlp_loss_backward", [_vp, _vp, _vp, _i32, _vp, _vp], C.c_int),
        ("ranc_mlp_adam_step", [_vp, C.c_float, C.c_float, C.c_float, C.c_float], C.c_int),
        ("ranc_mlp_destroy", [_vp], None),
        ("ranc_mlp_last_error", [_vp], C.c_char_p)):
    _f = getattr(_lib, _name)
    _f.argtypes, _f.restype = _args, _res

EXPORTED = ("ranc_mlp_create", "ranc_mlp_param_count", "ranc_mlp_get_params", "ranc_mlp_set_params",
            "ranc_mlp_forward", "ranc_mlp_loss_backward", "ranc_mlp_adam_step", "ranc_mlp_destroy",
            "ranc_mlp_last_error")


def _check(rc, h):
    if rc != 0:
        raise ranc.RancError(rc, _lib.ranc_mlp_last_error(h).decode())


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


class MLP:
    """Owning wrapper: dims = (inputs, hidden..., outputs)."""

    def __init__(self, dims, max_batch, seed=0, stream=0):
        self.dims = tuple(int(d) for d in dims)
        d = np.array(self.dims, dtype=np.int32)
        self.h = C.c_void_p()
        _check(_lib.ranc_mlp_create(len(dims) - 1, _p(d), int(max_batch), int(seed), C.c_void_p(int(stream)),
                                    C.byref(self.h)), None)
        n = C.c_int64()
        _check(_lib.ranc_mlp_param_count(self.h, C.byref(n)), self.h)
        self.n_params = n.value

    def get_params(self):
        out = np.zeros(self.n_params, np.float32)
        _check(_lib.ranc_mlp_get_params(self.h, _p(out)), self.h)
        return out

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        assert flat.size == self.n_params
        _check(_lib.ranc_mlp_set_params(self.h, _p(flat)), self.h)

    def forward(self, x_ptr, batch, y_ptr):
        _check(_lib.ranc_mlp_forward(self.h, C.c_void_p(int(x_ptr)), int(batch), C.c_void_p(int(y_ptr))), self.h)

    def loss_backward(self, x_ptr, t_ptr, batch, want_grads=False):
        loss = np.zeros(1, np.float32)
        grads = np.zeros(self.n_params, np.float32) if want_grads else None
        _check(_lib.ranc_mlp_loss_backward(self.h, C.c_void_p(int(x_ptr)), C.c_void_p(int(t_ptr)), int(batch),
                                           _p(loss), _p(grads) if want_grads else None), self.h)
        return float(loss[0]), grads

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(_lib.ranc_mlp_adam_step(self.h, lr, beta1, beta2, eps), self.h)

    def close(self):
        if self.h:
            _lib.ranc_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
