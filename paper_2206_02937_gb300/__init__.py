"""GB300 Compton pair-scatter library: thin Python binding of libcompton.so.

Every function below marshals arguments to the C ABI declared in
``include/compton.h`` (same names) and does nothing else: every step of the
path runs in the library's CUDA kernels.  Device buffers are torch CUDA
tensors, passed by ``data_ptr()``; streams are ``torch.cuda.Stream`` objects
(or None for the current stream).  The library must be built first
(``paper_2206_02937_gb300.buildlib.build()``); importing the binding without it
raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

from .buildlib import LIB, build  # noqa: F401

c_i32, c_i64, c_u32, c_u64, c_f32, c_f64, c_p = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                                 ctypes.c_uint64, ctypes.c_float, ctypes.c_double,
                                                 ctypes.c_void_p)

COMPTON_OK, COMPTON_EINVAL, COMPTON_ENOMEM, COMPTON_EBUSY, COMPTON_ETIMEOUT, COMPTON_ERANGE, \
    COMPTON_ENOTREADY, COMPTON_ECUDA, COMPTON_ENOMODEL = range(9)
MODE_PLAIN, MODE_MLP_FP32, MODE_MLP_BF16, MODE_MLP_FP8, MODE_PNET = range(5)
PNET_PARAMS = 337
FEATURES_MOMENTA, FEATURES_INVARIANTS = 0, 1


class compton_config(ctypes.Structure):
    _fields_ = [("n_cells", c_i64), ("max_particles", c_i64), ("w_over_v", c_f64), ("dt", c_f64),
                ("seed", c_u64), ("device", c_i32), ("gamma_fp64_threshold", c_f32),
                ("collide_fp64_threshold", c_f32), ("mem_budget_bytes", c_u64), ("max_train_batch", c_i64)]


class compton_species(ctypes.Structure):
    _fields_ = [("ux_dev", c_p), ("uy_dev", c_p), ("uz_dev", c_p), ("cell_dev", c_p), ("id_dev", c_p),
                ("n", c_i64), ("w_dev", c_p)]


class compton_pairs(ctypes.Structure):
    _fields_ = [("off_e_dev", c_p), ("off_g_dev", c_p), ("cell_info_dev", c_p), ("tile_cell_dev", c_p),
                ("n_pairs_dev", c_p), ("max_pairs", c_i64), ("n_cells", c_i64)]


class compton_stats(ctypes.Structure):
    _fields_ = [("pairs_tested", c_u64), ("scatters", c_u64), ("mlp_fallbacks", c_u64),
                ("error_flags", c_u64)]


class ComptonError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: status {status} ({strerror(status)})")


_lib = None

# (name, restype, argtypes) of every exported symbol; the CPU tests check
# that the built library exports each one.
SIGNATURES = {
    "compton_init": (c_i32, [ctypes.POINTER(compton_config), ctypes.POINTER(c_p)]),
    "compton_destroy": (c_i32, [c_p]),
    "compton_last_error": (ctypes.c_char_p, [c_p]),
    "compton_strerror": (ctypes.c_char_p, [c_i32]),
    "compton_check": (c_i32, [c_p, c_p]),
    "compton_get_stats": (c_i32, [c_p, ctypes.POINTER(compton_stats), c_i32, c_p]),
    "compton_bin_pairs": (c_i32, [c_p, ctypes.POINTER(compton_species), ctypes.POINTER(compton_species),
                                  ctypes.POINTER(compton_species), ctypes.POINTER(compton_species), c_u64,
                                  ctypes.POINTER(compton_pairs), c_p]),
    "compton_scatter_step": (c_i32, [c_p, ctypes.POINTER(compton_species), ctypes.POINTER(compton_species),
                                     ctypes.POINTER(compton_pairs), c_i32, c_u64, c_p, c_p, c_p]),
    "compton_scatter_pairs": (c_i32, [c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_i64, c_u64, c_u64, c_i32,
                                      c_p, c_p, c_p]),
    "compton_kn_ratio": (c_i32, [c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_i64, c_p, c_p]),
    "compton_kn_sample_angle": (c_i32, [c_p, c_p, c_p, c_i64, c_p, c_p, c_p, c_p]),
}


def lib():
    """Load libcompton.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise ImportError(f"libcompton.so is not built ({LIB}); run paper_2206_02937_gb300.buildlib.build()")
        L = ctypes.CDLL(LIB)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().compton_strerror(int(status)).decode()


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return c_p(stream.cuda_stream)


def _ptr(t):
    return c_p(0) if t is None else c_p(t.data_ptr())


def _check(st: int, what: str, ctx=None):
    if st != COMPTON_OK:
        err = ComptonError(st, what)
        if ctx is not None and st == COMPTON_ECUDA:
            err.args = (err.args[0] + ": " + lib().compton_last_error(ctx).decode(),)
        raise err


@dataclass
class Species:
    """One species as five torch CUDA tensors of equal length, plus optional
    per-particle weights over the cell volume (float32; None = the context's
    w_over_v for every particle)."""
    ux: "object"
    uy: "object"
    uz: "object"
    cell: "object"
    id: "object"
    w: "object" = None

    @property
    def n(self) -> int:
        return int(self.ux.shape[0])

    def c(self) -> compton_species:
        return compton_species(self.ux.data_ptr(), self.uy.data_ptr(), self.uz.data_ptr(),
                               self.cell.data_ptr(), self.id.data_ptr(), self.n,
                               None if self.w is None else self.w.data_ptr())

    @staticmethod
    def empty_like(s: "Species") -> "Species":
        import torch
        return Species(torch.empty_like(s.ux), torch.empty_like(s.uy), torch.empty_like(s.uz),
                       torch.empty_like(s.cell), torch.empty_like(s.id),
                       None if s.w is None else torch.empty_like(s.w))


def compton_init(n_cells: int, max_particles: int, w_over_v: float, dt: float, seed: int, device: int = 0,
                 gamma_fp64_threshold: float = 1.0e3, mem_budget_bytes: int = 0,
                 collide_fp64_threshold: float = 8.0, max_train_batch: int = 0) -> int:
    cfg = compton_config(n_cells, max_particles, w_over_v, dt, seed, device, gamma_fp64_threshold,
                         collide_fp64_threshold, mem_budget_bytes, max_train_batch)
    out = c_p()
    _check(lib().compton_init(ctypes.byref(cfg), ctypes.byref(out)), "compton_init")
    return out.value


def compton_destroy(ctx: int) -> None:
    _check(lib().compton_destroy(c_p(ctx)), "compton_destroy")


def compton_check(ctx: int, stream=None) -> int:
    """Returns the status (does not raise on ERANGE)."""
    return lib().compton_check(c_p(ctx), _stream_ptr(stream))


def compton_get_stats(ctx: int, reset: bool = False, stream=None) -> dict:
    s = compton_stats()
    _check(lib().compton_get_stats(c_p(ctx), ctypes.byref(s), int(reset), _stream_ptr(stream)),
           "compton_get_stats", ctx)
    return dict(pairs_tested=s.pairs_tested, scatters=s.scatters, mlp_fallbacks=s.mlp_fallbacks,
                error_flags=s.error_flags)


def compton_bin_pairs(ctx: int, e_in: Species, g_in: Species, e_out: Species, g_out: Species, step: int,
                      stream=None) -> compton_pairs:
    pairs = compton_pairs()
    ei, gi, eo, go = e_in.c(), g_in.c(), e_out.c(), g_out.c()
    _check(lib().compton_bin_pairs(c_p(ctx), ctypes.byref(ei), ctypes.byref(gi), ctypes.byref(eo),
                                   ctypes.byref(go), int(step), ctypes.byref(pairs), _stream_ptr(stream)),
           "compton_bin_pairs", ctx)
    return pairs


def compton_scatter_step(ctx: int, e: Species, g: Species, pairs: compton_pairs, mode: int, step: int,
                         prob_out=None, flag_out=None, stream=None) -> None:
    ec, gc = e.c(), g.c()
    _check(lib().compton_scatter_step(c_p(ctx), ctypes.byref(ec), ctypes.byref(gc), ctypes.byref(pairs),
                                      int(mode), int(step), _ptr(prob_out), _ptr(flag_out),
                                      _stream_ptr(stream)), "compton_scatter_step", ctx)


SIGNATURES["compton_scatter_step_ntc"] = (c_i32, [c_p, ctypes.POINTER(compton_species),
                                                  ctypes.POINTER(compton_species), ctypes.POINTER(compton_pairs),
                                                  c_u64, c_p])


def compton_scatter_step_ntc(ctx: int, e: Species, g: Species, pairs: compton_pairs, step: int,
                             stream=None) -> None:
    """No-Time-Counter collisions of the binned species, in place."""
    ec, gc = e.c(), g.c()
    _check(lib().compton_scatter_step_ntc(c_p(ctx), ctypes.byref(ec), ctypes.byref(gc), ctypes.byref(pairs),
                                          int(step), _stream_ptr(stream)), "compton_scatter_step_ntc", ctx)


def compton_scatter_pairs(ctx: int, u, k, n_dens, seed: int, step: int, mode: int = MODE_PLAIN,
                          prob_out=None, flag_out=None, stream=None) -> None:
    """u, k: (3, n) float32 CUDA tensors (rows contiguous), updated in place."""
    n = int(u.shape[1])
    _check(lib().compton_scatter_pairs(c_p(ctx), _ptr(u[0]), _ptr(u[1]), _ptr(u[2]), _ptr(k[0]), _ptr(k[1]),
                                       _ptr(k[2]), _ptr(n_dens), n, int(seed), int(step), int(mode),
                                       _ptr(prob_out), _ptr(flag_out), _stream_ptr(stream)),
           "compton_scatter_pairs", ctx)


def compton_kn_ratio(ctx: int, u, k, r_out, stream=None) -> None:
    n = int(u.shape[1])
    _check(lib().compton_kn_ratio(c_p(ctx), _ptr(u[0]), _ptr(u[1]), _ptr(u[2]), _ptr(k[0]), _ptr(k[1]),
                                  _ptr(k[2]), n, _ptr(r_out), _stream_ptr(stream)), "compton_kn_ratio", ctx)


def compton_kn_sample_angle(ctx: int, x, r, cth_out, sth_out, ratio_out, stream=None) -> None:
    n = int(x.shape[0])
    _check(lib().compton_kn_sample_angle(c_p(ctx), _ptr(x), _ptr(r), n, _ptr(cth_out), _ptr(sth_out),
                                         _ptr(ratio_out), _stream_ptr(stream)), "compton_kn_sample_angle", ctx)


SIGNATURES.update({
    "compton_mlp_set_params": (c_i32, [c_p, c_p, c_i64, c_p]),
    "compton_mlp_get_params": (c_i32, [c_p, c_p, c_i64]),
    "compton_mlp_calibrate": (c_i32, [c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_i64, c_p]),
    "compton_mlp_infer": (c_i32, [c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_i64, c_i32, c_p, c_p]),
    "compton_mlp_save": (c_i32, [c_p, c_p, ctypes.POINTER(ctypes.c_size_t)]),
    "compton_mlp_load": (c_i32, [c_p, c_p, ctypes.c_size_t]),
    "compton_mlp_train_step": (c_i32, [c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_i64, c_f32,
                                       ctypes.POINTER(c_f32), c_p]),
})

N_MLP_PARAMS = 12993


def _host_f32(a):
    import numpy as np
    return np.ascontiguousarray(a, dtype=np.float32)


def compton_mlp_set_params(ctx: int, theta, feature_scales=None) -> None:
    th = _host_f32(theta)
    fs = None if feature_scales is None else _host_f32(feature_scales)
    _check(lib().compton_mlp_set_params(c_p(ctx), c_p(th.ctypes.data), int(th.shape[0]),
                                        c_p(0) if fs is None else c_p(fs.ctypes.data)),
           "compton_mlp_set_params", ctx)


def compton_mlp_get_params(ctx: int):
    import numpy as np
    th = np.zeros(N_MLP_PARAMS, dtype=np.float32)
    _check(lib().compton_mlp_get_params(c_p(ctx), c_p(th.ctypes.data), N_MLP_PARAMS), "compton_mlp_get_params", ctx)
    return th


def compton_mlp_calibrate(ctx: int, u, k, stream=None) -> None:
    n = int(u.shape[1])
    _check(lib().compton_mlp_calibrate(c_p(ctx), _ptr(u[0]), _ptr(u[1]), _ptr(u[2]), _ptr(k[0]), _ptr(k[1]),
                                       _ptr(k[2]), n, _stream_ptr(stream)), "compton_mlp_calibrate", ctx)


def compton_mlp_infer(ctx: int, u, k, mode: int, r_out, stream=None) -> None:
    n = int(u.shape[1])
    _check(lib().compton_mlp_infer(c_p(ctx), _ptr(u[0]), _ptr(u[1]), _ptr(u[2]), _ptr(k[0]), _ptr(k[1]),
                                   _ptr(k[2]), n, int(mode), _ptr(r_out), _stream_ptr(stream)),
           "compton_mlp_infer", ctx)


def compton_mlp_save(ctx: int) -> bytes:
    n = ctypes.c_size_t(0)
    _check(lib().compton_mlp_save(c_p(ctx), c_p(0), ctypes.byref(n)), "compton_mlp_save", ctx)
    buf = ctypes.create_string_buffer(n.value)
    _check(lib().compton_mlp_save(c_p(ctx), ctypes.cast(buf, c_p), ctypes.byref(n)), "compton_mlp_save", ctx)
    return buf.raw[:n.value]


def compton_mlp_load(ctx: int, blob: bytes) -> None:
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(lib().compton_mlp_load(c_p(ctx), ctypes.cast(buf, c_p), len(blob)), "compton_mlp_load", ctx)


def compton_mlp_train_step(ctx: int, u, k, y, w, lr: float = 1e-3, want_loss: bool = True, stream=None):
    """One Adam step on a minibatch; returns the minibatch loss (synchronising) or None."""
    n = int(u.shape[1])
    loss = c_f32(0.0)
    _check(lib().compton_mlp_train_step(c_p(ctx), _ptr(u[0]), _ptr(u[1]), _ptr(u[2]), _ptr(k[0]), _ptr(k[1]),
                                        _ptr(k[2]), _ptr(y), _ptr(w), n, float(lr),
                                        ctypes.byref(loss) if want_loss else None, _stream_ptr(stream)),
           "compton_mlp_train_step", ctx)
    return float(loss.value) if want_loss else None


SIGNATURES["compton_mlp_get_grad"] = (c_i32, [c_p, c_p, c_i64])


def compton_mlp_get_grad(ctx: int):
    import numpy as np
    g = np.zeros(N_MLP_PARAMS, dtype=np.float32)
    _check(lib().compton_mlp_get_grad(c_p(ctx), c_p(g.ctypes.data), N_MLP_PARAMS), "compton_mlp_get_grad", ctx)
    return g


class compton_request(ctypes.Structure):
    _fields_ = [(nm, c_p) for nm in ("ux_in_dev", "uy_in_dev", "uz_in_dev", "kx_in_dev", "ky_in_dev", "kz_in_dev",
                                     "ux_out_dev", "uy_out_dev", "uz_out_dev", "kx_out_dev", "ky_out_dev",
                                     "kz_out_dev", "n_dens_dev")] + \
               [("n_dens", c_f32), ("n", c_i64), ("seed", c_u64), ("step", c_u64), ("mode", c_i32)]


class compton_result(ctypes.Structure):
    _fields_ = [("status", c_i32), ("scatters", c_u64), ("latency_s", c_f64), ("queue_s", c_f64)]


SIGNATURES.update({
    "compton_serve_start": (c_i32, [c_p, c_u64, c_i32]),
    "compton_serve_stop": (c_i32, [c_p]),
    "compton_submit": (c_i32, [c_p, ctypes.POINTER(compton_request), ctypes.POINTER(c_u64)]),
    "compton_poll": (c_i32, [c_p, c_u64, ctypes.POINTER(compton_result)]),
    "compton_serve_info": (c_i32, [c_p, ctypes.POINTER(c_u64), ctypes.POINTER(c_u64), ctypes.POINTER(c_u64)]),
})


def compton_serve_start(ctx: int, pool_bytes: int, max_active: int = 1024) -> None:
    _check(lib().compton_serve_start(c_p(ctx), int(pool_bytes), int(max_active)), "compton_serve_start", ctx)


def compton_serve_stop(ctx: int) -> None:
    _check(lib().compton_serve_stop(c_p(ctx)), "compton_serve_stop", ctx)


def compton_submit(ctx: int, u_in, k_in, u_out, k_out, n_dens, seed: int, step: int = 0,
                   mode: int = MODE_PLAIN) -> int:
    """u_in, k_in, u_out, k_out: (3, n) float32 CUDA tensors (rows contiguous);
    n_dens: a float or an (n,) float32 CUDA tensor.  Returns the ticket."""
    n = int(u_in.shape[1])
    dens_ptr, dens_val = (c_p(0), float(n_dens)) if isinstance(n_dens, (int, float)) else (_ptr(n_dens), 0.0)
    r = compton_request(*[_ptr(t) for t in (u_in[0], u_in[1], u_in[2], k_in[0], k_in[1], k_in[2],
                                            u_out[0], u_out[1], u_out[2], k_out[0], k_out[1], k_out[2])],
                        dens_ptr, dens_val, n, int(seed), int(step), int(mode))
    t = c_u64(0)
    _check(lib().compton_submit(c_p(ctx), ctypes.byref(r), ctypes.byref(t)), "compton_submit", ctx)
    return int(t.value)


def compton_poll(ctx: int, ticket: int):
    """None while the request is running, else a dict with its result."""
    res = compton_result()
    st = lib().compton_poll(c_p(ctx), int(ticket), ctypes.byref(res))
    if st == COMPTON_ENOTREADY:
        return None
    _check(st, "compton_poll", ctx)
    return dict(status=res.status, scatters=res.scatters, latency_s=res.latency_s, queue_s=res.queue_s)


def compton_serve_info(ctx: int) -> dict:
    a, b, c = c_u64(0), c_u64(0), c_u64(0)
    _check(lib().compton_serve_info(c_p(ctx), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "compton_serve_info", ctx)
    return dict(in_use=a.value, peak=b.value, pool=c.value)


SIGNATURES["compton_cell_offsets_noalloc"] = (c_i32, [c_p, c_i64, c_i64, c_p, c_p])


def compton_cell_offsets_noalloc(cell, n_cells: int, off_out, stream=None) -> None:
    """Per-cell offsets of one species (cell: int32 CUDA tensor; off_out:
    int32 CUDA tensor of at least n_cells + 1), with no device allocation."""
    import torch
    for name, t in (("cell", cell), ("off_out", off_out)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.int32 and t.is_contiguous()):
            raise ValueError(f"compton_cell_offsets_noalloc: {name} must be a contiguous int32 CUDA tensor")
    if off_out.numel() < int(n_cells) + 1:
        raise ValueError(f"compton_cell_offsets_noalloc: off_out holds {off_out.numel()} values, "
                         f"n_cells + 1 = {int(n_cells) + 1} needed")
    _check(lib().compton_cell_offsets_noalloc(_ptr(cell), int(cell.shape[0]), int(n_cells), _ptr(off_out),
                                              _stream_ptr(stream)), "compton_cell_offsets_noalloc")


SIGNATURES["compton_mlp_balance_weights"] = (c_i32, [c_p, c_p, c_i64, c_p, c_i32, c_p, c_p])


def compton_mlp_balance_weights(ctx: int, r, edges, w_out, stream=None) -> None:
    """r: float32 CUDA tensor; edges: n_bins + 1 increasing host floats."""
    import numpy as np
    e = np.ascontiguousarray(edges, dtype=np.float32)
    _check(lib().compton_mlp_balance_weights(c_p(ctx), _ptr(r), int(r.shape[0]), c_p(e.ctypes.data),
                                             int(e.shape[0] - 1), _ptr(w_out), _stream_ptr(stream)),
           "compton_mlp_balance_weights", ctx)


SIGNATURES["compton_mlp_set_train_precision"] = (c_i32, [c_p, c_i32])


def compton_mlp_set_train_precision(ctx: int, mode: int) -> None:
    """Training arithmetic: MODE_MLP_FP32 (CUDA cores, the default) or
    MODE_MLP_BF16 (tcgen05 tensor cores, BF16 operands, FP32 accumulation)."""
    _check(lib().compton_mlp_set_train_precision(c_p(ctx), int(mode)), "compton_mlp_set_train_precision", ctx)


SIGNATURES["compton_mlp_set_features"] = (c_i32, [c_p, c_i32])
SIGNATURES["compton_mlp_set_range"] = (c_i32, [c_p, c_f64, c_f64, c_f64])


def compton_mlp_set_range(ctx: int, gamma_max: float, eps_min: float, eps_max: float) -> None:
    """Training range of the network (outside it: analytic probability)."""
    _check(lib().compton_mlp_set_range(c_p(ctx), float(gamma_max), float(eps_min), float(eps_max)),
           "compton_mlp_set_range", ctx)


def compton_mlp_set_features(ctx: int, features: int) -> None:
    """Network inputs: FEATURES_MOMENTA (default) or FEATURES_INVARIANTS."""
    _check(lib().compton_mlp_set_features(c_p(ctx), int(features)), "compton_mlp_set_features", ctx)


SIGNATURES["compton_pnet_set_params"] = (c_i32, [c_p, c_p, c_i64, c_p, c_f64, c_f64, c_f64])
SIGNATURES["compton_pnet_get_params"] = (c_i32, [c_p, c_p, c_p, c_i64])
SIGNATURES["compton_pnet_infer"] = (c_i32, [c_p] * 7 + [c_i64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                                      c_p, c_p])
SIGNATURES["compton_pnet_train_step"] = (c_i32, [c_p] * 9 + [c_i64] + [ctypes.c_float] * 4 + [c_p, c_p])


def compton_pnet_set_params(ctx: int, theta, feature_scales=None, gamma_max: float = 1e3, eps_min: float = 1e-4,
                            eps_max: float = 1.0) -> None:
    """Load the paper network's 337 parameters (host array) and reset Adam."""
    import numpy as np
    t = np.ascontiguousarray(theta, dtype=np.float32)
    fs = None if feature_scales is None else np.ascontiguousarray(feature_scales, dtype=np.float32)
    _check(lib().compton_pnet_set_params(c_p(ctx), c_p(t.ctypes.data), int(t.shape[0]),
                                         None if fs is None else c_p(fs.ctypes.data), float(gamma_max),
                                         float(eps_min), float(eps_max)), "compton_pnet_set_params", ctx)


def compton_pnet_get_params(ctx: int):
    """(theta, grad of the last train step) as float32 host arrays."""
    import numpy as np
    t = np.zeros(PNET_PARAMS, np.float32)
    g = np.zeros(PNET_PARAMS, np.float32)
    _check(lib().compton_pnet_get_params(c_p(ctx), c_p(t.ctypes.data), c_p(g.ctypes.data), PNET_PARAMS),
           "compton_pnet_get_params", ctx)
    return t, g


def compton_pnet_infer(ctx: int, u, k, w_e: float, w_g: float, p_max: float, r_out, stream=None) -> None:
    """u, k: (3, n) float32 CUDA tensors; r_out: (n,) float32."""
    _check(lib().compton_pnet_infer(c_p(ctx), _ptr(u[0]), _ptr(u[1]), _ptr(u[2]), _ptr(k[0]), _ptr(k[1]),
                                    _ptr(k[2]), int(u.shape[1]), float(w_e), float(w_g), float(p_max),
                                    _ptr(r_out), _stream_ptr(stream)), "compton_pnet_infer", ctx)


def compton_pnet_train_step(ctx: int, u, k, y, w, w_e: float, w_g: float, p_max: float, lr: float,
                            want_loss: bool = True, stream=None):
    """One Adam step on the weighted MAE; returns the loss before the update
    (synchronising) when want_loss, else None."""
    loss = ctypes.c_float(0.0)
    _check(lib().compton_pnet_train_step(c_p(ctx), _ptr(u[0]), _ptr(u[1]), _ptr(u[2]), _ptr(k[0]), _ptr(k[1]),
                                         _ptr(k[2]), _ptr(y), None if w is None else _ptr(w), int(u.shape[1]),
                                         float(w_e), float(w_g), float(p_max), float(lr),
                                         ctypes.byref(loss) if want_loss else None, _stream_ptr(stream)),
           "compton_pnet_train_step", ctx)
    return float(loss.value) if want_loss else None


KERNEL_SLOTS = ("k_count", "k_scan", "k_place", "k_sort_gather", "k_pair_prob", "k_collide", "k_mlp", "k_ntc")

SIGNATURES["compton_kernel_timing"] = (c_i32, [c_p, c_i32])
SIGNATURES["compton_kernel_times"] = (c_i32, [c_p, c_p, c_p])


def compton_kernel_timing(ctx: int, enable: bool) -> None:
    """Start (restarting the counts) or stop per-kernel event timing."""
    _check(lib().compton_kernel_timing(c_p(ctx), 1 if enable else 0), "compton_kernel_timing", ctx)


def compton_kernel_times(ctx: int) -> dict:
    """Summed device time (ms) and launch count per kernel slot since timing
    was enabled (the last 64 launches of each slot)."""
    ms = (ctypes.c_double * len(KERNEL_SLOTS))()
    n = (ctypes.c_int64 * len(KERNEL_SLOTS))()
    _check(lib().compton_kernel_times(c_p(ctx), ms, n), "compton_kernel_times", ctx)
    return {name: {"ms": ms[i], "launches": n[i]} for i, name in enumerate(KERNEL_SLOTS)}


SIGNATURES["compton_debug_inject"] = (c_i32, [c_i64, c_i64, c_p])


def compton_debug_inject(skip: int, fail: int) -> int:
    """Arm host-side fault injection: the next `skip` checked CUDA calls pass,
    the `fail` after them report an error.  Returns the failures that were
    still pending."""
    pending = c_i64(0)
    _check(lib().compton_debug_inject(int(skip), int(fail), ctypes.byref(pending)), "compton_debug_inject")
    return int(pending.value)


SIGNATURES["compton_selftest_wait"] = (c_i32, [c_p, c_u64, c_p])


def compton_selftest_wait(ctx: int, timeout_ns: int, stream=None) -> None:
    _check(lib().compton_selftest_wait(c_p(ctx), int(timeout_ns), _stream_ptr(stream)), "compton_selftest_wait", ctx)
