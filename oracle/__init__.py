"""FP64 CPU oracle of the Compton pair-scatter step (arXiv 2206.02937).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (``paper_2206_02937_gb300``) and never imports it.

Two parts:
  * ``compton_oracle.c`` -- the physics step (Philox, binning and pairing,
    invariants, Klein-Nishina cross section, probability, Bernoulli trial,
    inverse-CDF sampling, boosts, momentum update), built with gcc into
    ``_build/liboracle.so`` and called through ctypes;
  * ``mlp.py`` -- the surrogate network's forward, backward and Adam in FP64
    numpy.

Every function cites the passage of the paper it follows; the pins that tie it
to something other than itself are in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "compton_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (FP64, no fused multiply-add contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        d, i32, i64, u32, u64 = (ctypes.c_double, ctypes.c_int32, ctypes.c_int64,
                                 ctypes.c_uint32, ctypes.c_uint64)
        P = ctypes.c_void_p
        L.or_philox4x32_10.argtypes = [P, P, P]
        L.or_philox4x32_10.restype = None
        L.or_kn_series_coef.argtypes = [ctypes.c_int]
        L.or_kn_series_coef.restype = d
        for name in ("or_kn_sigma",):
            getattr(L, name).argtypes = [d]
            getattr(L, name).restype = d
        for name in ("or_kn_dsigma_dt", "or_kn_cdf", "or_kn_sample_t"):
            getattr(L, name).argtypes = [d, d]
            getattr(L, name).restype = d
        L.or_invariants.argtypes = [P, P, P]
        L.or_invariants.restype = None
        L.or_boost_to_rest.argtypes = [P, d, P, P, P]
        L.or_boost_to_rest.restype = None
        L.or_boost_to_lab.argtypes = [P, d, P, P, P]
        L.or_boost_to_lab.restype = None
        L.or_onb.argtypes = [P, P, P]
        L.or_onb.restype = None
        L.or_scatter_event.argtypes = [P, P, d, d, u64, u64, u32, P, P, P, P, P]
        L.or_scatter_event.restype = None
        L.or_bernoulli_u0.argtypes = [u64, u64, u32]
        L.or_bernoulli_u0.restype = d
        L.or_collide.argtypes = [P, P, u64, u64, u32, P, P]
        L.or_collide.restype = None
        L.or_pair_key.argtypes = [u64, u64, u32, u32]
        L.or_pair_key.restype = u32
        L.or_sort_species.argtypes = [i64, P, P, i64, u64, u64, u32, P, P]
        L.or_sort_species.restype = ctypes.c_int
        L.or_step.argtypes = [i64, d, d, u64, u64,
                              i64, P, P, P, P, P,
                              i64, P, P, P, P, P,
                              P, P, P, P, P, P, P, P, P, P]
        L.or_step.restype = i64
        L.or_pairs.argtypes = [i64, P, P, P, P, P, P, P, d, u64, u64, P, P, P, P]
        L.or_pairs.restype = None
        L.or_ratio.argtypes = [i64, P, P, P, P, P, P, P]
        L.or_ratio.restype = None
        L.or_ntc_step.argtypes = [i64, d, d, u64, u64,
                                  i64, P, P, P, P, P,
                                  i64, P, P, P, P, P,
                                  P, P, P, P, P, P, P, P, P]
        L.or_ntc_step.restype = i64
        L.or_step_weighted.argtypes = [i64, d, d, u64, u64,
                                       i64, P, P, P, P, P, P,
                                       i64, P, P, P, P, P, P,
                                       P, P, P, P, P, P, P, P, P, P, P, P]
        L.or_step_weighted.restype = i64
        _ = (i32,)
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# Scalar building blocks (used by the pins)
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block function (Salmon et al., SC'11) on one counter."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def kn_sigma(x: float) -> float:
    """Klein-Nishina total cross section / sigma_T at rest-frame energy x (Sec. 3.2)."""
    return lib().or_kn_sigma(float(x))


def kn_series_coef(n: int) -> float:
    return lib().or_kn_series_coef(int(n))


def kn_dsigma_dt(x: float, t: float) -> float:
    return lib().or_kn_dsigma_dt(float(x), float(t))


def kn_cdf(x: float, t: float) -> float:
    return lib().or_kn_cdf(float(x), float(t))


def kn_sample_t(x: float, u: float) -> float:
    return lib().or_kn_sample_t(float(x), float(u))


def invariants(u, k):
    """(x, v): rest-frame photon energy and flux factor 1 - beta cos(psi) (Sec. 3.2)."""
    uu = np.ascontiguousarray(u, dtype=np.float64)
    kk = np.ascontiguousarray(k, dtype=np.float64)
    out = np.zeros(2)
    lib().or_invariants(_p(uu), _p(kk), _p(out))
    return float(out[0]), float(out[1])


def boost_to_rest(u, k):
    uu = np.ascontiguousarray(u, dtype=np.float64)
    kk = np.ascontiguousarray(k, dtype=np.float64)
    er = ctypes.c_double()
    kr = np.zeros(3)
    lib().or_boost_to_rest(_p(uu), float(np.linalg.norm(kk)), _p(kk), ctypes.byref(er), _p(kr))
    return er.value, kr


def boost_to_lab(u, eps_r, kr):
    uu = np.ascontiguousarray(u, dtype=np.float64)
    kk = np.ascontiguousarray(kr, dtype=np.float64)
    e = ctypes.c_double()
    k = np.zeros(3)
    lib().or_boost_to_lab(_p(uu), float(eps_r), _p(kk), ctypes.byref(e), _p(k))
    return e.value, k


def onb(n):
    nn = np.ascontiguousarray(n, dtype=np.float64)
    b1 = np.zeros(3)
    b2 = np.zeros(3)
    lib().or_onb(_p(nn), _p(b1), _p(b2))
    return b1, b2


def scatter_event(u, k, n_dens, dt, seed, step, ctr_id):
    """One pair event: returns (u_out, k_out, P, flag, x)."""
    uu = np.ascontiguousarray(u, dtype=np.float64)
    kk = np.ascontiguousarray(k, dtype=np.float64)
    uo = np.zeros(3)
    ko = np.zeros(3)
    P = ctypes.c_double()
    f = ctypes.c_int()
    x = ctypes.c_double()
    lib().or_scatter_event(_p(uu), _p(kk), float(n_dens), float(dt), int(seed), int(step),
                           int(ctr_id), _p(uo), _p(ko), ctypes.byref(P), ctypes.byref(f),
                           ctypes.byref(x))
    return uo, ko, P.value, f.value, x.value


def bernoulli_u0(seed, step, p) -> float:
    """The uniform the probability of pair p is compared with (Sec. 3.1)."""
    return float(lib().or_bernoulli_u0(int(seed), int(step), int(p)))


def angle_words(seed, step, p):
    """The two Philox words of pair p's scattering angles (stream 4)."""
    return philox4x32_10([int(p) & 0xFFFFFFFF, int(step) & 0xFFFFFFFF, 4, int(step) >> 32],
                         [int(seed) & 0xFFFFFFFF, int(seed) >> 32])[:2]


def collide(u, k, seed, step, ctr_id):
    """The collision of one pair with its own draws (always applied)."""
    uu = np.ascontiguousarray(u, dtype=np.float64)
    kk = np.ascontiguousarray(k, dtype=np.float64)
    uo = np.zeros(3)
    ko = np.zeros(3)
    lib().or_collide(_p(uu), _p(kk), int(seed), int(step), int(ctr_id), _p(uo), _p(ko))
    return uo, ko


def pair_key(seed, step, stream, pid) -> int:
    return int(lib().or_pair_key(int(seed), int(step), int(stream), int(pid)))


def sort_species(cell, pid, n_cells, seed, step, stream):
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    pid = np.ascontiguousarray(pid, dtype=np.uint32)
    n = cell.shape[0]
    perm = np.zeros(n, dtype=np.int64)
    off = np.zeros(n_cells + 1, dtype=np.int64)
    rc = lib().or_sort_species(n, _p(cell), _p(pid), n_cells, int(seed), int(step), int(stream),
                               _p(perm), _p(off))
    if rc != 0:
        raise ValueError("oracle: cell index out of range")
    return perm, off


# --------------------------------------------------------------------------
# Whole step and batch forms
# --------------------------------------------------------------------------
def step(n_cells, w_over_v, dt, seed, step_idx, e, g):
    """One step of the method (Sec. 3.1) on species dicts with keys
    ux,uy,uz (float32), cell (int32), id (uint32).  Photons use ux,uy,uz for
    their momentum k.  Returns a dict of FP64 results in sorted order."""
    def arr(s, key, dt_):
        return np.ascontiguousarray(s[key], dtype=dt_)

    ex, ey, ez = (arr(e, c, np.float32) for c in ("ux", "uy", "uz"))
    gx, gy, gz = (arr(g, c, np.float32) for c in ("ux", "uy", "uz"))
    ec, gc = arr(e, "cell", np.int32), arr(g, "cell", np.int32)
    ei, gi = arr(e, "id", np.uint32), arr(g, "id", np.uint32)
    ne, ng = ex.shape[0], gx.shape[0]
    mp = max(1, min(ne, ng))
    out = dict(
        e_out=np.zeros((3, ne)), g_out=np.zeros((3, ng)),
        e_perm=np.zeros(ne, dtype=np.int64), g_perm=np.zeros(ng, dtype=np.int64),
        e_off=np.zeros(n_cells + 1, dtype=np.int64), g_off=np.zeros(n_cells + 1, dtype=np.int64),
        pair_off=np.zeros(n_cells + 1, dtype=np.int64),
        P=np.zeros(mp), flag=np.zeros(mp, dtype=np.int32), x=np.zeros(mp))
    npairs = lib().or_step(int(n_cells), float(w_over_v), float(dt), int(seed), int(step_idx),
                           ne, _p(ex), _p(ey), _p(ez), _p(ec), _p(ei),
                           ng, _p(gx), _p(gy), _p(gz), _p(gc), _p(gi),
                           _p(out["e_out"]), _p(out["g_out"]), _p(out["e_perm"]), _p(out["g_perm"]),
                           _p(out["e_off"]), _p(out["g_off"]), _p(out["pair_off"]),
                           _p(out["P"]), _p(out["flag"]), _p(out["x"]))
    if npairs < 0:
        raise ValueError("oracle: bad input")
    for key in ("P", "flag", "x"):
        out[key] = out[key][:npairs]
    out["n_pairs"] = int(npairs)
    return out


def step_weighted(n_cells, w_over_v, dt, seed, step_idx, e, g):
    """One step with unequal macro-particle weights (or_step_weighted): the
    species dicts of step() with an optional "w" (float32 weight over the
    cell volume; absent = w_over_v).  Returns step()'s dict plus the sorted
    weights e_w, g_w and upd (bit 0: electron updated, bit 1: photon)."""
    def arr(s, key, dt_):
        return np.ascontiguousarray(s[key], dtype=dt_)

    ex, ey, ez = (arr(e, c, np.float32) for c in ("ux", "uy", "uz"))
    gx, gy, gz = (arr(g, c, np.float32) for c in ("ux", "uy", "uz"))
    ec, gc = arr(e, "cell", np.int32), arr(g, "cell", np.int32)
    ei, gi = arr(e, "id", np.uint32), arr(g, "id", np.uint32)
    ew = arr(e, "w", np.float32) if e.get("w") is not None else None
    gw = arr(g, "w", np.float32) if g.get("w") is not None else None
    ne, ng = ex.shape[0], gx.shape[0]
    mp = max(1, min(ne, ng))
    out = dict(
        e_out=np.zeros((3, ne)), g_out=np.zeros((3, ng)), e_w=np.zeros(ne), g_w=np.zeros(ng),
        e_perm=np.zeros(ne, dtype=np.int64), g_perm=np.zeros(ng, dtype=np.int64),
        e_off=np.zeros(n_cells + 1, dtype=np.int64), g_off=np.zeros(n_cells + 1, dtype=np.int64),
        pair_off=np.zeros(n_cells + 1, dtype=np.int64),
        P=np.zeros(mp), flag=np.zeros(mp, dtype=np.int32), upd=np.zeros(mp, dtype=np.int32))
    npairs = lib().or_step_weighted(int(n_cells), float(w_over_v), float(dt), int(seed), int(step_idx),
                                    ne, _p(ex), _p(ey), _p(ez), _p(ec), _p(ei), None if ew is None else _p(ew),
                                    ng, _p(gx), _p(gy), _p(gz), _p(gc), _p(gi), None if gw is None else _p(gw),
                                    _p(out["e_out"]), _p(out["g_out"]), _p(out["e_w"]), _p(out["g_w"]),
                                    _p(out["e_perm"]), _p(out["g_perm"]), _p(out["e_off"]), _p(out["g_off"]),
                                    _p(out["pair_off"]), _p(out["P"]), _p(out["flag"]), _p(out["upd"]))
    if npairs < 0:
        raise ValueError("oracle: bad input")
    for key in ("P", "flag", "upd"):
        out[key] = out[key][:npairs]
    out["n_pairs"] = int(npairs)
    return out


def ntc_step(n_cells, w_over_v, dt, seed, step_idx, e, g):
    """One step with No-Time-Counter candidate selection (Sec. 3.1) on the
    same species dicts as step().  Returns FP64 momenta in sorted order, the
    sort permutations and offsets, and per cell the candidate and collision
    counts and a flag for decisions within 1e-6 of their ratio."""
    def arr(s, key, dt_):
        return np.ascontiguousarray(s[key], dtype=dt_)

    ex, ey, ez = (arr(e, c, np.float32) for c in ("ux", "uy", "uz"))
    gx, gy, gz = (arr(g, c, np.float32) for c in ("ux", "uy", "uz"))
    ec, gc = arr(e, "cell", np.int32), arr(g, "cell", np.int32)
    ei, gi = arr(e, "id", np.uint32), arr(g, "id", np.uint32)
    ne, ng = ex.shape[0], gx.shape[0]
    out = dict(
        e_out=np.zeros((3, ne)), g_out=np.zeros((3, ng)),
        e_perm=np.zeros(ne, dtype=np.int64), g_perm=np.zeros(ng, dtype=np.int64),
        e_off=np.zeros(n_cells + 1, dtype=np.int64), g_off=np.zeros(n_cells + 1, dtype=np.int64),
        n_cand=np.zeros(n_cells, dtype=np.int64), n_coll=np.zeros(n_cells, dtype=np.int64),
        near=np.zeros(n_cells, dtype=np.int32))
    total = lib().or_ntc_step(int(n_cells), float(w_over_v), float(dt), int(seed), int(step_idx),
                              ne, _p(ex), _p(ey), _p(ez), _p(ec), _p(ei),
                              ng, _p(gx), _p(gy), _p(gz), _p(gc), _p(gi),
                              _p(out["e_out"]), _p(out["g_out"]), _p(out["e_perm"]), _p(out["g_perm"]),
                              _p(out["e_off"]), _p(out["g_off"]), _p(out["n_cand"]), _p(out["n_coll"]),
                              _p(out["near"]))
    if total < 0:
        raise ValueError("oracle: bad input")
    out["total_candidates"] = int(total)
    return out


def pairs(u, k, n_dens, dt, seed, step_idx):
    """Pre-paired events (pair i uses counter id i).  u, k: (3, n) float32;
    n_dens: (n,) float32.  Returns (u_out, k_out, P, flag) in FP64."""
    u = np.ascontiguousarray(u, dtype=np.float32)
    k = np.ascontiguousarray(k, dtype=np.float32)
    nd = np.ascontiguousarray(n_dens, dtype=np.float32)
    n = u.shape[1]
    uo = np.zeros((3, n))
    ko = np.zeros((3, n))
    P = np.zeros(n)
    flag = np.zeros(n, dtype=np.int32)
    lib().or_pairs(n, _p(u[0]), _p(u[1]), _p(u[2]), _p(k[0]), _p(k[1]), _p(k[2]), _p(nd),
                   float(dt), int(seed), int(step_idx), _p(uo), _p(ko), _p(P), _p(flag))
    return uo, ko, P, flag


def ratio(u, k) -> np.ndarray:
    """r = s(x) (1 - beta cos psi) / 2 per pair: the surrogate's target."""
    u = np.ascontiguousarray(u, dtype=np.float32)
    k = np.ascontiguousarray(k, dtype=np.float32)
    n = u.shape[1]
    r = np.zeros(n)
    lib().or_ratio(n, _p(u[0]), _p(u[1]), _p(u[2]), _p(k[0]), _p(k[1]), _p(k[2]), _p(r))
    return r
