"""CPU oracle of the residual-distribution Euler step (test infrastructure).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference legs may import this package.  The
product path (``paper_1705_02028_gb300``) never imports it, and this package
imports nothing from the product path.

The arithmetic lives in ``rd_oracle.cpp`` (plain C++17, templated on the
scalar type, built with ``-O2 -ffp-contract=off``); this module compiles it on
demand and wraps its C interface with numpy arrays.  ``exact.py`` holds the
closed-form solutions used by the physics pins.

Parity status of each function (what pins it is listed in the tests):
  run / run_ld / triangle_terms / stage2_terms / time_step / geometry /
  eigensystem / conserved: pinned (tests/test_oracle_*.py);
  run_tangent / dual_eval: pinned by the closed-form derivative rules of each
  dual-number operation and by central differences of run() with the same
  frozen dt sequence (tests/test_oracle_tangent.py).
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rd_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

N1, B2, LDA2, BMAX2, BMIN2, BX2 = 0, 1, 2, 3, 4, 5
SELECTIVE_LUMPING = 0x100
_BASE = {"N1": N1, "B2": B2, "LDA2": LDA2, "BMAX2": BMAX2, "BMIN2": BMIN2, "BX2": BX2}


def scheme_code(scheme) -> int:
    """Scheme name ("B2", "BMIN2", ...; suffix "_SL" for selective lumping) -> oracle code."""
    if not isinstance(scheme, str):
        return int(scheme)
    name, sl = (scheme[:-3], True) if scheme.endswith("_SL") else (scheme, False)
    return _BASE[name] | (SELECTIVE_LUMPING if sl else 0)


class _Schemes(dict):
    def __missing__(self, key):
        return scheme_code(key)


SCHEMES = _Schemes(_BASE)

_lib = None


def build(force: bool = False) -> str:
    """Compile rd_oracle.cpp into oracle/_build/liboracle.so (OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    cxx = os.environ.get("CXX") or shutil.which("g++") or "g++"
    base = [cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", _SRC]
    tmp = _LIB + ".tmp%d" % os.getpid()
    try:
        subprocess.run(base + ["-fopenmp", "-o", tmp], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i8p = ctypes.POINTER(ctypes.c_int8)
        mesh_args = [ctypes.c_int32, dp, ctypes.c_int32, i32p, i8p, ctypes.c_double, ctypes.c_double]
        for name in ("ora_run", "ora_run_ld"):
            f = getattr(_lib, name)
            f.argtypes = mesh_args + [dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int32, dp, dp, ctypes.c_int]
            f.restype = ctypes.c_int
        _lib.ora_run_tangent.argtypes = mesh_args + [dp, dp, ctypes.c_int, ctypes.c_double,
                                                     ctypes.c_double, ctypes.c_int32, dp, ctypes.c_int]
        _lib.ora_time_step.argtypes = mesh_args + [dp, ctypes.c_double, ctypes.c_double, dp]
        _lib.ora_geometry.argtypes = mesh_args + [dp, dp, dp, dp]
        _lib.ora_triangle_terms.argtypes = mesh_args + [dp, ctypes.c_double, ctypes.c_double] + [dp] * 8
        _lib.ora_triangle_terms_ld.argtypes = mesh_args + [dp, ctypes.c_double, ctypes.c_double] + [dp] * 4
        for f in (_lib.ora_stage2_terms, _lib.ora_stage2_terms_ld):
            f.argtypes = mesh_args + [dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int] + [dp] * 5
        _lib.ora_run_bc.argtypes = mesh_args + [dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_int32, dp, dp, ctypes.c_int,
                                                ctypes.POINTER(ctypes.c_uint8), ctypes.c_int32,
                                                ctypes.POINTER(ctypes.c_int32), ctypes.c_double, ctypes.c_int]
        _lib.ora_run_bc.restype = ctypes.c_int
        for name in ("ora_stage1_shares", "ora_stage1_shares_ld"):
            getattr(_lib, name).argtypes = mesh_args + [dp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                         dp, ctypes.c_int]
        _lib.ora_eigensystem.argtypes = [ctypes.c_double] * 6 + [dp] * 4
        _lib.ora_conserved.argtypes = mesh_args + [dp, dp]
        _lib.ora_dual_eval.argtypes = [ctypes.c_int] + [ctypes.c_double] * 4 + [dp]
        _lib.ora_num_threads.restype = ctypes.c_int
    return _lib


class OracleError(RuntimeError):
    pass


def _p(a, ct=ctypes.c_double):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _mesh_args(mesh):
    xy = np.ascontiguousarray(mesh.xy, dtype=np.float64)
    tri = np.ascontiguousarray(mesh.tri, dtype=np.int32)
    sh = None if mesh.shift is None else np.ascontiguousarray(mesh.shift, dtype=np.int8)
    keep = (xy, tri, sh)
    return keep, [mesh.nv, _p(xy), mesh.nt, _p(tri, ctypes.c_int32), _p(sh, ctypes.c_int8),
                  float(mesh.Lx), float(mesh.Ly)]


def _check(rc, what):
    if rc != 0:
        raise OracleError(f"{what} failed with status {rc}")


def num_threads() -> int:
    return int(lib().ora_num_threads())


def run(mesh, W0, scheme="B2", nsteps=1, cfl=0.8, gamma=1.4, eps=1e-6, dt_fixed=None,
        nthreads=1, long_double=False):
    """Advance W0 (4, nv) by nsteps; returns (W, dt per step)."""
    keep, margs = _mesh_args(mesh)
    W = np.ascontiguousarray(np.array(W0, dtype=np.float64, copy=True))
    dts = np.zeros(max(nsteps, 1))
    dtf = None if dt_fixed is None else np.ascontiguousarray(dt_fixed, dtype=np.float64)
    ghost = getattr(mesh, "ghost", None)
    walls = getattr(mesh, "walls", None)
    if ghost is not None or walls is not None:
        # boundary conditions of Sec. 3.5 (ghost vertices, reflecting walls)
        g = None if ghost is None else np.ascontiguousarray(ghost, dtype=np.uint8)
        wl = np.zeros((0, 2), np.int32) if walls is None else np.ascontiguousarray(walls, dtype=np.int32)
        rc = lib().ora_run_bc(*margs, _p(W), scheme_code(scheme), cfl, gamma, eps, nsteps, _p(dtf), _p(dts),
                              nthreads, _p(g, ctypes.c_uint8), len(wl), _p(wl, ctypes.c_int32),
                              float(getattr(mesh, "alpha", 0.75)), int(bool(long_double)))
        _check(rc, "ora_run_bc")
        del keep
        return W, dts[:nsteps]
    f = lib().ora_run_ld if long_double else lib().ora_run
    rc = f(*margs, _p(W), scheme_code(scheme), cfl, gamma, eps,
           nsteps, _p(dtf), _p(dts), nthreads)
    _check(rc, "ora_run")
    del keep
    return W, dts[:nsteps]


def run_tangent(mesh, W0, dW0, dts, scheme="B2", gamma=1.4, eps=1e-6, nthreads=1):
    """Forward-mode derivative of len(dts) steps with the dt sequence frozen."""
    keep, margs = _mesh_args(mesh)
    W = np.ascontiguousarray(np.array(W0, dtype=np.float64, copy=True))
    dW = np.ascontiguousarray(np.array(dW0, dtype=np.float64, copy=True))
    dtf = np.ascontiguousarray(dts, dtype=np.float64)
    rc = lib().ora_run_tangent(*margs, _p(W), _p(dW), scheme_code(scheme), gamma, eps, len(dtf),
                               _p(dtf), nthreads)
    _check(rc, "ora_run_tangent")
    del keep
    return W, dW


_DUAL_OPS = {"add": 0, "sub": 1, "mul": 2, "div": 3, "sqrt": 4, "fabs": 5, "neg": 6}


def dual_eval(op, a, da, b=0.0, db=0.0):
    """One operation of the oracle's dual-number type: returns (value, derivative)."""
    out = np.zeros(2)
    _check(lib().ora_dual_eval(_DUAL_OPS[op], float(a), float(da), float(b), float(db), _p(out)),
           "ora_dual_eval")
    return float(out[0]), float(out[1])


def time_step(mesh, W, cfl=0.8, gamma=1.4):
    keep, margs = _mesh_args(mesh)
    Wc = np.ascontiguousarray(W, dtype=np.float64)
    out = np.zeros(1)
    _check(lib().ora_time_step(*margs, _p(Wc), cfl, gamma, _p(out)), "ora_time_step")
    del keep
    return float(out[0])


def geometry(mesh):
    keep, margs = _mesh_args(mesh)
    V = np.zeros(mesh.nv)
    area = np.zeros(mesh.nt)
    lmax = np.zeros(mesh.nt)
    normals = np.zeros((mesh.nt, 3, 2))
    _check(lib().ora_geometry(*margs, _p(V), _p(area), _p(lmax), _p(normals)), "ora_geometry")
    del keep
    return dict(V=V, area=area, lmax=lmax, normals=normals)


def triangle_terms(mesh, W, gamma=1.4, eps=1e-6):
    keep, margs = _mesh_args(mesh)
    nt = mesh.nt
    Wc = np.ascontiguousarray(W, dtype=np.float64)
    out = dict(phiT=np.zeros((nt, 4)), phiN=np.zeros((nt, 3, 4)), phiLDA=np.zeros((nt, 3, 4)),
               phiB=np.zeros((nt, 3, 4)), beta=np.zeros((nt, 3, 4, 4)), theta=np.zeros((nt, 4)),
               Kp=np.zeros((nt, 3, 4, 4)), Km=np.zeros((nt, 3, 4, 4)))
    rc = lib().ora_triangle_terms(*margs, _p(Wc), gamma, eps, _p(out["phiT"]), _p(out["phiN"]),
                                  _p(out["phiLDA"]), _p(out["phiB"]), _p(out["beta"]),
                                  _p(out["theta"]), _p(out["Kp"]), _p(out["Km"]))
    _check(rc, "ora_triangle_terms")
    del keep
    return out


def triangle_terms_ld(mesh, W, gamma=1.4, eps=1e-6):
    """phi^T, phi^N, phi^LDA, phi^B evaluated in long double (returned as double)."""
    keep, margs = _mesh_args(mesh)
    nt = mesh.nt
    Wc = np.ascontiguousarray(W, dtype=np.float64)
    out = dict(phiT=np.zeros((nt, 4)), phiN=np.zeros((nt, 3, 4)), phiLDA=np.zeros((nt, 3, 4)),
               phiB=np.zeros((nt, 3, 4)))
    rc = lib().ora_triangle_terms_ld(*margs, _p(Wc), gamma, eps, _p(out["phiT"]), _p(out["phiN"]),
                                     _p(out["phiLDA"]), _p(out["phiB"]))
    _check(rc, "ora_triangle_terms_ld")
    del keep
    return out


def stage1_shares(mesh, W, scheme="B2", gamma=1.4, eps=1e-6, nthreads=1, long_double=False):
    """Stage-1 (forward-Euler) shares of any scheme at state W: (nt, 3, 4)."""
    keep, margs = _mesh_args(mesh)
    Wc = np.ascontiguousarray(W, dtype=np.float64)
    out = np.zeros((mesh.nt, 3, 4))
    f = lib().ora_stage1_shares_ld if long_double else lib().ora_stage1_shares
    _check(f(*margs, _p(Wc), gamma, eps, scheme_code(scheme), _p(out), nthreads), "ora_stage1_shares")
    del keep
    return out


def stage2_terms(mesh, Wn, Ws, dt, gamma=1.4, eps=1e-6, scheme="B2", long_double=False):
    keep, margs = _mesh_args(mesh)
    nt = mesh.nt
    a = np.ascontiguousarray(Wn, dtype=np.float64)
    b = np.ascontiguousarray(Ws, dtype=np.float64)
    out = dict(PhiT=np.zeros((nt, 4)), PhiN=np.zeros((nt, 3, 4)), PhiLDA=np.zeros((nt, 3, 4)),
               Phi=np.zeros((nt, 3, 4)), theta=np.zeros((nt, 4)))
    f = lib().ora_stage2_terms_ld if long_double else lib().ora_stage2_terms
    rc = f(*margs, _p(a), _p(b), dt, gamma, eps, scheme_code(scheme),
                                _p(out["PhiT"]), _p(out["PhiN"]), _p(out["PhiLDA"]), _p(out["Phi"]),
                                _p(out["theta"]))
    _check(rc, "ora_stage2_terms")
    del keep
    return out


def eigensystem(u, v, h, nx, ny, gamma=1.4):
    K = np.zeros((4, 4))
    lam = np.zeros(4)
    R = np.zeros((4, 4))
    L = np.zeros((4, 4))
    _check(lib().ora_eigensystem(u, v, h, gamma, nx, ny, _p(K), _p(lam), _p(R), _p(L)),
           "ora_eigensystem")
    return K, lam, R, L


def conserved(mesh, W):
    keep, margs = _mesh_args(mesh)
    Wc = np.ascontiguousarray(W, dtype=np.float64)
    out = np.zeros(4)
    _check(lib().ora_conserved(*margs, _p(Wc), _p(out)), "ora_conserved")
    del keep
    return out
