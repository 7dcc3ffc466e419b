"""Thin Python binding of the C ABI in include/rd.h (argument marshalling only).

Every step of the solver runs in the CUDA library ``_lib/librd.so``; this
module converts numpy arrays to pointers, installs PyTorch's caching allocator
as the library's device allocator, and hands the library a PyTorch CUDA stream.
There is no CPU fallback: if the library or a GPU is missing, every entry point
raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

RD_OK, RD_EINVAL, RD_ENOMEM, RD_ECUDA, RD_ENONPHYSICAL, RD_ETIMEOUT, RD_ENOTSUP = range(7)
SCHEMES = {"N1": 0, "B2": 1, "LDA2": 2, "BMAX2": 3, "BMIN2": 4, "BX2": 5}
LUMPING = {"global": 0, "selective": 1}
PRECISIONS = {"fp64": 0, "fp32": 1, "df64": 2}
ORDERS = {"none": 0, "morton": 1, "rcm": 2}

_lib = None
_alloc_refs = None


class RDError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        msg = _lib.rd_strerror(status).decode() if _lib is not None else str(status)
        super().__init__(f"{what}: {msg} (status {status})")


class MeshgenParams(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("max_circumradius", ctypes.c_double),
                ("quality", ctypes.c_double), ("nx0", ctypes.c_int32), ("ny0", ctypes.c_int32),
                ("max_vertices", ctypes.c_int32), ("max_rounds", ctypes.c_int32),
                ("max_flip_rounds", ctypes.c_int32), ("reserved", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class Params(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int32), ("precision", ctypes.c_int32), ("cfl", ctypes.c_double),
                ("gamma", ctypes.c_double), ("eps_fix", ctypes.c_double), ("lumping", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


_dp = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i8p = ctypes.POINTER(ctypes.c_int8)
_vp = ctypes.c_void_p

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

# name -> (restype, argtypes)
_SIGS = {
    "rd_set_allocator": (ctypes.c_int, [ALLOC_FN, FREE_FN, _vp]),
    "rd_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "rd_version": (ctypes.c_int, []),
    "rd_mesh_create": (ctypes.c_int, [ctypes.c_int32, _dp, ctypes.c_int32, _i32p, _i8p, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int32, _vp, ctypes.POINTER(_vp)]),
    "rd_mesh_destroy": (None, [_vp]),
    "rd_mesh_permutation": (ctypes.c_int, [_vp, _i32p, _i32p]),
    "rd_mesh_sizes": (ctypes.c_int, [_vp, _i32p, _i32p]),
    "rd_mesh_set_boundary": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint8), ctypes.c_int32, _i32p,
                                            ctypes.c_double]),
    "rd_meshgen_run": (ctypes.c_int, [_vp, _vp, _vp]),
    "rd_meshgen_sizes": (ctypes.c_int, [_vp, _i32p, _i32p, _i32p, _i32p]),
    "rd_meshgen_times": (ctypes.c_int, [_vp, _dp]),
    "rd_meshgen_get": (ctypes.c_int, [_vp, _dp, _i32p, ctypes.POINTER(ctypes.c_int8), ctypes.POINTER(ctypes.c_int64)]),
    "rd_meshgen_domain": (ctypes.c_int, [_vp, _dp, _dp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "rd_meshgen_destroy": (None, [_vp]),
    "rd_state_init": (ctypes.c_int, [_vp, _dp, ctypes.POINTER(Params), ctypes.POINTER(_vp)]),
    "rd_state_set": (ctypes.c_int, [_vp, _dp]),
    "rd_step": (ctypes.c_int, [_vp, _dp]),
    "rd_run": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_double, _i32p]),
    "rd_get_state": (ctypes.c_int, [_vp, _dp]),
    "rd_conserved_totals": (ctypes.c_int, [_vp, _dp]),
    "rd_get_time": (ctypes.c_int, [_vp, _dp, ctypes.POINTER(ctypes.c_int64)]),
    "rd_get_dt": (ctypes.c_int, [_vp, _dp]),
    "rd_state_destroy": (None, [_vp]),
    "rd_state_triangle_shares": (ctypes.c_int, [_vp, ctypes.c_int32, _dp, _dp]),
    "rd_cfl_dt": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, _vp,
                                 ctypes.c_double, ctypes.c_double, _vp, _vp]),
    "rd_cfl_dt_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp,
                                         _vp, ctypes.c_double, ctypes.c_double, _vp, _vp]),
    "rd_state_profile": (ctypes.c_int, [_vp, ctypes.c_int32, _dp, _i32p]),
    "rd_count_flops": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _dp]),
    "rd_probe_fma_peak": (ctypes.c_int, [ctypes.c_int32, _dp]),
    "rd_math_eval": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, _vp, _vp, _vp]),
    "rd_batch_create": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(_vp), ctypes.POINTER(_dp),
                                       ctypes.POINTER(Params), ctypes.POINTER(_vp)]),
    "rd_batch_run": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "rd_batch_get_state": (ctypes.c_int, [_vp, ctypes.c_int32, _dp]),
    "rd_batch_get_dt": (ctypes.c_int, [_vp, _dp]),
    "rd_batch_destroy": (None, [_vp]),
    "rd_state_autotune": (ctypes.c_int, [_vp, _i32p, _i32p]),
    "rd_state_launch_shapes": (ctypes.c_int, [_vp, _i32p, _i32p, _i32p]),
    "rd_state_set_launch_shapes": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "rd_state_stage_shapes": (ctypes.c_int, [_vp, ctypes.c_int32, _i32p, _i32p]),
    "rd_state_set_stage_shapes": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "rd_state_set_tiling": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32]),
    "rd_state_set_tiling_ex": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "rd_state_get_tiling_flags": (ctypes.c_int, [_vp, _i32p]),
    "rd_state_get_tiling": (ctypes.c_int, [_vp, _i32p, _i32p, _i32p]),
    "rd_adjoint_forward": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, _dp]),
    "rd_adjoint_backward": (ctypes.c_int, [_vp, _dp, _dp]),
    "rd_run_fixed_dt": (ctypes.c_int, [_vp, ctypes.c_int32, _dp]),
    "rd_state_branch_masks": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "rd_batch_get_time": (ctypes.c_int, [_vp, _dp, ctypes.POINTER(ctypes.c_int64)]),
    "rd_batch_sizes": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "rd_batch_autotune": (ctypes.c_int, [_vp, _i32p, _i32p]),
    "rd_batch_profile": (ctypes.c_int, [_vp, ctypes.c_int32, _dp]),
    "rd_partition_plan": (ctypes.c_int, [ctypes.c_int32, _dp, ctypes.c_int32, _i32p, _i8p, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _i32p,
                                         _i32p, _i32p, _i32p, _i32p, _i32p, _i32p, _i32p, _i32p]),
    "rd_part_create": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, _dp, ctypes.POINTER(Params),
                                      ctypes.POINTER(_vp)]),
    "rd_part_sizes": (ctypes.c_int, [_vp, _i32p]),
    "rd_part_lists": (ctypes.c_int, [_vp, _i32p, _i32p, _i32p]),
    "rd_part_phase": (ctypes.c_int, [_vp, ctypes.c_int32, _vp]),
    "rd_part_dt_device": (ctypes.c_int, [_vp, ctypes.POINTER(_vp)]),
    "rd_part_get_dt": (ctypes.c_int, [_vp, _dp]),
    "rd_part_set_dt": (ctypes.c_int, [_vp, ctypes.c_double]),
    "rd_part_get_owned": (ctypes.c_int, [_vp, _dp]),
    "rd_part_status": (ctypes.c_int, [_vp, _dp, ctypes.POINTER(ctypes.c_int64)]),
    "rd_part_destroy": (None, [_vp]),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load librd.so (building it in-tree if needed).  Raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"CUDA library {_build.LIB} is missing; run build() first")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc, what):
    if rc != RD_OK:
        raise RDError(rc, what)


def _ptr(a, ct=ctypes.c_double):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ct))


def _require_gpu():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the residual-distribution library needs a CUDA GPU; none is available")
    return torch


def use_torch_allocator():
    """Route the library's device allocations through PyTorch's caching allocator."""
    global _alloc_refs
    if _alloc_refs is not None:
        return
    torch = _require_gpu()
    lib = load()

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      int(stream or 0))
        except Exception:
            return None

    def _free(ptr, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    refs = (ALLOC_FN(_alloc), FREE_FN(_free))
    _check(lib.rd_set_allocator(refs[0], refs[1], None), "rd_set_allocator")
    _alloc_refs = refs


def count_flops(scheme: str, stage: int):
    """Counted (add, mul, div, sqrt) of one triangle in a stage's triangle kernel."""
    lib = load()
    out = np.zeros(4)
    _check(lib.rd_count_flops(SCHEMES[scheme], int(stage), _ptr(out)), "rd_count_flops")
    return dict(add=out[0], mul=out[1], div=out[2], sqrt=out[3], total=float(out.sum()))


def probe_fma_peak(precision: str = "fp64") -> float:
    """Measured FMA throughput of the current GPU in flop/s."""
    _require_gpu()
    lib = load()
    out = ctypes.c_double()
    _check(lib.rd_probe_fma_peak(PRECISIONS[precision], ctypes.byref(out)), "rd_probe_fma_peak")
    return out.value


MATH_FNS = {"rcp": 0}


def math_eval(fn: str, x):
    """The triangle kernels' arithmetic helper `fn` applied element-wise to a float64
    CUDA tensor x (rd_math_eval); returns a new tensor."""
    torch = _require_gpu()
    lib = load()
    x = x.contiguous()
    out = torch.empty_like(x)
    st = torch.cuda.current_stream(x.device)
    _check(lib.rd_math_eval(MATH_FNS[fn], x.numel(), _vp(x.data_ptr()), _vp(out.data_ptr()),
                            _vp(st.cuda_stream)), "rd_math_eval")
    return out


def cfl_dt(W, tri, lmax, V, csr_ptr, csr_ent, precision="fp64", gamma=1.4, cfl=0.8, stream=None,
           entry="rd_cfl_dt") -> float:
    """CFL time step of a state held in torch CUDA tensors (rd_cfl_dt).

    W (4, nv), lmax (nt,), V (nv,): float64 or float32 CUDA tensors; tri (3, nt),
    csr_ptr (nv+1,), csr_ent (3 nt,): int32 CUDA tensors (caller-owned)."""
    torch = _require_gpu()
    lib = load()
    nv, nt = int(W.shape[1]), int(tri.shape[1])
    out = torch.zeros(1, dtype=torch.float64, device=W.device)
    st = stream if stream is not None else torch.cuda.current_stream(W.device)
    rc = getattr(lib, entry)(nv, nt, PRECISIONS[precision], W.data_ptr(), tri.data_ptr(), lmax.data_ptr(),
                             V.data_ptr(), csr_ptr.data_ptr(), csr_ent.data_ptr(), float(gamma), float(cfl),
                             out.data_ptr(), _vp(st.cuda_stream))
    _check(rc, entry)
    return float(out.item())


def _params(scheme, precision, cfl, gamma, eps_fix, lumping="global") -> Params:
    """Scheme name ("B2", "BMIN2", ...; the suffix "_SL" selects selective lumping) -> rd_params."""
    if isinstance(scheme, str) and scheme.endswith("_SL"):
        scheme, lumping = scheme[:-3], "selective"
    return Params(SCHEMES[scheme] if isinstance(scheme, str) else int(scheme),
                  PRECISIONS[precision] if isinstance(precision, str) else int(precision),
                  float(cfl), float(gamma), float(eps_fix),
                  LUMPING[lumping] if isinstance(lumping, str) else int(lumping), 0)


class Mesh:
    """Device mesh store (rd_mesh_create) built from an inputs.Mesh-like object."""

    def __init__(self, mesh, reorder: str = "morton", stream=None, allocator: str = "torch"):
        torch = _require_gpu()
        lib = load()
        if allocator == "torch":
            use_torch_allocator()
        self._stream = stream if stream is not None else torch.cuda.Stream()
        self.nv, self.nt = int(mesh.nv), int(mesh.nt)
        xy = np.ascontiguousarray(mesh.xy, dtype=np.float64)
        tri = np.ascontiguousarray(mesh.tri, dtype=np.int32)
        sh = None if mesh.shift is None else np.ascontiguousarray(mesh.shift, dtype=np.int8)
        h = _vp()
        rc = lib.rd_mesh_create(self.nv, _ptr(xy), self.nt, _ptr(tri, ctypes.c_int32), _ptr(sh, ctypes.c_int8),
                                float(mesh.Lx), float(mesh.Ly), ORDERS[reorder],
                                _vp(self._stream.cuda_stream), ctypes.byref(h))
        _check(rc, "rd_mesh_create")
        self.handle = h
        self.states = []
        self.has_boundary = False
        ghost, walls = getattr(mesh, "ghost", None), getattr(mesh, "walls", None)
        if ghost is not None or walls is not None:
            self.set_boundary(ghost, walls, getattr(mesh, "alpha", 0.75))

    def set_boundary(self, ghost=None, walls=None, alpha: float = 0.75):
        """Ghost vertices ([nv] flags) and reflecting walls ([n][2] (triangle, corner)), Sec. 3.5."""
        g = None if ghost is None else np.ascontiguousarray(ghost, dtype=np.uint8)
        w = np.zeros((0, 2), np.int32) if walls is None else np.ascontiguousarray(walls, dtype=np.int32)
        _check(_lib.rd_mesh_set_boundary(self.handle, _ptr(g, ctypes.c_uint8), len(w), _ptr(w, ctypes.c_int32),
                                         float(alpha)), "rd_mesh_set_boundary")
        self.has_boundary = bool(len(w)) or (g is not None and bool(g.any()))

    @property
    def stream(self):
        return self._stream

    def permutation(self):
        vp = np.empty(self.nv, dtype=np.int32)
        tp = np.empty(self.nt, dtype=np.int32)
        _check(_lib.rd_mesh_permutation(self.handle, _ptr(vp, ctypes.c_int32), _ptr(tp, ctypes.c_int32)),
               "rd_mesh_permutation")
        return vp, tp

    def close(self):
        if getattr(self, "handle", None):
            for s in list(self.states):
                s.close()
            _lib.rd_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class State:
    """Solver state on one mesh (rd_state_init ... rd_state_destroy)."""

    def __init__(self, mesh: Mesh, W, scheme="B2", precision="fp64", cfl=0.8, gamma=1.4, eps_fix=1e-6,
                 lumping="global"):
        load()
        self.mesh = mesh
        self.scheme = scheme
        self.params = _params(scheme, precision, cfl, gamma, eps_fix, lumping)
        Wc = np.ascontiguousarray(W, dtype=np.float64)
        if Wc.shape != (4, mesh.nv):
            raise ValueError(f"W must have shape (4, {mesh.nv})")
        h = _vp()
        _check(_lib.rd_state_init(mesh.handle, _ptr(Wc), ctypes.byref(self.params), ctypes.byref(h)),
               "rd_state_init")
        self.handle = h
        mesh.states.append(self)

    def step(self, return_dt: bool = False):
        dt = ctypes.c_double(0.0)
        _check(_lib.rd_step(self.handle, ctypes.byref(dt) if return_dt else None), "rd_step")
        return dt.value if return_dt else None

    def run(self, n_steps: int, t_end: float = 0.0) -> int:
        done = ctypes.c_int32(0)
        _check(_lib.rd_run(self.handle, int(n_steps), float(t_end), ctypes.byref(done)), "rd_run")
        return done.value

    def get(self, out=None) -> np.ndarray:
        W = out if out is not None else np.empty((4, self.mesh.nv), dtype=np.float64)
        _check(_lib.rd_get_state(self.handle, _ptr(W)), "rd_get_state")
        return W

    def set(self, W):
        Wc = np.ascontiguousarray(W, dtype=np.float64)
        _check(_lib.rd_state_set(self.handle, _ptr(Wc)), "rd_state_set")

    def conserved(self) -> np.ndarray:
        out = np.zeros(4)
        _check(_lib.rd_conserved_totals(self.handle, _ptr(out)), "rd_conserved_totals")
        return out

    def time(self):
        t = ctypes.c_double()
        n = ctypes.c_int64()
        _check(_lib.rd_get_time(self.handle, ctypes.byref(t), ctypes.byref(n)), "rd_get_time")
        return t.value, n.value

    def dt(self) -> float:
        d = ctypes.c_double()
        _check(_lib.rd_get_dt(self.handle, ctypes.byref(d)), "rd_get_dt")
        return d.value

    def triangle_shares(self, which: str = "B"):
        w = {"N": 0, "LDA": 1, "B": 2}[which]
        out = np.empty((self.mesh.nt, 3, 4))
        cfl = np.empty(self.mesh.nt)
        _check(_lib.rd_state_triangle_shares(self.handle, w, _ptr(out), _ptr(cfl)), "rd_state_triangle_shares")
        return out, cfl

    def profile(self, n_steps: int):
        """Mean per-kernel milliseconds over n_steps real steps (CUDA events on the mesh stream)."""
        ms = np.zeros(6)
        n = ctypes.c_int32(0)
        _check(_lib.rd_state_profile(self.handle, int(n_steps), _ptr(ms), ctypes.byref(n)), "rd_state_profile")
        names = ["tri_stage1", "gather_cfl", "update1", "tri_stage2", "update2", "commit"]
        if self.tiling()[0] > 0:
            names[0:2] = ["tile_stage1", "tile_bnd1"]
            if str(self.scheme).split("_")[0] not in ("N1", "BX2") and not self.mesh.has_boundary:
                names[3:5] = ["tile_stage2", "tile_bnd2"]
        return dict(zip(names, ms.tolist())), n.value

    def run_fixed_dt(self, dts):
        """Steps with a prescribed dt sequence (rd_run_fixed_dt)."""
        d = np.ascontiguousarray(dts, dtype=np.float64)
        _check(_lib.rd_run_fixed_dt(self.handle, len(d), _ptr(d)), "rd_run_fixed_dt")

    def adjoint_forward(self, n_steps: int, ckpt_every: int = 20) -> np.ndarray:
        """Rollout of n_steps recording dt and checkpoints; returns the dt sequence."""
        dts = np.empty(int(n_steps))
        _check(_lib.rd_adjoint_forward(self.handle, int(n_steps), int(ckpt_every), _ptr(dts)),
               "rd_adjoint_forward")
        return dts

    def adjoint_backward(self, dL_dW_final) -> np.ndarray:
        """dL/dW0 of the last adjoint_forward rollout (dt sequence held fixed)."""
        g = np.ascontiguousarray(dL_dW_final, dtype=np.float64)
        out = np.empty((4, self.mesh.nv))
        _check(_lib.rd_adjoint_backward(self.handle, _ptr(g), _ptr(out)), "rd_adjoint_backward")
        return out

    def branch_masks(self):
        """Per-triangle branch masks of the next step (stage 1, stage 2)."""
        m1 = np.zeros(self.mesh.nt, dtype=np.uint64)
        m2 = np.zeros(self.mesh.nt, dtype=np.uint64)
        _check(_lib.rd_state_branch_masks(self.handle, _ptr(m1, ctypes.c_uint64), _ptr(m2, ctypes.c_uint64)),
               "rd_state_branch_masks")
        return m1, m2

    def autotune(self):
        """Pick the fastest launch shapes for this state (rd_state_autotune)."""
        tb, vb = ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.rd_state_autotune(self.handle, ctypes.byref(tb), ctypes.byref(vb)), "rd_state_autotune")
        return tb.value, vb.value

    def launch_shapes(self):
        """(triangle block, vertex block, DF64 kernel variant) in use (rd_state_launch_shapes)."""
        tb, vb, oc = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.rd_state_launch_shapes(self.handle, ctypes.byref(tb), ctypes.byref(vb), ctypes.byref(oc)),
               "rd_state_launch_shapes")
        return tb.value, vb.value, oc.value

    def set_launch_shapes(self, tri_block: int, vtx_block: int, df_variant: int = 2):
        """The same triangle block and DF64 variant for both stages (rd_state_set_launch_shapes)."""
        _check(_lib.rd_state_set_launch_shapes(self.handle, int(tri_block), int(vtx_block), int(df_variant)),
               "rd_state_set_launch_shapes")

    def stage_shapes(self, stage: int):
        """(triangle block, DF64 kernel variant) of stage 1 or 2 (rd_state_stage_shapes)."""
        tb, oc = ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.rd_state_stage_shapes(self.handle, int(stage), ctypes.byref(tb), ctypes.byref(oc)),
               "rd_state_stage_shapes")
        return tb.value, oc.value

    def set_stage_shapes(self, stage: int, tri_block: int, df_variant: int = 2):
        _check(_lib.rd_state_set_stage_shapes(self.handle, int(stage), int(tri_block), int(df_variant)),
               "rd_state_set_stage_shapes")

    def set_tiling(self, tile_triangles: int, threads: int = 128, stage_geometry: bool = False):
        """Tiled step with tiles of `tile_triangles` triangles (0: untiled); rd_state_set_tiling_ex,
        with the tile's geometry staged in shared memory when stage_geometry."""
        _check(_lib.rd_state_set_tiling_ex(self.handle, int(tile_triangles), int(threads), 1 if stage_geometry else 0),
               "rd_state_set_tiling_ex")

    def tiling_flags(self) -> int:
        out = ctypes.c_int32()
        _check(_lib.rd_state_get_tiling_flags(self.handle, ctypes.byref(out)), "rd_state_get_tiling_flags")
        return out.value

    def tiling(self):
        """(tile_triangles, threads, boundary vertices) of the current tiling; zeros when untiled."""
        tt, bt, nb = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.rd_state_get_tiling(self.handle, ctypes.byref(tt), ctypes.byref(bt), ctypes.byref(nb)),
               "rd_state_get_tiling")
        return tt.value, bt.value, nb.value

    def close(self):
        if getattr(self, "handle", None):
            _lib.rd_state_destroy(self.handle)
            self.handle = None
            if self in self.mesh.states:
                self.mesh.states.remove(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent meshes advanced together (rd_batch_create ... rd_batch_destroy)."""

    def __init__(self, meshes, states, scheme="B2", precision="fp64", cfl=0.8, gamma=1.4, eps_fix=1e-6,
                 lumping="global"):
        load()
        self.meshes = list(meshes)
        self.params = _params(scheme, precision, cfl, gamma, eps_fix, lumping)
        self._W = [np.ascontiguousarray(W, dtype=np.float64) for W in states]
        for m, W in zip(self.meshes, self._W):
            if W.shape != (4, m.nv):
                raise ValueError("each state must have shape (4, nv) of its mesh")
        n = len(self.meshes)
        hs = (_vp * n)(*[m.handle for m in self.meshes])
        ws = (_dp * n)(*[_ptr(W) for W in self._W])
        h = _vp()
        _check(_lib.rd_batch_create(n, hs, ws, ctypes.byref(self.params), ctypes.byref(h)), "rd_batch_create")
        self.handle = h
        self._W = None

    @property
    def n_mesh(self):
        return len(self.meshes)

    def sizes(self):
        nv, nt = ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.rd_batch_sizes(self.handle, ctypes.byref(nv), ctypes.byref(nt)), "rd_batch_sizes")
        return nv.value, nt.value

    def run(self, n_steps: int):
        _check(_lib.rd_batch_run(self.handle, int(n_steps)), "rd_batch_run")

    def get(self, m: int) -> np.ndarray:
        W = np.empty((4, self.meshes[m].nv))
        _check(_lib.rd_batch_get_state(self.handle, int(m), _ptr(W)), "rd_batch_get_state")
        return W

    def dt(self) -> np.ndarray:
        out = np.empty(self.n_mesh)
        _check(_lib.rd_batch_get_dt(self.handle, _ptr(out)), "rd_batch_get_dt")
        return out

    def time(self):
        t = np.empty(self.n_mesh)
        n = np.empty(self.n_mesh, dtype=np.int64)
        _check(_lib.rd_batch_get_time(self.handle, _ptr(t), _ptr(n, ctypes.c_int64)), "rd_batch_get_time")
        return t, n

    def autotune(self):
        tb, vb = ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.rd_batch_autotune(self.handle, ctypes.byref(tb), ctypes.byref(vb)), "rd_batch_autotune")
        return tb.value, vb.value

    def profile(self, n_steps: int):
        ms = np.zeros(6)
        _check(_lib.rd_batch_profile(self.handle, int(n_steps), _ptr(ms)), "rd_batch_profile")
        names = ("tri_stage1", "gather_cfl", "update1", "tri_stage2", "update2", "commit")
        return dict(zip(names, ms.tolist()))

    def close(self):
        if getattr(self, "handle", None):
            _lib.rd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rollout(state: "State", W0, n_steps: int, ckpt_every: int = 20):
    """Differentiable rollout: W_final = F^{n_steps}(W0) as a torch.autograd.Function.

    W0 is a float64 CPU tensor of shape (4, nv) in the caller's vertex order; the
    forward pass records the dt sequence (held fixed by the backward pass, which
    runs the library's hand-written adjoint kernels with checkpoints every
    `ckpt_every` steps)."""
    import torch

    class _Rollout(torch.autograd.Function):
        @staticmethod
        def forward(ctx, w0):
            state.set(w0.detach().cpu().numpy())
            ctx.dts = state.adjoint_forward(n_steps, ckpt_every)
            return torch.from_numpy(state.get())

        @staticmethod
        def backward(ctx, grad_out):
            g0 = state.adjoint_backward(grad_out.detach().cpu().numpy())
            return torch.from_numpy(g0)

    return _Rollout.apply(W0)


def meshgen(max_circumradius: float, Lx: float = 1.0, Ly: float = 1.0, quality: float = 2.0 ** 0.5,
            nx0: int = 4, ny0: int = 4, max_vertices: int | None = None, seed: int = 7,
            max_rounds: int = 10000, max_flip_rounds: int = 10000, stream=None):
    """Periodic Delaunay refinement on the GPU (rd_meshgen_run).  Returns (mesh, info):
    an inputs.Mesh of the generated triangulation (xy, tri, shift, periods) and a dict
    with the integer coordinates, round / flip counts, per-phase times and the status."""
    torch = _require_gpu()
    lib = load()
    from . import inputs
    if max_vertices is None:
        # about 1.3 vertices per (R^2) of area for beta <= sqrt 2 meshes, with headroom
        max_vertices = int(4.0 * Lx * Ly / (max_circumradius ** 2)) + 4 * nx0 * ny0 + 1024
    p = MeshgenParams(float(Lx), float(Ly), float(max_circumradius), float(quality), int(nx0), int(ny0),
                      int(max_vertices), int(max_rounds), int(max_flip_rounds), 0, int(seed))
    st = stream if stream is not None else torch.cuda.Stream()
    h = _vp()
    rc = lib.rd_meshgen_run(ctypes.byref(p), _vp(st.cuda_stream), ctypes.byref(h))
    if not h:
        _check(rc, "rd_meshgen_run")
    try:
        nv, nt, rounds, flips = (ctypes.c_int32() for _ in range(4))
        _check(lib.rd_meshgen_sizes(h, ctypes.byref(nv), ctypes.byref(nt), ctypes.byref(rounds), ctypes.byref(flips)),
               "rd_meshgen_sizes")
        nv, nt = nv.value, nt.value
        xy = np.empty((nv, 2))
        tri = np.empty((nt, 3), dtype=np.int32)
        shift = np.empty((nt, 3, 2), dtype=np.int8)
        xyu = np.empty((nv, 2), dtype=np.int64)
        _check(lib.rd_meshgen_get(h, _ptr(xy), _ptr(tri, ctypes.c_int32), _ptr(shift, ctypes.c_int8),
                                  _ptr(xyu, ctypes.c_int64)), "rd_meshgen_get")
        ms = np.zeros(5)
        _check(lib.rd_meshgen_times(h, _ptr(ms)), "rd_meshgen_times")
        lx, ly = ctypes.c_double(), ctypes.c_double()
        px, py = ctypes.c_int64(), ctypes.c_int64()
        _check(lib.rd_meshgen_domain(h, ctypes.byref(lx), ctypes.byref(ly), ctypes.byref(px), ctypes.byref(py)),
               "rd_meshgen_domain")
    finally:
        lib.rd_meshgen_destroy(h)
    mesh = inputs.Mesh(xy=xy, tri=tri, shift=shift, Lx=lx.value, Ly=ly.value,
                       orig_vertex=np.arange(nv, dtype=np.int64))
    info = dict(status=rc, rounds=rounds.value, flips=flips.value, xy_units=xyu, Px=px.value, Py=py.value,
                unit=lx.value / px.value,
                ms=dict(zip(("quality_locate", "cavities", "insert", "flips", "total"), ms.tolist())))
    return mesh, info


# ---------------------------------------------------------------------------
# vertex-partitioned step (rd_partition_plan, rd_part_*)
# ---------------------------------------------------------------------------
PART_PACK_W, PART_UNPACK_W, PART_STAGE1, PART_UPDATE1, PART_PACK_WS, PART_UNPACK_WS, PART_STAGE2 = range(7)


def partition_plan(mesh, n_parts: int, part: int, reorder: str = "morton") -> dict:
    """Plan of one part of a vertex partition, computed on the host (no GPU needed)."""
    lib = load()
    xy = np.ascontiguousarray(mesh.xy, dtype=np.float64)
    tri = np.ascontiguousarray(mesh.tri, dtype=np.int32)
    sh = None if mesh.shift is None else np.ascontiguousarray(mesh.shift, dtype=np.int8)
    args = (int(mesh.nv), _ptr(xy), int(mesh.nt), _ptr(tri, ctypes.c_int32), _ptr(sh, ctypes.c_int8),
            float(mesh.Lx), float(mesh.Ly), ORDERS[reorder], int(n_parts), int(part))
    sizes = np.zeros(4, dtype=np.int32)
    i32 = lambda a: _ptr(a, ctypes.c_int32)
    _check(lib.rd_partition_plan(*args, i32(sizes), *([None] * 8)), "rd_partition_plan")
    n_own, n_gh, nlt, n_send = (int(x) for x in sizes)
    out = dict(n_owned=n_own, n_ghost=n_gh, n_local_tri=nlt, n_send=n_send,
               local_vertices=np.empty(n_own + n_gh, np.int32), local_triangles=np.empty(nlt, np.int32),
               local_corners=np.empty((3, nlt), np.int32), csr_ptr=np.empty(n_own + 1, np.int32),
               csr_ent=np.empty(0, np.int32), send_ptr=np.empty(n_parts + 1, np.int32),
               send_idx=np.empty(n_send, np.int32), recv_ptr=np.empty(n_parts + 1, np.int32))
    _check(lib.rd_partition_plan(*args, i32(sizes), None, None, None, i32(out["csr_ptr"]), None, None, None, None),
           "rd_partition_plan")
    out["csr_ent"] = np.empty(int(out["csr_ptr"][-1]), np.int32)
    _check(lib.rd_partition_plan(*args, i32(sizes), i32(out["local_vertices"]), i32(out["local_triangles"]),
                                 i32(out["local_corners"]), i32(out["csr_ptr"]), i32(out["csr_ent"]),
                                 i32(out["send_ptr"]), i32(out["send_idx"]), i32(out["recv_ptr"])),
           "rd_partition_plan")
    return out


class Part:
    """One part of a vertex-partitioned state (rd_part_create ... rd_part_destroy)."""

    def __init__(self, mesh: Mesh, n_parts: int, part: int, W, scheme="B2", precision="fp64", cfl=0.8, gamma=1.4,
                 eps_fix=1e-6, lumping="global"):
        torch = _require_gpu()
        load()
        self.mesh = mesh
        self.n_parts, self.part = int(n_parts), int(part)
        self.params = _params(scheme, precision, cfl, gamma, eps_fix, lumping)
        self.two_stage = self.params.scheme != SCHEMES["N1"]
        Wc = np.ascontiguousarray(W, dtype=np.float64)
        if Wc.shape != (4, mesh.nv):
            raise ValueError(f"W must have shape (4, {mesh.nv})")
        h = _vp()
        _check(_lib.rd_part_create(mesh.handle, self.n_parts, self.part, _ptr(Wc), ctypes.byref(self.params),
                                   ctypes.byref(h)), "rd_part_create")
        self.handle = h
        sz = np.zeros(4, dtype=np.int32)
        _check(_lib.rd_part_sizes(h, _ptr(sz, ctypes.c_int32)), "rd_part_sizes")
        self.n_owned, self.n_ghost, self.n_local_tri, self.n_send = (int(x) for x in sz)
        self.local_vertices = np.empty(self.n_owned + self.n_ghost, np.int32)
        self.send_ptr = np.empty(self.n_parts + 1, np.int32)
        self.recv_ptr = np.empty(self.n_parts + 1, np.int32)
        _check(_lib.rd_part_lists(h, _ptr(self.local_vertices, ctypes.c_int32), _ptr(self.send_ptr, ctypes.c_int32),
                                  _ptr(self.recv_ptr, ctypes.c_int32)), "rd_part_lists")
        dtype = torch.float32 if self.params.precision == PRECISIONS["fp32"] else torch.float64
        dev = torch.device("cuda", torch.cuda.current_device())
        self.send_buf = torch.empty((max(self.n_send, 1), 4), dtype=dtype, device=dev)
        self.recv_buf = torch.empty((max(self.n_ghost, 1), 4), dtype=dtype, device=dev)
        dp = _vp()
        _check(_lib.rd_part_dt_device(h, ctypes.byref(dp)), "rd_part_dt_device")
        self._dt_ptr = dp.value

    def phase(self, ph: int, buf=None):
        _check(_lib.rd_part_phase(self.handle, int(ph), _vp(buf.data_ptr()) if buf is not None else None),
               "rd_part_phase")

    def dt_tensor(self):
        """A one-element float64 CUDA tensor viewing this part's dt in place (for an all-reduce)."""
        import torch

        class _View:
            pass
        v = _View()
        v.__cuda_array_interface__ = {"shape": (1,), "typestr": "<f8", "data": (self._dt_ptr, False), "version": 3}
        return torch.as_tensor(v, device=torch.device("cuda", torch.cuda.current_device()))

    def get_dt(self) -> float:
        out = ctypes.c_double()
        _check(_lib.rd_part_get_dt(self.handle, ctypes.byref(out)), "rd_part_get_dt")
        return out.value

    def set_dt(self, dt: float):
        _check(_lib.rd_part_set_dt(self.handle, float(dt)), "rd_part_set_dt")

    def owned(self) -> np.ndarray:
        W = np.empty((4, self.n_owned))
        _check(_lib.rd_part_get_owned(self.handle, _ptr(W)), "rd_part_get_owned")
        return W

    def status(self):
        t, n = ctypes.c_double(), ctypes.c_int64()
        _check(_lib.rd_part_status(self.handle, ctypes.byref(t), ctypes.byref(n)), "rd_part_status")
        return t.value, n.value

    def close(self):
        if getattr(self, "handle", None):
            _lib.rd_part_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _exchange_local(parts, pack, unpack):
    """Ghost exchange between parts that share one device: each part packs its
    send list, then copies the slice part q needs into q's receive buffer."""
    import torch
    for p in parts:
        p.phase(pack, p.send_buf)
    torch.cuda.synchronize()
    for q in parts:
        for p in parts:
            a, b = int(p.send_ptr[q.part]), int(p.send_ptr[q.part + 1])
            c, d = int(q.recv_ptr[p.part]), int(q.recv_ptr[p.part + 1])
            if b > a:
                q.recv_buf[c:d].copy_(p.send_buf[a:b])
    torch.cuda.synchronize()
    for q in parts:
        q.phase(unpack, q.recv_buf)


def run_parts_local(parts, n_steps: int):
    """Advance all parts of one partitioned state held on this device by n_steps
    (the exchange is a device copy between the parts' buffers; dt is the minimum
    of the parts' dt, taken through the host)."""
    import torch
    for _ in range(int(n_steps)):
        _exchange_local(parts, PART_PACK_W, PART_UNPACK_W)
        for p in parts:
            p.phase(PART_STAGE1)
        dt = min(p.get_dt() for p in parts)
        for p in parts:
            p.set_dt(dt)
            p.phase(PART_UPDATE1)
        if parts[0].two_stage:
            _exchange_local(parts, PART_PACK_WS, PART_UNPACK_WS)
            for p in parts:
                p.phase(PART_STAGE2)
    torch.cuda.synchronize()
    for p in parts:
        p.status()


def run_part_distributed(part: Part, n_steps: int, group=None):
    """Advance this rank's part by n_steps with torch.distributed: ghost states
    through point-to-point send/recv with every peer that shares vertices with
    this part, dt through an in-place all-reduce (min) on the device.  Every
    rank of the group runs this with its own part of the same partition."""
    import torch
    import torch.distributed as dist

    def exchange(pack, unpack):
        part.phase(pack, part.send_buf)
        torch.cuda.current_stream().wait_stream(part.mesh.stream)
        ops = []
        for q in range(part.n_parts):
            if q == part.part:
                continue
            a, b = int(part.send_ptr[q]), int(part.send_ptr[q + 1])
            c, d = int(part.recv_ptr[q]), int(part.recv_ptr[q + 1])
            if b > a:
                ops.append(dist.P2POp(dist.isend, part.send_buf[a:b], q, group))
            if d > c:
                ops.append(dist.P2POp(dist.irecv, part.recv_buf[c:d], q, group))
        if ops:
            for w in dist.batch_isend_irecv(ops):
                w.wait()
        part.mesh.stream.wait_stream(torch.cuda.current_stream())
        part.phase(unpack, part.recv_buf)

    dt = part.dt_tensor()
    for _ in range(int(n_steps)):
        exchange(PART_PACK_W, PART_UNPACK_W)
        part.phase(PART_STAGE1)
        torch.cuda.current_stream().wait_stream(part.mesh.stream)
        dist.all_reduce(dt, op=dist.ReduceOp.MIN, group=group)
        part.mesh.stream.wait_stream(torch.cuda.current_stream())
        part.phase(PART_UPDATE1)
        if part.two_stage:
            exchange(PART_PACK_WS, PART_UNPACK_WS)
            part.phase(PART_STAGE2)
    torch.cuda.synchronize()
