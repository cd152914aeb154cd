"""ctypes binding of libcutcell.so (include/cutcell.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Importing works without a GPU; creating a model needs the built
library and a CUDA device, and fails loudly otherwise (there is no CPU path).
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcutcell.so")

CC_OK, CC_EINVAL, CC_ECUDA, CC_EGEOM, CC_ENUMERIC, CC_ENOMEM, CC_ESTATE, CC_ETIMEOUT = range(8)
CC_FP64, CC_FP32 = 0, 1
CC_RHOP, CC_PP, CC_MX, CC_MY, CC_MZ, CC_UB = range(6)
STATUS = {0: "CC_OK", 1: "CC_EINVAL", 2: "CC_ECUDA", 3: "CC_EGEOM", 4: "CC_ENUMERIC", 5: "CC_ENOMEM",
          6: "CC_ESTATE", 7: "CC_ETIMEOUT"}
HOST_GZ = 2

# every entry point of include/cutcell.h
EXPORTS = ("cc_create", "cc_destroy", "cc_last_error", "cc_set_terrain", "cc_build_geometry",
           "cc_get_geometry", "cc_get_stencils", "cc_get_groups", "cc_init_state", "cc_upload_state",
           "cc_download_state", "cc_step", "cc_diagnostics", "cc_synchronize", "cc_last_launch_count",
           "cc_profile_enable", "cc_profile_read", "cc_profile_reset", "cc_create_refined",
           "cc_refine_mass", "cc_domain_count", "cc_create_refined_blocks", "cc_domain_block", "cc_autotune", "cc_get_schedule", "cc_set_schedule",
           "cc_get_warp_roles", "cc_set_warp_roles",
           "cc_graphs_enable", "cc_inject_wait_timeout", "cc_upload_state_async", "cc_download_state_async",
           "cc_save", "cc_load",
           "cc_set_terrain_analytic", "cc_get_terrain", "cc_download_derived", "cc_error_norms", "cc_cbcm_cubes",
           "cc_mass_sum_noalloc", "cc_noalloc_last_error", "cc_upload_state_f32", "cc_download_state_f32",
           "cc_upload_state_f32_async", "cc_download_state_f32_async", "cc_fma_peak",
           "cc_state_elems", "cc_upload_all_async", "cc_upload_all_f32_async")
CC_NOALLOC_MAX_PARTS = 1024
CC_HILL_BELL, CC_HILL_ELLIPSOID, CC_HILL_COSINE = range(3)
HILL_KINDS = {"bell": CC_HILL_BELL, "ellipsoid": CC_HILL_ELLIPSOID, "hemisphere": CC_HILL_ELLIPSOID,
              "cosine": CC_HILL_COSINE}
# derived output fields: corner velocity components, cell theta'
CC_U, CC_V, CC_W, CC_THETA_P = range(4)
CC_K_FULL, CC_K_GROUPS, CC_K_DIAGNOSE, CC_K_REFINE = range(4)
KERNEL_NAMES = {CC_K_FULL: "k_full", CC_K_GROUPS: "k_groups", CC_K_DIAGNOSE: "k_diag", CC_K_REFINE: "refinement"}


class CCConfig(ct.Structure):
    _fields_ = [("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int),
                ("dx", ct.c_double), ("dy", ct.c_double), ("dz", ct.c_double),
                ("dt", ct.c_double),
                ("U", ct.c_double), ("N", ct.c_double), ("theta0", ct.c_double),
                ("p_surf", ct.c_double), ("p0", ct.c_double), ("g", ct.c_double),
                ("R", ct.c_double), ("cp", ct.c_double),
                ("ra_nu", ct.c_double), ("c4", ct.c_double), ("sponge_frac", ct.c_double),
                ("tau_max", ct.c_double), ("bc_slip", ct.c_int)]


class CCBox(ct.Structure):
    _fields_ = [("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int), ("ox", ct.c_int), ("oy", ct.c_int)]


class CCDiag(ct.Structure):
    _fields_ = [("mass", ct.c_double), ("mass_comp", ct.c_double), ("max_u", ct.c_double),
                ("max_w", ct.c_double), ("nonfinite", ct.c_longlong), ("steps", ct.c_longlong),
                ("heat", ct.c_double), ("heat_comp", ct.c_double)]


class CCCube(ct.Structure):
    _fields_ = [("level", ct.c_int), ("ci", ct.c_int), ("cj", ct.c_int), ("ck", ct.c_int)]


class CutcellError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load libcutcell.so; raise if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ct.CDLL(path)
    vp, i, d = ct.c_void_p, ct.c_int, ct.c_double
    L.cc_create.argtypes = [ct.POINTER(CCConfig), i, i, vp, ct.POINTER(vp)]
    L.cc_destroy.argtypes = [vp]
    L.cc_last_error.restype = ct.c_char_p
    L.cc_last_error.argtypes = [vp]
    L.cc_set_terrain.argtypes = [vp, i, vp]
    L.cc_set_terrain_analytic.argtypes = [vp, i, i, vp]
    L.cc_get_terrain.argtypes = [vp, i, vp]
    L.cc_download_derived.argtypes = [vp, i, i, i, vp]
    L.cc_error_norms.argtypes = [vp, i, vp, i, i, d, vp]
    L.cc_cbcm_cubes.argtypes = [i, i, i, i, d, i, vp, vp, i, ct.POINTER(i)]
    L.cc_build_geometry.argtypes = [vp]
    L.cc_get_geometry.argtypes = [vp, i] + [vp] * 7
    L.cc_get_stencils.argtypes = [vp, i] + [vp] * 8
    L.cc_get_groups.argtypes = [vp, i, ct.POINTER(i), ct.POINTER(i), vp, vp, vp]
    L.cc_init_state.argtypes = [vp]
    L.cc_upload_state.argtypes = [vp, i, i, i, vp]
    L.cc_download_state.argtypes = [vp, i, i, i, vp]
    L.cc_upload_state_async.argtypes = [vp, i, i, i, vp]
    L.cc_download_state_async.argtypes = [vp, i, i, i, vp]
    for fn in ("cc_upload_state_f32", "cc_download_state_f32", "cc_upload_state_f32_async",
               "cc_download_state_f32_async"):
        getattr(L, fn).argtypes = [vp, i, i, i, vp]
    L.cc_state_elems.argtypes = [vp, ct.POINTER(ct.c_longlong)]
    L.cc_upload_all_async.argtypes = [vp, vp]
    L.cc_upload_all_f32_async.argtypes = [vp, vp]
    L.cc_step.argtypes = [vp, i]
    L.cc_diagnostics.argtypes = [vp, i, ct.POINTER(CCDiag)]
    L.cc_synchronize.argtypes = [vp]
    L.cc_last_launch_count.restype = ct.c_longlong
    L.cc_last_launch_count.argtypes = [vp]
    L.cc_profile_enable.argtypes = [vp, i]
    L.cc_profile_read.argtypes = [vp, i, ct.POINTER(d), ct.POINTER(ct.c_longlong)]
    L.cc_profile_reset.argtypes = [vp]
    L.cc_create_refined.argtypes = [ct.POINTER(CCConfig), i, ct.POINTER(CCBox), i, vp, ct.POINTER(vp)]
    L.cc_create_refined_blocks.argtypes = [ct.POINTER(CCConfig), i, ct.POINTER(CCBox), i, ct.POINTER(i), i,
                                           ct.POINTER(i), i, vp, ct.POINTER(vp)]
    L.cc_domain_block.argtypes = [vp, i, ct.POINTER(i), ct.POINTER(i), ct.POINTER(i)]
    L.cc_refine_mass.argtypes = [vp, i, ct.POINTER(d)]
    L.cc_domain_count.restype = i
    L.cc_domain_count.argtypes = [vp]
    L.cc_autotune.argtypes = [vp, i]
    L.cc_graphs_enable.argtypes = [vp, i]
    L.cc_inject_wait_timeout.argtypes = [vp, i]
    L.cc_save.argtypes = [vp, ct.c_char_p]
    L.cc_load.argtypes = [vp, ct.c_char_p]
    L.cc_get_schedule.argtypes = [vp, i, ct.POINTER(i), ct.POINTER(i)]
    L.cc_set_schedule.argtypes = [vp, i, i, i]
    L.cc_get_warp_roles.argtypes = [vp, i, ct.POINTER(i)]
    L.cc_set_warp_roles.argtypes = [vp, i, i]
    L.cc_mass_sum_noalloc.argtypes = [vp, i, vp, ct.c_longlong, i, vp, vp]
    L.cc_noalloc_last_error.restype = ct.c_char_p
    L.cc_fma_peak.argtypes = [i, i, vp, ct.POINTER(ct.c_double)]
    L.cc_noalloc_last_error.argtypes = []
    _lib = L
    return L


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ct.c_void_p)


def config_from(cfg) -> CCConfig:
    c = CCConfig()
    for name, _ in CCConfig._fields_:
        setattr(c, name, getattr(cfg, name))
    return c


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return None


def mass_sum_noalloc(rho_ptr: int, precision: int, volume_ptr: int, n: int, nparts: int, out_ptr: int,
                     stream=None) -> int:
    """cc_mass_sum_noalloc on caller-owned device buffers (raw pointers).

    For callers that cannot allocate device memory: the library allocates
    nothing for this call.  Returns the status; raises on errors."""
    L = load()
    if stream is None:
        stream = _current_stream()
    st = L.cc_mass_sum_noalloc(ct.c_void_p(rho_ptr), precision, ct.c_void_p(volume_ptr), int(n), int(nparts),
                               ct.c_void_p(out_ptr), stream)
    if st != CC_OK:
        raise CutcellError(st, L.cc_noalloc_last_error().decode())
    return st


def fma_peak(precision: int, iters: int = 1 << 16, stream=None) -> float:
    """cc_fma_peak: the measured fused multiply-add rate of the current GPU
    in flop/s (2 per fused multiply-add)."""
    L = load()
    if stream is None:
        stream = _current_stream()
    out = ct.c_double(0.0)
    st = L.cc_fma_peak(int(precision), int(iters), stream, ct.byref(out))
    if st != CC_OK:
        raise CutcellError(st, "cc_fma_peak failed")
    return out.value


class Model:
    """Ensemble of periodic domains advanced on the GPU through the C ABI."""

    def __init__(self, cfgs, precision: int = CC_FP64, stream=None):
        self.L = load()
        if not isinstance(cfgs, (list, tuple)):
            cfgs = [cfgs]
        self.cfgs = list(cfgs)
        arr = (CCConfig * len(cfgs))(*[config_from(c) for c in cfgs])
        self._arr = arr
        if stream is None:
            stream = _current_stream()
        self.stream = stream
        h = ct.c_void_p()
        st = self.L.cc_create(arr, len(cfgs), precision, stream, ct.byref(h))
        if st != CC_OK:
            raise CutcellError(st, self.L.cc_last_error(None).decode())
        self.h = h
        self.precision = precision

    def _check(self, st):
        if st != CC_OK:
            raise CutcellError(st, self.L.cc_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.L.cc_destroy(self.h)
            self.h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- set-up
    def set_terrain(self, d: int, h: np.ndarray):
        h = np.ascontiguousarray(h, dtype=np.float64)
        c = self.cfgs[d]
        assert h.shape == (c.ny, c.nx)
        self._check(self.L.cc_set_terrain(self.h, d, _p(h)))

    def set_terrain_analytic(self, d: int, kind, h0: float, a: float, xc: float | None = None,
                             yc: float | None = None):
        """Hill evaluated on the GPU at the corners of domain d (centred on the
        domain by default); kind is CC_HILL_* or a name of HILL_KINDS."""
        c = self.cfgs[d]
        k = HILL_KINDS[kind] if isinstance(kind, str) else int(kind)
        xc = 0.5 * c.nx * c.dx if xc is None else xc
        yc = 0.5 * c.ny * c.dy if yc is None else yc
        prm = np.array([h0, a, xc, yc], np.float64)
        self._check(self.L.cc_set_terrain_analytic(self.h, d, k, _p(prm)))

    def terrain(self, d: int = 0) -> np.ndarray:
        c = self.cfgs[d]
        out = np.zeros((c.ny, c.nx))
        self._check(self.L.cc_get_terrain(self.h, d, _p(out)))
        return out

    def build_geometry(self):
        self._check(self.L.cc_build_geometry(self.h))

    def geometry(self, d: int = 0) -> dict:
        c = self.cfgs[d]
        cs = (c.nz, c.ny, c.nx)
        out = dict(vf=np.zeros(cs), ax=np.zeros(cs), ay=np.zeros(cs), az=np.zeros((c.nz + 1, c.ny, c.nx)),
                   cls=np.zeros(cs, np.int8), root=np.zeros(cs, np.int32),
                   vcls=np.zeros((c.nz + 1 + 2 * HOST_GZ, c.ny, c.nx), np.int8))
        self._check(self.L.cc_get_geometry(self.h, d, *[_p(out[k]) for k in
                                                         ("vf", "ax", "ay", "az", "cls", "root", "vcls")]))
        return out

    def stencils(self, d: int = 0) -> dict:
        c = self.cfgs[d]
        q = (c.ny, c.nx)
        ps = (c.nz + 1 + 2 * HOST_GZ, c.ny, c.nx)
        out = dict(bK=np.zeros(q, np.int32), bI=np.zeros(q, np.int32), bJ=np.zeros(q, np.int32),
                   ba=np.zeros(q), bb=np.zeros(q), bn=np.zeros(q + (3,)), mK=np.zeros(ps, np.int32),
                   mg=np.zeros(ps))
        self._check(self.L.cc_get_stencils(self.h, d, *[_p(out[k]) for k in
                                                         ("bK", "bI", "bJ", "ba", "bb", "bn", "mK", "mg")]))
        return out

    def groups(self, d: int = 0):
        ng, nm = ct.c_int(), ct.c_int()
        self._check(self.L.cc_get_groups(self.h, d, ct.byref(ng), ct.byref(nm), None, None, None))
        host = np.zeros(ng.value, np.int32)
        start = np.zeros(ng.value + 1, np.int32)
        mem = np.zeros(nm.value, np.int32)
        self._check(self.L.cc_get_groups(self.h, d, ct.byref(ng), ct.byref(nm), _p(host), _p(start), _p(mem)))
        return host, start, mem

    # ---------------------------------------------------------------- state
    def init_state(self):
        self._check(self.L.cc_init_state(self.h))

    def _shape(self, d, field):
        c = self.cfgs[d]
        if field in (CC_RHOP, CC_PP):
            return (c.nz, c.ny, c.nx)
        if field == CC_UB:
            return (c.ny, c.nx, 3)
        return (c.nz + 1 + 2 * HOST_GZ, c.ny, c.nx)

    def download(self, d: int, field: int, level: int = 1, out: np.ndarray | None = None,
                 dtype=np.float64) -> np.ndarray:
        """One field in the host layout, as FP64 or (FP32 models) FP32."""
        shape = self._shape(d, field)
        if out is None:
            out = np.zeros(shape, dtype)
        assert out.shape == shape and out.dtype in (np.float64, np.float32) and out.flags.c_contiguous
        fn = self.L.cc_download_state_f32 if out.dtype == np.float32 else self.L.cc_download_state
        self._check(fn(self.h, d, field, level, _p(out)))
        return out

    def derived(self, d: int, which: int, level: int = 1) -> np.ndarray:
        """Corner velocity component (CC_U, CC_V, CC_W; corners K = 0 .. nz)
        or the cell potential-temperature perturbation (CC_THETA_P)."""
        c = self.cfgs[d]
        shape = (c.nz, c.ny, c.nx) if which == CC_THETA_P else (c.nz + 1, c.ny, c.nx)
        out = np.zeros(shape)
        self._check(self.L.cc_download_derived(self.h, d, which, level, _p(out)))
        return out

    def download_ptr(self, d: int, field: int, level: int, ptr: int, wait: bool = True, f32: bool = False):
        if f32:
            fn = self.L.cc_download_state_f32 if wait else self.L.cc_download_state_f32_async
        else:
            fn = self.L.cc_download_state if wait else self.L.cc_download_state_async
        self._check(fn(self.h, d, field, level, ct.c_void_p(ptr)))

    def upload(self, d: int, field: int, level: int, a: np.ndarray):
        """One field from a host array; FP32 arrays go through the FP32 calls
        (FP32 models only), anything else as FP64."""
        if a.dtype != np.float32:
            a = np.ascontiguousarray(a, dtype=np.float64)
        a = np.ascontiguousarray(a)
        assert a.shape == self._shape(d, field)
        fn = self.L.cc_upload_state_f32 if a.dtype == np.float32 else self.L.cc_upload_state
        self._check(fn(self.h, d, field, level, _p(a)))

    def upload_ptr(self, d: int, field: int, level: int, ptr: int, wait: bool = True, f32: bool = False):
        if f32:
            fn = self.L.cc_upload_state_f32 if wait else self.L.cc_upload_state_f32_async
        else:
            fn = self.L.cc_upload_state if wait else self.L.cc_upload_state_async
        self._check(fn(self.h, d, field, level, ct.c_void_p(ptr)))

    def state_elems(self) -> int:
        """Elements of the whole two-time-level state in one host buffer
        (cc_state_elems: every domain, fields rho', p', rho u, rho v, rho w,
        levels 0 then 1, host layouts back to back)."""
        n = ct.c_longlong(0)
        self._check(self.L.cc_state_elems(self.h, ct.byref(n)))
        return int(n.value)

    def upload_all_ptr(self, ptr: int, f32: bool = False):
        """cc_upload_all_async / cc_upload_all_f32_async: the whole state from
        the host buffer at ptr, queued on the model's stream (the buffer stays
        valid until synchronize)."""
        fn = self.L.cc_upload_all_f32_async if f32 else self.L.cc_upload_all_async
        self._check(fn(self.h, ct.c_void_p(ptr)))

    def step(self, n: int = 1):
        self._check(self.L.cc_step(self.h, int(n)))

    def synchronize(self):
        self._check(self.L.cc_synchronize(self.h))

    def diagnostics(self, d: int = 0, check: bool = True) -> dict:
        g = CCDiag()
        st = self.L.cc_diagnostics(self.h, d, ct.byref(g))
        if check:
            self._check(st)
        return dict(mass=g.mass, mass_comp=g.mass_comp, max_u=g.max_u, max_w=g.max_w,
                    nonfinite=g.nonfinite, steps=g.steps, heat=g.heat, heat_comp=g.heat_comp, status=st)

    @property
    def last_launch_count(self) -> int:
        return int(self.L.cc_last_launch_count(self.h))

    def profile(self, on: bool = True):
        self._check(self.L.cc_profile_enable(self.h, 1 if on else 0))

    def profile_reset(self):
        self._check(self.L.cc_profile_reset(self.h))

    def autotune(self, reps: int = 3) -> list:
        """Time every full-cell schedule on the current state and keep the
        fastest (per level of a refined model); returns the schedules."""
        self._check(self.L.cc_autotune(self.h, int(reps)))
        return [self.schedule(d) for d in range(len(self.cfgs))]

    def save(self, path: str):
        """Checkpoint the whole state to a file (cc_save)."""
        self._check(self.L.cc_save(self.h, os.fsencode(path)))

    def load(self, path: str):
        """Resume from a checkpoint written by a model of the same set-up."""
        self._check(self.L.cc_load(self.h, os.fsencode(path)))

    def graphs(self, on: bool = True):
        self._check(self.L.cc_graphs_enable(self.h, 1 if on else 0))

    def inject_wait_timeout(self, on: bool = True):
        """Make every bounded TMA wait of the refined-box stencil run out (the
        step watchdog's test)."""
        self._check(self.L.cc_inject_wait_timeout(self.h, 1 if on else 0))

    def schedule(self, d: int = 0) -> tuple:
        ty, items = ct.c_int(), ct.c_int()
        self._check(self.L.cc_get_schedule(self.h, d, ct.byref(ty), ct.byref(items)))
        return ty.value, items.value

    def set_schedule(self, d: int, tile_y: int, items_per_launch: int):
        self._check(self.L.cc_set_schedule(self.h, d, int(tile_y), int(items_per_launch)))

    def warp_roles(self, d: int = 0) -> int:
        nr = ct.c_int()
        self._check(self.L.cc_get_warp_roles(self.h, d, ct.byref(nr)))
        return nr.value

    def set_warp_roles(self, d: int, roles: int):
        self._check(self.L.cc_set_warp_roles(self.h, d, int(roles)))

    def profile_read(self, kernel: int):
        ms, n = ct.c_double(), ct.c_longlong()
        self._check(self.L.cc_profile_read(self.h, kernel, ct.byref(ms), ct.byref(n)))
        return ms.value, n.value


def error_norms(a: "Model", da: int, b: "Model", db: int, which: int, zmin: float = float("-inf")):
    """(L1, L2, N) of a corner velocity component of domain da of model a
    against the finer domain db of model b at the coincident corners above
    zmin (cc_error_norms)."""
    out = np.zeros(3)
    a._check(a.L.cc_error_norms(a.h, da, b.h, db, which, float(zmin), _p(out)))
    return out[0], out[1], int(out[2])


def cbcm_cubes(nx0: int, ny0: int, nz0: int, cube: int, H: float, nlev: int, h_finest: np.ndarray):
    """Block-structured cube layout (cc_cbcm_cubes): a list of (level, ci,
    cj, ck), sorted by (level, ck, cj, ci)."""
    L = load()
    h = np.ascontiguousarray(h_finest, dtype=np.float64)
    n = ct.c_int()
    st = L.cc_cbcm_cubes(nx0, ny0, nz0, cube, H, nlev, _p(h), None, 0, ct.byref(n))
    if st != CC_OK:
        raise CutcellError(st, "cube layout: invalid arguments")
    arr = (CCCube * max(1, n.value))()
    st = L.cc_cbcm_cubes(nx0, ny0, nz0, cube, H, nlev, _p(h), ct.cast(arr, ct.c_void_p), n.value, ct.byref(n))
    if st != CC_OK:
        raise CutcellError(st, "cube layout failed")
    return [(c.level, c.ci, c.cj, c.ck) for c in arr[:n.value]]


class _Level:
    """Sizes of one level of a refined model (what Model's accessors read)."""

    def __init__(self, base, l: int, box=None):
        f = 2.0 ** -l
        self.nx, self.ny, self.nz = (base.nx, base.ny, base.nz) if box is None else tuple(box[:3])
        self.dx, self.dy, self.dz, self.dt = base.dx * f, base.dy * f, base.dz * f, base.dt * f


class RefinedModel(Model):
    """Block-structured refinement advanced on the GPU through the C ABI:
    cc_create_refined_blocks (levels as domains 0 .. nlev-1; with cuts the
    finest level as sibling blocks, domains nlev-1 ..), cc_step (one cycle of
    level 0 per step), cc_refine_mass."""

    def __init__(self, base, boxes, precision: int = CC_FP64, stream=None, xcuts=(), ycuts=()):
        self.L = load()
        self.base = base
        self.boxes = [tuple(b) for b in boxes]
        self.cfgs = [_Level(base, 0)] + [_Level(base, l + 1, b) for l, b in enumerate(self.boxes)]
        cb = config_from(base)
        arr = (CCBox * max(1, len(self.boxes)))(*[CCBox(*b) for b in self.boxes])
        self._arr = (cb, arr)
        if stream is None:
            stream = _current_stream()
        self.stream = stream
        h = ct.c_void_p()
        xc = (ct.c_int * max(1, len(xcuts)))(*xcuts)
        yc = (ct.c_int * max(1, len(ycuts)))(*ycuts)
        st = self.L.cc_create_refined_blocks(ct.byref(cb), len(self.boxes) + 1, arr, len(xcuts), xc, len(ycuts), yc,
                                             precision, stream, ct.byref(h))
        if st != CC_OK:
            raise CutcellError(st, self.L.cc_last_error(None).decode())
        self.h = h
        self.precision = precision
        # per domain: (level, block origin x, y); the finest level's blocks
        # replace its single entry in cfgs
        self.blocks = []
        for d in range(self.L.cc_domain_count(self.h)):
            lv, ox, oy = ct.c_int(), ct.c_int(), ct.c_int()
            self._check(self.L.cc_domain_block(self.h, d, ct.byref(lv), ct.byref(ox), ct.byref(oy)))
            self.blocks.append((lv.value, ox.value, oy.value))
        self._nlev = len(self.boxes) + 1
        fine = self.boxes[-1]
        xs, ys = [0, *xcuts, fine[0]], [0, *ycuts, fine[1]]
        self.cfgs = self.cfgs[:-1] + [_Level(base, self._nlev - 1, (xs[a + 1] - xs[a], ys[b + 1] - ys[b], fine[2]))
                                      for b in range(len(ys) - 1) for a in range(len(xs) - 1)]

    @property
    def nlev(self) -> int:
        return self._nlev

    @property
    def ndom(self) -> int:
        return len(self.cfgs)

    def level_domains(self, lev: int) -> list:
        return [d for d, b in enumerate(self.blocks) if b[0] == lev]

    def set_level_terrain(self, lev: int, h: np.ndarray):
        """Corner heights of a whole level (its box's corners), cut into its blocks."""
        for d in self.level_domains(lev):
            _, ox, oy = self.blocks[d]
            c = self.cfgs[d]
            self.set_terrain(d, np.ascontiguousarray(h[oy:oy + c.ny, ox:ox + c.nx]))

    def download_level(self, lev: int, field: int, level: int = 1) -> np.ndarray:
        """One field of a whole level in the host layout of its box, stitched
        from its blocks."""
        ds = self.level_domains(lev)
        parts = [(self.blocks[d], self.download(d, field, level)) for d in ds]
        ny = max(b[2] + a.shape[-2 if field != CC_UB else 0] for b, a in parts)
        nx = max(b[1] + a.shape[-1 if field != CC_UB else 1] for b, a in parts)
        first = parts[0][1]
        if field == CC_UB:
            out = np.zeros((ny, nx, 3), first.dtype)
            for (_, ox, oy), a in parts:
                out[oy:oy + a.shape[0], ox:ox + a.shape[1]] = a
        else:
            out = np.zeros(first.shape[:-2] + (ny, nx), first.dtype)
            for (_, ox, oy), a in parts:
                out[..., oy:oy + a.shape[-2], ox:ox + a.shape[-1]] = a
        return out

    def mass(self, both: bool = True) -> float:
        out = ct.c_double()
        self._check(self.L.cc_refine_mass(self.h, 1 if both else 0, ct.byref(out)))
        return out.value
