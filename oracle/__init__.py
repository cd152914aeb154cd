"""ctypes wrapper of the plain FP64 CPU oracle (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The product path never does.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
SRC = os.path.join(HERE, "oracle.c")

OK, EINVAL, EGEOM = 0, 1, 3
F_RHOP, F_PP, F_MX, F_MY, F_MZ, F_UB = range(6)
# derived output fields: corner velocity components, cell theta'
D_U, D_V, D_W, D_THETA = range(4)
# cell classes and corner classes
C_UG, C_FULL, C_CUT, C_ABS = 0, 1, 2, 3
V_UG, V_PRED, V_MF, V_LID = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None


class Params(ct.Structure):
    _fields_ = [("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int),
                ("dx", ct.c_double), ("dy", ct.c_double), ("dz", ct.c_double),
                ("dt", ct.c_double),
                ("U", ct.c_double), ("N", ct.c_double), ("theta0", ct.c_double),
                ("p_surf", ct.c_double), ("p0", ct.c_double), ("g", ct.c_double),
                ("R", ct.c_double), ("cp", ct.c_double),
                ("ra_nu", ct.c_double), ("c4", ct.c_double), ("sponge_frac", ct.c_double),
                ("tau_max", ct.c_double), ("bc_slip", ct.c_int), ("ztop", ct.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, FP64, no contraction, OpenMP)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True, cwd=HERE)
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ct.CDLL(LIB)
            L.oc_create.restype = ct.c_void_p
            L.oc_create.argtypes = [ct.POINTER(Params), ct.c_void_p, ct.POINTER(ct.c_int)]
            L.oc_destroy.argtypes = [ct.c_void_p]
            L.oc_init_state.argtypes = [ct.c_void_p]
            L.oc_step.argtypes = [ct.c_void_p, ct.c_int]
            L.oc_dims.argtypes = [ct.c_void_p] + [ct.POINTER(ct.c_long)] * 3 + [ct.POINTER(ct.c_int)]
            L.oc_get_state.argtypes = [ct.c_void_p, ct.c_int, ct.c_int, ct.c_void_p]
            L.oc_set_state.argtypes = [ct.c_void_p, ct.c_int, ct.c_int, ct.c_void_p]
            L.oc_get_state_padded.argtypes = [ct.c_void_p, ct.c_int, ct.c_int, ct.c_void_p]
            L.oc_padding.argtypes = [ct.c_void_p] + [ct.POINTER(ct.c_int)] * 4
            L.oc_padding.restype = None
            L.oc_get_geometry.argtypes = [ct.c_void_p] + [ct.c_void_p] * 10
            L.oc_get_points.argtypes = [ct.c_void_p] + [ct.c_void_p] * 9
            L.oc_get_base.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                      ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]
            L.oc_base_len.argtypes = [ct.c_void_p]
            L.oc_mass.restype = ct.c_double
            L.oc_mass.argtypes = [ct.c_void_p, ct.c_int]
            L.oc_nsteps.argtypes = [ct.c_void_p]
            L.oc_heat.restype = ct.c_double
            L.oc_heat.argtypes = [ct.c_void_p, ct.c_int]
            L.oc_get_derived.argtypes = [ct.c_void_p, ct.c_int, ct.c_int, ct.c_void_p]
            L.oc_error_norms.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_double, ct.c_void_p]
            L.oc_line_int.restype = ct.c_double
            L.oc_line_int.argtypes = [ct.c_double] * 4
            L.oc_line_frac.restype = ct.c_double
            L.oc_line_frac.argtypes = [ct.c_double] * 3
            L.oc_col_int.restype = ct.c_double
            L.oc_col_int.argtypes = [ct.c_double] * 7 + [ct.c_int]
            L.oc_refine_create.restype = ct.c_void_p
            L.oc_refine_create.argtypes = [ct.POINTER(Params), ct.c_int, ct.c_void_p, ct.c_void_p,
                                           ct.POINTER(ct.c_int)]
            L.oc_refine_destroy.argtypes = [ct.c_void_p]
            L.oc_refine_init.argtypes = [ct.c_void_p]
            L.oc_refine_step.argtypes = [ct.c_void_p, ct.c_int]
            L.oc_refine_level.restype = ct.c_void_p
            L.oc_refine_level.argtypes = [ct.c_void_p, ct.c_int]
            L.oc_refine_mass.restype = ct.c_double
            L.oc_refine_mass.argtypes = [ct.c_void_p, ct.c_int]
            FN = ct.CFUNCTYPE(ct.c_double, ct.c_double, ct.c_void_p)
            L.oc_gauss_legendre8.restype = ct.c_double
            L.oc_gauss_legendre8.argtypes = [FN, ct.c_void_p, ct.c_double, ct.c_double]
            L._FN = FN
            _lib = L
        return _lib


def params_from(cfg) -> Params:
    p = Params()
    for name, _ in Params._fields_:
        setattr(p, name, getattr(cfg, name, 0.0 if name == "ztop" else None))
    return p


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ct.c_void_p)


class OracleError(RuntimeError):
    pass


class Model:
    """One periodic single-level domain advanced by the oracle."""

    def __init__(self, cfg, h: np.ndarray | None = None):
        self.cfg = cfg
        L = lib()
        if h is None:
            h = cfg.heights()
        h = np.ascontiguousarray(h, dtype=np.float64)
        assert h.shape == (cfg.ny, cfg.nx)
        self.h = h
        self._p = params_from(cfg)
        st = ct.c_int(0)
        self._m = L.oc_create(ct.byref(self._p), _ptr(h), ct.byref(st))
        if not self._m:
            raise OracleError(f"oracle create failed with status {st.value}")
        nc, np_, nq, gz = ct.c_long(), ct.c_long(), ct.c_long(), ct.c_int()
        L.oc_dims(self._m, ct.byref(nc), ct.byref(np_), ct.byref(nq), ct.byref(gz))
        self.ncell, self.ncorner, self.ncol, self.gz = nc.value, np_.value, nq.value, gz.value

    def __del__(self):
        m = getattr(self, "_m", None)
        if m:
            lib().oc_destroy(m)
            self._m = None

    # shapes
    @property
    def cell_shape(self):
        return (self.cfg.nz, self.cfg.ny, self.cfg.nx)

    @property
    def corner_shape(self):
        return (self.cfg.nz + 1 + 2 * self.gz, self.cfg.ny, self.cfg.nx)

    def geometry(self) -> dict:
        c = self.cfg
        out = dict(vf=np.zeros(self.ncell), ax=np.zeros(self.ncell), ay=np.zeros(self.ncell),
                   az=np.zeros(self.ncol * (c.nz + 1)), cls=np.zeros(self.ncell, np.int8),
                   root=np.zeros(self.ncell, np.int32), vg=np.zeros(self.ncell),
                   hc=np.zeros(self.ncol), gx=np.zeros(self.ncol), gy=np.zeros(self.ncol))
        lib().oc_get_geometry(self._m, *[_ptr(out[k]) for k in
                                         ("vf", "ax", "ay", "az", "cls", "root", "vg", "hc", "gx", "gy")])
        for k in ("vf", "ax", "ay", "cls", "root", "vg"):
            out[k] = out[k].reshape(self.cell_shape)
        out["az"] = out["az"].reshape((c.nz + 1, c.ny, c.nx))
        for k in ("hc", "gx", "gy"):
            out[k] = out[k].reshape((c.ny, c.nx))
        return out

    def points(self) -> dict:
        c = self.cfg
        out = dict(vcls=np.zeros(self.ncorner, np.int8), bK=np.zeros(self.ncol, np.int32),
                   bI=np.zeros(self.ncol, np.int32), bJ=np.zeros(self.ncol, np.int32),
                   ba=np.zeros(self.ncol), bb=np.zeros(self.ncol), bn=np.zeros(3 * self.ncol),
                   mK=np.zeros(self.ncorner, np.int32), mg=np.zeros(self.ncorner))
        lib().oc_get_points(self._m, *[_ptr(out[k]) for k in
                                       ("vcls", "bK", "bI", "bJ", "ba", "bb", "bn", "mK", "mg")])
        out["vcls"] = out["vcls"].reshape(self.corner_shape)
        out["mK"] = out["mK"].reshape(self.corner_shape)
        out["mg"] = out["mg"].reshape(self.corner_shape)
        for k in ("bK", "bI", "bJ", "ba", "bb"):
            out[k] = out[k].reshape((c.ny, c.nx))
        out["bn"] = out["bn"].reshape((c.ny, c.nx, 3))
        return out

    def base(self):
        nb = lib().oc_base_len(self._m)
        rhob, pb = np.zeros(nb), np.zeros(nb)
        koff, n = ct.c_int(), ct.c_int()
        lib().oc_get_base(self._m, _ptr(rhob), _ptr(pb), ct.byref(koff), ct.byref(n))
        return rhob, pb, koff.value

    def init_state(self):
        lib().oc_init_state(self._m)

    def step(self, n: int = 1):
        lib().oc_step(self._m, int(n))

    @property
    def nsteps(self) -> int:
        return lib().oc_nsteps(self._m)

    def field(self, f: int, level: int = 1) -> np.ndarray:
        if f in (F_RHOP, F_PP):
            a = np.zeros(self.ncell)
            shape = self.cell_shape
        elif f == F_UB:
            a = np.zeros(3 * self.ncol)
            shape = (self.cfg.ny, self.cfg.nx, 3)
        else:
            a = np.zeros(self.ncorner)
            shape = self.corner_shape
        st = lib().oc_get_state(self._m, f, level, _ptr(a))
        if st != OK:
            raise OracleError(f"get_state {f} {level} -> {st}")
        return a.reshape(shape)

    def set_field(self, f: int, level: int, a: np.ndarray):
        a = np.ascontiguousarray(a, dtype=np.float64).ravel()
        st = lib().oc_set_state(self._m, f, level, _ptr(a))
        if st != OK:
            raise OracleError(f"set_state {f} {level} -> {st}")

    def padded(self, f: int, level: int = 1):
        """The whole padded array of prognostic field f at time level `level`
        ((nz + 2G, ny + 2G, nx + 2G); cell or corner (i, j, k) at
        [k + G, j + G, i + G]) and the padding G."""
        g, nx, ny, nz = (ct.c_int() for _ in range(4))
        lib().oc_padding(self._m, ct.byref(g), ct.byref(nx), ct.byref(ny), ct.byref(nz))
        a = np.zeros(nz.value * ny.value * nx.value)
        st = lib().oc_get_state_padded(self._m, f, level, _ptr(a))
        if st != OK:
            raise OracleError(f"get_state_padded {f} {level} -> {st}")
        return a.reshape((nz.value, ny.value, nx.value)), g.value

    def mass(self, level: int = 1) -> float:
        return lib().oc_mass(self._m, level)

    def heat(self, level: int = 1) -> float:
        return lib().oc_heat(self._m, level)

    def derived(self, which: int, level: int = 1) -> np.ndarray:
        c = self.cfg
        shape = self.cell_shape if which == D_THETA else (c.nz + 1, c.ny, c.nx)
        a = np.zeros(int(np.prod(shape)))
        st = lib().oc_get_derived(self._m, which, level, _ptr(a))
        if st != OK:
            raise OracleError(f"get_derived {which} {level} -> {st}")
        return a.reshape(shape)


def error_norms(a: Model, b: Model, which: int, zmin: float):
    """(L1, L2, N) of a corner velocity component of model a against the
    finer model b at the coincident corners above zmin."""
    out = np.zeros(3)
    st = lib().oc_error_norms(a._m, b._m, which, float(zmin), _ptr(out))
    if st != OK:
        raise OracleError(f"error_norms -> {st}")
    return out[0], out[1], int(out[2])


def line_int(z, ha, hb, length):
    return lib().oc_line_int(z, ha, hb, length)


def line_frac(z, ha, hb):
    return lib().oc_line_frac(z, ha, hb)


def col_int(z, h00, h10, h01, h11, dx, dy, kind):
    return lib().oc_col_int(z, h00, h10, h01, h11, dx, dy, kind)


def gauss_legendre8(f, a, b):
    L = lib()
    cb = L._FN(lambda s, _ctx: f(s))
    return L.oc_gauss_legendre8(cb, None, a, b)


class Box(ct.Structure):
    _fields_ = [("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int), ("ox", ct.c_int), ("oy", ct.c_int)]


class _LevelView(Model):
    """A level owned by a Refine driver (not destroyed by itself)."""

    def __init__(self, owner, ptr, cfg):
        self._owner = owner
        self.cfg = cfg
        self._m = ptr
        nc, np_, nq, gz = ct.c_long(), ct.c_long(), ct.c_long(), ct.c_int()
        lib().oc_dims(self._m, ct.byref(nc), ct.byref(np_), ct.byref(nq), ct.byref(gz))
        self.ncell, self.ncorner, self.ncol, self.gz = nc.value, np_.value, nq.value, gz.value

    def __del__(self):
        pass


class Refine:
    """Block-structured refinement: level 0 = cfg (periodic, lid), levels
    1.. = boxes (nx, ny, nz, ox, oy) in cells of that level; h_finest = corner
    heights of the finest level over I, J = -4 .. n+4 ((ny+9) x (nx+9))."""

    def __init__(self, cfg, boxes, h_finest=None):
        L = lib()
        self.cfg = cfg
        self.boxes = [tuple(b) for b in boxes]
        self._p = params_from(cfg)
        nlev = 1 + len(boxes)
        arr = (Box * max(1, len(boxes)))(*[Box(*b) for b in boxes])
        self._arr = arr
        hp = None
        if h_finest is not None:
            h_finest = np.ascontiguousarray(h_finest, dtype=np.float64)
            hp = _ptr(h_finest)
        st = ct.c_int(0)
        self._r = L.oc_refine_create(ct.byref(self._p), nlev, ct.cast(arr, ct.c_void_p), hp, ct.byref(st))
        if not self._r:
            raise OracleError(f"refine create failed with status {st.value}")
        self.nlev = nlev
        self.levels = []
        for l in range(nlev):
            import dataclasses
            f = 2.0 ** -l
            if l == 0:
                c = cfg
            else:
                nx, ny, nz, ox, oy = self.boxes[l - 1]
                c = dataclasses.replace(cfg, nx=nx, ny=ny, nz=nz, dx=cfg.dx * f, dy=cfg.dy * f, dz=cfg.dz * f,
                                        dt=cfg.dt * f)
            self.levels.append(_LevelView(self, L.oc_refine_level(self._r, l), c))

    def __del__(self):
        r = getattr(self, "_r", None)
        if r:
            lib().oc_refine_destroy(r)
            self._r = None

    def init_state(self):
        lib().oc_refine_init(self._r)

    def step(self, n: int = 1):
        lib().oc_refine_step(self._r, int(n))

    def mass(self, both: bool = True) -> float:
        return lib().oc_refine_mass(self._r, 1 if both else 0)
