"""B300 nodal DG acoustic solver with Pade HABC and edge/corner compatibility.

Thin ctypes binding of the C ABI declared in ``include/dgh.h`` (libdgh.so,
built in-tree for sm_103a).  Every step of the time integration runs in the
library's CUDA kernels; this module only marshals arguments.  There is no
CPU fallback: constructing a solver without the built library or without a
CUDA device raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdgh.so")
CHECKED_LIB_PATH = os.path.join(_HERE, "libdgh_checked.so")   # index-checked build (tests)

DGH_OK = 0
BC_HABC = 0
BC_DIRICHLET = 1
PREC_FP32 = 0
PREC_BF16_TC = 1
PREC_FP16_TC = 2
PREC_SPLIT_BF16 = 3
PREC_FP32_CUDA = 4     # FP32 CUDA-core contractions at every order
PREC_SPLIT_TF32 = 5    # split-TF32 tensor-core contractions (N <= 4; PREC_FP32's kernel at N = 4 on large meshes)

_ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "EUNSTABLE", -5: "ETIMEOUT", -6: "ESTATE",
           -7: "EUNSUPPORTED", -8: "EBOUNDS"}
DGH_EINVAL = -1
DGH_ENOMEM = -2
DGH_ECUDA = -3
DGH_EUNSTABLE = -4
DGH_ETIMEOUT = -5
DGH_ESTATE = -6
DGH_EUNSUPPORTED = -7
DGH_EBOUNDS = -8


class DghError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("dgh error %d (%s): %s" % (code, _ERRORS.get(code, "?"), msg))
        self.code = code


class _Desc(ctypes.Structure):
    _fields_ = [
        ("order", ctypes.c_int32), ("habc_order", ctypes.c_int32), ("bc", ctypes.c_int32 * 6),
        ("precision", ctypes.c_int32), ("reserved0", ctypes.c_int32),
        ("n_vertices", ctypes.c_int64), ("n_cells", ctypes.c_int64),
        ("vertices", ctypes.POINTER(ctypes.c_double)), ("cells", ctypes.POINTER(ctypes.c_int32)),
        ("c", ctypes.POINTER(ctypes.c_double)), ("rho", ctypes.POINTER(ctypes.c_double)),
        ("dt", ctypes.c_double), ("cfl", ctypes.c_double),
    ]


class _Info(ctypes.Structure):
    _fields_ = [
        ("order", ctypes.c_int32), ("habc_order", ctypes.c_int32), ("Np", ctypes.c_int32),
        ("Np2", ctypes.c_int32), ("Np1", ctypes.c_int32), ("n_corners", ctypes.c_int32),
        ("n_cells", ctypes.c_int64), ("n_tris", ctypes.c_int64), ("n_lines", ctypes.c_int64),
        ("n_bfaces", ctypes.c_int64), ("ndof", ctypes.c_int64), ("step_count", ctypes.c_int64),
        ("dt", ctypes.c_double), ("time", ctypes.c_double), ("device_bytes", ctypes.c_int64),
    ]


MLP_NPARAM = 4673
MLP_IN = 6


class _TrainCfg(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("batch", ctypes.c_int64), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("seed", ctypes.c_uint64)]


class _Launch(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int32) for f in
                ("tile2", "tile1", "cta3_per_sm", "grid3", "grid2", "grid1", "occ3", "sms", "thr2", "thr1",
                 "sm3_div", "split3", "kern3")]


_lib = None


def load_library(path=LIB_PATH):
    """Load libdgh.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libdgh.so not built: run paper_1610_05023_b300/build.py (nvcc, sm_103a)")
    lib = ctypes.CDLL(path)
    P, D = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
    sig = {
        "dgh_create": (ctypes.c_int, [ctypes.POINTER(_Desc), P, ctypes.POINTER(P)]),
        "dgh_plan": (ctypes.c_int, [ctypes.POINTER(_Desc), ctypes.POINTER(_Info)]),
        "dgh_destroy": (None, [P]),
        "dgh_last_error": (ctypes.c_char_p, [P]),
        "dgh_get_info": (ctypes.c_int, [P, ctypes.POINTER(_Info)]),
        "dgh_get_nodes": (ctypes.c_int, [P, ctypes.c_int, D, ctypes.c_size_t]),
        "dgh_init_gaussian": (ctypes.c_int, [P, D, ctypes.c_double, ctypes.c_double]),
        "dgh_set_state": (ctypes.c_int, [P, ctypes.c_int, D, ctypes.c_size_t]),
        "dgh_get_state": (ctypes.c_int, [P, ctypes.c_int, D, ctypes.c_size_t]),
        "dgh_set_state_f32": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(ctypes.c_float), ctypes.c_size_t]),
        "dgh_get_state_f32": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(ctypes.c_float), ctypes.c_size_t]),
        "dgh_get_fields": (ctypes.c_int, [P, ctypes.c_int, D, ctypes.c_size_t]),
        "dgh_set_time": (ctypes.c_int, [P, ctypes.c_double]),
        "dgh_init_fields": (ctypes.c_int, [P, D, ctypes.c_size_t]),
        "dgh_set_material": (ctypes.c_int, [P, D, D, ctypes.c_size_t]),
        "dgh_set_material_layers": (ctypes.c_int, [P, ctypes.c_int, D, D, D]),
        "dgh_add_point_source": (ctypes.c_int, [P, D, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
        "dgh_step": (ctypes.c_int, [P, ctypes.c_int64]),
        "dgh_set_watchdog": (ctypes.c_int, [P, ctypes.c_int64, ctypes.c_double]),
        "dgh_sync": (ctypes.c_int, [P]),
        "dgh_is_checked_build": (ctypes.c_int, []),
        "dgh_time_kernels": (ctypes.c_int, [P, ctypes.c_int64, D]),
        "dgh_get_energy": (ctypes.c_int, [P, D]),
        "dgh_get_error_energy": (ctypes.c_int, [P, D, ctypes.c_size_t, D]),
        "dgh_get_energy_noalloc": (ctypes.c_int, [P, ctypes.c_void_p, P]),
        "dgh_save_state": (ctypes.c_int, [P, P, ctypes.POINTER(ctypes.c_size_t)]),
        "dgh_load_state": (ctypes.c_int, [P, P, ctypes.c_size_t]),
        "dgh_get_launch": (ctypes.c_int, [P, ctypes.POINTER(_Launch)]),
        "dgh_set_launch": (ctypes.c_int, [P, ctypes.POINTER(_Launch)]),
        "dgh_tune": (ctypes.c_int, [P, ctypes.c_int, D, D]),
        "dgh_batch_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(P)]),
        "dgh_batch_plan": (ctypes.c_int, [ctypes.POINTER(_Desc), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(_Info), ctypes.POINTER(ctypes.c_int)]),
        "dgh_batch_destroy": (None, [P]),
        "dgh_batch_last_error": (ctypes.c_char_p, [P]),
        "dgh_batch_count": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "dgh_batch_stream": (ctypes.c_int, [P, ctypes.POINTER(P)]),
        "dgh_batch_step": (ctypes.c_int, [P, ctypes.c_int64]),
        "dgh_batch_sync": (ctypes.c_int, [P]),
        "dgh_batch_get_info": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(_Info)]),
        "dgh_batch_get_state": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, D, ctypes.c_size_t]),
        "dgh_batch_get_energy": (ctypes.c_int, [P, ctypes.c_int, D]),
        "dgh_batch_get_launch": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(_Launch)]),
        "dgh_batch_tune": (ctypes.c_int, [P, ctypes.c_int, D, D]),
        "dgh_selftest_wait": (ctypes.c_int, [P, ctypes.c_int64]),
        "dgh_selftest_throw": (ctypes.c_int, [ctypes.c_int]),
        "dgh_fp32_probe": (ctypes.c_int, [D, D]),
        "dgh_clear_error": (ctypes.c_int, [P]),
        "dgh_closure_set_weights": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_float), ctypes.c_size_t]),
        "dgh_closure_record": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int64,
                                              ctypes.c_uint64]),
        "dgh_closure_samples": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_float), ctypes.c_int64,
                                               ctypes.POINTER(ctypes.c_int64)]),
        "dgh_closure_eval": (ctypes.c_int, [ctypes.POINTER(ctypes.c_float), ctypes.c_size_t,
                                            ctypes.POINTER(ctypes.c_float), ctypes.c_int64,
                                            ctypes.POINTER(ctypes.c_float)]),
        "dgh_mlp_loss_grad": (ctypes.c_int, [ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                             ctypes.POINTER(ctypes.c_float), ctypes.c_int64, D,
                                             ctypes.POINTER(ctypes.c_float)]),
        "dgh_mlp_train": (ctypes.c_int, [ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), ctypes.c_int64,
                                         ctypes.POINTER(_TrainCfg), ctypes.POINTER(ctypes.c_float), D, D]),
        "dgh_closure_train": (ctypes.c_int, [P, ctypes.POINTER(_TrainCfg), ctypes.POINTER(ctypes.c_float), D, D]),
        "dgh_closure_train_homogeneous": (ctypes.c_int, [P, ctypes.POINTER(_TrainCfg), ctypes.POINTER(ctypes.c_float),
                                                         D, D]),
        "dgh_closure_fit_homogeneous": (ctypes.c_int, [ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                                       ctypes.c_int64, ctypes.POINTER(_TrainCfg),
                                                       ctypes.POINTER(ctypes.c_float), D, D]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None and a.shape != shape:
        raise ValueError("expected shape %s, got %s" % (shape, a.shape))
    return a


def _lib_check(rc):
    if rc != DGH_OK:
        raise DghError(rc, load_library().dgh_last_error(None).decode())


def fp32_probe():
    """Measured FP32 CUDA-core TFLOP/s (scalar FFMA, packed FP32x2 FMA) of the current device."""
    lib = load_library()
    a, b = ctypes.c_double(), ctypes.c_double()
    _lib_check(lib.dgh_fp32_probe(ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def closure_eval(w, X):
    """The correction [n] of the device inference kernel for weights w (4673
    values: MLP(x) - MLP(0); 4680: the homogeneous form), features X [n][6]."""
    lib = load_library()
    w = _f32(w)
    X = _f32(X)
    y = np.empty(X.shape[0], np.float32)
    _lib_check(lib.dgh_closure_eval(_fptr(w), w.size, _fptr(X), X.shape[0], _fptr(y)))
    return y


def _train_cfg(steps=2000, batch=4096, lr=1e-3, seed=1, beta1=0.9, beta2=0.999, eps=1e-8):
    return _TrainCfg(int(steps), int(batch), float(lr), float(beta1), float(beta2), float(eps), int(seed))


def closure_fit_homogeneous(X, Y, **train_kw):
    """Train the homogeneous closure (dgh_closure_fit_homogeneous): returns
    (the 4680 values for Solver.closure_set_weights, minibatch MSE history,
    final MSE), the losses in relative-target units.  Keyword arguments as
    mlp_train."""
    lib = load_library()
    X, Y = _f32(X), _f32(Y)
    cfg = _train_cfg(**train_kw)
    w = np.empty(MLP_NPARAM + MLP_IN + 1, np.float32)
    hist = np.empty(max(int(cfg.steps), 1))
    fin = ctypes.c_double()
    _lib_check(lib.dgh_closure_fit_homogeneous(_fptr(X), _fptr(Y), X.shape[0], ctypes.byref(cfg), _fptr(w),
                                               _dptr(hist), ctypes.byref(fin)))
    return w, hist[:int(cfg.steps)], fin.value


def mlp_loss_grad(w, X, Y):
    """(loss, grad) of loss = mean (MLP(X) - Y)^2 / 2 by the device training kernels."""
    lib = load_library()
    w, X, Y = _f32(w, (MLP_NPARAM,)), _f32(X), _f32(Y)
    loss = ctypes.c_double()
    g = np.empty(MLP_NPARAM, np.float32)
    _lib_check(lib.dgh_mlp_loss_grad(_fptr(w), _fptr(X), _fptr(Y), X.shape[0], ctypes.byref(loss), _fptr(g)))
    return loss.value, g


def mlp_train(X, Y, steps=2000, batch=4096, lr=1e-3, seed=1, beta1=0.9, beta2=0.999, eps=1e-8):
    """Adam on the GPU; returns (weights for raw features, minibatch MSE history, final MSE)."""
    lib = load_library()
    X, Y = _f32(X), _f32(Y)
    cfg = _TrainCfg(int(steps), int(batch), float(lr), float(beta1), float(beta2), float(eps), int(seed))
    w = np.empty(MLP_NPARAM, np.float32)
    hist = np.empty(max(int(steps), 1))
    fin = ctypes.c_double()
    _lib_check(lib.dgh_mlp_train(_fptr(X), _fptr(Y), X.shape[0], ctypes.byref(cfg), _fptr(w), _dptr(hist),
                                 ctypes.byref(fin)))
    return w, hist[:int(steps)], fin.value


def _make_desc(VX, EToV, N, P, bc, c, rho, dt, cfl, precision=PREC_FP32):
    VX = np.ascontiguousarray(VX, dtype=np.float64)
    EToV = np.ascontiguousarray(EToV, dtype=np.int32)
    K = EToV.shape[0]
    c = np.ascontiguousarray(np.broadcast_to(np.asarray(c, np.float64), (K,)))
    rho = np.ascontiguousarray(np.broadcast_to(np.asarray(rho, np.float64), (K,)))
    d = _Desc()
    d.order, d.habc_order = int(N), int(P)
    for i in range(6):
        d.bc[i] = int(bc[i])
    d.precision = int(precision)
    d.n_vertices, d.n_cells = VX.shape[0], K
    d.vertices = _dptr(VX)
    d.cells = EToV.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    d.c, d.rho = _dptr(c), _dptr(rho)
    d.dt, d.cfl = float(dt), float(cfl)
    return d, (VX, EToV, c, rho)   # keep the arrays alive with the descriptor


def plan(VX, EToV, N, P, bc=(BC_HABC,) * 6, c=1.0, rho=1.0, dt=0.0, cfl=1.0, precision=PREC_FP32):
    """Host-only set-up (no GPU): sizes, ndof and time step of a problem."""
    lib = load_library()
    d, _keep = _make_desc(VX, EToV, N, P, bc, c, rho, dt, cfl, precision)
    i = _Info()
    rc = lib.dgh_plan(ctypes.byref(d), ctypes.byref(i))
    if rc != DGH_OK:
        raise DghError(rc, lib.dgh_last_error(None).decode())
    return {f: getattr(i, f) for f, _ in _Info._fields_}


def batch_plan(problems):
    """Host-only grouping of a batch (no GPU).  problems: a list of dicts with
    the keyword arguments of plan().  Returns (group_of, group_infos)."""
    lib = load_library()
    descs = (_Desc * len(problems))()
    keep = []
    for i, kw in enumerate(problems):
        kw = dict(kw)
        d, k = _make_desc(kw.pop("VX"), kw.pop("EToV"), kw.pop("N"), kw.pop("P"), kw.pop("bc", (BC_HABC,) * 6),
                          kw.pop("c", 1.0), kw.pop("rho", 1.0), kw.pop("dt", 0.0), kw.pop("cfl", 1.0),
                          kw.pop("precision", PREC_FP32))
        if kw:
            raise TypeError("unknown keys %s" % sorted(kw))
        descs[i] = d
        keep.append(k)
    gof = (ctypes.c_int * len(problems))()
    infos = (_Info * len(problems))()
    ng = ctypes.c_int()
    rc = lib.dgh_batch_plan(descs, len(problems), gof, infos, ctypes.byref(ng))
    if rc != DGH_OK:
        raise DghError(rc, lib.dgh_last_error(None).decode())
    return list(gof), [{f: getattr(infos[g], f) for f, _ in _Info._fields_} for g in range(ng.value)]


class Solver:
    """One DG + HABC problem on the current CUDA device.

    VX [Nv,3] vertex coordinates, EToV [K,4] cell vertex ids, N polynomial
    degree, P HABC order (0 = basic ABC), bc six codes (BC_HABC /
    BC_DIRICHLET for -x,+x,-y,+y,-z,+z), c and rho per cell (or scalars),
    dt > 0 fixed step (else cfl * the min-over-cells rule), stream a
    torch.cuda.Stream, an integer cudaStream_t or None, precision one of
    PREC_FP32 (the FP32 contract, with the faster of its two kernels:
    split-TF32 tensor-core products at N = 4 with >= 65,536 cells, FP32 CUDA
    cores otherwise), PREC_FP32_CUDA (FP32 CUDA cores at every order),
    PREC_SPLIT_TF32 (split TF32, N <= 4), PREC_BF16_TC,
    PREC_FP16_TC, PREC_SPLIT_BF16 (the precision form's tensor-core products
    of the 3D volume and lift terms).
    """

    def __init__(self, VX, EToV, N, P, bc=(BC_HABC,) * 6, c=1.0, rho=1.0, dt=0.0, cfl=1.0, stream=None,
                 precision=PREC_FP32):
        lib = load_library()
        d, _keep = _make_desc(VX, EToV, N, P, bc, c, rho, dt, cfl, precision)
        if stream is None:
            sptr = None
        elif isinstance(stream, int):
            sptr = stream
        else:
            sptr = stream.cuda_stream
        self.stream = stream
        h = ctypes.c_void_p()
        rc = lib.dgh_create(ctypes.byref(d), ctypes.c_void_p(sptr) if sptr else None, ctypes.byref(h))
        if rc != DGH_OK:
            raise DghError(rc, lib.dgh_last_error(None).decode())
        self._h = h
        self._lib = lib
        self.precision = int(precision)
        self.N, self.P = int(N), int(P)

    # ------------------------------------------------------------ helpers
    def _check(self, rc):
        if rc != DGH_OK:
            raise DghError(rc, self._lib.dgh_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.dgh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------ API
    @property
    def info(self):
        i = _Info()
        self._check(self._lib.dgh_get_info(self._h, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in _Info._fields_}

    def shape(self, level):
        i = self.info
        if level == 3:
            return (i["n_cells"], 4, i["Np"])
        if level == 2:
            return (i["n_tris"], self.P, 3, i["Np2"])
        if level == 1:
            return (i["n_lines"], self.P * self.P, 2, i["Np1"])
        raise ValueError("level must be 3, 2 or 1")

    def nodes(self, level):
        i = self.info
        n = {3: (i["n_cells"], i["Np"]), 2: (i["n_tris"], i["Np2"]), 1: (i["n_lines"], i["Np1"])}[level]
        out = np.empty(n + (3,))
        self._check(self._lib.dgh_get_nodes(self._h, level, _dptr(out), out.size))
        return out

    def init_gaussian(self, x0, width, amp=1.0):
        x = np.ascontiguousarray(x0, dtype=np.float64)
        self._check(self._lib.dgh_init_gaussian(self._h, _dptr(x), float(width), float(amp)))

    def set_state(self, level, arr):
        """Time-stepped variables of a level (canonical layout).  A float32
        array goes through dgh_set_state_f32 unchanged (half the bytes);
        anything else is taken as float64 (dgh_set_state)."""
        if isinstance(arr, np.ndarray) and arr.dtype == np.float32:
            a = np.ascontiguousarray(arr)
            if a.shape != self.shape(level):
                raise ValueError("state shape %s != %s" % (a.shape, self.shape(level)))
            self._check(self._lib.dgh_set_state_f32(self._h, level, _fptr(a), a.size))
            return
        a = np.ascontiguousarray(arr, dtype=np.float64)
        if a.shape != self.shape(level):
            raise ValueError("state shape %s != %s" % (a.shape, self.shape(level)))
        self._check(self._lib.dgh_set_state(self._h, level, _dptr(a), a.size))

    def get_state(self, level, out=None, dtype=np.float64):
        """Time-stepped variables of a level (canonical layout); out: an
        optional C-contiguous float64 or float32 array of the right shape to
        fill (e.g. in pinned host memory), else a new array of dtype.  float32
        reads the device state unchanged (dgh_get_state_f32)."""
        shape = self.shape(level)
        if out is None:
            out = np.empty(shape, dtype=dtype)
        if out.dtype not in (np.float64, np.float32) or out.shape != shape or not out.flags.c_contiguous:
            raise ValueError("out must be a C-contiguous float64 or float32 array of shape %s" % (shape,))
        if out.dtype == np.float32:
            self._check(self._lib.dgh_get_state_f32(self._h, level, _fptr(out), out.size))
        else:
            self._check(self._lib.dgh_get_state(self._h, level, _dptr(out), out.size))
        return out

    def get_fields(self, level):
        out = np.empty(self.shape(level))
        self._check(self._lib.dgh_get_fields(self._h, level, _dptr(out), out.size))
        return out

    def set_time(self, t):
        self._check(self._lib.dgh_set_time(self._h, float(t)))

    def init_fields(self, q3):
        """Initial state from 3D fields [K][4][Np] (canonical order); auxiliary
        fields, time and step count to zero."""
        q = np.ascontiguousarray(q3, dtype=np.float64)
        self._check(self._lib.dgh_init_fields(self._h, _dptr(q), q.size))

    def set_material(self, c, rho):
        """New material (c, rho per cell); the state carries over."""
        K = self.info["n_cells"]
        cc = np.ascontiguousarray(np.broadcast_to(np.asarray(c, np.float64), (K,)))
        rr = np.ascontiguousarray(np.broadcast_to(np.asarray(rho, np.float64), (K,)))
        self._check(self._lib.dgh_set_material(self._h, _dptr(cc), _dptr(rr), K))

    def set_material_layers(self, z_top, c, rho):
        """Horizontal layers bottom to top: layer l holds cell centroids with
        z < z_top[l]; len(c) = len(rho) = len(z_top) + 1."""
        z = np.ascontiguousarray(z_top, dtype=np.float64)
        cc = np.ascontiguousarray(c, dtype=np.float64)
        rr = np.ascontiguousarray(rho, dtype=np.float64)
        if cc.size != z.size + 1 or rr.size != cc.size:
            raise ValueError("need len(c) == len(rho) == len(z_top) + 1")
        self._check(self._lib.dgh_set_material_layers(self._h, int(cc.size), _dptr(z) if z.size else None,
                                                      _dptr(cc), _dptr(rr)))

    def set_watchdog(self, every, energy_limit=0.0):
        """Energy watchdog (dgh_set_watchdog): every `every` steps, step()
        raises DghError (EUNSTABLE) if the 3D energy is not finite or exceeds
        energy_limit (> 0).  every = 0 turns it off."""
        self._check(self._lib.dgh_set_watchdog(self._h, int(every), float(energy_limit)))

    def add_point_source(self, xs, f_peak, t_s, amp=1.0):
        x = np.ascontiguousarray(xs, dtype=np.float64)
        self._check(self._lib.dgh_add_point_source(self._h, _dptr(x), float(f_peak), float(t_s), float(amp)))

    def step(self, n=1):
        self._check(self._lib.dgh_step(self._h, int(n)))

    def time_kernels(self, nsteps):
        """Mean launch duration (ms) of the 3D, 2D, 1D, 0D stage kernels and of
        a step, from CUDA events around every launch (advances the solution)."""
        out = np.zeros(5)
        self._check(self._lib.dgh_time_kernels(self._h, int(nsteps), _dptr(out)))
        return {"k3d": out[0], "k2d": out[1], "k1d": out[2], "k0d": out[3], "step": out[4]}

    def sync(self):
        self._check(self._lib.dgh_sync(self._h))

    def selftest_wait(self, limit=1000):
        """Return code of the bounded-wait self-test (DGH_ETIMEOUT = -5 expected)."""
        return self._lib.dgh_selftest_wait(self._h, int(limit))

    def clear_error(self):
        self._check(self._lib.dgh_clear_error(self._h))

    def energy(self):
        e = ctypes.c_double()
        self._check(self._lib.dgh_get_energy(self._h, ctypes.byref(e)))
        return e.value

    def error_energy(self, ref3):
        """Energy of (3D fields - ref3), ref3 [K][4][Np] FP64 (device reduction, FP64)."""
        r = np.ascontiguousarray(ref3, dtype=np.float64)
        if r.shape != self.shape(3):
            raise ValueError("reference shape %s != %s" % (r.shape, self.shape(3)))
        e = ctypes.c_double()
        self._check(self._lib.dgh_get_error_energy(self._h, _dptr(r), r.size, ctypes.byref(e)))
        return e.value

    def energy_noalloc(self, d_out, stream=None):
        """Energy written to the device double at address d_out (an int), with no
        allocation inside the call (see dgh_get_energy_noalloc); asynchronous.
        A stream other than the solver's is first made to wait for the work
        already enqueued on the solver's stream."""
        sptr = stream if isinstance(stream, int) or stream is None else stream.cuda_stream
        self._check(self._lib.dgh_get_energy_noalloc(self._h, ctypes.c_void_p(d_out),
                                                     ctypes.c_void_p(sptr) if sptr else None))

    def save_state(self):
        size = ctypes.c_size_t(0)
        self._check(self._lib.dgh_save_state(self._h, None, ctypes.byref(size)))
        buf = ctypes.create_string_buffer(size.value)
        self._check(self._lib.dgh_save_state(self._h, ctypes.cast(buf, ctypes.c_void_p), ctypes.byref(size)))
        return buf.raw

    def load_state(self, blob):
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        self._check(self._lib.dgh_load_state(self._h, ctypes.cast(buf, ctypes.c_void_p), len(blob)))

    def closure_set_weights(self, w):
        """Enable the learned closure with weights w (4673, or 4680 for the
        homogeneous form), or disable it (None)."""
        if w is None:
            self._check(self._lib.dgh_closure_set_weights(self._h, None, 0))
            return
        w = _f32(w)
        self._check(self._lib.dgh_closure_set_weights(self._h, _fptr(w), w.size))

    def closure_record(self, shadow_order=2, every=1, fraction=1.0, max_samples=1 << 20, seed=0):
        """Add a shadow HABC chain of order shadow_order driven one-way by this
        solver's 3D traces and record training rows on every `every`-th step
        from a hashed fraction of the boundary face nodes (dgh_closure_record)."""
        self._check(self._lib.dgh_closure_record(self._h, int(shadow_order), int(every), float(fraction),
                                                 int(max_samples), int(seed)))

    def closure_train(self, homogeneous=False, **train_kw):
        """Train the closure on this solver's recorded rows (dgh_closure_train,
        or dgh_closure_train_homogeneous); returns (weights, minibatch MSE
        history, final MSE) like mlp_train / closure_fit_homogeneous."""
        cfg = _train_cfg(**train_kw)
        w = np.empty(MLP_NPARAM + (MLP_IN + 1 if homogeneous else 0), np.float32)
        hist = np.empty(max(int(cfg.steps), 1))
        fin = ctypes.c_double()
        fn = self._lib.dgh_closure_train_homogeneous if homogeneous else self._lib.dgh_closure_train
        self._check(fn(self._h, ctypes.byref(cfg), _fptr(w), _dptr(hist), ctypes.byref(fin)))
        return w, hist[:int(cfg.steps)], fin.value

    def closure_samples(self, max_rows=None):
        """Recorded rows [n][7]: 6 features and the target.  Open-loop rows
        (closure off): the shadow chain's features, r^-_this - r^-_shadow.
        Closed-loop rows (closure on): this chain's features, r^-_shadow -
        r^-_this."""
        cnt = ctypes.c_int64()
        self._check(self._lib.dgh_closure_samples(self._h, None, 0, ctypes.byref(cnt)))
        n = cnt.value if max_rows is None else min(cnt.value, int(max_rows))
        out = np.empty((n, 7), np.float32)
        self._check(self._lib.dgh_closure_samples(self._h, _fptr(out), n, ctypes.byref(cnt)))
        return out

    @property
    def launch(self):
        """Launch shape (tile2, tile1, cta3_per_sm and the derived grids)."""
        o = _Launch()
        self._check(self._lib.dgh_get_launch(self._h, ctypes.byref(o)))
        return {f: getattr(o, f) for f, _ in _Launch._fields_}

    def set_launch(self, tile2=None, tile1=None, cta3_per_sm=None, thr2=None, thr1=None, sm3_div=None, split3=None):
        cur = self.launch
        o = _Launch()
        o.tile2 = cur["tile2"] if tile2 is None else int(tile2)
        o.tile1 = cur["tile1"] if tile1 is None else int(tile1)
        o.cta3_per_sm = cur["cta3_per_sm"] if cta3_per_sm is None else int(cta3_per_sm)
        o.thr2 = cur["thr2"] if thr2 is None else int(thr2)
        o.thr1 = cur["thr1"] if thr1 is None else int(thr1)
        o.sm3_div = cur["sm3_div"] if sm3_div is None else int(sm3_div)
        o.split3 = cur["split3"] if split3 is None else int(split3)
        self._check(self._lib.dgh_set_launch(self._h, ctypes.byref(o)))

    def tune(self, steps=5, cache=None):
        """Autotune the launch shape (results unchanged); returns (ms/step
        before, after).  With cache (a JSON file path), a shape stored for the
        same key (tune_cache_key) is applied instead of searching, and a new
        search result is stored."""
        key = tune_cache_key(self.info, self.precision) if cache else None
        if cache:
            hit = tune_cache_load(cache).get(key)
            if hit is not None:
                self.set_launch(**{k: hit[k] for k in TUNABLE if k in hit})
                return hit["ms_before"], hit["ms_after"]
        a, b = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.dgh_tune(self._h, int(steps), ctypes.byref(a), ctypes.byref(b)))
        if cache:
            L = self.launch
            tune_cache_store(cache, key, dict({k: L[k] for k in TUNABLE}, ms_before=a.value, ms_after=b.value))
        return a.value, b.value


TUNABLE = ("tile2", "tile1", "cta3_per_sm", "thr2", "thr1", "sm3_div", "split3")


def tune_cache_key(info, precision):
    """Key of a tuned launch shape in a tuning cache: the orders, the
    precision mode and the sizes of every level (a cache file belongs to one
    machine and build)."""
    return "N%d_P%d_prec%d_K%d_T%d_L%d_C%d" % (info["order"], info["habc_order"], int(precision), info["n_cells"],
                                               info["n_tris"], info["n_lines"], info["n_corners"])


def tune_cache_load(path):
    """The cache {key: shape}; empty when the file does not exist."""
    import json
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def tune_cache_store(path, key, shape):
    """Adds or replaces one entry (written to a temporary file, then renamed)."""
    import json
    data = tune_cache_load(path)
    data[key] = shape
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


class Batch:
    """Independent problems stepped together (see dgh_batch_create): a snapshot
    of the given Solver objects, grouped by (N, P), one graph per step."""

    def __init__(self, solvers):
        lib = load_library()
        arr = (ctypes.c_void_p * len(solvers))(*[s._h.value for s in solvers])
        h = ctypes.c_void_p()
        rc = lib.dgh_batch_create(arr, len(solvers), ctypes.byref(h))
        if rc != DGH_OK:
            raise DghError(rc, lib.dgh_batch_last_error(None).decode())
        self._h, self._lib = h, lib
        self._P = [s.P for s in solvers]

    def _check(self, rc):
        if rc != DGH_OK:
            raise DghError(rc, self._lib.dgh_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.dgh_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def counts(self):
        n, g = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.dgh_batch_count(self._h, ctypes.byref(n), ctypes.byref(g)))
        return n.value, g.value

    @property
    def stream_handle(self):
        """The batch's cudaStream_t as an int (all its device work runs there)."""
        p = ctypes.c_void_p()
        self._check(self._lib.dgh_batch_stream(self._h, ctypes.byref(p)))
        return p.value

    def info(self, i):
        o = _Info()
        self._check(self._lib.dgh_batch_get_info(self._h, int(i), ctypes.byref(o)))
        return {f: getattr(o, f) for f, _ in _Info._fields_}

    def shape(self, i, level):
        d = self.info(i)
        P = self._P[i]
        return {3: (d["n_cells"], 4, d["Np"]), 2: (d["n_tris"], P, 3, d["Np2"]),
                1: (d["n_lines"], P * P, 2, d["Np1"])}[level]

    def step(self, n=1):
        self._check(self._lib.dgh_batch_step(self._h, int(n)))

    def sync(self):
        self._check(self._lib.dgh_batch_sync(self._h))

    def get_state(self, i, level):
        out = np.empty(self.shape(i, level))
        self._check(self._lib.dgh_batch_get_state(self._h, int(i), level, _dptr(out), out.size))
        return out

    def energy(self, i):
        e = ctypes.c_double()
        self._check(self._lib.dgh_batch_get_energy(self._h, int(i), ctypes.byref(e)))
        return e.value

    def launch(self, group):
        o = _Launch()
        self._check(self._lib.dgh_batch_get_launch(self._h, int(group), ctypes.byref(o)))
        return {f: getattr(o, f) for f, _ in _Launch._fields_}

    def tune(self, steps=5):
        a, b = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.dgh_batch_tune(self._h, int(steps), ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value
