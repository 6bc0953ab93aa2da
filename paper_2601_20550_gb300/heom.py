"""ctypes binding of libheom2dvs (argument marshalling only).

Every function here forwards to the C entry point of the same name in
include/heom2dvs.h; all arithmetic of the method runs in the library's CUDA
kernels.  The library is loaded from this package directory and its absence is
an error: there is no CPU fallback.
"""
import copy
import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libheom2dvs.so")

FP64, FP32, TC = 0, 1, 2
STATUS = {0: "HEOM_OK", -1: "HEOM_EINVAL", -2: "HEOM_ENOMEM", -3: "HEOM_ECUDA",
          -4: "HEOM_EUNSTABLE", -5: "HEOM_ETIMEOUT", -6: "HEOM_ENOTCONV",
          -7: "HEOM_ENONFINITE", -8: "HEOM_ECKPT"}


class HeomError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class heom_mode(ct.Structure):
    _fields_ = [("potential", ct.c_int), ("omega_cm", ct.c_double), ("g3_cm", ct.c_double),
                ("morse_D_cm", ct.c_double), ("n_levels", ct.c_int), ("n_prim", ct.c_int),
                ("q_min", ct.c_double), ("q_max", ct.c_double), ("zeta_cm", ct.c_double),
                ("gamma_cm", ct.c_double), ("V_LL", ct.c_double), ("V_SL", ct.c_double),
                ("mu1", ct.c_double), ("mu2", ct.c_double), ("K_pade", ct.c_int)]


class heom_pair(ct.Structure):
    _fields_ = [("s", ct.c_int), ("t", ct.c_int), ("g_st_cm", ct.c_double),
                ("g_s2t_cm", ct.c_double), ("g_st2_cm", ct.c_double), ("mu_st", ct.c_double)]


class heom_model(ct.Structure):
    _fields_ = [("n_modes", ct.c_int), ("modes", ct.POINTER(heom_mode)), ("n_pairs", ct.c_int),
                ("pairs", ct.POINTER(heom_pair)), ("T_K", ct.c_double), ("depth_L", ct.c_int),
                ("precision", ct.c_int)]


class heom_grid(ct.Structure):
    _fields_ = [("dt_fs", ct.c_double), ("steps_per_sample", ct.c_int), ("n1", ct.c_int),
                ("n3", ct.c_int), ("n_t2", ct.c_int), ("t2_fs", ct.POINTER(ct.c_double))]


class heom_hier_info(ct.Structure):
    _fields_ = [("d", ct.c_int), ("n_ado", ct.c_int), ("n_exp", ct.c_int), ("n_modes", ct.c_int),
                ("precision", ct.c_int), ("beta", ct.c_double)]


_lib = None
_P = ct.c_void_p
_D = ct.POINTER(ct.c_double)


def lib():
    """Load libheom2dvs.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libheom2dvs.so not found at %s; run __graft_entry__.build()" % LIB_PATH)
    L = ct.CDLL(LIB_PATH)
    sig = {
        "heom_build_hierarchy": [ct.POINTER(heom_model), ct.POINTER(_P)],
        "heom_get_info": [_P, ct.POINTER(heom_hier_info)],
        "heom_get_operators": [_P, _D, _D, _D, _D, ct.POINTER(ct.c_int32)],
        "heom_get_mode": [_P, ct.c_int, _D, _D],
        "heom_equilibrate": [_P, ct.c_double, ct.c_double, ct.c_double, ct.POINTER(_P)],
        "heom_state_create": [_P, ct.c_int, ct.c_int, ct.POINTER(_P)],
        "heom_state_upload": [_P, _D],
        "heom_state_download": [_P, _D],
        "heom_state_copy_out": [_P, _D],
        "heom_propagate": [_P, _P, ct.c_double, ct.c_int64],
        "heom_kick": [_P, _P, ct.c_int],
        "heom_trace": [_P, _P, ct.c_int, _D],
        "heom_response_2d": [_P, _P, ct.POINTER(heom_grid), _D, _D, _D],
        "heom_response_1d": [_P, _P, ct.c_double, ct.c_int, ct.c_int, _D, _D],
        "heom_propagate_dev": [_P, _P, _P, _P, ct.c_int, ct.c_int, ct.c_double, ct.c_int64, _P],
        "heom_response_2d_rows": [_P, _P, ct.POINTER(heom_grid), ct.c_int, ct.c_int, _D, _D],
        "heom_response_2d_batched": [ct.POINTER(_P), ct.POINTER(_P), ct.c_int, ct.POINTER(heom_grid), _D, _D, _D],
        "heom_response_2d_grad": [_P, _P, ct.POINTER(heom_grid), _D, ct.c_int, _D, _D],
        "heom_steady_state": [_P, ct.c_double, ct.c_int, ct.c_int, ct.c_double, ct.c_int, ct.POINTER(_P),
                              ct.POINTER(ct.c_int)],
        "heom_get_tuning": [_P, ct.c_int, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int64), ct.POINTER(ct.c_int),
                            ct.POINTER(ct.c_int)],
        "heom_state_broadcast": [_P, _P],
        "heom_spectrum_2d": [_D, _D, ct.c_int, ct.c_int, ct.c_int, ct.c_double, _D],
        "heom_trace_dev": [_P, _P, ct.c_int, ct.c_int, ct.c_int, _P, _P],
        "heom_kick_dev": [_P, _P, _P, ct.c_int, ct.c_int, ct.c_int, _P],
        "heom_state_export_dev": [_P, _P, _P],
        "heom_propagate_noalloc": [_P, _P, ct.c_int, ct.c_double, ct.c_int64, _P],
        "heom_state_import_dev": [_P, _P, _P],
        "heom_set_wait_limit_ns": [_P, ct.c_uint64],
        "heom_ckpt_write": [ct.c_char_p, _P, ct.c_uint64],
        "heom_ckpt_read": [ct.c_char_p, _P, ct.c_uint64],
        "heom_ckpt_verify": [ct.c_char_p, ct.POINTER(ct.c_uint64)],
        "heom_state_save": [_P, ct.c_char_p],
        "heom_state_load": [_P, ct.c_char_p],
        "heom_debug_force_tc_shape": [ct.c_int],
        "heom_tc_shape_count": [],
        "heom_tc_shape_params": [ct.c_int, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int), ct.POINTER(ct.c_int),
                                 ct.POINTER(ct.c_int)],
        "heom_get_tc_shape": [_P, ct.c_int64, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int), ct.POINTER(ct.c_int),
                              ct.POINTER(ct.c_int)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ct.c_int
    L.heom_free_hier.argtypes = [_P]
    L.heom_free_hier.restype = None
    L.heom_free_state.argtypes = [_P]
    L.heom_free_state.restype = None
    L.heom_last_error.restype = ct.c_char_p
    L.heom_launch_count.restype = ct.c_uint64
    L.heom_source_tag.restype = ct.c_char_p
    L.heom_state_device_ptr.argtypes = [_P]
    L.heom_state_device_ptr.restype = _P
    L.heom_state_branches.argtypes = [_P]
    L.heom_state_branches.restype = ct.c_int
    L.heom_debug_fail_alloc.argtypes = [ct.c_int64]
    L.heom_debug_fail_alloc.restype = None
    _lib = L
    return L


def _check(rc, allow=()):
    if rc != 0 and rc not in allow:
        raise HeomError(rc, lib().heom_last_error().decode())
    return rc


def _dptr(a):
    return a.ctypes.data_as(_D) if a is not None else None


POTENTIAL = {"cubic": 0, "harmonic": 0, "morse": 1}


def marshal_model(model, precision=FP64):
    """heom_model struct from a model dictionary (keeps the arrays alive on the struct)."""
    modes = (heom_mode * len(model["modes"]))()
    for i, md in enumerate(model["modes"]):
        modes[i] = heom_mode(POTENTIAL[md["potential"]], md["omega_cm"], md["g3_cm"],
                             md["morse_D_cm"], md["n_levels"], md["n_prim"], md["q_min"],
                             md["q_max"], md["zeta_cm"], md["gamma_cm"], md["V_LL"], md["V_SL"],
                             md["mu1"], md["mu2"], md["K_pade"])
    npair = len(model["pairs"])
    pairs = (heom_pair * max(1, npair))()
    for i, pr in enumerate(model["pairs"]):
        pairs[i] = heom_pair(pr["s"], pr["t"], pr["g_st_cm"], pr["g_s2t_cm"], pr["g_st2_cm"],
                             pr["mu_st"])
    m = heom_model(len(model["modes"]), modes, npair, pairs, model["T_K"], model["depth_L"],
                   precision)
    m._keep = (modes, pairs)
    return m


def marshal_grid(grid):
    t2 = np.ascontiguousarray(grid["t2_fs"], dtype=np.float64)
    g = heom_grid(grid["dt_fs"], grid["steps_per_sample"], grid["n1"], grid["n3"], len(t2),
                  t2.ctypes.data_as(_D))
    g._keep = t2
    return g


class Hier:
    """Owning wrapper of a heom_hier handle."""

    def __init__(self, handle):
        self.h = handle
        info = heom_hier_info()
        _check(lib().heom_get_info(self.h, ct.byref(info)))
        self.d, self.n_ado, self.n_exp = info.d, info.n_ado, info.n_exp
        self.n_modes, self.precision, self.beta = info.n_modes, info.precision, info.beta

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.heom_free_hier(self.h)
            self.h = None


class State:
    """Owning wrapper of a heom_state handle."""

    def __init__(self, handle, hier, branches, precision):
        self.h, self.hier, self.branches, self.precision = handle, hier, branches, precision

    @property
    def shape(self):
        return (self.branches, self.hier.n_ado, self.hier.d, self.hier.d)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.heom_free_state(self.h)
            self.h = None


def heom_build_hierarchy(model, precision=FP64):
    m = marshal_model(model, precision)
    out = _P()
    _check(lib().heom_build_hierarchy(ct.byref(m), ct.byref(out)))
    return Hier(out)


def heom_get_operators(h):
    d, D, N = h.d, h.n_exp, h.n_ado
    H = np.zeros((d, d))
    mu = np.zeros((d, d))
    mup = np.zeros((d, d))
    bath = np.zeros((D, 4))
    ado = np.zeros((N, D), dtype=np.int32)
    _check(lib().heom_get_operators(h.h, _dptr(H), _dptr(mu), _dptr(mup), _dptr(bath),
                                    ado.ctypes.data_as(ct.POINTER(ct.c_int32))))
    return {"H": H, "mu": mu, "mu_plus": mup, "bath": bath, "ado": ado}


def heom_get_mode(h, s, n):
    E = np.zeros(n)
    qk = np.zeros((4, n, n))
    _check(lib().heom_get_mode(h.h, s, _dptr(E), _dptr(qk)))
    return E, qk


def heom_state_create(h, branches, precision=FP64):
    out = _P()
    _check(lib().heom_state_create(h.h, branches, precision, ct.byref(out)))
    return State(out, h, branches, precision)


def heom_state_upload(s, arr):
    a = np.ascontiguousarray(arr, dtype=np.complex128)
    if a.shape != s.shape:
        raise ValueError("state shape %s, array %s" % (s.shape, a.shape))
    _check(lib().heom_state_upload(s.h, a.ctypes.data_as(_D)))


def heom_state_download(s):
    a = np.zeros(s.shape, dtype=np.complex128)
    _check(lib().heom_state_download(s.h, a.ctypes.data_as(_D)))
    return a


def heom_state_copy_out(s):
    """The state as [branches][n_ado][d][d] complex128 in the product eigenbasis."""
    a = np.zeros(s.shape, dtype=np.complex128)
    _check(lib().heom_state_copy_out(s.h, a.ctypes.data_as(_D)))
    return a


def heom_equilibrate(h, dt_fs, t_max_fs, tol=0.0):
    out = _P()
    rc = _check(lib().heom_equilibrate(h.h, dt_fs, t_max_fs, tol, ct.byref(out)), allow=(-6,))
    s = State(out, h, 1, FP64)
    s.converged = rc == 0
    return s


def heom_propagate(h, s, dt_fs, n_steps):
    _check(lib().heom_propagate(h.h, s.h, dt_fs, int(n_steps)))


def heom_kick(h, s, which):
    _check(lib().heom_kick(h.h, s.h, which))


def heom_trace(h, s, order):
    out = np.zeros(s.branches, dtype=np.complex128)
    _check(lib().heom_trace(h.h, s.h, order, out.ctypes.data_as(_D)))
    return out


def heom_response_2d(h, rho_eq, grid):
    g = marshal_grid(grid)
    shape = (len(grid["t2_fs"]), grid["n1"], grid["n3"])
    RI = np.zeros(shape, dtype=np.complex128)
    RII = np.zeros(shape, dtype=np.complex128)
    SC = np.zeros(shape)
    _check(lib().heom_response_2d(h.h, rho_eq.h, ct.byref(g), RI.ctypes.data_as(_D),
                                  RII.ctypes.data_as(_D), SC.ctypes.data_as(_D)))
    return RI, RII, SC


def heom_response_2d_batched(hiers, eqs, grid):
    """R_I, R_II, S_C of shape (n_sets, n_t2, n1, n3) for several parameter sets."""
    g = marshal_grid(grid)
    n = len(hiers)
    shape = (n, len(grid["t2_fs"]), grid["n1"], grid["n3"])
    RI = np.zeros(shape, dtype=np.complex128)
    RII = np.zeros(shape, dtype=np.complex128)
    SC = np.zeros(shape)
    harr = (_P * n)(*[x.h for x in hiers])
    earr = (_P * n)(*[x.h for x in eqs])
    _check(lib().heom_response_2d_batched(harr, earr, n, ct.byref(g), RI.ctypes.data_as(_D),
                                          RII.ctypes.data_as(_D), SC.ctypes.data_as(_D)))
    return RI, RII, SC


N_THETA = 12


def _theta_slot(model, i):
    """(dict, key) of gradient parameter i in a model description, or None."""
    grp, k = divmod(i, 3)
    if grp == 1:
        return (model["pairs"][k], "g_s2t_cm") if k < len(model["pairs"]) else None
    if k >= len(model["modes"]):
        return None
    md = model["modes"][k]
    if grp == 0:
        return (md, "morse_D_cm") if md["potential"] == "morse" else (md, "g3_cm")
    return (md, "V_SL") if grp == 2 else (md, "gamma_cm")


def theta_of(model):
    """The twelve gradient parameters of a model description (dtheta order of heom_response_2d_grad)."""
    th = np.zeros(N_THETA)
    for i in range(N_THETA):
        s = _theta_slot(model, i)
        if s is not None:
            th[i] = s[0][s[1]]
    return th


def with_theta(model, theta):
    """Copy of a model description with the twelve parameters replaced."""
    out = copy.deepcopy(model)
    for i in range(N_THETA):
        s = _theta_slot(out, i)
        if s is not None:
            s[0][s[1]] = float(theta[i])
    return out


def heom_response_2d_grad(h, rho_eq, grid, S_ref, ckpt_every=64):
    """(loss, dtheta[12]) of the squared misfit of S_C against S_ref [n_t2][n1][n3]."""
    g = marshal_grid(grid)
    S = np.ascontiguousarray(S_ref, dtype=np.float64).reshape(len(grid["t2_fs"]), grid["n1"], grid["n3"])
    loss = np.zeros(1)
    dth = np.zeros(12)
    _check(lib().heom_response_2d_grad(h.h, rho_eq.h, ct.byref(g), S.ctypes.data_as(_D), int(ckpt_every),
                                       loss.ctypes.data_as(_D), dth.ctypes.data_as(_D)))
    return float(loss[0]), dth


def heom_response_2d_rows(h, rho_eq, grid, j0, j1):
    g = marshal_grid(grid)
    shape = (len(grid["t2_fs"]), j1 - j0, grid["n3"])
    RI = np.zeros(shape, dtype=np.complex128)
    RII = np.zeros(shape, dtype=np.complex128)
    _check(lib().heom_response_2d_rows(h.h, rho_eq.h, ct.byref(g), j0, j1, RI.ctypes.data_as(_D),
                                       RII.ctypes.data_as(_D)))
    return RI, RII


def heom_spectrum_2d(R_I, R_II, dtau_fs):
    """S_C from R_I, R_II of shape (n_t2, n1, n3) (device Fourier sums)."""
    RI = np.ascontiguousarray(R_I, dtype=np.complex128)
    RII = np.ascontiguousarray(R_II, dtype=np.complex128)
    SC = np.zeros(RI.shape)
    _check(lib().heom_spectrum_2d(RI.ctypes.data_as(_D), RII.ctypes.data_as(_D), RI.shape[0],
                                  RI.shape[1], RI.shape[2], dtau_fs, SC.ctypes.data_as(_D)))
    return SC


def heom_state_broadcast(src, dst):
    _check(lib().heom_state_broadcast(src.h, dst.h))


def heom_state_device_ptr(s):
    return int(lib().heom_state_device_ptr(s.h) or 0)


def heom_state_export_dev(s, dst_ptr, stream_ptr=0):
    _check(lib().heom_state_export_dev(s.h, _P(dst_ptr), _P(stream_ptr)))


def heom_state_import_dev(s, src_ptr, stream_ptr=0):
    _check(lib().heom_state_import_dev(s.h, _P(src_ptr), _P(stream_ptr)))


def heom_trace_dev(h, state_ptr, branches, precision, order, out_ptr, stream_ptr):
    _check(lib().heom_trace_dev(h.h, _P(state_ptr), branches, precision, order, _P(out_ptr),
                                _P(stream_ptr)))


def heom_kick_dev(h, in_ptr, out_ptr, branches, precision, which, stream_ptr):
    _check(lib().heom_kick_dev(h.h, _P(in_ptr), _P(out_ptr), branches, precision, which,
                               _P(stream_ptr)))


def heom_response_1d(h, rho_eq, dt_fs, m, n):
    R1 = np.zeros(n, dtype=np.complex128)
    I = np.zeros(n)
    _check(lib().heom_response_1d(h.h, rho_eq.h, dt_fs, m, n, R1.ctypes.data_as(_D), _dptr(I)))
    return R1, I


def heom_propagate_dev(h, state_ptr, scratch_a_ptr, scratch_b_ptr, branches, precision, dt_fs,
                       n_steps, stream_ptr):
    """Device-pointer propagation (pointers as ints, e.g. torch tensor.data_ptr())."""
    _check(lib().heom_propagate_dev(h.h, _P(state_ptr), _P(scratch_a_ptr), _P(scratch_b_ptr),
                                    branches, precision, dt_fs, int(n_steps), _P(stream_ptr)))


def heom_propagate_noalloc(h, state_ptr, branches, dt_fs, n_steps, stream_ptr=0):
    """Allocation-free FP64 propagation of a device state (scratch in a static device array)."""
    _check(lib().heom_propagate_noalloc(h.h, _P(state_ptr), branches, dt_fs, int(n_steps),
                                        _P(stream_ptr)))


def heom_steady_state(h, tol=1e-12, restart=40, max_iter=4000, dt_fs=0.5, steps_per_matvec=0):
    """(rho_eq State, Arnoldi steps) of the Krylov steady-state solve."""
    out = _P()
    its = ct.c_int(0)
    rc = _check(lib().heom_steady_state(h.h, float(tol), int(restart), int(max_iter), float(dt_fs),
                                        int(steps_per_matvec), ct.byref(out), ct.byref(its)), allow=(-6,))
    s = State(out, h, 1, FP64)
    s.converged = rc == 0
    return s, its.value


def heom_get_tuning(h):
    """[(kind, elements, block, grid)] launch shapes the autotuner chose for hierarchy h."""
    L = lib()
    n = L.heom_get_tuning(h.h, 0, None, None, None, None)
    kind, el = (ct.c_int * max(n, 1))(), (ct.c_int64 * max(n, 1))()
    blk, grd = (ct.c_int * max(n, 1))(), (ct.c_int * max(n, 1))()
    L.heom_get_tuning(h.h, n, kind, el, blk, grd)
    return [(kind[i], el[i], blk[i], grd[i]) for i in range(n)]


def heom_ckpt_write(path, arr):
    """Write a contiguous numpy array's bytes to a checkpoint file."""
    a = np.ascontiguousarray(arr)
    _check(lib().heom_ckpt_write(os.fsencode(path), a.ctypes.data_as(_P), a.nbytes))


def heom_ckpt_read(path, out):
    """Fill the contiguous numpy array ``out`` from a checkpoint file (integrity checked)."""
    if not out.flags["C_CONTIGUOUS"]:
        raise ValueError("out must be C-contiguous")
    _check(lib().heom_ckpt_read(os.fsencode(path), out.ctypes.data_as(_P), out.nbytes))
    return out


def heom_ckpt_verify(path):
    """Payload size of an intact checkpoint file (raises HeomError otherwise)."""
    n = ct.c_uint64(0)
    _check(lib().heom_ckpt_verify(os.fsencode(path), ct.byref(n)))
    return n.value


def heom_state_save(s, path):
    _check(lib().heom_state_save(s.h, os.fsencode(path)))


def heom_state_load(s, path):
    _check(lib().heom_state_load(s.h, os.fsencode(path)))


def heom_set_wait_limit_ns(h, ns):
    """Time limit (ns) of every device-side wait of h's tensor-core stage kernel."""
    _check(lib().heom_set_wait_limit_ns(h.h, int(ns)))


def heom_debug_fail_alloc(after):
    """Make device allocations fail after `after` more successes (after < 0: off)."""
    lib().heom_debug_fail_alloc(int(after))


def heom_source_tag():
    """SHA-256 tag (16 hex digits) of the tensor-core stage kernels' source the library was built from."""
    return lib().heom_source_tag().decode()


def heom_tc_shape_params(shape):
    """(rows per thread, row groups, ADOs per block, flags) of coupling-kernel shape `shape`."""
    r, g, a, f = ct.c_int(0), ct.c_int(0), ct.c_int(0), ct.c_int(0)
    _check(lib().heom_tc_shape_params(int(shape), ct.byref(r), ct.byref(g), ct.byref(a), ct.byref(f)))
    return r.value, g.value, a.value, f.value


def heom_tc_shape_count():
    """Number of coupling-kernel shapes of the tensor-core path (valid: 0 .. count - 1)."""
    return int(lib().heom_tc_shape_count())


def heom_debug_force_tc_shape(shape):
    """Force the tensor-core path's coupling-kernel shape (0-16), or -1 to tune again."""
    _check(lib().heom_debug_force_tc_shape(int(shape)))


def heom_get_tc_shape(h, elements):
    """(rows per thread, row groups, ADOs per block, flags) tuned for `elements`, or None;
    flags bit 0: bulk L2 prefetch, bit 1: two neighbour sources in flight per thread."""
    r, g, a, p = ct.c_int(0), ct.c_int(0), ct.c_int(0), ct.c_int(0)
    if lib().heom_get_tc_shape(h.h, int(elements), ct.byref(r), ct.byref(g), ct.byref(a), ct.byref(p)) != 1:
        return None
    return r.value, g.value, a.value, p.value


def heom_launch_count():
    return int(lib().heom_launch_count())


def heom_last_error():
    return lib().heom_last_error().decode()


def spectrum_2d(model, grid, precision=FP64):
    """Whole 2D procedure through the C ABI: build, equilibrate, R_I/R_II, S_C."""
    h = heom_build_hierarchy(model, precision)
    eq = heom_equilibrate(h, grid["dt_fs"], grid["t_eq_fs"], 0.0)
    RI, RII, SC = heom_response_2d(h, eq, grid)
    return h, eq, RI, RII, SC
