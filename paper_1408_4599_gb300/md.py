"""ctypes binding of the C ABI in ``include/md.h`` (libmdgpu.so).

Argument marshalling only: every step of the method runs in the CUDA
kernels behind the ABI.  Loading fails loudly when the library is missing;
there is no CPU fallback.  Arrays may be numpy arrays (host) or torch
tensors (host or CUDA); CUDA streams are passed as torch streams or raw
``cudaStream_t`` integers.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmdgpu.so")

MD_OK = 0
STATUS = {0: "MD_OK", -1: "MD_ERR_ARG", -2: "MD_ERR_BOX", -3: "MD_ERR_STATE", -4: "MD_ERR_CUDA", -5: "MD_ERR_OOM",
          -6: "MD_ERR_NONFINITE", -7: "MD_ERR_OVERFLOW", -8: "MD_ERR_TIMEOUT", -9: "MD_ERR_UNSUPPORTED"}
KERNEL_KINDS = ("integrate", "bin", "pack", "force", "kinetic", "batch", "adjoint", "other")

dp = C.POINTER(C.c_double)
ip = C.POINTER(C.c_int32)


class md_component(C.Structure):
    _fields_ = [("n_lj", C.c_int32), ("lj_pos", dp), ("lj_type", ip), ("lj_mass", dp),
                ("n_chg", C.c_int32), ("chg_pos", dp), ("chg_q", dp),
                ("n_dip", C.c_int32), ("dip_pos", dp), ("dip_axis", dp), ("dip_mu", dp),
                ("n_quad", C.c_int32), ("quad_pos", dp), ("quad_axis", dp), ("quad_Q", dp)]


class md_site_types(C.Structure):
    _fields_ = [("n_types", C.c_int32), ("eps", dp), ("sigma", dp), ("xi", dp), ("eta", dp),
                ("n_comp", C.c_int32), ("comp", C.POINTER(md_component))]


class md_options(C.Structure):
    _fields_ = [("eps_rf", C.c_double), ("lj_shift", C.c_int32), ("lj_lrc", C.c_int32),
                ("deterministic", C.c_int32), ("half_shell", C.c_int32), ("cell_div", C.c_int32)]


class md_observables(C.Structure):
    _fields_ = [("U_pot", C.c_double), ("U_lrc", C.c_double), ("U_rf_self", C.c_double),
                ("K_trans", C.c_double), ("K_rot", C.c_double), ("W", C.c_double), ("W_lrc", C.c_double),
                ("W_xx", C.c_double), ("W_yy", C.c_double), ("W_zz", C.c_double), ("T", C.c_double),
                ("P", C.c_double), ("time", C.c_double), ("step", C.c_int64), ("n_mol_pairs", C.c_int64),
                ("n_site_pairs", C.c_int64), ("n_examined", C.c_int64), ("n_molecules", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class md_batch_tuning(C.Structure):
    _fields_ = [("chunk", C.c_int32), ("grid_pct", C.c_int32), ("test_width", C.c_int32),
                ("half_min_occ", C.c_double), ("ms", C.c_float), ("default_ms", C.c_float),
                ("from_cache", C.c_int32), ("key", C.c_char * 160)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["key"] = self.key.decode()
        return d


class md_kernel_times(C.Structure):
    _fields_ = [("launches", C.c_int64 * 8), ("ms", C.c_double * 8)]

    def as_dict(self):
        return {k: {"launches": int(self.launches[i]), "ms": float(self.ms[i])} for i, k in enumerate(KERNEL_KINDS)}


_lib = None

# Every symbol include/md.h declares (checked by the CPU test suite).
EXPORTS = ("md_create", "md_set_molecules", "md_compute_forces", "md_step", "md_energy_virial",
           "md_get_molecules", "md_get_forces", "md_n_molecules", "md_sync", "md_profile", "md_kernel_times_get",
           "md_destroy", "md_status_str", "md_last_error", "md_n_params", "md_get_params", "md_set_params",
           "md_param_grad", "md_batch_create", "md_batch_set_molecules", "md_batch_compute_forces", "md_batch_step",
           "md_batch_energy_virial", "md_batch_get_molecules", "md_batch_get_forces", "md_batch_tune",
           "md_batch_destroy", "md_batch_last_error", "md_batch_set_thermostat", "md_kinetic_noalloc",
           "md_fp32_peak", "md_batch_tune_tiles")


def lib():
    """The loaded libmdgpu.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() (no CPU fallback exists)")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        i32, i64 = C.c_int32, C.c_int64
        L.md_create.argtypes = [dp, C.c_double, C.POINTER(md_site_types), C.POINTER(md_options), C.POINTER(vp)]
        L.md_set_molecules.argtypes = [vp, i64, ip, vp, vp, vp, vp, i32, vp]
        L.md_compute_forces.argtypes = [vp, vp]
        L.md_step.argtypes = [vp, i32, C.c_double, C.c_double, vp]
        L.md_energy_virial.argtypes = [vp, C.POINTER(md_observables)]
        L.md_get_molecules.argtypes = [vp, vp, vp, vp, vp, i32, vp]
        L.md_get_forces.argtypes = [vp, vp, vp, i32, vp]
        L.md_n_molecules.argtypes = [vp]
        L.md_n_molecules.restype = i64
        L.md_sync.argtypes = [vp, vp]
        L.md_profile.argtypes = [vp, i32]
        L.md_kernel_times_get.argtypes = [vp, C.POINTER(md_kernel_times)]
        L.md_n_params.argtypes = [vp]
        L.md_n_params.restype = i32
        L.md_get_params.argtypes = [vp, dp]
        L.md_set_params.argtypes = [vp, dp, i32]
        L.md_param_grad.argtypes = [vp, i32, i64, vp, vp, i32, dp, dp, dp, vp]
        L.md_batch_create.argtypes = [i32, dp, C.c_double, C.POINTER(md_site_types), C.POINTER(md_options),
                                      C.POINTER(vp)]
        L.md_batch_set_molecules.argtypes = [vp, C.POINTER(i64), vp, vp, vp, vp, i32, vp]
        L.md_batch_compute_forces.argtypes = [vp, vp]
        L.md_batch_step.argtypes = [vp, i32, C.c_double, i32, vp]
        L.md_batch_energy_virial.argtypes = [vp, C.POINTER(md_observables), vp]
        L.md_batch_get_molecules.argtypes = [vp, vp, vp, vp, vp, i32, vp]
        L.md_batch_get_forces.argtypes = [vp, vp, vp, i32, vp]
        L.md_batch_tune.argtypes = [vp, vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(C.c_float)]
        L.md_batch_set_thermostat.argtypes = [vp, dp, vp]
        L.md_batch_tune_tiles.argtypes = [vp, vp, C.c_char_p, C.POINTER(md_batch_tuning)]
        L.md_batch_destroy.argtypes = [vp]
        L.md_batch_destroy.restype = None
        L.md_batch_last_error.argtypes = [vp]
        L.md_batch_last_error.restype = C.c_char_p
        for name in ("md_batch_create", "md_batch_set_molecules", "md_batch_compute_forces", "md_batch_step",
                     "md_batch_energy_virial", "md_batch_get_molecules", "md_batch_get_forces", "md_batch_tune",
                     "md_batch_set_thermostat", "md_batch_tune_tiles"):
            getattr(L, name).restype = C.c_int
        L.md_kinetic_noalloc.argtypes = [i64, vp, vp, vp, vp, vp, C.c_double, dp, C.c_double, vp, vp]
        L.md_kinetic_noalloc.restype = C.c_int
        L.md_fp32_peak.argtypes = [i32, dp, vp]
        L.md_fp32_peak.restype = C.c_int
        L.md_destroy.argtypes = [vp]
        L.md_destroy.restype = None
        L.md_status_str.argtypes = [C.c_int]
        L.md_status_str.restype = C.c_char_p
        L.md_last_error.argtypes = [vp]
        L.md_last_error.restype = C.c_char_p
        for name in ("md_create", "md_set_molecules", "md_compute_forces", "md_step", "md_energy_virial",
                     "md_get_molecules", "md_get_forces", "md_sync", "md_profile", "md_kernel_times_get",
                     "md_get_params", "md_set_params", "md_param_grad"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


class MDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def _check(code, handle=None):
    if code != MD_OK:
        msg = lib().md_last_error(handle).decode() if handle else lib().md_status_str(code).decode()
        raise MDError(code, msg)


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return C.c_void_p(0)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(a, out=False):
    """(pointer, on_device, keepalive) of a numpy array or torch tensor (FP64,
    contiguous).  A host input of another dtype or layout is passed as a
    converted copy; an output (out=True) must already be a writable
    C-contiguous float64 array, since the library writes through the pointer
    and a copy would silently drop the result."""
    if a is None:
        return None, 0, None
    if isinstance(a, np.ndarray):
        if out:
            if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or not a.flags["WRITEABLE"]:
                raise ValueError("output arrays passed to the MD ABI must be writable C-contiguous float64")
        else:
            a = np.ascontiguousarray(a, dtype=np.float64)
        return C.c_void_p(a.ctypes.data), 0, a
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("tensors passed to the MD ABI must be contiguous float64")
        return C.c_void_p(a.data_ptr()), int(a.is_cuda), a
    raise TypeError(f"unsupported array type {type(a)}")


def _side(entries):
    """The on_device flag shared by every given (pointer, on_device, keep)
    entry of _ptr.  The library takes one flag per call for all of its
    pointers, so host arrays mixed with CUDA tensors are refused (a host
    pointer would be handed to a kernel as a device address), and so are
    CUDA tensors on a device other than the current one (the library
    launches on the current device)."""
    live = [e for e in entries if e[0] is not None]
    sides = {e[1] for e in live}
    if len(sides) > 1:
        raise ValueError("all arrays of one call must live on the same side (host or device)")
    dev = sides.pop() if sides else 0
    if dev:
        import torch
        cur = torch.cuda.current_device()
        for e in live:
            if e[2].device.index != cur:
                raise ValueError(f"CUDA tensor on {e[2].device}, but the current device is cuda:{cur}")
    return dev


def _need_rows(n, w, **arrays):
    """Every given array (numpy or torch) must have shape (n, w): the library
    reads or writes exactly n rows of w doubles through each pointer."""
    for name, a in arrays.items():
        if a is not None and tuple(a.shape) != (n, w):
            raise ValueError(f"{name} has shape {tuple(a.shape)}, expected ({n}, {w})")


class Model:
    """C structs (md_site_types + md_component) for an mdgen model dict; the
    numpy buffers are kept alive as long as this object."""

    def __init__(self, md: dict):
        self._keep = []
        t = md_site_types()
        eps = self._arr(md["lj_types"]["eps"])
        sig = self._arr(md["lj_types"]["sigma"])
        T = len(md["lj_types"]["eps"])
        t.n_types = T
        t.eps, t.sigma = eps, sig
        t.xi = self._arr(np.asarray(md["xi"], float).ravel()) if md.get("xi") is not None else None
        t.eta = self._arr(np.asarray(md["eta"], float).ravel()) if md.get("eta") is not None else None
        c = md_component()
        lj = md["lj"]
        c.n_lj = len(lj)
        c.lj_pos = self._arr([x for s in lj for x in s["pos"]])
        c.lj_type = self._iarr([s["type"] for s in lj])
        c.lj_mass = self._arr([s["mass"] for s in lj])
        ch = md["charges"]
        c.n_chg = len(ch)
        c.chg_pos = self._arr([x for s in ch for x in s["pos"]])
        c.chg_q = self._arr([s["q"] for s in ch])
        dd = md["dipoles"]
        c.n_dip = len(dd)
        c.dip_pos = self._arr([x for s in dd for x in s["pos"]])
        c.dip_axis = self._arr([x for s in dd for x in s["axis"]])
        c.dip_mu = self._arr([s["mu"] for s in dd])
        qq = md["quads"]
        c.n_quad = len(qq)
        c.quad_pos = self._arr([x for s in qq for x in s["pos"]])
        c.quad_axis = self._arr([x for s in qq for x in s["axis"]])
        c.quad_Q = self._arr([s["Q"] for s in qq])
        self.comp = (md_component * 1)(c)
        t.n_comp = 1
        t.comp = self.comp
        self.types = t

    def _arr(self, v):
        a = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
        if a.size == 0:
            a = np.zeros(1)
        self._keep.append(a)
        return a.ctypes.data_as(dp)

    def _iarr(self, v):
        a = np.ascontiguousarray(np.asarray(v, dtype=np.int32))
        if a.size == 0:
            a = np.zeros(1, dtype=np.int32)
        self._keep.append(a)
        return a.ctypes.data_as(ip)


# ------------------------------------------------------- C-ABI functions
def md_create(box, cutoff, model: dict, eps_rf=math.inf, lj_shift=0, lj_lrc=0, deterministic=1, half_shell=0,
              cell_div=1):
    """Returns (handle, Model) -- keep the Model alive with the handle."""
    M = Model(model)
    b = (C.c_double * 3)(*[float(x) for x in box])
    o = md_options(float(eps_rf), int(lj_shift), int(lj_lrc), int(deterministic), int(half_shell), int(cell_div))
    h = C.c_void_p()
    _check(lib().md_create(b, float(cutoff), C.byref(M.types), C.byref(o), C.byref(h)))
    return h, M


def md_set_molecules(h, r, q, v=None, j=None, stream=None):
    rp, dev, k1 = _ptr(r)
    qp, dq, k2 = _ptr(q)
    vp, dv, k3 = _ptr(v)
    jp, dj, k4 = _ptr(j)
    dev = _side([(rp, dev, k1), (qp, dq, k2), (vp, dv, k3), (jp, dj, k4)])
    n = (k1.shape[0] if k1 is not None else 0)
    _need_rows(n, 3, r=k1, v=k3, j=k4)
    _need_rows(n, 4, q=k2)
    _check(lib().md_set_molecules(h, n, None, rp, vp, qp, jp, dev, _stream_ptr(stream)), h)


def md_compute_forces(h, stream=None):
    _check(lib().md_compute_forces(h, _stream_ptr(stream)), h)


def md_step(h, n_steps, dt, T_target=0.0, stream=None):
    _check(lib().md_step(h, int(n_steps), float(dt), float(T_target), _stream_ptr(stream)), h)


def md_energy_virial(h) -> dict:
    o = md_observables()
    _check(lib().md_energy_virial(h, C.byref(o)), h)
    return o.as_dict()


def md_get_molecules(h, r=None, v=None, q=None, j=None, stream=None):
    """Fills the given arrays (host numpy or device tensors); with no
    arrays given, returns host numpy copies of r, v, q, j."""
    if r is None and v is None and q is None and j is None:
        n = lib().md_n_molecules(h)
        r, v, q, j = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 4)), np.zeros((n, 3))
    ptrs = [_ptr(a, out=True) for a in (r, v, q, j)]
    dev = _side(ptrs)
    n = lib().md_n_molecules(h)
    _need_rows(n, 3, r=r, v=v, j=j)
    _need_rows(n, 4, q=q)
    _check(lib().md_get_molecules(h, *[p[0] for p in ptrs], dev, _stream_ptr(stream)), h)
    return r, v, q, j


def md_get_forces(h, F=None, tau=None, stream=None):
    if F is None and tau is None:
        n = lib().md_n_molecules(h)
        F, tau = np.zeros((n, 3)), np.zeros((n, 3))
    pf, pt = _ptr(F, out=True), _ptr(tau, out=True)
    dev = _side([pf, pt])
    _need_rows(lib().md_n_molecules(h), 3, F=F, tau=tau)
    _check(lib().md_get_forces(h, pf[0], pt[0], dev, _stream_ptr(stream)), h)
    return F, tau


def md_sync(h, stream=None):
    _check(lib().md_sync(h, _stream_ptr(stream)), h)


def md_profile(h, enable=True):
    _check(lib().md_profile(h, int(enable)), h)


def md_kernel_times_get(h) -> dict:
    t = md_kernel_times()
    _check(lib().md_kernel_times_get(h, C.byref(t)), h)
    return t.as_dict()


def md_n_params(h) -> int:
    return int(lib().md_n_params(h))


def md_get_params(h) -> np.ndarray:
    th = np.zeros(md_n_params(h))
    _check(lib().md_get_params(h, th.ctypes.data_as(dp)), h)
    return th


def md_set_params(h, theta):
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
    _check(lib().md_set_params(h, th.ctypes.data_as(dp), int(th.shape[0])), h)


def md_param_grad(h, r_all, q_all, stream=None):
    """(dU/dtheta, dW/dtheta, <U>, <W>) over the configurations r_all
    (n_cfg x n x 3) and q_all (n_cfg x n x 4), host arrays or device tensors."""
    rp, dev, rk = _ptr(r_all)
    qp, dq, qk = _ptr(q_all)
    dev = _side([(rp, dev, rk), (qp, dq, qk)])
    if len(rk.shape) != 3 or rk.shape[2] != 3 or tuple(qk.shape) != (rk.shape[0], rk.shape[1], 4):
        raise ValueError(f"r_all {tuple(rk.shape)} and q_all {tuple(qk.shape)} must be n_cfg x n x 3 and x 4")
    n_cfg, n = int(rk.shape[0]), int(rk.shape[1])
    P = md_n_params(h)
    dU, dW, means = np.zeros(P), np.zeros(P), np.zeros(2)
    _check(lib().md_param_grad(h, n_cfg, n, rp, qp, dev, dU.ctypes.data_as(dp), dW.ctypes.data_as(dp),
                               means.ctypes.data_as(dp), _stream_ptr(stream)), h)
    return dU, dW, float(means[0]), float(means[1])


def md_kinetic_noalloc(v, q, j, F, tau, mass, moments, dt, K_out, stream=None):
    """K_out (device float64 tensor of 2) <- (K_trans, K_rot); allocates nothing."""
    ptrs = [_ptr(a) for a in (v, q, j, F, tau)] + [_ptr(K_out, out=True)]
    if min(p[1] for p in ptrs) != 1:
        raise ValueError("md_kinetic_noalloc takes device tensors only")
    _side(ptrs)  # one device, the current one (the file-scope scratch is per device)
    I = (C.c_double * 3)(*[float(x) for x in moments])
    n = ptrs[0][2].shape[0]
    _need_rows(n, 3, v=v, j=j, F=F, tau=tau)
    _need_rows(n, 4, q=q)
    if K_out.numel() < 2:
        raise ValueError("K_out must hold 2 doubles")
    _check(lib().md_kinetic_noalloc(n, *[p[0] for p in ptrs[:5]], float(mass), I, float(dt), ptrs[5][0],
                                    _stream_ptr(stream)))


def md_fp32_peak(paired=False, stream=None):
    """(FLOP/s, ms) of the FMA-chain peak kernel: scalar FMA, or with paired
    the two-wide fma.rn.f32x2."""
    out = np.zeros(2)
    _check(lib().md_fp32_peak(int(bool(paired)), out.ctypes.data_as(dp), _stream_ptr(stream)))
    return float(out[0]), float(out[1])


def md_destroy(h):
    if h:
        lib().md_destroy(h)


class System:
    """Owning wrapper: one md_system handle plus its model structs."""

    def __init__(self, cfg: dict, deterministic=1, half_shell=0, cell_div=1):
        self.cfg = cfg
        self.h, self._model = md_create(cfg["box"], cfg["rc"], cfg["model"], cfg.get("eps_rf", math.inf),
                                        cfg.get("lj_shift", 0), cfg.get("lj_lrc", 0), deterministic, half_shell,
                                        cell_div)

    def set(self, r, q, v=None, j=None, stream=None):
        md_set_molecules(self.h, r, q, v, j, stream)
        return self

    def compute_forces(self, stream=None):
        md_compute_forces(self.h, stream)

    def step(self, n_steps, dt, T_target=0.0, stream=None):
        md_step(self.h, n_steps, dt, T_target, stream)

    def observables(self):
        return md_energy_virial(self.h)

    def molecules(self, **kw):
        return md_get_molecules(self.h, **kw)

    def forces(self, **kw):
        return md_get_forces(self.h, **kw)

    def params(self):
        return md_get_params(self.h)

    def set_params(self, theta):
        md_set_params(self.h, theta)

    def param_grad(self, r_all, q_all, stream=None):
        return md_param_grad(self.h, r_all, q_all, stream)

    def close(self):
        if self.h:
            md_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _bcheck(code, handle):
    if code != MD_OK:
        raise MDError(code, lib().md_batch_last_error(handle).decode() if handle else lib().md_status_str(code).decode())


class Batch:
    """Owning wrapper of an md_batch: replicas of one model (cfgs share the
    model dict, the cut-off and the options)."""

    def __init__(self, cfgs, half_shell=1):
        c0 = cfgs[0]
        self.cfgs = cfgs
        self._model = Model(c0["model"])
        boxes = np.ascontiguousarray(np.array([c["box"] for c in cfgs], dtype=np.float64))
        o = md_options(float(c0.get("eps_rf", math.inf)), int(c0.get("lj_shift", 0)), int(c0.get("lj_lrc", 0)), 0,
                       int(half_shell))
        h = C.c_void_p()
        _check(lib().md_batch_create(len(cfgs), boxes.ctypes.data_as(dp), float(c0["rc"]), C.byref(self._model.types),
                                     C.byref(o), C.byref(h)))
        self.h = h
        self.n_per = np.array([c["r"].shape[0] for c in cfgs], dtype=np.int64)

    def set(self, r=None, q=None, v=None, j=None, stream=None):
        """Concatenated state; by default the cfgs' own r, q, v, j."""
        if r is None:
            r = np.concatenate([c["r"] for c in self.cfgs])
            q = np.concatenate([c["q"] for c in self.cfgs])
            v = np.concatenate([c["v"] for c in self.cfgs])
            j = np.concatenate([c["j"] for c in self.cfgs])
        ptrs = [_ptr(a) for a in (r, v, q, j)]
        nt = int(self.n_per.sum())
        _need_rows(nt, 3, r=ptrs[0][2], v=ptrs[1][2], j=ptrs[3][2])
        _need_rows(nt, 4, q=ptrs[2][2])
        dev = _side(ptrs)
        n = self.n_per.ctypes.data_as(C.POINTER(C.c_int64))
        _bcheck(lib().md_batch_set_molecules(self.h, n, ptrs[0][0], ptrs[1][0], ptrs[2][0], ptrs[3][0], dev,
                                             _stream_ptr(stream)), self.h)
        return self

    def compute_forces(self, stream=None):
        _bcheck(lib().md_batch_compute_forces(self.h, _stream_ptr(stream)), self.h)

    def step(self, n_steps, dt, use_graph=True, stream=None):
        _bcheck(lib().md_batch_step(self.h, int(n_steps), float(dt), int(bool(use_graph)), _stream_ptr(stream)),
                self.h)

    def observables(self, stream=None):
        out = (md_observables * len(self.cfgs))()
        _bcheck(lib().md_batch_energy_virial(self.h, out, _stream_ptr(stream)), self.h)
        return [o.as_dict() for o in out]

    def molecules(self, stream=None):
        n = int(self.n_per.sum())
        r, v, q, j = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 4)), np.zeros((n, 3))
        ptrs = [_ptr(a) for a in (r, v, q, j)]
        _bcheck(lib().md_batch_get_molecules(self.h, *[p[0] for p in ptrs], 0, _stream_ptr(stream)), self.h)
        return r, v, q, j

    def forces(self, stream=None):
        n = int(self.n_per.sum())
        F, tau = np.zeros((n, 3)), np.zeros((n, 3))
        _bcheck(lib().md_batch_get_forces(self.h, _ptr(F)[0], _ptr(tau)[0], 0, _stream_ptr(stream)), self.h)
        return F, tau

    def set_thermostat(self, T_target=None, stream=None):
        """Per-replica NVT targets (sequence of n_sys; <= 0 or None: NVE)."""
        if T_target is None:
            _bcheck(lib().md_batch_set_thermostat(self.h, None, _stream_ptr(stream)), self.h)
            return
        t = np.ascontiguousarray(np.asarray(T_target, dtype=np.float64))
        if t.shape != (len(self.cfgs),):
            raise ValueError("one target per replica")
        _bcheck(lib().md_batch_set_thermostat(self.h, t.ctypes.data_as(dp), _stream_ptr(stream)), self.h)

    def tune(self, stream=None):
        bc, bg, bm = C.c_int32(), C.c_int32(), C.c_float()
        _bcheck(lib().md_batch_tune(self.h, _stream_ptr(stream), C.byref(bc), C.byref(bg), C.byref(bm)), self.h)
        return {"chunk": bc.value, "grid_pct": bg.value, "force_ms": bm.value}

    def tune_tiles(self, cache_path=None, stream=None):
        """Tile autotuner (md_batch_tune_tiles); cache_path: optional text
        file of earlier choices.  Returns the md_batch_tuning as a dict."""
        t = md_batch_tuning()
        p = cache_path.encode() if cache_path else None
        _bcheck(lib().md_batch_tune_tiles(self.h, _stream_ptr(stream), p, C.byref(t)), self.h)
        return t.as_dict()

    def close(self):
        if self.h:
            lib().md_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
