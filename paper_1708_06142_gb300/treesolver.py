"""Thin ctypes binding of libtreesolver.so (the C ABI in include/treesolver.h).

Argument marshalling only: every step of the method runs in the library's CUDA kernels.  Device
buffers are torch CUDA tensors (PyTorch provides memory and streams); the library never sees a torch
type, only raw pointers.  There is no CPU fallback: if the shared library is missing this module
raises at import of the library.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

NB = 8
NCB = 512

TS_OK = 0
STATUS_NAMES = {0: "TS_OK", 1: "TS_ERR_INVALID_ARG", 2: "TS_ERR_UNSUPPORTED", 3: "TS_ERR_OUT_OF_MEMORY",
                4: "TS_ERR_CUDA", 5: "TS_ERR_NOT_BUILT", 6: "TS_ERR_STACK_OVERFLOW", 7: "TS_ERR_TIMEOUT",
                8: "TS_ERR_NUMERIC"}
TS_MAC_BH, TS_MAC_APE, TS_MAC_MPE, TS_MAC_SUMSQ = 0, 1, 2, 3
TS_PREC_FP64, TS_PREC_FP32_KAHAN = 0, 1


class TSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class TSMesh(C.Structure):
    _fields_ = [("nblocks", C.c_int32), ("level", C.c_void_p), ("child", C.c_void_p), ("lo", C.c_void_p),
                ("size", C.c_void_p), ("bc", C.c_int32 * 3)]


class TSGravityParams(C.Structure):
    _fields_ = [("mac", C.c_int32), ("theta", C.c_double), ("safe_box", C.c_double), ("a_lim", C.c_double),
                ("a_old_dev", C.c_void_p), ("eps_rel", C.c_double), ("G", C.c_double),
                ("precision", C.c_int32), ("ewald", C.c_int32), ("zero_mean", C.c_int32), ("accel", C.c_int32),
                ("queue_max", C.c_int32)]


class TSShieldParams(C.Structure):
    _fields_ = [("k_av", C.c_double), ("k_h2", C.c_double), ("b5", C.c_double), ("k_co", C.c_double),
                ("co_n_co", C.c_int32), ("co_n_h2", C.c_int32), ("co_table", C.c_void_p),
                ("co_lg_co", C.c_double * 2), ("co_lg_h2", C.c_double * 2)]


class TSSurrogateParams(C.Structure):
    _fields_ = [("b_min", C.c_double), ("b_max", C.c_double), ("n_samples", C.c_int64), ("steps", C.c_int32),
                ("batch", C.c_int32), ("lr", C.c_double), ("seed", C.c_uint64), ("z_power", C.c_double)]


class TSErrorStats(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_nonfinite", C.c_int64), ("a_ref_max", C.c_double), ("phi_ref_max", C.c_double),
                ("e_a_median", C.c_double), ("e_a_p99", C.c_double), ("e_a_max", C.c_double),
                ("e_phi_median", C.c_double), ("e_phi_p99", C.c_double), ("e_phi_max", C.c_double)]


class TSColumnParams(C.Structure):
    _fields_ = [("n_side", C.c_int32), ("theta", C.c_double), ("safe_box", C.c_double), ("max_dist", C.c_double),
                ("table_ntheta", C.c_int32), ("table_nphi", C.c_int32), ("table_npsi", C.c_int32),
                ("table_nsub", C.c_int32), ("table_psi_min", C.c_double), ("table_psi_max", C.c_double)]


# every symbol the header declares, with (restype, argtypes)
_P = C.c_void_p
SIGNATURES = {
    "ts_create": (C.c_int, [C.POINTER(_P), C.c_int, _P]),
    "ts_destroy": (C.c_int, [_P]),
    "ts_last_error": (C.c_char_p, []),
    "ts_tree_build": (C.c_int, [_P, C.POINTER(TSMesh), _P]),
    "ts_tree_fp64_records": (C.c_int, [_P, C.c_int32]),
    "ts_mesh_info": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "ts_block_moments": (C.c_int, [_P, _P, _P]),
    "ts_ewald_field": (C.c_int, [_P, C.c_int32, C.c_char_p]),
    "ts_ewald_table_get": (C.c_int, [_P, C.POINTER(C.c_int32), _P, _P]),
    "ts_ewald_taylor_get": (C.c_int, [_P, _P, _P]),
    "ts_gravity_params_default": (None, [C.POINTER(TSGravityParams)]),
    "ts_gravity_walk": (C.c_int, [_P, C.POINTER(TSGravityParams), _P, _P]),
    "ts_column_params_default": (None, [C.POINTER(TSColumnParams)]),
    "ts_column_walk": (C.c_int, [_P, C.POINTER(TSColumnParams), _P]),
    "ts_noderay_table_get": (C.c_int, [_P, _P, _P]),
    "ts_column_av": (C.c_int, [_P, C.c_int64, C.c_int32, _P, C.c_double, _P]),
    "ts_column_quantities": (C.c_int, [_P, C.c_int32, _P]),
    "ts_column_shielding": (C.c_int, [_P, C.c_int64, C.c_int32, _P, _P, _P]),
    "ts_sync": (C.c_int, [_P]),
    "ts_stats": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "ts_surrogate_train": (C.c_int, [_P, _P, C.POINTER(C.c_double)]),
    "ts_surrogate_get": (C.c_int, [_P, _P, _P, _P]),
    "ts_surrogate_set": (C.c_int, [_P, _P, _P, _P]),
    "ts_gravity_walk_range": (C.c_int, [_P, _P, C.c_int32, C.c_int32, _P, _P]),
    "ts_walk_block_counts": (C.c_int, [_P, _P]),
    "ts_potential_sums": (C.c_int, [_P, C.c_int32, _P, C.c_int32, C.c_int32, _P]),
    "ts_potential_shift": (C.c_int, [_P, C.c_int32, _P, C.c_int32, C.c_int32, C.c_double]),
    "ts_surrogate_save": (C.c_int, [_P, C.c_char_p]),
    "ts_surrogate_load": (C.c_int, [_P, C.c_char_p]),
    "ts_surrogate_eval": (C.c_int, [_P, C.c_int64, _P, _P]),
    "ts_surrogate_grad": (C.c_int, [_P, C.c_int64, _P, _P, _P, C.POINTER(C.c_double)]),
    "ts_batch_create": (C.c_int, [C.POINTER(_P), _P, C.c_int32]),
    "ts_batch_destroy": (C.c_int, [_P]),
    "ts_batch_run": (C.c_int, [_P, C.POINTER(TSGravityParams), _P, _P, C.POINTER(TSColumnParams), _P, _P, C.c_int32]),
    "ts_batch_set_tuning": (C.c_int, [_P, C.c_int32, C.c_int32]),
    "ts_batch_set_mode": (C.c_int, [_P, C.c_int32, C.c_int32]),
    "ts_batch_sync": (C.c_int, [_P, _P, C.POINTER(C.c_double)]),
    "ts_autotune_walk": (C.c_int, [_P, C.POINTER(TSGravityParams), _P, _P, C.POINTER(C.c_int32), _P]),
    "ts_zero_mean_noalloc": (C.c_int, [C.c_int32, _P, _P, C.c_int64, _P]),
    "ts_walk_counters": (C.c_int, [_P, _P]),
    "ts_set_walk_grouping": (C.c_int, [_P, C.c_int32, C.c_int32]),
    "ts_error_metrics": (C.c_int, [_P, C.c_int32, C.c_int64, _P, _P, _P, _P, C.c_int32, _P, _P]),
    "ts_peak_probe": (C.c_int, [C.c_int32, C.c_int32, _P]),
    "ts_gravity_walk_abu": (C.c_int, [_P, _P, C.c_double, C.c_double, _P, _P, _P]),
    "ts_block_workload": (C.c_int, [_P, _P]),
    "ts_version": (C.c_char_p, []),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(f"libtreesolver.so not built ({path}); run __graft_entry__.build()")
    L = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(st):
    if st != TS_OK:
        raise TSError(st, _lib.ts_last_error().decode())


def _dptr(t, dtype=None, numel=None, name="buffer"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


class TreeSolver:
    """One library context: one mesh, its tree, Ewald and node-ray tables, on one device/stream."""

    def __init__(self, device: int = 0, stream=None):
        load()
        self._ctx = C.c_void_p()
        s = C.c_void_p(stream.cuda_stream) if stream is not None else None
        _check(_lib.ts_create(C.byref(self._ctx), device, s))
        self.device = device
        self.stream = stream
        self.ncell = 0
        self._mesh_keep = None

    def close(self):
        if self._ctx:
            _lib.ts_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def make_mesh(mesh):
        level = np.ascontiguousarray(mesh.level, dtype=np.int32)
        child = np.ascontiguousarray(mesh.child, dtype=np.int32)
        lo = np.ascontiguousarray(mesh.lo, dtype=np.float64)
        size = np.ascontiguousarray(mesh.size, dtype=np.float64)
        m = TSMesh(mesh.nblocks, level.ctypes.data, child.ctypes.data, lo.ctypes.data, size.ctypes.data,
                   (C.c_int32 * 3)(*mesh.bc))
        return m, (level, child, lo, size)

    def tree_build(self, mesh, density):
        """mesh: inputs.Mesh or None (keep the previous mesh); density: CUDA float64 [ncell]."""
        import torch
        if mesh is not None:
            m, keep = self.make_mesh(mesh)
            _check(_lib.ts_tree_build(self._ctx, C.byref(m), _dptr(density, torch.float64, mesh.ncell, "density")))
            self._mesh_keep = keep
            self.ncell = mesh.ncell
        else:
            _check(_lib.ts_tree_build(self._ctx, None, _dptr(density, torch.float64, self.ncell, "density")))
        self.lq = 1

    def fp64_records(self, enabled: bool):
        """Whether later tree builds write the FP64 records that only FP64 walks read."""
        _check(_lib.ts_tree_fp64_records(self._ctx, 1 if enabled else 0))

    def column_quantities(self, q):
        """Extra mapped quantities for the current tree: q a CUDA float64 [nq, ncell] (nq <= 2) of
        densities, or None; later column walks write [ncell, 1 + nq, N_PIX]."""
        import torch
        if q is None:
            _check(_lib.ts_column_quantities(self._ctx, 0, None))
            self.lq = 1
            return
        nq = q.shape[0]
        _check(_lib.ts_column_quantities(self._ctx, nq, _dptr(q, torch.float64, nq * self.ncell, "quantities")))
        self.lq = 1 + nq

    def column_shielding(self, cols, out, k_av=1.0, k_h2=1.0, b5=3.0, k_co=1.0, co_table=None, lg_co=(0.0, 1.0),
                         lg_h2=(0.0, 1.0)):
        """(A_V, <f_H2>, <f_CO>) per cell from l_q = 3 maps cols [n, 3, npix] into out [n, 3]."""
        import torch
        n, lq, npix = cols.shape
        if lq != 3:
            raise ValueError("cols must hold the total, H2 and CO maps")
        p = TSShieldParams()
        p.k_av, p.k_h2, p.b5, p.k_co = k_av, k_h2, b5, k_co
        tab = None
        if co_table is not None:
            tab = np.ascontiguousarray(co_table, dtype=np.float64)
            p.co_n_co, p.co_n_h2 = tab.shape
            p.co_table = tab.ctypes.data
        p.co_lg_co[0], p.co_lg_co[1] = lg_co
        p.co_lg_h2[0], p.co_lg_h2[1] = lg_h2
        _check(_lib.ts_column_shielding(self._ctx, n, npix, _dptr(cols, torch.float32, n * 3 * npix, "columns"),
                                        C.byref(p), _dptr(out, torch.float32, 3 * n, "out")))

    def mesh_info(self):
        n, l, b = C.c_int64(), C.c_int32(), C.c_int32()
        _check(_lib.ts_mesh_info(self._ctx, C.byref(n), C.byref(l), C.byref(b)))
        return n.value, l.value, b.value

    def block_moments(self, nblocks):
        mass, com = np.zeros(nblocks), np.zeros((nblocks, 3))
        _check(_lib.ts_block_moments(self._ctx, mass.ctypes.data, com.ctypes.data))
        return mass, com

    def ewald_field(self, n: int = 64, cache_path: str | None = None):
        _check(_lib.ts_ewald_field(self._ctx, n, cache_path.encode() if cache_path else None))

    def ewald_table(self):
        n = C.c_int32()
        ext = np.zeros(3)
        _check(_lib.ts_ewald_table_get(self._ctx, C.byref(n), ext.ctypes.data, None))
        tab = np.zeros((n.value, n.value, n.value, 4))
        _check(_lib.ts_ewald_table_get(self._ctx, C.byref(n), ext.ctypes.data, tab.ctypes.data))
        return tab, ext

    @staticmethod
    def gravity_params(mac="bh", theta=0.5, safe_box=1.2, a_lim=0.0, a_old=None, eps_rel=0.0, G=1.0,
                       precision="fp32", zero_mean=False, ewald="table", accel="direct", queue_max=0):
        p = TSGravityParams()
        _lib.ts_gravity_params_default(C.byref(p))
        p.ewald = {"table": 0, "mlp": 1, "taylor": 2}[ewald]
        p.mac = {"bh": TS_MAC_BH, "ape": TS_MAC_APE, "mpe": TS_MAC_MPE, "sumsq": TS_MAC_SUMSQ}[mac]
        p.theta, p.safe_box, p.a_lim, p.eps_rel, p.G = theta, safe_box, a_lim, eps_rel, G
        p.a_old_dev = _dptr(a_old, name="a_old").value if a_old is not None else None
        p.precision = TS_PREC_FP64 if precision == "fp64" else TS_PREC_FP32_KAHAN
        p.zero_mean = int(bool(zero_mean))
        p.accel = {"direct": 0, "numdiff": 1}[accel]
        p.queue_max = int(queue_max)
        return p

    def gravity_walk(self, pot, acc, params: TSGravityParams | None = None, **kw):
        """pot: CUDA [ncell], acc: CUDA [ncell, 3]; float32 (fp32) or float64 (fp64)."""
        import torch
        p = params if params is not None else self.gravity_params(**kw)
        dt = torch.float64 if p.precision == TS_PREC_FP64 else torch.float32
        _check(_lib.ts_gravity_walk(self._ctx, C.byref(p), _dptr(pot, dt, self.ncell, "pot"),
                                    _dptr(acc, dt, 3 * self.ncell, "acc")))

    def gravity_walk_range(self, pot, acc, leaf_begin, leaf_end, params: TSGravityParams | None = None, **kw):
        """Walk of the cells of leaf-blocks [leaf_begin, leaf_end) into the full-size pot / acc."""
        import torch
        p = params if params is not None else self.gravity_params(**kw)
        dt = torch.float64 if p.precision == TS_PREC_FP64 else torch.float32
        _check(_lib.ts_gravity_walk_range(self._ctx, C.byref(p), int(leaf_begin), int(leaf_end),
                                          _dptr(pot, dt, self.ncell, "pot"), _dptr(acc, dt, 3 * self.ncell, "acc")))

    def walk_block_counts(self):
        """Interactions of every leaf-block in its latest range walk (int64 [nleaf])."""
        n = self.ncell // 512
        out = np.zeros(n, dtype=np.int64)
        _check(_lib.ts_walk_block_counts(self._ctx, out.ctypes.data))
        return out

    def potential_sums(self, pot, leaf_begin, leaf_end):
        """(sum dV phi, sum dV) in FP64 over the cells of the range."""
        import torch
        prec = TS_PREC_FP64 if pot.dtype == torch.float64 else TS_PREC_FP32_KAHAN
        out = np.zeros(2)
        _check(_lib.ts_potential_sums(self._ctx, prec, _dptr(pot, pot.dtype, self.ncell, "pot"), int(leaf_begin),
                                      int(leaf_end), out.ctypes.data))
        return out

    def potential_shift(self, pot, leaf_begin, leaf_end, shift):
        import torch
        prec = TS_PREC_FP64 if pot.dtype == torch.float64 else TS_PREC_FP32_KAHAN
        _check(_lib.ts_potential_shift(self._ctx, prec, _dptr(pot, pot.dtype, self.ncell, "pot"), int(leaf_begin),
                                       int(leaf_end), float(shift)))

    @staticmethod
    def column_params(n_side=2, theta=0.5, safe_box=1.2, max_dist=0.0, ntheta=0, nphi=0, npsi=0, nsub=0,
                      psi_min=0.0, psi_max=0.0):
        p = TSColumnParams()
        _lib.ts_column_params_default(C.byref(p))
        p.n_side, p.theta, p.safe_box, p.max_dist = n_side, theta, safe_box, max_dist
        p.table_ntheta, p.table_nphi, p.table_npsi, p.table_nsub = ntheta, nphi, npsi, nsub
        p.table_psi_min, p.table_psi_max = psi_min, psi_max
        return p

    def column_walk(self, cols, params: TSColumnParams | None = None, **kw):
        import torch
        p = params if params is not None else self.column_params(**kw)
        npix = 12 * p.n_side * p.n_side
        lq = getattr(self, "lq", 1)
        _check(_lib.ts_column_walk(self._ctx, C.byref(p), _dptr(cols, torch.float32, self.ncell * lq * npix, "columns")))

    def ewald_taylor_table(self):
        """FP64 first-order Taylor table [n, n, n, 10] = (C, A_c, Jxx, Jxy, Jxz, Jyy, Jyz, Jzz)."""
        n = C.c_int32()
        _check(_lib.ts_ewald_taylor_get(self._ctx, C.byref(n), None))
        t = np.zeros((n.value, n.value, n.value, 10))
        _check(_lib.ts_ewald_taylor_get(self._ctx, C.byref(n), t.ctypes.data))
        return t

    def column_av(self, cols, k=1.0, av=None):
        """Mean visual extinction per cell (eq. av) of a float32 CUDA column map [n, npix]; returns
        (or fills) a float32 CUDA tensor [n]."""
        import torch
        n, npix = cols.shape
        if av is None:
            av = torch.empty(n, dtype=torch.float32, device=cols.device)
        _check(_lib.ts_column_av(self._ctx, n, npix, _dptr(cols, torch.float32, n * npix, "columns"), float(k),
                                 _dptr(av, torch.float32, n, "av")))
        return av

    def noderay_table(self):
        dims = (C.c_int32 * 4)()
        _check(_lib.ts_noderay_table_get(self._ctx, dims, None))
        t = np.zeros(tuple(dims))
        _check(_lib.ts_noderay_table_get(self._ctx, dims, t.ctypes.data))
        return t

    # ---- learned Ewald correction (2P1I)
    def surrogate_train(self, b_min=0.5, b_max=2.0, n_samples=1 << 20, steps=1000000, batch=4096, lr=3e-3, seed=1,
                        z_power=2.0):
        p = TSSurrogateParams(b_min, b_max, n_samples, steps, batch, lr, seed, z_power)
        loss = C.c_double()
        _check(_lib.ts_surrogate_train(self._ctx, C.byref(p), C.byref(loss)))
        return loss.value

    def surrogate_get(self):
        params, norm, br = np.zeros(8900, dtype=np.float32), np.zeros(8, dtype=np.float32), np.zeros(2)
        _check(_lib.ts_surrogate_get(self._ctx, params.ctypes.data, norm.ctypes.data, br.ctypes.data))
        return params, norm, br

    def surrogate_set(self, params, norm, b_range):
        params = np.ascontiguousarray(params, dtype=np.float32)
        norm = np.ascontiguousarray(norm, dtype=np.float32)
        br = np.ascontiguousarray(b_range, dtype=np.float64)
        _check(_lib.ts_surrogate_set(self._ctx, params.ctypes.data, norm.ctypes.data, br.ctypes.data))

    def surrogate_save(self, path):
        """Write the trained network to a versioned file with a content hash."""
        _check(_lib.ts_surrogate_save(self._ctx, os.fsencode(path)))

    def surrogate_load(self, path):
        """Read a network written by surrogate_save (a damaged file raises TSError, status 1)."""
        _check(_lib.ts_surrogate_load(self._ctx, os.fsencode(path)))

    def surrogate_eval(self, feat, out):
        import torch
        n = feat.shape[0]
        _check(_lib.ts_surrogate_eval(self._ctx, n, _dptr(feat, torch.float32, 4 * n, "feat"),
                                      _dptr(out, torch.float32, 4 * n, "out")))

    def surrogate_grad(self, feat, targ):
        import torch
        n = feat.shape[0]
        g = np.zeros(8900, dtype=np.float32)
        loss = C.c_double()
        _check(_lib.ts_surrogate_grad(self._ctx, n, _dptr(feat, torch.float32, 4 * n, "feat"),
                                      _dptr(targ, torch.float32, 4 * n, "targ"), g.ctypes.data, C.byref(loss)))
        return loss.value, g

    def set_walk_grouping(self, precision="fp32", targets_per_lane=2):
        _check(_lib.ts_set_walk_grouping(self._ctx, TS_PREC_FP64 if precision == "fp64" else TS_PREC_FP32_KAHAN,
                                         targets_per_lane))

    def walk_counters(self):
        out = np.zeros(4, dtype=np.int64)
        _check(_lib.ts_walk_counters(self._ctx, out.ctypes.data))
        return dict(interactions=int(out[0]), mac_tests=int(out[1]), pops=int(out[2]), active_lanes=int(out[3]))

    def gravity_walk_abu(self, pot, acc, a_tol, phi_tol=0.0, params: TSGravityParams | None = None, **kw):
        """Adaptive Block Update: pot/acc hold the previous solution on input, the new one on output.
        Returns the number of leaf-blocks walked in full (synchronises the stream)."""
        import torch
        p = params if params is not None else self.gravity_params(**kw)
        dt = torch.float64 if p.precision == TS_PREC_FP64 else torch.float32
        n = C.c_int32()
        _check(_lib.ts_gravity_walk_abu(self._ctx, C.byref(p), a_tol, phi_tol, _dptr(pot, dt, self.ncell, "pot"),
                                        _dptr(acc, dt, 3 * self.ncell, "acc"), C.byref(n)))
        return n.value

    def block_workload(self):
        w = np.zeros(self.ncell // 512)
        _check(_lib.ts_block_workload(self._ctx, w.ctypes.data))
        return w

    def error_metrics(self, pot=None, acc=None, pot_ref=None, acc_ref=None, mod_const=False, e_out=None):
        """Sec. 3 eq. ea accuracy of (pot, acc) against FP64 references on the device: returns a dict
        of the ts_error_stats fields.  pot/acc are float32 or float64 CUDA tensors ([n], [n, 3]);
        e_out (optional, float64 [2, n]) receives e_a and e_phi per entry."""
        import torch
        x = acc if acc is not None else pot
        if x is None:
            raise ValueError("error_metrics needs pot or acc")
        n = x.shape[0]
        dt = x.dtype
        prec = TS_PREC_FP64 if dt == torch.float64 else TS_PREC_FP32_KAHAN
        P = lambda t, k, nm, d: _dptr(t, d, k * n, nm) if t is not None else None
        st = TSErrorStats()
        _check(_lib.ts_error_metrics(self._ctx, prec, n, P(pot, 1, "pot", dt), P(acc, 3, "acc", dt),
                                     P(pot_ref, 1, "pot_ref", torch.float64), P(acc_ref, 3, "acc_ref", torch.float64),
                                     1 if mod_const else 0, P(e_out, 2, "e_out", torch.float64), C.byref(st)))
        return {k: getattr(st, k) for k, _ in TSErrorStats._fields_}

    def sync(self):
        _check(_lib.ts_sync(self._ctx))

    def stats(self):
        i, m, ms = C.c_int64(), C.c_int64(), C.c_double()
        _check(_lib.ts_stats(self._ctx, C.byref(i), C.byref(m), C.byref(ms)))
        return dict(interactions=i.value, mac_tests=m.value, walk_ms=ms.value)


def peak_probe(device=0, kind="fp32"):
    """Measured FMA throughput (TFLOP/s) of the device: kind "fp32", "fp32x2" (packed) or "fp64"."""
    v = C.c_double()
    _check(load().ts_peak_probe(device, {"fp32": 0, "fp32x2": 1, "fp64": 2}[kind], C.byref(v)))
    return v.value


def version() -> str:
    return load().ts_version().decode()


def zero_mean_noalloc(pot, weights=None, stream=None):
    """Subtract the (weighted) mean of a CUDA float32 potential in place, without any allocation by
    the library (for callers that may not allocate device memory).  Runs on `stream`, by default
    torch's current stream of the potential's device, so that it is ordered after the caller's own
    writes of pot and weights."""
    import torch
    load()
    n = pot.numel()
    if weights is not None and weights.device != pot.device:
        raise ValueError(f"weights on {weights.device}, potential on {pot.device}: both must be on one GPU")
    w = _dptr(weights, torch.float64, n, "weights") if weights is not None else None
    if stream is None:
        stream = torch.cuda.current_stream(pot.device)
    s = C.c_void_p(stream.cuda_stream)
    _check(_lib.ts_zero_mean_noalloc(pot.device.index or 0, _dptr(pot, torch.float32, n, "pot"), w, n, s))


def autotune_walk(ts: TreeSolver, pot, acc, params: TSGravityParams):
    """Time the walk with 1, 2 and 4 targets per lane; keep the fastest.  Returns (best, [ms x3])."""
    import torch
    best = C.c_int32()
    ms = np.zeros(3)
    dt = torch.float64 if params.precision == TS_PREC_FP64 else torch.float32
    _check(_lib.ts_autotune_walk(ts._ctx, C.byref(params), _dptr(pot, dt, ts.ncell, "pot"),
                                 _dptr(acc, dt, 3 * ts.ncell, "acc"), C.byref(best), ms.ctypes.data))
    return best.value, ms


class Batch:
    """Many independent grids (one TreeSolver each, same device) walked by one persistent kernel."""

    def __init__(self, solvers):
        load()
        self.solvers = list(solvers)
        arr = (C.c_void_p * len(self.solvers))(*[s._ctx.value for s in self.solvers])
        self._b = C.c_void_p()
        _check(_lib.ts_batch_create(C.byref(self._b), arr, len(self.solvers)))

    def close(self):
        if self._b:
            _lib.ts_batch_destroy(self._b)
            self._b = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tuning(self, items_per_dequeue=4, ctas_per_sm=0):
        _check(_lib.ts_batch_set_tuning(self._b, items_per_dequeue, ctas_per_sm))

    def set_mode(self, mode=0, nstreams=8):
        """0: persistent per-class kernels; 1: per-grid kernels spread over nstreams streams."""
        _check(_lib.ts_batch_set_mode(self._b, mode, nstreams))

    def run(self, gravity=None, pots=None, accs=None, column=None, cols=None, densities=None, use_graph=True):
        """gravity/column: TSGravityParams / TSColumnParams or None; lists of CUDA tensors per grid."""
        import torch
        n = len(self.solvers)

        def ptrs(ts, dtype, numels, name):
            return (C.c_void_p * n)(*[_dptr(t, dtype, k, name).value for t, k in zip(ts, numels)])

        nc = [s.ncell for s in self.solvers]
        p_pot = p_acc = p_cols = p_den = None
        if gravity is not None:
            p_pot = ptrs(pots, torch.float32, nc, "pot")
            p_acc = ptrs(accs, torch.float32, [3 * k for k in nc], "acc")
        if column is not None:
            npix = 12 * column.n_side ** 2
            p_cols = ptrs(cols, torch.float32, [npix * k for k in nc], "columns")
        if densities is not None:
            p_den = ptrs(densities, torch.float64, nc, "density")
        _check(_lib.ts_batch_run(self._b, C.byref(gravity) if gravity is not None else None, p_pot, p_acc,
                                 C.byref(column) if column is not None else None, p_cols, p_den, int(use_graph)))

    def sync(self):
        out = np.zeros(5, dtype=np.int64)
        ms = C.c_double()
        _check(_lib.ts_batch_sync(self._b, out.ctypes.data, C.byref(ms)))
        return dict(interactions=int(out[0]), mac_tests=int(out[1]), column_interactions=int(out[2]),
                    items=int(out[3]), cells=int(out[4]), ms=ms.value)
