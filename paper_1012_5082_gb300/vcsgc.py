"""Thin Python binding of the C ABI in ``include/vcsgc.h`` (ctypes).

The module functions carry the C names and only marshal arguments: every
step of the method runs in ``libvcsgc.so``'s CUDA kernels.  ``Context`` is a
small convenience wrapper over the same calls.  There is no CPU fallback: if
the library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK = 0
ERR = {-1: "INVALID_ARG", -2: "CUDA", -3: "TABLE_RANGE", -4: "NONFINITE", -5: "SCHEDULE",
       -6: "TIMEOUT", -7: "NOMEM", -8: "STATE", -9: "OVERFLOW"}
SCHED_BLOCKS, SCHED_SUBLATTICE, SCHED_SPATIAL, SCHED_OVERLAP = 0, 1, 2, 3
PREC_FP64, PREC_MIXED = 0, 1
MLP_IN = 10
MLP_NPARAM = 4929


class VcsgcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"vcsgc error {code} ({ERR.get(code, '?')}): {msg}")
        self.code = code


class Lattice(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("a", C.c_double), ("n", C.c_int64), ("x", C.c_void_p), ("y", C.c_void_p),
                ("z", C.c_void_p), ("box", C.c_double * 3)]


class EamTables(C.Structure):
    _fields_ = [("nr", C.c_int32), ("dr", C.c_double), ("nrho", C.c_int32), ("drho", C.c_double),
                ("rc", C.c_double), ("pair", C.c_void_p * 3), ("dpair", C.c_void_p * 3),
                ("dens", C.c_void_p * 2), ("ddens", C.c_void_p * 2), ("embed", C.c_void_p * 2),
                ("dembed", C.c_void_p * 2)]


class Options(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("c0", C.c_double), ("kappa_units", C.c_int32),
                ("schedule", C.c_int32), ("sched", C.c_int32 * 6), ("precision", C.c_int32),
                ("n_replicas", C.c_int32), ("phi_r", C.c_void_p), ("kappa_r", C.c_void_p),
                ("T_r", C.c_void_p), ("seed_r", C.c_void_p), ("c0_r", C.c_void_p),
                ("mass", C.c_double * 2), ("dt", C.c_double), ("gamma", C.c_double),
                ("T_md", C.c_double), ("skin", C.c_double), ("md_seed", C.c_uint64),
                ("stream", C.c_void_p), ("device", C.c_int32)]


class Observables(C.Structure):
    _fields_ = [("n_sites", C.c_int64), ("n_b", C.c_int64), ("c", C.c_double),
                ("energy", C.c_double), ("energy_per_atom", C.c_double), ("steps", C.c_int64),
                ("trials", C.c_int64), ("local_accepts", C.c_int64), ("global_trials", C.c_int64),
                ("global_accepts", C.c_int64), ("flips", C.c_int64), ("near_ties", C.c_int64),
                ("acc_local", C.c_double), ("acc_global", C.c_double), ("mean_c", C.c_double),
                ("var_c", C.c_double), ("dmu_est", C.c_double), ("sweeps", C.c_double),
                ("kappa_p", C.c_double), ("dmu0", C.c_double), ("stage1_accepts", C.c_int64)]


_lib = None
EXPORTS = ["vcsgc_default_options", "vcsgc_init", "vcsgc_steps", "vcsgc_sweep", "vcsgc_steps_per_sweep",
           "md_steps", "vcsgc_hybrid", "observables", "vcsgc_get_types", "vcsgc_set_types",
           "vcsgc_get_rho", "vcsgc_delta_e", "vcsgc_energy", "vcsgc_forces", "vcsgc_get_md",
           "vcsgc_set_velocities", "vcsgc_kinetic_energy", "vcsgc_neighbours", "vcsgc_last_error",
           "vcsgc_free", "vcsgc_profile_steps", "vcsgc_neighbour_list_noalloc", "vcsgc_batch_init",
           "vcsgc_autotune", "vcsgc_features", "vcsgc_mlp_create", "vcsgc_mlp_set_params",
           "vcsgc_mlp_get_params", "vcsgc_mlp_forward", "vcsgc_mlp_grad", "vcsgc_mlp_train",
           "vcsgc_mlp_last_error", "vcsgc_mlp_free", "vcsgc_set_surrogate", "vcsgc_observables_all",
           "vcsgc_get_types_all", "vcsgc_set_types_all", "vcsgc_multi_init", "vcsgc_multi_sweep",
           "vcsgc_multi_steps", "vcsgc_multi_steps_per_sweep", "vcsgc_multi_observables",
           "vcsgc_multi_get_types", "vcsgc_multi_set_types", "vcsgc_multi_delta_e", "vcsgc_multi_energy",
           "vcsgc_multi_last_error", "vcsgc_multi_free", "vcsgc_set_ensemble", "vcsgc_md_state",
           "vcsgc_minimize", "vcsgc_save", "vcsgc_load", "vcsgc_set_launch", "vcsgc_get_launch",
           "vcsgc_philox", "vcsgc_cluster_sizes", "vcsgc_set_schedule", "vcsgc_autotune_schedule",
           "vcsgc_multi_set_surrogate", "vcsgc_multi_features"]


def lib():
    """Load libvcsgc.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libvcsgc.so is missing; the CUDA path cannot run")
        L = C.CDLL(path)
        P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        sig = {
            "vcsgc_default_options": (I32, [P]),
            "vcsgc_init": (I32, [C.POINTER(C.c_void_p), P, P, P, D, D, D, P]),
            "vcsgc_steps": (I32, [P, I64]),
            "vcsgc_sweep": (I32, [P, I64]),
            "vcsgc_steps_per_sweep": (I32, [P, P]),
            "md_steps": (I32, [P, I64]),
            "vcsgc_hybrid": (I32, [P, I64, I64, I64]),
            "observables": (I32, [P, I32, P]),
            "vcsgc_get_types": (I32, [P, I32, P]),
            "vcsgc_set_types": (I32, [P, I32, P]),
            "vcsgc_get_rho": (I32, [P, I32, P]),
            "vcsgc_delta_e": (I32, [P, I32, P, I64, P]),
            "vcsgc_energy": (I32, [P, I32, P]),
            "vcsgc_forces": (I32, [P, P, P, P]),
            "vcsgc_get_md": (I32, [P, P, P, P, P, P, P]),
            "vcsgc_set_velocities": (I32, [P, P, P, P]),
            "vcsgc_kinetic_energy": (I32, [P, P]),
            "vcsgc_neighbours": (I32, [P, I64, P, I32, P]),
            "vcsgc_profile_steps": (I32, [P, I64, P, P]),
            "vcsgc_neighbour_list_noalloc": (I32, [I64, P, P, P, P, D, I32, P, P, P]),
            "vcsgc_batch_init": (I32, [C.POINTER(C.c_void_p), I32, P, D, P, P, P, P, P, P]),
            "vcsgc_autotune": (I32, [P, I64, P]),
            "vcsgc_last_error": (C.c_char_p, [P]),
            "vcsgc_free": (None, [P]),
            "vcsgc_features": (I32, [P, P, P]),
            "vcsgc_mlp_create": (I32, [C.POINTER(C.c_void_p), P, P]),
            "vcsgc_mlp_set_params": (I32, [P, P]),
            "vcsgc_mlp_get_params": (I32, [P, P]),
            "vcsgc_mlp_forward": (I32, [P, P, I64, P]),
            "vcsgc_mlp_grad": (I32, [P, P, P, I64, P, P]),
            "vcsgc_mlp_train": (I32, [P, P, P, I64, I64, I64, D, C.c_uint64, P]),
            "vcsgc_mlp_last_error": (C.c_char_p, [P]),
            "vcsgc_mlp_free": (None, [P]),
            "vcsgc_set_surrogate": (I32, [P, P]),
            "vcsgc_observables_all": (I32, [P, P]),
            "vcsgc_get_types_all": (I32, [P, P]),
            "vcsgc_set_types_all": (I32, [P, P]),
            "vcsgc_set_ensemble": (I32, [P, I32, D, D, D, I32]),
            "vcsgc_save": (I32, [P, C.c_char_p]),
            "vcsgc_load": (I32, [P, C.c_char_p]),
            "vcsgc_md_state": (I32, [P, P]),
            "vcsgc_minimize": (I32, [P, D, I64, P, P]),
            "vcsgc_multi_init": (I32, [C.POINTER(C.c_void_p), P, P, P, I32, P, P, P, P, P, P, P, I32]),
            "vcsgc_multi_sweep": (I32, [P, I64]),
            "vcsgc_multi_steps": (I32, [P, I64]),
            "vcsgc_multi_steps_per_sweep": (I32, [P, P]),
            "vcsgc_multi_observables": (I32, [P, I32, P]),
            "vcsgc_multi_get_types": (I32, [P, I32, P]),
            "vcsgc_multi_set_types": (I32, [P, I32, P]),
            "vcsgc_multi_delta_e": (I32, [P, I32, P, P, I64, P]),
            "vcsgc_multi_energy": (I32, [P, I32, P]),
            "vcsgc_multi_set_surrogate": (I32, [P, P]),
            "vcsgc_multi_features": (I32, [P, P, P]),
            "vcsgc_multi_last_error": (C.c_char_p, [P]),
            "vcsgc_multi_free": (None, [P]),
            "vcsgc_set_launch": (I32, [P, I32, I32, I32]),
            "vcsgc_get_launch": (I32, [P, P, P, P]),
            "vcsgc_philox": (I32, [P, P, P, I64]),
            "vcsgc_cluster_sizes": (I32, [P, P]),
            "vcsgc_set_schedule": (I32, [P, I32, P]),
            "vcsgc_autotune_schedule": (I32, [P, I32, P, P, I64, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(rc, ctx=None):
    if rc != OK:
        msg = lib().vcsgc_last_error(ctx)
        raise VcsgcError(rc, msg.decode() if msg else "")


# ------------------------------------------------- C-named entry points
def vcsgc_default_options():
    o = Options()
    _check(lib().vcsgc_default_options(C.byref(o)))
    return o


def vcsgc_init(lattice, types, eam, phi, kappa, T, options=None):
    """Returns the context handle; the caller frees it with vcsgc_free."""
    h = C.c_void_p()
    rc = lib().vcsgc_init(C.byref(h), C.byref(lattice), _ptr(types), C.byref(eam), phi, kappa, T,
                          C.byref(options) if options is not None else None)
    _check(rc, None)
    return h


def vcsgc_steps(ctx, n):
    _check(lib().vcsgc_steps(ctx, int(n)), ctx)


def vcsgc_sweep(ctx, n):
    _check(lib().vcsgc_sweep(ctx, int(n)), ctx)


def md_steps(ctx, n):
    _check(lib().md_steps(ctx, int(n)), ctx)


def observables(ctx, replica=0):
    o = Observables()
    _check(lib().observables(ctx, int(replica), C.byref(o)), ctx)
    return {f: getattr(o, f) for f, _ in Observables._fields_}


def vcsgc_free(ctx):
    lib().vcsgc_free(ctx)


def vcsgc_neighbour_list_noalloc(n, d_x, d_y, d_z, box, rl, K, d_nbr, d_cnt, stream=None):
    """Device pointers in and out (integers, e.g. torch tensor data_ptr());
    returns the status code."""
    b = (C.c_double * 3)(*[float(v) for v in box])
    return lib().vcsgc_neighbour_list_noalloc(int(n), C.c_void_p(d_x), C.c_void_p(d_y),
                                              C.c_void_p(d_z), b, float(rl), int(K),
                                              C.c_void_p(d_nbr), C.c_void_p(d_cnt),
                                              C.c_void_p(stream) if stream else None)


def vcsgc_philox(ctr, key):
    """Philox4x32-10 words of the device generator: ctr [n, 4] and key [n, 2]
    uint32 in, [n, 4] uint32 out."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    assert c.shape[0] == k.shape[0]
    out = np.zeros_like(c)
    _check(lib().vcsgc_philox(_ptr(c), _ptr(k), _ptr(out), c.shape[0]))
    return out


def vcsgc_features(ctx, d_X, d_Y):
    """Device pointers (integers) of the caller's [rows][10] and [rows] float
    buffers."""
    _check(lib().vcsgc_features(ctx, C.c_void_p(d_X), C.c_void_p(d_Y)), ctx)


def vcsgc_set_surrogate(ctx, mlp):
    _check(lib().vcsgc_set_surrogate(ctx, mlp), ctx)


def _check_mlp(rc, m):
    if rc != OK:
        msg = lib().vcsgc_mlp_last_error(m) if m else b""
        raise VcsgcError(rc, msg.decode() if msg else "")


def vcsgc_mlp_create(params, stream=None):
    p = np.ascontiguousarray(params, dtype=np.float32)
    assert p.shape == (MLP_NPARAM,)
    h = C.c_void_p()
    _check_mlp(lib().vcsgc_mlp_create(C.byref(h), _ptr(p), stream), None)
    return h


def vcsgc_mlp_forward(mlp, d_X, n, d_out):
    _check_mlp(lib().vcsgc_mlp_forward(mlp, C.c_void_p(d_X), int(n), C.c_void_p(d_out)), mlp)


def vcsgc_mlp_grad(mlp, d_X, d_Y, n):
    g = np.zeros(MLP_NPARAM, dtype=np.float32)
    loss = C.c_double()
    _check_mlp(lib().vcsgc_mlp_grad(mlp, C.c_void_p(d_X), C.c_void_p(d_Y), int(n), _ptr(g), C.byref(loss)), mlp)
    return g, loss.value


def vcsgc_mlp_train(mlp, d_X, d_Y, n, batch, steps, lr, seed):
    hist = np.zeros(max(1, int(steps)), dtype=np.float64)
    _check_mlp(lib().vcsgc_mlp_train(mlp, C.c_void_p(d_X), C.c_void_p(d_Y), int(n), int(batch), int(steps),
                                     float(lr), int(seed), _ptr(hist)), mlp)
    return hist[:int(steps)]


def vcsgc_mlp_get_params(mlp):
    p = np.zeros(MLP_NPARAM, dtype=np.float32)
    _check_mlp(lib().vcsgc_mlp_get_params(mlp, _ptr(p)), mlp)
    return p


def vcsgc_mlp_set_params(mlp, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    assert p.shape == (MLP_NPARAM,)
    _check_mlp(lib().vcsgc_mlp_set_params(mlp, _ptr(p)), mlp)


def vcsgc_mlp_free(mlp):
    lib().vcsgc_mlp_free(mlp)


class Surrogate:
    """The delayed-acceptance surrogate network (vcsgc_mlp_*); inputs and
    outputs are CUDA float32 torch tensors."""

    def __init__(self, params, stream=None):
        self.h = vcsgc_mlp_create(params, None if stream is None else getattr(stream, "cuda_stream", stream))

    def close(self):
        if getattr(self, "h", None):
            vcsgc_mlp_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def params(self):
        return vcsgc_mlp_get_params(self.h)

    @params.setter
    def params(self, p):
        vcsgc_mlp_set_params(self.h, p)

    def forward(self, X):
        import torch
        X = X.contiguous()
        out = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
        vcsgc_mlp_forward(self.h, X.data_ptr(), X.shape[0], out.data_ptr())
        return out

    def grad(self, X, Y):
        X, Y = X.contiguous(), Y.contiguous()
        return vcsgc_mlp_grad(self.h, X.data_ptr(), Y.data_ptr(), X.shape[0])

    def train(self, X, Y, *, batch=4096, steps=1000, lr=1e-3, seed=1):
        X, Y = X.contiguous(), Y.contiguous()
        return vcsgc_mlp_train(self.h, X.data_ptr(), Y.data_ptr(), X.shape[0], batch, steps, lr, seed)


# ----------------------------------------------------------- convenience
def _eam_struct(tables, keep):
    E = EamTables()
    E.nr, E.dr, E.nrho, E.drho, E.rc = tables.nr, tables.dr, tables.nrho, tables.drho, tables.rc

    def arr(a):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=np.float64)
        keep.append(a)
        return a.ctypes.data

    for q in range(3):
        E.pair[q] = arr(tables.pair[q])
        E.dpair[q] = arr(tables.dpair[q])
    for q in range(2):
        E.dens[q] = arr(tables.dens[q])
        E.ddens[q] = arr(tables.ddens[q])
        E.embed[q] = arr(tables.embed[q])
        E.dembed[q] = arr(tables.dembed[q])
    return E


class Context:
    """Owns one C context; keeps the host arrays passed at init alive."""

    def __init__(self, lattice, types, tables, phi, kappa, T, *, seed=1, c0=-1.0, kappa_units=0,
                 schedule=SCHED_SUBLATTICE, sched=(4, 4, 4, 0, 0, 0), n_replicas=1, phi_r=None,
                 kappa_r=None, T_r=None, seed_r=None, c0_r=None, masses=(55.845, 63.546), dt=2.0,
                 gamma=0.01, T_md=-1.0, skin=0.3, md_seed=12345, stream=None, device=-1,
                 precision=0):
        self._keep = []
        L = Lattice()
        if lattice.cells is not None and getattr(lattice, "rigid", True):
            L.kind = 0
            L.nx, L.ny, L.nz = lattice.cells
            L.a = lattice.a
        else:
            L.kind = 1
            xs = [np.ascontiguousarray(v, dtype=np.float64) for v in (lattice.x, lattice.y, lattice.z)]
            self._keep += xs
            L.n = xs[0].shape[0]
            L.x, L.y, L.z = (v.ctypes.data for v in xs)
            for q in range(3):
                L.box[q] = float(lattice.box[q])
        E = EamTables()
        E.nr, E.dr, E.nrho, E.drho, E.rc = tables.nr, tables.dr, tables.nrho, tables.drho, tables.rc

        def arr(a):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64)
            self._keep.append(a)
            return a.ctypes.data

        for q in range(3):
            E.pair[q] = arr(tables.pair[q])
            E.dpair[q] = arr(tables.dpair[q])
        for q in range(2):
            E.dens[q] = arr(tables.dens[q])
            E.ddens[q] = arr(tables.ddens[q])
            E.embed[q] = arr(tables.embed[q])
            E.dembed[q] = arr(tables.dembed[q])
        o = vcsgc_default_options()
        o.seed = seed
        o.c0 = c0
        o.kappa_units = kappa_units
        o.schedule = schedule
        for q in range(6):
            o.sched[q] = sched[q] if q < len(sched) else 0
        o.n_replicas = n_replicas
        o.precision = precision
        for name, val, dt_ in (("phi_r", phi_r, np.float64), ("kappa_r", kappa_r, np.float64),
                               ("T_r", T_r, np.float64), ("seed_r", seed_r, np.uint64),
                               ("c0_r", c0_r, np.float64)):
            if val is not None:
                a = np.ascontiguousarray(val, dtype=dt_)
                self._keep.append(a)
                setattr(o, name, a.ctypes.data)
        o.mass[0], o.mass[1] = masses
        o.dt, o.gamma, o.T_md, o.skin, o.md_seed = dt, gamma, T_md, skin, md_seed
        if stream is not None:
            o.stream = getattr(stream, "cuda_stream", stream)
        o.device = device
        t = np.ascontiguousarray(types, dtype=np.uint8)
        self.n_replicas = n_replicas
        self.h = vcsgc_init(L, t, E, phi, kappa, T, o)
        self.n = int(t.shape[-1]) if t.ndim > 1 else int(t.shape[0]) // n_replicas
        self._keep = []

    def close(self):
        if getattr(self, "h", None):
            vcsgc_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def steps(self, n):
        vcsgc_steps(self.h, n)

    def sweep(self, n):
        vcsgc_sweep(self.h, n)

    @property
    def steps_per_sweep(self):
        v = C.c_int64()
        _check(lib().vcsgc_steps_per_sweep(self.h, C.byref(v)), self.h)
        return v.value

    def md_steps(self, n):
        md_steps(self.h, n)

    def hybrid(self, n_cycles, n_md, n_mc):
        _check(lib().vcsgc_hybrid(self.h, int(n_cycles), int(n_md), int(n_mc)), self.h)

    def observables(self, replica=0):
        return observables(self.h, replica)

    def types(self, replica=0):
        out = np.zeros(self.n, dtype=np.uint8)
        _check(lib().vcsgc_get_types(self.h, int(replica), _ptr(out)), self.h)
        return out

    def set_types(self, t, replica=0):
        t = np.ascontiguousarray(t, dtype=np.uint8)
        _check(lib().vcsgc_set_types(self.h, int(replica), _ptr(t)), self.h)

    def _total_sites(self):
        return int(sum(self.sizes)) if hasattr(self, "sizes") else self.n * self.n_replicas

    def types_all(self, out=None):
        """Every replica's species back to back (vcsgc_get_types_all); out: a
        contiguous uint8 array of the total size (e.g. pinned), or None."""
        if out is None:
            out = np.zeros(self._total_sites(), dtype=np.uint8)
        assert out.dtype == np.uint8 and out.flags.c_contiguous and out.size == self._total_sites()
        _check(lib().vcsgc_get_types_all(self.h, _ptr(out)), self.h)
        return out

    def set_types_all(self, t):
        t = np.ascontiguousarray(t, dtype=np.uint8)
        assert t.size == self._total_sites()
        _check(lib().vcsgc_set_types_all(self.h, _ptr(t)), self.h)

    def observables_all(self):
        R = self.n_replicas
        arr = (Observables * R)()
        _check(lib().vcsgc_observables_all(self.h, arr), self.h)
        return [{f: getattr(o, f) for f, _ in Observables._fields_} for o in arr]

    def rho(self, replica=0):
        out = np.zeros(self.n, dtype=np.float64)
        _check(lib().vcsgc_get_rho(self.h, int(replica), _ptr(out)), self.h)
        return out

    def delta_e(self, sites, replica=0):
        s = np.ascontiguousarray(sites, dtype=np.int64)
        out = np.zeros(s.shape[0], dtype=np.float64)
        _check(lib().vcsgc_delta_e(self.h, int(replica), _ptr(s), s.shape[0], _ptr(out)), self.h)
        return out

    def energy(self, replica=0):
        v = C.c_double()
        _check(lib().vcsgc_energy(self.h, int(replica), C.byref(v)), self.h)
        return v.value

    def forces(self):
        f = [np.zeros(self.n) for _ in range(3)]
        _check(lib().vcsgc_forces(self.h, *(_ptr(a) for a in f)), self.h)
        return f

    def md_state(self):
        a = [np.zeros(self.n) for _ in range(6)]
        _check(lib().vcsgc_get_md(self.h, *(_ptr(q) for q in a)), self.h)
        return a

    def positions(self):
        a = [np.zeros(self.n) for _ in range(3)]
        _check(lib().vcsgc_get_md(self.h, *(_ptr(q) for q in a), None, None, None), self.h)
        return a

    def set_velocities(self, v):
        vv = [np.ascontiguousarray(q, dtype=np.float64) for q in v]
        _check(lib().vcsgc_set_velocities(self.h, *(_ptr(q) for q in vv)), self.h)

    def kinetic_energy(self):
        v = C.c_double()
        _check(lib().vcsgc_kinetic_energy(self.h, C.byref(v)), self.h)
        return v.value

    def save(self, path):
        _check(lib().vcsgc_save(self.h, os.fsencode(path)), self.h)

    def load(self, path):
        _check(lib().vcsgc_load(self.h, os.fsencode(path)), self.h)

    def set_ensemble(self, kind, t_damp=100.0, p_damp=1000.0, p_ext_bar=0.0, chain=3):
        """kind: 'langevin', 'nvt' or 'npt' (Nose-Hoover chains, MTK barostat)."""
        k = {"langevin": 0, "nvt": 1, "npt": 2}[kind]
        _check(lib().vcsgc_set_ensemble(self.h, k, float(t_damp), float(p_damp), float(p_ext_bar), int(chain)),
               self.h)

    def ensemble_state(self):
        out = np.zeros(9)
        _check(lib().vcsgc_md_state(self.h, _ptr(out)), self.h)
        keys = ("kinetic", "potential", "temperature", "pressure_bar", "volume", "conserved", "lx", "ly", "lz")
        return dict(zip(keys, out.tolist()))

    def minimize(self, ftol=1e-4, max_iter=1000):
        it = C.c_int64()
        fm = C.c_double()
        _check(lib().vcsgc_minimize(self.h, float(ftol), int(max_iter), C.byref(it), C.byref(fm)), self.h)
        return {"converged": fm.value < ftol, "iterations": it.value, "fmax": fm.value}

    def profile_steps(self, n):
        """Device time (ms) of the propose and commit kernels over n steps."""
        a, b = C.c_double(), C.c_double()
        _check(lib().vcsgc_profile_steps(self.h, int(n), C.byref(a), C.byref(b)), self.h)
        return a.value, b.value

    def set_launch(self, form=0, block=128, variant=1):
        """Launch shape of the fused colour step (vcsgc_set_launch): form 0
        with variant = row prefetch, form 1 with variant = CTAs per cluster."""
        _check(lib().vcsgc_set_launch(self.h, int(form), int(block), int(variant)), self.h)

    def set_schedule(self, kind, sched):
        """Switch the colour schedule between colour steps (vcsgc_set_schedule)."""
        sc = np.ascontiguousarray(sched, dtype=np.int32)
        assert sc.shape == (6,)
        _check(lib().vcsgc_set_schedule(self.h, int(kind), _ptr(sc)), self.h)

    def autotune_schedule(self, candidates, sweeps=2):
        """candidates: [(kind, sched6), ...]; returns (best index, accepted
        flips per second of each candidate)."""
        kinds = np.ascontiguousarray([k for k, _ in candidates], dtype=np.int32)
        sc = np.ascontiguousarray([list(s) for _, s in candidates], dtype=np.int32).reshape(-1)
        scores = np.zeros(len(candidates))
        best = C.c_int32()
        _check(lib().vcsgc_autotune_schedule(self.h, len(candidates), _ptr(kinds), _ptr(sc), int(sweeps),
                                             _ptr(scores), C.byref(best)), self.h)
        return best.value, scores

    def cluster_sizes(self):
        """Cluster sizes of the cluster-resident form these lattices allow."""
        m = C.c_int32()
        _check(lib().vcsgc_cluster_sizes(self.h, C.byref(m)), self.h)
        return [1 << q for q in range(5) if m.value >> q & 1]

    def get_launch(self):
        f, b, p = C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().vcsgc_get_launch(self.h, C.byref(f), C.byref(b), C.byref(p)), self.h)
        return f.value, b.value, p.value

    def autotune(self, steps=64):
        """Pick the fused colour step's block size by timing (real steps)."""
        b = C.c_int32()
        _check(lib().vcsgc_autotune(self.h, int(steps), C.byref(b)), self.h)
        return b.value

    def features(self):
        """(X [rows, 10], Y [rows]) CUDA float32 tensors of every site of every
        replica (vcsgc_features)."""
        import torch
        rows = int(sum(self.sizes)) if hasattr(self, "sizes") else self.n * self.n_replicas
        X = torch.empty((rows, MLP_IN), dtype=torch.float32, device="cuda")
        Y = torch.empty(rows, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        vcsgc_features(self.h, X.data_ptr(), Y.data_ptr())
        return X, Y

    def set_surrogate(self, surrogate):
        """Delayed acceptance with a copy of surrogate's weights (None: off)."""
        vcsgc_set_surrogate(self.h, None if surrogate is None else surrogate.h)

    def neighbours(self, i, cap=256):
        out = np.zeros(cap, dtype=np.int32)
        cnt = C.c_int32()
        _check(lib().vcsgc_neighbours(self.h, int(i), _ptr(out), cap, C.byref(cnt)), self.h)
        return out[:min(cnt.value, cap)].copy()


class Batch(Context):
    """Rigid BCC lattices of different sizes advanced by one launch per colour
    step (vcsgc_batch_init).  types: list of per-replica species arrays."""

    def __init__(self, cells, types, tables, phi, kappa, T, *, a=2.855, seed=1, c0=-1.0,
                 seed_r=None, c0_r=None, sched=(4, 4, 4), stream=None, device=-1, precision=0):
        self._keep = []
        cells = np.ascontiguousarray(cells, dtype=np.int32).reshape(-1, 3)
        R = cells.shape[0]
        t = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.uint8) for x in types]))
        E = _eam_struct(tables, self._keep)
        o = vcsgc_default_options()
        o.seed = seed
        o.c0 = c0
        o.schedule = SCHED_SUBLATTICE
        for q in range(3):
            o.sched[q] = sched[q]
        o.precision = precision
        for name, val, dt_ in (("seed_r", seed_r, np.uint64), ("c0_r", c0_r, np.float64)):
            if val is not None:
                arr_ = np.ascontiguousarray(val, dtype=dt_)
                self._keep.append(arr_)
                setattr(o, name, arr_.ctypes.data)
        if stream is not None:
            o.stream = getattr(stream, "cuda_stream", stream)
        o.device = device
        ph = np.ascontiguousarray(np.broadcast_to(phi, (R,)), dtype=np.float64)
        ka = np.ascontiguousarray(np.broadcast_to(kappa, (R,)), dtype=np.float64)
        TT = np.ascontiguousarray(np.broadcast_to(T, (R,)), dtype=np.float64)
        h = C.c_void_p()
        rc = lib().vcsgc_batch_init(C.byref(h), R, _ptr(cells), float(a), _ptr(t), C.byref(E),
                                    _ptr(ph), _ptr(ka), _ptr(TT), C.byref(o))
        _check(rc, None)
        self.h = h
        self.n_replicas = R
        self.sizes = [int(2 * c[0] * c[1] * c[2]) for c in cells]
        self.n = self.sizes[0]
        self._keep = []

    def types(self, replica=0):
        out = np.zeros(self.sizes[replica], dtype=np.uint8)
        _check(lib().vcsgc_get_types(self.h, int(replica), _ptr(out)), self.h)
        return out

    def rho(self, replica=0):
        out = np.zeros(self.sizes[replica], dtype=np.float64)
        _check(lib().vcsgc_get_rho(self.h, int(replica), _ptr(out)), self.h)
        return out


# ------------------------------------------------------------ multicomponent
class MultiTables(C.Structure):
    _fields_ = [("K", C.c_int32), ("nr", C.c_int32), ("dr", C.c_double), ("nrho", C.c_int32),
                ("drho", C.c_double), ("rc", C.c_double),
                ("pair", C.c_void_p * 10), ("dpair", C.c_void_p * 10),
                ("dens", C.c_void_p * 4), ("ddens", C.c_void_p * 4),
                ("embed", C.c_void_p * 4), ("dembed", C.c_void_p * 4)]


class MultiObs(C.Structure):
    _fields_ = [("n_sites", C.c_int64), ("K", C.c_int32), ("pad", C.c_int32), ("n", C.c_int64 * 4),
                ("c", C.c_double * 4), ("energy", C.c_double), ("energy_per_atom", C.c_double),
                ("steps", C.c_int64), ("trials", C.c_int64), ("local_accepts", C.c_int64),
                ("global_trials", C.c_int64), ("global_accepts", C.c_int64), ("flips", C.c_int64),
                ("near_ties", C.c_int64), ("acc_local", C.c_double), ("acc_global", C.c_double),
                ("mean_c", C.c_double * 4), ("var_c", C.c_double * 4), ("dmu_est", C.c_double * 4),
                ("kappa_p", C.c_double * 4), ("dmu0", C.c_double * 4), ("sweeps", C.c_double),
                ("stage1_accepts", C.c_int64)]


class Multi:
    """K-species (K <= 4) colour step on R replicas of one rigid BCC lattice
    (vcsgc_multi_init).  tables: EAMTables with K = len(tables.dens) species
    and K (K + 1) / 2 pair tables in the order (0,0), (0,1), ..., (K-1,K-1).
    types: (R, N) or (N,) species; phi, kappa, c0: (R, K-1) or broadcastable;
    T: (R,) or scalar."""

    def __init__(self, lattice, types, tables, phi, kappa, T, *, c0=-1.0, seed_r=None, period=(4, 4, 4),
                 n_replicas=None, stream=None, device=-1):
        keep = []
        K = len(tables.dens)
        t = np.asarray(types, dtype=np.uint8)
        R = n_replicas or (t.shape[0] if t.ndim == 2 else 1)
        N = lattice.n
        t = np.ascontiguousarray(np.broadcast_to(t.reshape(-1, N), (R, N)), dtype=np.uint8)
        E = MultiTables()
        E.K, E.nr, E.dr, E.nrho, E.drho, E.rc = K, tables.nr, tables.dr, tables.nrho, tables.drho, tables.rc

        def ptr(a):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64)
            keep.append(a)
            return a.ctypes.data

        for q in range(len(tables.pair)):
            E.pair[q] = ptr(tables.pair[q])
            E.dpair[q] = ptr(tables.dpair[q])
        for q in range(K):
            E.dens[q] = ptr(tables.dens[q])
            E.ddens[q] = ptr(tables.ddens[q])
            E.embed[q] = ptr(tables.embed[q])
            E.dembed[q] = ptr(tables.dembed[q])
        if lattice.cells is None:
            raise ValueError("the multicomponent form needs a rigid lattice")
        L = Lattice()
        L.kind = 0
        L.nx, L.ny, L.nz = lattice.cells
        L.a = lattice.a
        L.n = N
        ph = np.ascontiguousarray(np.broadcast_to(phi, (R, K - 1)), dtype=np.float64)
        ka = np.ascontiguousarray(np.broadcast_to(kappa, (R, K - 1)), dtype=np.float64)
        cc = np.ascontiguousarray(np.broadcast_to(c0, (R, K - 1)), dtype=np.float64)
        TT = np.ascontiguousarray(np.broadcast_to(T, (R,)), dtype=np.float64)
        sr = None if seed_r is None else np.ascontiguousarray(seed_r, dtype=np.uint64)
        per = np.ascontiguousarray(period, dtype=np.int32)
        st = None if stream is None else getattr(stream, "cuda_stream", stream)
        h = C.c_void_p()
        rc = lib().vcsgc_multi_init(C.byref(h), C.byref(L), _ptr(t), C.byref(E), R, _ptr(ph), _ptr(ka), _ptr(TT),
                                    _ptr(cc), _ptr(sr), _ptr(per), st, int(device))
        if rc != OK:
            msg = lib().vcsgc_multi_last_error(None)
            raise VcsgcError(rc, msg.decode() if msg else "")
        self.h = h
        self.K, self.R, self.n = K, R, N
        spw = C.c_int64()
        self._chk(lib().vcsgc_multi_steps_per_sweep(self.h, C.byref(spw)))
        self.steps_per_sweep = spw.value

    def _chk(self, rc):
        if rc != OK:
            msg = lib().vcsgc_multi_last_error(self.h)
            raise VcsgcError(rc, msg.decode() if msg else "")

    def sweep(self, n=1):
        self._chk(lib().vcsgc_multi_sweep(self.h, int(n)))

    def steps(self, n):
        self._chk(lib().vcsgc_multi_steps(self.h, int(n)))

    def observables(self, r=0):
        o = MultiObs()
        self._chk(lib().vcsgc_multi_observables(self.h, int(r), C.byref(o)))
        K = o.K
        out = {}
        for f, _ in MultiObs._fields_:
            v = getattr(o, f)
            out[f] = [v[a] for a in range(K)] if isinstance(v, C.Array) else v
        return out

    def types(self, r=0):
        out = np.zeros(self.n, dtype=np.uint8)
        self._chk(lib().vcsgc_multi_get_types(self.h, int(r), _ptr(out)))
        return out

    def set_types(self, t, r=0):
        tt = np.ascontiguousarray(t, dtype=np.uint8)
        assert tt.shape == (self.n,)
        self._chk(lib().vcsgc_multi_set_types(self.h, int(r), _ptr(tt)))

    def delta_e(self, sites, to, r=0):
        s = np.ascontiguousarray(sites, dtype=np.int64)
        tt = np.ascontiguousarray(np.broadcast_to(to, s.shape), dtype=np.uint8)
        out = np.zeros(s.shape[0])
        self._chk(lib().vcsgc_multi_delta_e(self.h, int(r), _ptr(s), _ptr(tt), s.shape[0], _ptr(out)))
        return out

    def energy(self, r=0):
        e = C.c_double()
        self._chk(lib().vcsgc_multi_energy(self.h, int(r), C.byref(e)))
        return e.value

    def set_surrogate(self, surrogate):
        """Delayed acceptance (K = 2, species-dependent densities) with a copy
        of surrogate's weights (None: off); vcsgc_multi_set_surrogate."""
        self._chk(lib().vcsgc_multi_set_surrogate(self.h, None if surrogate is None else surrogate.h))

    def features(self):
        """(X [R N, 10], Y [R N]) CUDA float32 tensors of every site of every
        replica (vcsgc_multi_features)."""
        import torch
        rows = self.n * self.R
        X = torch.empty((rows, MLP_IN), dtype=torch.float32, device="cuda")
        Y = torch.empty(rows, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        self._chk(lib().vcsgc_multi_features(self.h, X.data_ptr(), Y.data_ptr()))
        return X, Y

    def close(self):
        if getattr(self, "h", None):
            lib().vcsgc_multi_free(self.h)
            self.h = None

    def __del__(self):
        self.close()
