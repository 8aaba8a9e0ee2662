"""ctypes binding of the serial FP64 CPU oracle (``vcsgc_oracle.c``, and
``vcsgc_multi.c`` for the multicomponent generalisation).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain reference the CUDA path
is checked against: only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  The product path never
calls it, and it imports nothing from the CUDA package.

``build()`` compiles the C sources with gcc into ``oracle/liboracle.so``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "vcsgc_oracle.c")
HDR = os.path.join(HERE, "vcsgc_oracle.h")
SRCS = [SRC, os.path.join(HERE, "vcsgc_multi.c")]
HDRS = [HDR, os.path.join(HERE, "vcsgc_multi.h"), os.path.join(HERE, "orc_internal.h")]
LIB = os.path.join(HERE, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle if the shared object is missing or stale."""
    stale = (not os.path.exists(LIB) or
             os.path.getmtime(LIB) < max(os.path.getmtime(f) for f in SRCS + HDRS))
    if force or stale:
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, *SRCS, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class EamIn(C.Structure):
    _fields_ = [("nr", C.c_int32), ("dr", C.c_double), ("nrho", C.c_int32),
                ("drho", C.c_double), ("rc", C.c_double),
                ("pair", C.c_void_p * 3), ("dpair", C.c_void_p * 3),
                ("dens", C.c_void_p * 2), ("ddens", C.c_void_p * 2),
                ("embed", C.c_void_p * 2), ("dembed", C.c_void_p * 2)]


class Obs(C.Structure):
    _fields_ = [("n_sites", C.c_int64), ("n_b", C.c_int64), ("energy", C.c_double),
                ("steps", C.c_int64), ("trials", C.c_int64), ("local_accepts", C.c_int64),
                ("global_trials", C.c_int64), ("global_accepts", C.c_int64),
                ("flips", C.c_int64), ("near_ties", C.c_int64), ("sum_c", C.c_double),
                ("sum_c2", C.c_double), ("stage1_accepts", C.c_int64)]

MLP_IN = 10
MLP_H = 64
MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P, D, I64, I32, U64 = C.c_void_p, C.c_double, C.c_int64, C.c_int, C.c_uint64
        sig = {
            "orc_create": (P, [I64, P, P, P, P, P, P, I32]),
            "orc_free": (None, [P]),
            "orc_set_params": (I32, [P, D, D, D, I32, D, U64]),
            "orc_schedule_blocks": (I32, [P] + [I32] * 9),
            "orc_schedule_sublattice": (I32, [P] + [I32] * 6),
            "orc_schedule_spatial": (I32, [P] + [I32] * 6),
            "orc_schedule_overlap": (I32, [P] + [I32] * 9),
            "orc_schedule_weights": (I32, [P, P]),
            "orc_track_trials": (I32, [P, I32]),
            "orc_trial_counts": (None, [P, P]),
            "orc_schedule_min_separation": (D, [P]),
            "orc_schedule_info": (I64, [P, P, P]),
            "orc_schedule_export": (None, [P, P, P, P]),
            "orc_parallel_steps": (I32, [P, I64]),
            "orc_serial_steps": (I32, [P, I64, I32]),
            "orc_delta_e": (D, [P, I64]),
            "orc_delta_e_full": (D, [P, I64]),
            "orc_energy_full": (D, [P]),
            "orc_flip": (None, [P, I64]),
            "orc_get_types": (None, [P, P]),
            "orc_set_types": (None, [P, P]),
            "orc_get_rho": (None, [P, P]),
            "orc_get_obs": (None, [P, P]),
            "orc_reset_counters": (None, [P]),
            "orc_neighbour_count": (I64, [P, I64]),
            "orc_neighbour": (None, [P, I64, I64, P, P, P]),
            "orc_philox": (None, [P, P, P]),
            "orc_u01": (D, [C.c_uint32, C.c_uint32]),
            "orc_below": (U64, [C.c_uint32, C.c_uint32, U64]),
            "orc_spline": (I32, [P, I32, D, P, P]),
            "orc_forces": (None, [P, P, P, P]),
            "orc_set_md": (None, [P, P, P, P, D, D, D, D, D, U64]),
            "orc_md_steps": (I32, [P, I64]),
            "orc_get_md": (None, [P, P, P, P, P, P, P]),
            "orc_kinetic_energy": (D, [P]),
            "orc_hybrid_cycles": (I32, [P, I64, I64, I64]),
            "orc_run_histogram": (I32, [P, I64, I32, P, P]),
            "orc_set_shells": (I32, [P, I32, P, D]),
            "orc_descriptor": (I32, [P, I64, P]),
            "orc_mlp_eval": (D, [P, P]),
            "orc_set_surrogate": (I32, [P, I32, P]),
            "orc_surrogate": (D, [P, I64]),
            "orc_set_ensemble": (I32, [P, I32, D, D, D, I32]),
            "orc_virial": (D, [P]),
            "orc_md_state": (None, [P, P]),
            "orc_minimize": (I32, [P, D, I64, P, P]),
            "orcm_tri": (I32, [I32, I32, I32]),
            "orcm_create": (P, [I64, P, P, P, P, P, P]),
            "orcm_free": (None, [P]),
            "orcm_set_params": (I32, [P, P, P, D, P, U64]),
            "orcm_schedule_sublattice": (I32, [P] + [I32] * 6),
            "orcm_schedule_blocks": (I32, [P] + [I32] * 9),
            "orcm_parallel_steps": (I32, [P, I64]),
            "orcm_run_histogram": (I32, [P, I64, P, P]),
            "orcm_energy_full": (D, [P]),
            "orcm_delta_e": (D, [P, I64, I32]),
            "orcm_delta_e_full": (D, [P, I64, I32]),
            "orcm_get_types": (None, [P, P]),
            "orcm_set_types": (None, [P, P]),
            "orcm_get_rho": (None, [P, P]),
            "orcm_get_obs": (None, [P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def philox(ctr, key):
    """Philox4x32-10 block: four uint32 counter words, two key words."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_p(c), _p(k), _p(out))
    return out


def u01(lo, hi):
    return lib().orc_u01(int(lo), int(hi))


def below(lo, hi, m):
    return lib().orc_below(int(lo), int(hi), int(m))


def mlp_eval(params, x):
    """The surrogate MLP (FP64) at one raw descriptor x (10 counts)."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    assert p.shape == (MLP_NPARAM,) and xx.shape == (MLP_IN,)
    return lib().orc_mlp_eval(_p(p), _p(xx))


class System:
    """One VC-SGC system held by the oracle."""

    def __init__(self, lattice, types, tables, brute=False):
        self._keep = []
        x, y, z = (np.ascontiguousarray(v, dtype=np.float64) for v in (lattice.x, lattice.y, lattice.z))
        box = np.ascontiguousarray(lattice.box, dtype=np.float64)
        t = np.ascontiguousarray(types, dtype=np.uint8)
        e = EamIn()
        e.nr, e.dr, e.nrho, e.drho, e.rc = tables.nr, tables.dr, tables.nrho, tables.drho, tables.rc

        def ptr(a):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64)
            self._keep.append(a)
            return a.ctypes.data

        for q in range(3):
            e.pair[q] = ptr(tables.pair[q])
            e.dpair[q] = ptr(tables.dpair[q])
        for q in range(2):
            e.dens[q] = ptr(tables.dens[q])
            e.ddens[q] = ptr(tables.ddens[q])
            e.embed[q] = ptr(tables.embed[q])
            e.dembed[q] = ptr(tables.dembed[q])
        self.n = int(x.shape[0])
        self.h = lib().orc_create(self.n, _p(x), _p(y), _p(z), _p(box), _p(t), C.byref(e),
                                  1 if brute else 0)
        if not self.h:
            raise ValueError("oracle: invalid system")
        self._keep = []

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_free(self.h)
            self.h = None

    # ---- parameters and schedules
    def set_params(self, phi, kappa, T, kappa_units=0, c0=-1.0, seed=0):
        if lib().orc_set_params(self.h, phi, kappa, T, kappa_units, c0, seed):
            raise ValueError("oracle: bad parameters")

    def schedule_blocks(self, cells, block, colours=(2, 2, 2)):
        if lib().orc_schedule_blocks(self.h, *cells, *block, *colours):
            raise ValueError("oracle: block schedule does not divide the lattice")

    def schedule_sublattice(self, cells, period=(4, 4, 4)):
        if lib().orc_schedule_sublattice(self.h, *cells, *period):
            raise ValueError("oracle: sublattice schedule does not divide the lattice")

    def schedule_spatial(self, blocks, colours=(2, 2, 2)):
        if lib().orc_schedule_spatial(self.h, *blocks, *colours):
            raise ValueError("oracle: spatial schedule does not divide")

    def schedule_overlap(self, cells, cell, gap):
        """Overlapping, position-weighted domains: cells of `cell` lattice
        cells, same-colour domains `gap` lattice cells apart (Sec. III A)."""
        if lib().orc_schedule_overlap(self.h, *cells, *cell, *gap):
            raise ValueError("oracle: overlapping schedule does not divide the lattice")

    def schedule_weights(self):
        """Pick weights parallel to schedule_tables()'s sites, or None."""
        col, dom, sites = self.schedule_tables()
        wt = np.zeros(len(sites), dtype=np.int64)
        return wt if lib().orc_schedule_weights(self.h, _p(wt)) else None

    def track_trials(self, on=True):
        if lib().orc_track_trials(self.h, int(bool(on))):
            raise MemoryError("oracle: trial counters")

    def trial_counts(self):
        out = np.zeros(self.n, dtype=np.int64)
        lib().orc_trial_counts(self.h, _p(out))
        return out

    def schedule_min_separation(self):
        return lib().orc_schedule_min_separation(self.h)

    def schedule_tables(self):
        nc = C.c_int64()
        dpc = C.c_int64()
        nd = lib().orc_schedule_info(self.h, C.byref(nc), C.byref(dpc))
        col = np.zeros(nc.value + 1, dtype=np.int64)
        dom = np.zeros(nd + 1, dtype=np.int64)
        lib().orc_schedule_export(self.h, _p(col), _p(dom), None)
        sites = np.zeros(int(dom[-1]), dtype=np.int64)
        lib().orc_schedule_export(self.h, _p(col), _p(dom), _p(sites))
        return col, dom, sites

    # ---- sampling
    def parallel_steps(self, n):
        if lib().orc_parallel_steps(self.h, int(n)):
            raise RuntimeError("oracle: no schedule")

    def serial_steps(self, n, mode=0):
        if lib().orc_serial_steps(self.h, int(n), int(mode)):
            raise RuntimeError("oracle: serial mode 2 needs a surrogate")

    def run_histogram(self, n_steps, mode=-1):
        """Histogram of n_B after each of n_steps steps, and the mean energy."""
        hist = np.zeros(self.n + 1, dtype=np.int64)
        se = C.c_double(0.0)
        if lib().orc_run_histogram(self.h, int(n_steps), int(mode), _p(hist), C.byref(se)):
            raise RuntimeError("oracle: no schedule")
        return hist, se.value / max(1, n_steps)

    # ---- delayed acceptance
    def set_shells(self, radii, tol=1e-6):
        r = np.ascontiguousarray(radii, dtype=np.float64)
        if lib().orc_set_shells(self.h, len(r), _p(r), float(tol)):
            raise ValueError("oracle: bad shells")

    def descriptor(self, i):
        out = np.zeros(MLP_IN)
        if lib().orc_descriptor(self.h, int(i), _p(out)):
            raise ValueError("oracle: the descriptor needs 5 shells")
        return out

    def set_surrogate(self, kind, params=None):
        """kind: 'off', 'mlp' (params: MLP_NPARAM values) or 'exact'."""
        k = {"off": 0, "mlp": 1, "exact": 2}[kind]
        p = None
        if params is not None:
            p = np.ascontiguousarray(params, dtype=np.float64)
            assert p.shape == (MLP_NPARAM,)
        if lib().orc_set_surrogate(self.h, k, None if p is None else _p(p)):
            raise ValueError("oracle: bad surrogate (MLP needs 5 shells and parameters)")
        self._params = p

    def surrogate(self, i):
        return lib().orc_surrogate(self.h, int(i))

    # ---- energies
    def delta_e(self, i):
        return lib().orc_delta_e(self.h, int(i))

    def delta_e_full(self, i):
        return lib().orc_delta_e_full(self.h, int(i))

    def energy_full(self):
        return lib().orc_energy_full(self.h)

    def flip(self, i):
        lib().orc_flip(self.h, int(i))

    # ---- state
    @property
    def types(self):
        out = np.zeros(self.n, dtype=np.uint8)
        lib().orc_get_types(self.h, _p(out))
        return out

    def set_types(self, t):
        t = np.ascontiguousarray(t, dtype=np.uint8)
        lib().orc_set_types(self.h, _p(t))

    @property
    def rho(self):
        out = np.zeros(self.n, dtype=np.float64)
        lib().orc_get_rho(self.h, _p(out))
        return out

    def set_ensemble(self, kind, t_damp=100.0, p_damp=1000.0, p_ext_bar=0.0, chain=3):
        """kind: 'langevin', 'nvt' or 'npt' (Nose-Hoover chains, MTK barostat)."""
        k = {"langevin": 0, "nvt": 1, "npt": 2}[kind]
        if lib().orc_set_ensemble(self.h, k, float(t_damp), float(p_damp), float(p_ext_bar), int(chain)):
            raise ValueError("oracle: bad ensemble parameters")

    def virial(self):
        return lib().orc_virial(self.h)

    def ensemble_state(self):
        out = np.zeros(9)
        lib().orc_md_state(self.h, _p(out))
        keys = ("kinetic", "potential", "temperature", "pressure_bar", "volume", "conserved", "lx", "ly", "lz")
        return dict(zip(keys, out.tolist()))

    def minimize(self, ftol=1e-4, max_iter=1000):
        it = C.c_int64()
        fm = C.c_double()
        rc = lib().orc_minimize(self.h, float(ftol), int(max_iter), C.byref(it), C.byref(fm))
        if rc < 0:
            raise MemoryError("oracle: minimize")
        return {"converged": rc == 0, "iterations": it.value, "fmax": fm.value}

    def obs(self):
        o = Obs()
        lib().orc_get_obs(self.h, C.byref(o))
        return {f: getattr(o, f) for f, _ in Obs._fields_}

    def reset_counters(self):
        lib().orc_reset_counters(self.h)

    def neighbours(self, i):
        k = lib().orc_neighbour_count(self.h, int(i))
        out = []
        j = C.c_int64()
        r = C.c_double()
        d = np.zeros(3)
        for q in range(k):
            lib().orc_neighbour(self.h, int(i), q, C.byref(j), C.byref(r), _p(d))
            out.append((j.value, r.value, d.copy()))
        return out

    def spline(self, which, x):
        v = C.c_double()
        dv = C.c_double()
        if lib().orc_spline(self.h, int(which), float(x), C.byref(v), C.byref(dv)):
            raise ValueError("oracle: spline argument out of range")
        return v.value, dv.value

    # ---- MD
    def forces(self):
        f = [np.zeros(self.n) for _ in range(3)]
        lib().orc_forces(self.h, *(_p(a) for a in f))
        return f

    def set_md(self, v, masses, dt, gamma, T, seed):
        vv = [np.ascontiguousarray(a, dtype=np.float64) for a in v]
        lib().orc_set_md(self.h, *(_p(a) for a in vv), masses[0], masses[1], dt, gamma, T, seed)

    def md_steps(self, n):
        if lib().orc_md_steps(self.h, int(n)):
            raise RuntimeError("oracle: md not set up")

    def md_state(self):
        a = [np.zeros(self.n) for _ in range(6)]
        lib().orc_get_md(self.h, *(_p(q) for q in a))
        return a

    def kinetic_energy(self):
        return lib().orc_kinetic_energy(self.h)

    def hybrid_cycles(self, n_cycles, n_md, n_mc):
        if lib().orc_hybrid_cycles(self.h, int(n_cycles), int(n_md), int(n_mc)):
            raise RuntimeError("oracle: hybrid cycle failed")


# ------------------------------------------------------------ multicomponent
MULTI_MAX_K = 4


class MultiEamIn(C.Structure):
    _fields_ = [("K", C.c_int32), ("nr", C.c_int32), ("dr", C.c_double), ("nrho", C.c_int32),
                ("drho", C.c_double), ("rc", C.c_double),
                ("pair", C.c_void_p * 10), ("dpair", C.c_void_p * 10),
                ("dens", C.c_void_p * 4), ("ddens", C.c_void_p * 4),
                ("embed", C.c_void_p * 4), ("dembed", C.c_void_p * 4)]


class MultiObs(C.Structure):
    _fields_ = [("n_sites", C.c_int64), ("K", C.c_int32), ("pad", C.c_int32), ("n", C.c_int64 * 4),
                ("energy", C.c_double), ("steps", C.c_int64), ("trials", C.c_int64),
                ("local_accepts", C.c_int64), ("global_trials", C.c_int64), ("global_accepts", C.c_int64),
                ("flips", C.c_int64), ("near_ties", C.c_int64), ("sum_c", C.c_double * 4),
                ("sum_c2", C.c_double * 4)]


class MultiSystem:
    """K-species VC-SGC system held by the multicomponent oracle.  tables:
    an EAMTables with K = len(tables.dens) species and K (K + 1) / 2 pair
    tables in the order (0,0), (0,1), ..., (K-1,K-1)."""

    def __init__(self, lattice, types, tables):
        keep = []
        x, y, z = (np.ascontiguousarray(v, dtype=np.float64) for v in (lattice.x, lattice.y, lattice.z))
        box = np.ascontiguousarray(lattice.box, dtype=np.float64)
        t = np.ascontiguousarray(types, dtype=np.uint8)
        K = len(tables.dens)
        assert len(tables.pair) == K * (K + 1) // 2
        e = MultiEamIn()
        e.K, e.nr, e.dr, e.nrho, e.drho, e.rc = K, tables.nr, tables.dr, tables.nrho, tables.drho, tables.rc

        def ptr(a):
            a = np.ascontiguousarray(a, dtype=np.float64)
            keep.append(a)
            return a.ctypes.data

        for q in range(len(tables.pair)):
            e.pair[q] = ptr(tables.pair[q])
            e.dpair[q] = ptr(tables.dpair[q])
        for q in range(K):
            e.dens[q] = ptr(tables.dens[q])
            e.ddens[q] = ptr(tables.ddens[q])
            e.embed[q] = ptr(tables.embed[q])
            e.dembed[q] = ptr(tables.dembed[q])
        self.n = int(x.shape[0])
        self.K = K
        self.h = lib().orcm_create(self.n, _p(x), _p(y), _p(z), _p(box), _p(t), C.byref(e))
        if not self.h:
            raise ValueError("oracle: invalid multicomponent system")

    def __del__(self):
        if getattr(self, "h", None):
            lib().orcm_free(self.h)
            self.h = None

    def set_params(self, phi, kappa, T, c0=None, seed=1):
        """phi, kappa, c0: one value per solute species 1..K-1 (c0 < 0 or
        None: the current concentration)."""
        m = self.K - 1
        ph = np.ascontiguousarray(np.broadcast_to(phi, (m,)), dtype=np.float64)
        ka = np.ascontiguousarray(np.broadcast_to(kappa, (m,)), dtype=np.float64)
        cc = np.ascontiguousarray(np.broadcast_to(-1.0 if c0 is None else c0, (m,)), dtype=np.float64)
        if lib().orcm_set_params(self.h, _p(ph), _p(ka), float(T), _p(cc), int(seed) & (2**64 - 1)):
            raise ValueError("oracle: bad parameters")

    def schedule_sublattice(self, cells, period=(4, 4, 4)):
        if lib().orcm_schedule_sublattice(self.h, *cells, *period):
            raise ValueError("oracle: sublattice schedule does not divide the lattice")

    def schedule_blocks(self, cells, block, colours=(2, 2, 2)):
        if lib().orcm_schedule_blocks(self.h, *cells, *block, *colours):
            raise ValueError("oracle: block schedule does not divide the lattice")

    def parallel_steps(self, n):
        if lib().orcm_parallel_steps(self.h, int(n)):
            raise RuntimeError("oracle: no schedule")

    def run_histogram(self, n_steps):
        """Joint histogram of the solute counts (shape (N+1,)*(K-1), axis q
        = species q+1) after each of n_steps steps, and the mean energy."""
        nb = (self.n + 1) ** (self.K - 1)
        hist = np.zeros(nb, dtype=np.int64)
        se = C.c_double(0.0)
        if lib().orcm_run_histogram(self.h, int(n_steps), _p(hist), C.byref(se)):
            raise RuntimeError("oracle: no schedule")
        # bin = n_1 + (N+1) (n_2 + (N+1) n_3): C order puts n_1 last
        return hist.reshape((self.n + 1,) * (self.K - 1)).transpose(), se.value / max(1, n_steps)

    def energy_full(self):
        return lib().orcm_energy_full(self.h)

    def delta_e(self, i, b):
        return lib().orcm_delta_e(self.h, int(i), int(b))

    def delta_e_full(self, i, b):
        return lib().orcm_delta_e_full(self.h, int(i), int(b))

    @property
    def types(self):
        out = np.zeros(self.n, dtype=np.uint8)
        lib().orcm_get_types(self.h, _p(out))
        return out

    def set_types(self, t):
        tt = np.ascontiguousarray(t, dtype=np.uint8)
        assert tt.shape == (self.n,) and tt.max(initial=0) < self.K
        lib().orcm_set_types(self.h, _p(tt))

    def rho(self):
        out = np.zeros(self.n)
        lib().orcm_get_rho(self.h, _p(out))
        return out

    def obs(self):
        o = MultiObs()
        lib().orcm_get_obs(self.h, C.byref(o))
        K = o.K
        return {"n_sites": o.n_sites, "K": K, "n": [o.n[a] for a in range(K)], "energy": o.energy,
                "steps": o.steps, "trials": o.trials, "local_accepts": o.local_accepts,
                "global_trials": o.global_trials, "global_accepts": o.global_accepts, "flips": o.flips,
                "near_ties": o.near_ties, "sum_c": [o.sum_c[a] for a in range(K)],
                "sum_c2": [o.sum_c2[a] for a in range(K)]}
