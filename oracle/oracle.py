"""Python front end of the CPU oracle.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It reads a mechanism JSON with the
standard ``json`` module, packs it into the flat arrays of ``oracle.cpp``
and calls the C functions through ``ctypes``.  Nothing here is shared with
the CUDA path.

Functions follow the paper's reaction-system and source-term definitions
(Sec. 2.3, eq. (sourceeq)) and the constant-pressure 0D reactor (Sec. 2.2);
the per-function references are in ``oracle.cpp``.

Parity status: rates, Jacobian and integrator are pinned by the tests in
``tests/test_oracle.py`` (closed forms, invariants, equilibrium by Gibbs
minimisation, finite differences, convergence orders).
"""
from __future__ import annotations

import ctypes as C
import json
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "_build", "liboracle.so")


def build(force: bool = False) -> str:
    """Compile oracle.cpp into a shared library (g++, OpenMP)."""
    src = os.path.join(_HERE, "oracle.cpp")
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(src):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class _OMech(C.Structure):
    _fields_ = [("N", C.c_int), ("M", C.c_int),
                ("W", C.c_void_p), ("nasa", C.c_void_p),
                ("nreac", C.c_void_p), ("reac", C.c_void_p),
                ("nprod", C.c_void_p), ("prod", C.c_void_p),
                ("type", C.c_void_p), ("rev", C.c_void_p),
                ("A", C.c_void_p), ("b", C.c_void_p), ("Ea", C.c_void_p),
                ("eff", C.c_void_p), ("A0", C.c_void_p), ("b0", C.c_void_p),
                ("Ea0", C.c_void_p), ("troe", C.c_void_p)]


_TYPES = {"elementary": 0, "three-body": 1, "falloff-troe": 2}
_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i, p = C.c_double, C.c_int, C.c_void_p
        _lib.or_integrate.argtypes = [p, C.c_int64, p, p, p, d, d, d, d, i, p, p, i]
        _lib.or_rates.argtypes = [p, d, d, p, p, p, p, p, p]
        _lib.or_rhs.argtypes = [p, d, p, p, p]
        _lib.or_rhs_v.argtypes = [p, d, p, p, p]
        _lib.or_jac_v.argtypes = [p, d, p, p]
        _lib.or_integrate_v.argtypes = [p, C.c_int64, p, p, p, d, d, d, d, i, p, p, i]
        _lib.or_jac.argtypes = [p, d, p, p]
        _lib.or_thermo.argtypes = [p, d, p, p, p]
        _lib.or_ros_replay.argtypes = [p, d, p, i, p]
        _lib.or_ros_step.argtypes = [p, d, p, d, p, p]
        _lib.or_ros_replay_dir.argtypes = [p, d, p, i, p, d, p, d, p, p, p]
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


class Mech:
    """Mechanism packed for the oracle (arrays kept alive by this object)."""

    def __init__(self, mech: dict | str):
        if isinstance(mech, str):
            with open(mech) as f:
                mech = json.load(f)
        self.json = mech
        sp = mech["species"]
        names = [s["name"] for s in sp]
        self.names = names
        N, M = len(sp), len(mech["reactions"])
        self.N, self.M = N, M
        self.W = np.array([s["W"] for s in sp], dtype=np.float64)
        self.nasa = np.array([s["nasa7"] for s in sp], dtype=np.float64).reshape(N, 7)
        self.nreac = np.zeros(M, np.int32)
        self.nprod = np.zeros(M, np.int32)
        self.reac = np.zeros((M, 3), np.int32)
        self.prod = np.zeros((M, 3), np.int32)
        self.type = np.zeros(M, np.int32)
        self.rev = np.zeros(M, np.int32)
        self.A = np.zeros(M)
        self.b = np.zeros(M)
        self.Ea = np.zeros(M)
        self.eff = np.ones((M, N))
        self.A0 = np.zeros(M)
        self.b0 = np.zeros(M)
        self.Ea0 = np.zeros(M)
        self.troe = np.zeros((M, 4))
        self.nu = np.zeros((N, M))  # net stoichiometry nu'' - nu' (test helper)
        for j, r in enumerate(mech["reactions"]):
            for side, cnt, arr, sgn in (("reactants", self.nreac, self.reac, -1),
                                        ("products", self.nprod, self.prod, 1)):
                lst = []
                for name, v in r[side].items():
                    lst += [names.index(name)] * int(v)
                    self.nu[names.index(name), j] += sgn * v
                if len(lst) > 3:
                    raise ValueError("more than 3 species on one side")
                cnt[j] = len(lst)
                arr[j, :len(lst)] = lst
            self.type[j] = _TYPES[r["type"]]
            self.rev[j] = 1 if r.get("reversible", True) else 0
            self.A[j], self.b[j], self.Ea[j] = r["A"], r["b"], r["Ea"]
            for name, e in r.get("efficiencies", {}).items():
                self.eff[j, names.index(name)] = e
            if r["type"] == "falloff-troe":
                lo = r["low"]
                self.A0[j], self.b0[j], self.Ea0[j] = lo["A"], lo["b"], lo["Ea"]
                t = r["troe"]
                self.troe[j] = [t["alpha"], t["T3"], t["T1"], t["T2"]]
        self._s = _OMech(N, M, *[_ptr(a) for a in (
            self.W, self.nasa, self.nreac, self.reac, self.nprod, self.prod, self.type, self.rev,
            self.A, self.b, self.Ea, self.eff, self.A0, self.b0, self.Ea0, self.troe)])
        self.ref = C.byref(self._s)
        elements = mech.get("elements", [])
        self.elements = elements
        self.elem = np.array([[s["composition"].get(e, 0) for s in sp] for e in elements],
                             dtype=np.float64).reshape(len(elements), N)

    # -- single-cell definitions ------------------------------------------
    def thermo(self, T):
        cp, h, s = (np.zeros(self.N) for _ in range(3))
        _load().or_thermo(self.ref, float(T), _ptr(cp), _ptr(h), _ptr(s))
        return cp, h, s

    def rates(self, T, p, Y):
        Y = np.ascontiguousarray(Y, dtype=np.float64)
        w = np.zeros(self.N)
        q, kf, kr = (np.zeros(self.M) for _ in range(3))
        rho = C.c_double()
        _load().or_rates(self.ref, float(T), float(p), _ptr(Y), _ptr(w), C.addressof(rho),
                         _ptr(q), _ptr(kf), _ptr(kr))
        return {"wdot": w, "rho": rho.value, "q": q, "kf": kf, "kr": kr}

    def rhs(self, p, y):
        y = np.ascontiguousarray(y, dtype=np.float64)
        f = np.zeros(self.N + 1)
        q = C.c_double()
        _load().or_rhs(self.ref, float(p), _ptr(y), _ptr(f), C.addressof(q))
        return f, q.value

    def ignition(self, T, p, Y, dt, nsteps, grid=4, rtol=1e-10):
        """nsteps consecutive steps of dt (the repeated CFD step of the 0D
        ignition runs, Sec. 4.1) from (T, p, Y); the ignition delay is the time
        of [dT/dt]_max (Sec. 4.1), here over a grid of dt/grid.  Returns the
        final T, Y, the grid time of the largest dT/dt per cell and that rate."""
        T = np.array(T, dtype=np.float64)
        Y = np.array(Y, dtype=np.float64)
        p = np.asarray(p, dtype=np.float64)
        n = T.shape[0]
        best = np.full(n, -np.inf)
        tbest = np.zeros(n)
        h = dt / grid
        for k in range(nsteps * grid):
            for c in range(n):
                fT = self.rhs(p[c], np.r_[T[c], Y[:, c]])[0][0]
                if fT > best[c]:
                    best[c] = fT
                    tbest[c] = k * h
            T, Y, st, _ = self.integrate(T, p, Y, h, rtol=rtol)
            if np.any(st != 0):
                raise RuntimeError("oracle integration failed")
        return T, Y, tbest, best

    def jac(self, p, y):
        y = np.ascontiguousarray(y, dtype=np.float64)
        n = self.N + 1
        J = np.zeros((n, n))
        _load().or_jac(self.ref, float(p), _ptr(y), _ptr(J))
        return J

    # -- integration --------------------------------------------------------
    def integrate(self, T, p, Y, dt, rtol=1e-10, atolY=1e-20, atolT=1e-10, max_steps=100000,
                  threads=None, constant_volume=False):
        """Integrate cells over dt.  Y is species-major [N, ncells].  Returns
        (T, Y, status, nsteps) as new arrays.  constant_volume: each cell's
        density is fixed from its initial (p, T, Y) and its internal energy is
        conserved (Sec. 2.2's constant-volume reactor); otherwise p is fixed and
        the enthalpy conserved."""
        T = np.array(T, dtype=np.float64, copy=True)
        p = np.ascontiguousarray(p, dtype=np.float64)
        Y = np.array(Y, dtype=np.float64, copy=True, order="C")
        n = T.shape[0]
        status = np.zeros(n, np.int32)
        nst = np.zeros(n, np.int32)
        if threads is None:
            threads = os.cpu_count() or 1
        fn = _load().or_integrate_v if constant_volume else _load().or_integrate
        fn(self.ref, n, _ptr(T), _ptr(p), _ptr(Y), float(dt), rtol, atolY, atolT, int(max_steps),
           _ptr(status), _ptr(nst), int(threads))
        return T, Y, status, nst

    def rhs_v(self, rho, y):
        """Constant-volume right-hand side at density rho [g/cm^3]: (f, qdot)."""
        y = np.ascontiguousarray(y, dtype=np.float64)
        f = np.zeros(self.N + 1)
        q = C.c_double()
        _load().or_rhs_v(self.ref, float(rho), _ptr(y), _ptr(f), C.addressof(q))
        return f, q.value

    def jac_v(self, rho, y):
        y = np.ascontiguousarray(y, dtype=np.float64)
        n = self.N + 1
        J = np.zeros((n, n))
        _load().or_jac_v(self.ref, float(rho), _ptr(y), _ptr(J))
        return J

    def density(self, T, p, Y):
        """Ideal-gas density [g/cm^3] from T [K], p [Pa], Y (species-major)."""
        Y = np.asarray(Y, dtype=np.float64)
        sumYW = (Y / self.W[:, None]).sum(axis=0) if Y.ndim == 2 else float(np.sum(Y / self.W))
        return 10.0 * np.asarray(p) / (8.314462618e7 * np.asarray(T) * sumYW)

    def internal_energy_mass(self, T, Y):
        """Mixture specific internal energy [J/kg]: u = h - R T sum_k Y_k / W_k."""
        return self.enthalpy_mass(T, Y) - 8.314462618 * T * float(np.sum(np.asarray(Y) / (self.W * 1e-3)))

    def ros_step(self, p, y, h):
        y = np.ascontiguousarray(y, dtype=np.float64)
        yn = np.zeros_like(y)
        e = np.zeros_like(y)
        rc = _load().or_ros_step(self.ref, float(p), _ptr(y), float(h), _ptr(yn), _ptr(e))
        if rc != 0:
            raise RuntimeError("LU failure")
        return yn, e

    def ros_replay(self, p, y0, hs):
        y = np.array(y0, dtype=np.float64, copy=True)
        hs = np.ascontiguousarray(hs, dtype=np.float64)
        rc = _load().or_ros_replay(self.ref, float(p), _ptr(y), len(hs), _ptr(hs))
        if rc != 0:
            raise RuntimeError("LU failure")
        return y

    def ros_replay_dir(self, p, y0, hs, wT=0.0, wY=None, wQ=0.0, dy0=None, dlnA=None):
        y0 = np.ascontiguousarray(y0, dtype=np.float64)
        hs = np.ascontiguousarray(hs, dtype=np.float64)
        wY = None if wY is None else np.ascontiguousarray(wY, dtype=np.float64)
        dy0 = None if dy0 is None else np.ascontiguousarray(dy0, dtype=np.float64)
        dlnA = None if dlnA is None else np.ascontiguousarray(dlnA, dtype=np.float64)
        out = C.c_double()
        rc = _load().or_ros_replay_dir(self.ref, float(p), _ptr(y0), len(hs), _ptr(hs), float(wT),
                                       None if wY is None else _ptr(wY), float(wQ),
                                       None if dy0 is None else _ptr(dy0),
                                       None if dlnA is None else _ptr(dlnA), C.addressof(out))
        if rc != 0:
            raise RuntimeError("LU failure")
        return out.value

    # -- helpers used by pins ------------------------------------------------
    def enthalpy_mass(self, T, Y):
        """Mixture specific enthalpy [J/kg] at (T, Y)."""
        _, h, _ = self.thermo(T)
        return float(np.sum(Y * h * 8.314462618 * T / (self.W * 1e-3)))


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
