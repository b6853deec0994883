"""ctypes front end of the FP64 CPU oracle (gbo.c).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The CUDA path never imports this
package and this package never imports the CUDA path.

`build()` compiles gbo.c with gcc (-O2, no fast-math) into oracle/_build/.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gbo.c")
_OUT = os.path.join(_HERE, "_build", "libgbo.so")
_lib = None

KE = 332.0522173
KB = 0.0019872043
FARADAY = 23.0605478
LN10 = 2.302585092994045684


class Params(C.Structure):
    _fields_ = [(k, C.c_double) for k in (
        "alpha", "beta", "gamma", "offset", "eps_in", "eps_out",
        "bond_k", "bond_r0", "rep_k", "rep_sigma", "dt", "friction", "mass", "kT", "kappa",
        "rgbmax", "cut")]


def default_params(**kw) -> Params:
    """OBC parameters alpha, beta, gamma = 1.0, 0.8, 4.85, offset 0.09 A,
    eps_in 1, eps_out 78.5, no salt (kappa = 0), no cutoffs (rgbmax = cut = 0);
    MD driver constants (bond k 300 about 1.5 A, soft repulsion k 100 below
    2.5 A, 2 fs, 10 / ps, 12 amu, 300 K)."""
    d = dict(alpha=1.0, beta=0.8, gamma=4.85, offset=0.09, eps_in=1.0, eps_out=78.5,
             bond_k=300.0, bond_r0=1.5, rep_k=100.0, rep_sigma=2.5, dt=0.002, friction=10.0,
             mass=12.0, kT=KB * 300.0, kappa=0.0, rgbmax=0.0, cut=0.0)
    d.update(kw)
    return Params(**d)


def build(force: bool = False) -> str:
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i64, i32, u64 = C.c_double, C.c_int64, C.c_int32, C.c_uint64
        P = C.c_void_p
        _lib.gbo_hct_pair.restype = d
        _lib.gbo_hct_pair.argtypes = [d, d, d]
        _lib.gbo_hct_pair_dr.restype = d
        _lib.gbo_hct_pair_dr.argtypes = [d, d, d]
        _lib.gbo_hct_pair_cut.restype = d
        _lib.gbo_hct_pair_cut.argtypes = [d, d, d, d]
        _lib.gbo_hct_pair_dr_cut.restype = d
        _lib.gbo_hct_pair_dr_cut.argtypes = [d, d, d, d]
        _lib.gbo_philox4x64.argtypes = [P, P, P]
        _lib.gbo_born_radii.argtypes = [i64, P, P, P, C.POINTER(Params), P, P, P, P]
        _lib.gbo_born_radii_subset.argtypes = [i64, P, P, P, C.POINTER(Params), P, i64, P]
        _lib.gbo_energy_fixed_radii.argtypes = [i64, P, P, P, C.POINTER(Params), P]
        _lib.gbo_energy_forces.argtypes = [i64, P, P, P, P, C.POINTER(Params), P, P, P, P, P]
        _lib.gbo_restraints.argtypes = [i64, P, C.POINTER(Params), P, P]
        _lib.gbo_mc_step.argtypes = [i32, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P,
                                     P, P, d, u64, u64, i32, C.POINTER(Params), P, P, P, P, P, P]
        _lib.gbo_mc_sweep.argtypes = [i32, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P,
                                      P, P, d, u64, u64, i32, C.POINTER(Params), P, P, P, P, P]
        _lib.gbo_exchange.argtypes = [i32, i32, i32, i32, P, P, P, i32, u64, u64, d, i32, P, P]
        _lib.gbo_normals.argtypes = [u64, u64, u64, u64, P]
        _lib.gbo_forces_all.argtypes = [i32, P, P, P, P, P, C.POINTER(Params), P, P]
        _lib.gbo_md_step.argtypes = [i32, P, P, P, P, P, P, C.POINTER(Params), P, u64, u64, P]
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def hct_pair(r: float, a: float, s: float) -> float:
    return lib().gbo_hct_pair(r, a, s)


def hct_pair_cut(r: float, a: float, s: float, rc: float) -> float:
    return lib().gbo_hct_pair_cut(float(r), float(a), float(s), float(rc))


def hct_pair_dr_cut(r: float, a: float, s: float, rc: float) -> float:
    return lib().gbo_hct_pair_dr_cut(float(r), float(a), float(s), float(rc))


def hct_pair_dr(r: float, a: float, s: float) -> float:
    return lib().gbo_hct_pair_dr(r, a, s)


def philox4x64(counter, key) -> np.ndarray:
    c = np.asarray(counter, dtype=np.uint64)
    k = np.asarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().gbo_philox4x64(_p(c), _p(k), _p(out))
    return out


def born_radii(x, rho, screen, p: Optional[Params] = None):
    """Returns dict(I, psi, R, dRdpsi) for one molecule."""
    p = p or default_params()
    x, rho, screen = _d(x).reshape(-1, 3), _d(rho), _d(screen)
    n = rho.size
    out = {k: np.zeros(n) for k in ("I", "psi", "R", "dRdpsi")}
    lib().gbo_born_radii(n, _p(x), _p(rho), _p(screen), C.byref(p), _p(out["I"]),
                         _p(out["psi"]), _p(out["R"]), _p(out["dRdpsi"]))
    return out


def born_radii_subset(x, rho, screen, idx, p: Optional[Params] = None) -> np.ndarray:
    """Born radii of the listed atoms only (O(N) each)."""
    p = p or default_params()
    x, rho, screen = _d(x).reshape(-1, 3), _d(rho), _d(screen)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros(idx.size)
    lib().gbo_born_radii_subset(rho.size, _p(x), _p(rho), _p(screen), C.byref(p), _p(idx), idx.size,
                                _p(out))
    return out


def energy_fixed_radii(x, q, R, p: Optional[Params] = None) -> np.ndarray:
    p = p or default_params()
    x, q, R = _d(x).reshape(-1, 3), _d(q), _d(R)
    E = np.zeros(2)
    lib().gbo_energy_fixed_radii(q.size, _p(x), _p(q), _p(R), C.byref(p), _p(E))
    return E


def energy_forces(x, q, rho, screen, p: Optional[Params] = None):
    """One molecule: dict(E=[E_GB, E_Coul], F (n,3), phi (n), R, dEdR)."""
    p = p or default_params()
    x, q, rho, screen = _d(x).reshape(-1, 3), _d(q), _d(rho), _d(screen)
    n = q.size
    E = np.zeros(2)
    F = np.zeros((n, 3))
    phi, R, dEdR = np.zeros(n), np.zeros(n), np.zeros(n)
    lib().gbo_energy_forces(n, _p(x), _p(q), _p(rho), _p(screen), C.byref(p), _p(E), _p(F),
                            _p(phi), _p(R), _p(dEdR))
    return dict(E=E, F=F, phi=phi, R=R, dEdR=dEdR)


def energy(x, q, rho, screen, p: Optional[Params] = None) -> float:
    """E_GB + E_Coul of one molecule (Born radii recomputed)."""
    p = p or default_params()
    x, q, rho, screen = _d(x).reshape(-1, 3), _d(q), _d(rho), _d(screen)
    E = np.zeros(2)
    lib().gbo_energy_forces(q.size, _p(x), _p(q), _p(rho), _p(screen), C.byref(p), _p(E),
                            None, None, None, None)
    return float(E.sum())


def restraints(x, p: Optional[Params] = None):
    p = p or default_params()
    x = _d(x).reshape(-1, 3)
    E = np.zeros(2)
    F = np.zeros_like(x)
    lib().gbo_restraints(x.shape[0], _p(x), C.byref(p), _p(E), _p(F))
    return E, F


def batch_arrays(batch):
    """float64 copies of a synth.Batch's packed inputs: x (N,3), q, rho, screen, atom_off."""
    xyzq = batch.xyzq().astype(np.float64)
    rs = batch.rad_screen().astype(np.float64)
    return (np.ascontiguousarray(xyzq[:, :3]), np.ascontiguousarray(xyzq[:, 3]),
            np.ascontiguousarray(rs[:, 0]), np.ascontiguousarray(rs[:, 1]),
            batch.atom_off.astype(np.int64))


def batch_energy_forces(batch, p: Optional[Params] = None, with_phi: bool = False):
    """Per replica energy/forces for a whole synth.Batch (FP32 inputs cast to FP64)."""
    x, q, rho, scr, off = batch_arrays(batch)
    E = np.zeros((batch.n_rep, 2))
    F = np.zeros_like(x)
    R = np.zeros_like(q)
    phi = np.zeros_like(q) if with_phi else None
    for r in range(batch.n_rep):
        a, b = off[r], off[r + 1]
        o = energy_forces(x[a:b], q[a:b], rho[a:b], scr[a:b], p)
        E[r] = o["E"]
        F[a:b] = o["F"]
        R[a:b] = o["R"]
        if with_phi:
            phi[a:b] = o["phi"]
    return dict(E=E, F=F, R=R, phi=phi)


def mc_step(batch_off, x, q, R, tables, states, pH, E, kT, seed, step, kind,
            p: Optional[Params] = None):
    """One protonation (kind 0) or redox (kind 1) attempt per replica.

    q and states are updated in place (float64 / int32 arrays).  Returns dict
    with dG, acc, thresh (= -kT ln u), site, new_state per replica."""
    p = p or default_params()
    M = len(batch_off) - 1
    out = dict(dG=np.zeros(M), acc=np.zeros(M, np.uint8), thresh=np.zeros(M),
               site=np.zeros(M, np.int32), new_state=np.zeros(M, np.int32))
    t = tables
    lib().gbo_mc_step(
        M, _p(np.ascontiguousarray(batch_off, np.int64)), _p(x), _p(q), _p(R),
        _p(t["site_off"]), _p(t["site_kind"]), _p(t["site_nstates"]), _p(t["site_atom_off"]),
        _p(t["site_atom_idx"]), _p(t["site_state_off"]), _p(t["site_q_off"]), _p(t["q_state"]),
        _p(t["G_ref"]), _p(t["n_H"]), _p(t["n_e"]), _p(t["pKa_ref"]), _p(t["E0_ref"]),
        _p(np.ascontiguousarray(pH, np.float64)), _p(np.ascontiguousarray(E, np.float64)),
        float(kT), int(seed), int(step), int(kind), C.byref(p), _p(states), _p(out["dG"]),
        _p(out["acc"]), _p(out["thresh"]), _p(out["site"]), _p(out["new_state"]))
    return out


def mc_sweep(batch_off, x, q, R, tables, states, pH, E, kT, seed, step, kind,
             p: Optional[Params] = None):
    """Per-residue sweep (Sec. III.A.2): one attempt for every site of the
    kind, in random order.  q and states are updated in place.  Returns dict of
    per-site arrays: dG, acc (1 accepted, 0 rejected, 2 not of this kind),
    thresh (= -kT ln u), visit (position in the replica's sweep, -1 if not)."""
    p = p or default_params()
    M = len(batch_off) - 1
    S = int(tables["n_sites"])
    out = dict(dG=np.zeros(S), acc=np.zeros(S, np.uint8), thresh=np.zeros(S),
               visit=np.zeros(S, np.int32))
    t = tables
    lib().gbo_mc_sweep(
        M, _p(np.ascontiguousarray(batch_off, np.int64)), _p(x), _p(q), _p(R),
        _p(t["site_off"]), _p(t["site_kind"]), _p(t["site_nstates"]), _p(t["site_atom_off"]),
        _p(t["site_atom_idx"]), _p(t["site_state_off"]), _p(t["site_q_off"]), _p(t["q_state"]),
        _p(t["G_ref"]), _p(t["n_H"]), _p(t["n_e"]), _p(t["pKa_ref"]), _p(t["E0_ref"]),
        _p(np.ascontiguousarray(pH, np.float64)), _p(np.ascontiguousarray(E, np.float64)),
        float(kT), int(seed), int(step), int(kind), C.byref(p), _p(states), _p(out["dG"]),
        _p(out["acc"]), _p(out["thresh"]), _p(out["visit"]))
    return out


def exchange(values, rep_at_slot, n_count, dim, attempt, seed, kT, wrap=True,
             n_ladders=1, ladder_len=None, ladder_stride=None, slot_stride=1):
    """Neighbour exchange; rep_at_slot (int32) is updated in place."""
    values = _d(values)
    ladder_len = ladder_len or values.size
    ladder_stride = ladder_len if ladder_stride is None else ladder_stride
    n_count = np.ascontiguousarray(n_count, np.int32)
    delta = np.zeros(n_ladders * ladder_len)
    acc = np.zeros(n_ladders * ladder_len, np.uint8)
    lib().gbo_exchange(n_ladders, ladder_len, ladder_stride, slot_stride, _p(values),
                       _p(rep_at_slot), _p(n_count), int(dim), int(attempt), int(seed),
                       float(kT), int(wrap), _p(delta), _p(acc))
    return delta, acc


def normals(seed, r, step, atom) -> np.ndarray:
    z = np.zeros(4)
    lib().gbo_normals(int(seed), int(r), int(step), int(atom), _p(z))
    return z


def forces_all(atom_off, x, q, rho, screen, p: Optional[Params] = None):
    p = p or default_params()
    M = len(atom_off) - 1
    F = np.zeros_like(x)
    E = np.zeros((M, 4))
    lib().gbo_forces_all(M, _p(atom_off), _p(x), _p(q), _p(rho), _p(screen), C.byref(p),
                         _p(F), _p(E))
    return F, E


def md_step(atom_off, x, v, q, rho, screen, F, seed, step, p: Optional[Params] = None):
    """One BAOAB step for every replica; x, v, F updated in place. Returns E (M,4)."""
    p = p or default_params()
    M = len(atom_off) - 1
    E = np.zeros((M, 4))
    lib().gbo_md_step(M, _p(atom_off), _p(x), _p(v), _p(q), _p(rho), _p(screen), C.byref(p),
                      _p(F), int(seed), int(step), _p(E))
    return E


def site_reference_energies(batch, p: Optional[Params] = None) -> np.ndarray:
    """G_ref(s) = E_elec(q(s)) - E_elec(q(0)) for every site state at the
    starting conformation of its replica (other sites in state 0)."""
    p = p or default_params()
    x, q, rho, scr, off = batch_arrays(batch)
    t = batch.site_tables()
    G = np.zeros(t["site_state_off"][-1])
    for r in range(batch.n_rep):
        a, b = off[r], off[r + 1]
        R = born_radii(x[a:b], rho[a:b], scr[a:b], p)["R"]
        base = energy_fixed_radii(x[a:b], q[a:b], R, p).sum()
        for s in range(t["site_off"][r], t["site_off"][r + 1]):
            na = t["site_atom_off"][s + 1] - t["site_atom_off"][s]
            idx = t["site_atom_idx"][t["site_atom_off"][s]:t["site_atom_off"][s + 1]]
            for k in range(t["site_nstates"][s]):
                qq = q[a:b].copy()
                qo = t["site_q_off"][s] + k * na
                qq[idx] = t["q_state"][qo:qo + na].astype(np.float64)
                G[t["site_state_off"][s] + k] = energy_fixed_radii(x[a:b], qq, R, p).sum() - base
    return G
