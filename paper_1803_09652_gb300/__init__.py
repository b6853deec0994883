"""Python binding of libgbremd (GB300 CUDA kernels behind a C ABI).

Argument marshalling only: every step of the hot path runs in the CUDA
library.  Torch supplies device memory and streams.  There is no CPU
fallback: importing works anywhere, but the first call raises if the shared
library has not been built or no CUDA device is present.

Call names follow the C ABI in include/gbremd.h:
    Context.born_radii       -> gb_born_radii
    Context.energy_forces    -> gb_energy_forces
    Context.mc_step          -> redox_ph_mc_step
    eremd_exchange           -> eremd_exchange
    Context.md_init / md_segment -> gb_md_init / gb_md_segment
    Context.md_segment_host  -> gb_md_segment_host
Replica ensembles split over processes: shard.ShardedSimulation.
"""
from __future__ import annotations

import ctypes as C
import os
import re
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(_PKG)
HEADER = os.path.join(ROOT, "include", "gbremd.h")
LIB_PATH = os.path.join(_PKG, "_build", "libgbremd.so")

KE = 332.0522173
KB = 0.0019872043
FARADAY = 23.0605478

GB_OK = 0
MAX_SITE_ATOMS = 128      # per titratable site (shared-memory rows of the MC kernel)
ERRORS = {-1: "GB_ERR_INVALID_ARG", -2: "GB_ERR_CUDA", -3: "GB_ERR_TIMEOUT",
          -4: "GB_ERR_NONFINITE", -5: "GB_ERR_NOMEM"}


class GBError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [(k, C.c_float) for k in
                ("alpha", "beta", "gamma", "offset", "eps_in", "eps_out", "rep_k", "rep_sigma",
                 "kappa", "rgbmax", "cut")]


def default_params(**kw) -> Params:
    """OBC alpha, beta, gamma = 1.0, 0.8, 4.85; offset 0.09 A; eps 1 / 78.5;
    soft repulsion off; no salt (kappa = 0); no cutoffs (rgbmax = cut = 0)."""
    d = dict(alpha=1.0, beta=0.8, gamma=4.85, offset=0.09, eps_in=1.0, eps_out=78.5,
             rep_k=0.0, rep_sigma=0.0, kappa=0.0, rgbmax=0.0, cut=0.0)
    d.update(kw)
    return Params(**d)


_P = C.c_void_p


class Sites(C.Structure):
    _fields_ = [("n_rep", C.c_int32), ("n_sites", C.c_int32), ("site_off_host", _P),
                ("site_off", _P), ("site_kind", _P), ("site_nstates", _P), ("site_atom_off", _P),
                ("site_atom_idx", _P), ("site_state_off", _P), ("site_q_off", _P), ("q_state", _P),
                ("G_ref", _P), ("n_H", _P), ("n_e", _P), ("pKa_ref", _P), ("E0_ref", _P)]


class MDState(C.Structure):
    _fields_ = [("xyzq", _P), ("vel", _P), ("force", _P), ("rad_screen", _P), ("R", _P),
                ("state", _P), ("pH", _P), ("E", _P), ("grid", _P), ("E_ladder", _P),
                ("pH_ladder", _P), ("n_E", C.c_int32), ("n_pH", C.c_int32),
                ("dt", C.c_double), ("friction", C.c_double), ("mass", C.c_double),
                ("kT", C.c_double), ("bond_k", C.c_float), ("bond_r0", C.c_float),
                ("seed", C.c_uint64), ("step", C.c_uint64), ("attempt", C.c_uint64),
                ("mc_every", C.c_int32), ("ex_every", C.c_int32), ("ex_dim", C.c_int32),
                ("wrap", C.c_int32), ("mc_mode", C.c_int32), ("ex_count", _P), ("occ_count", _P),
                ("occ_stride", C.c_int32), ("rep_base", C.c_int64)]


class MDHost(C.Structure):
    """gb_md_host: host arrays mirroring an MD state's device buffers."""
    _fields_ = [("xyzq", _P), ("vel", _P), ("force", _P), ("state", _P), ("pH", _P), ("E", _P),
                ("grid", _P), ("n_sites", C.c_int32)]


_lib = None


def exported_names() -> list:
    """Function names declared in include/gbremd.h."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(\w+)\s*\(", src, flags=re.M)))


def load(path: Optional[str] = None):
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libgbremd.so not built ({p}); run __graft_entry__.build()")
    lib = C.CDLL(p)
    i32, u64, d = C.c_int32, C.c_uint64, C.c_double
    sig = {
        "gb_ctx_create": [C.POINTER(_P), i32, _P, C.POINTER(Params), i32],
        "gb_ctx_destroy": [_P],
        "gb_sync_status": [_P, _P],
        "gb_autotune": [_P, _P, _P, _P],
        "gb_set_tiles": [_P, i32, i32],
        "gb_set_reg_cap": [_P, i32, i32],
        "gb_get_reg_caps": [_P, _P],
        "gb_get_tiles": [_P, C.POINTER(i32), C.POINTER(i32)],
        "gb_born_radii": [_P, _P, _P, _P, _P],
        "gb_energy_forces": [_P, _P, _P, _P, _P, _P, _P, _P, _P],
        "redox_ph_mc_step": [_P, C.POINTER(Sites), _P, _P, _P, _P, d, u64, u64, i32, _P, _P, _P, _P],
        "redox_ph_mc_sweep": [_P, C.POINTER(Sites), _P, _P, _P, _P, d, u64, u64, i32, _P, _P, _P, _P],
        "eremd_exchange": [i32, i32, i32, i32, _P, _P, _P, i32, u64, u64, d, i32, _P, _P, _P, _P],
        "gb_count_bound": [C.POINTER(Sites), _P, i32, _P, _P],
        "gb_md_init": [_P, C.POINTER(MDState), _P],
        "gb_md_segment": [_P, C.POINTER(MDState), C.POINTER(Sites), C.c_int64, _P],
        "gb_md_segment_host": [_P, C.POINTER(MDState), C.POINTER(Sites), C.c_int64, C.POINTER(MDHost), _P],
        "gb_set_profiling": [_P, i32],
        "gb_pass_times": [_P, C.POINTER(C.c_double)],
        "gb_set_persistent": [_P, i32],
        "gb_set_wait_limit": [_P, C.c_int64],
        "gb_autotune_md": [_P, C.POINTER(MDState), C.POINTER(Sites), C.c_int64, _P],
        "gb_persist_times": [_P, C.POINTER(C.c_double)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.gb_last_error.argtypes = [_P]
    lib.gb_last_error.restype = C.c_char_p
    if path is None:
        _lib = lib
    return lib


def _check(rc: int, ctx=None):
    if rc != GB_OK:
        msg = load().gb_last_error(ctx).decode(errors="replace")
        raise GBError(rc, msg)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class SiteTables:
    """Device copies of a site table (see synth.Batch.site_tables) plus the
    gb_sites struct that points at them."""

    def __init__(self, tables: dict, n_rep: int, device):
        import torch
        self.t = {}
        for k, v in tables.items():
            if k == "n_sites":
                continue
            a = np.asarray(v)
            dt = {np.dtype(np.int32): torch.int32, np.dtype(np.float32): torch.float32,
                  np.dtype(np.float64): torch.float64}[a.dtype]
            self.t[k] = torch.as_tensor(a.copy(), dtype=dt, device=device) if a.size else \
                torch.zeros(1, dtype=dt, device=device)
        sizes = np.diff(np.asarray(tables["site_atom_off"]))
        if sizes.size and (sizes.max() > MAX_SITE_ATOMS or sizes.min() < 1):
            raise ValueError(f"each site needs 1..{MAX_SITE_ATOMS} atoms")
        if np.any(np.asarray(tables["site_nstates"]) < 2):
            raise ValueError("each site needs at least two states")
        self.site_off_host = np.ascontiguousarray(tables["site_off"], dtype=np.int32)
        s = Sites()
        s.n_rep = n_rep
        s.n_sites = int(tables["n_sites"])
        s.site_off_host = self.site_off_host.ctypes.data
        for k in ("site_off", "site_kind", "site_nstates", "site_atom_off", "site_atom_idx",
                  "site_state_off", "site_q_off", "q_state", "G_ref", "n_H", "n_e", "pKa_ref",
                  "E0_ref"):
            setattr(s, k, self.t[k].data_ptr())
        self.struct = s

    def set_G_ref(self, G):
        import torch
        self.t["G_ref"].copy_(torch.as_tensor(np.asarray(G, np.float64)))


class Context:
    """A gb_ctx for a fixed batch layout (atom offsets)."""

    def __init__(self, atom_off: Sequence[int], params: Optional[Params] = None, device: int = 0):
        self.lib = load()
        self.atom_off = np.ascontiguousarray(atom_off, dtype=np.int64)
        self.M = int(self.atom_off.size - 1)
        self.N = int(self.atom_off[-1])
        self.params = params or default_params()
        self.device = device
        h = _P()
        rc = self.lib.gb_ctx_create(C.byref(h), self.M, self.atom_off.ctypes.data,
                                    C.byref(self.params), device)
        _check(rc, None)
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.gb_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- pair passes ----------------------------------------------------------------
    def born_radii(self, xyzq, rad, R_out=None, stream=None):
        import torch
        if R_out is None:
            R_out = torch.empty(self.N, dtype=torch.float32, device=xyzq.device)
        _check(self.lib.gb_born_radii(self.h, _ptr(xyzq), _ptr(rad), _ptr(R_out), _stream(stream)), self.h)
        return R_out

    def energy_forces(self, xyzq, rad, want=("R", "F", "E", "dEdq", "F_fixed"), stream=None):
        """Returns a dict with the requested outputs (torch tensors)."""
        import torch
        dev = xyzq.device
        out = {}
        if "R" in want:
            out["R"] = torch.empty(self.N, dtype=torch.float32, device=dev)
        if "F" in want:
            out["F"] = torch.empty((self.N, 3), dtype=torch.float32, device=dev)
        if "F_fixed" in want:
            out["F_fixed"] = torch.empty((3, self.N), dtype=torch.int64, device=dev)
        if "E" in want:
            out["E"] = torch.empty((self.M, 3), dtype=torch.float64, device=dev)
        if "dEdq" in want:
            out["dEdq"] = torch.empty(self.N, dtype=torch.float64, device=dev)
        rc = self.lib.gb_energy_forces(self.h, _ptr(xyzq), _ptr(rad), _ptr(out.get("R")),
                                       _ptr(out.get("F_fixed")), _ptr(out.get("F")),
                                       _ptr(out.get("E")), _ptr(out.get("dEdq")), _stream(stream))
        _check(rc, self.h)
        return out

    def sync_status(self, stream=None):
        _check(self.lib.gb_sync_status(self.h, _stream(stream)), self.h)

    def autotune(self, xyzq, rad, stream=None):
        _check(self.lib.gb_autotune(self.h, _ptr(xyzq), _ptr(rad), _stream(stream)), self.h)
        return self.tiles()

    def set_tiles(self, warps_per_block: int, tiles_per_task: int):
        _check(self.lib.gb_set_tiles(self.h, warps_per_block, tiles_per_task), self.h)

    def set_reg_cap(self, min_blocks: int, pass_index: int = -1):
        """Register cap (1, 3 or 4 blocks of 256 threads per SM) of one pair
        pass (0 Born, 1 energy, 2 chain) or of all three (-1)."""
        _check(self.lib.gb_set_reg_cap(self.h, int(pass_index), int(min_blocks)), self.h)

    def reg_caps(self):
        caps = (C.c_int32 * 3)()
        _check(self.lib.gb_get_reg_caps(self.h, caps), self.h)
        return tuple(caps)

    def tiles(self):
        w, t = C.c_int32(), C.c_int32()
        _check(self.lib.gb_get_tiles(self.h, C.byref(w), C.byref(t)), self.h)
        return int(w.value), int(t.value)

    # -- Monte Carlo ----------------------------------------------------------------
    def mc_step(self, sites: SiteTables, xyzq, R, pH, E, kT, seed, step, kind, state,
                dG_out=None, acc_out=None, stream=None):
        import torch
        dev = xyzq.device
        if dG_out is None:
            dG_out = torch.empty(self.M, dtype=torch.float64, device=dev)
        if acc_out is None:
            acc_out = torch.empty(self.M, dtype=torch.uint8, device=dev)
        rc = self.lib.redox_ph_mc_step(self.h, C.byref(sites.struct), _ptr(xyzq), _ptr(R), _ptr(pH),
                                       _ptr(E), float(kT), int(seed), int(step), int(kind),
                                       _ptr(state), _ptr(dG_out), _ptr(acc_out), _stream(stream))
        _check(rc, self.h)
        return dG_out, acc_out

    def mc_sweep(self, sites: SiteTables, xyzq, R, pH, E, kT, seed, step, kind, state,
                 dG_out=None, acc_out=None, stream=None):
        """Per-residue sweep: one attempt for every site of the kind (per-site
        outputs; acc 2 marks sites of the other kind)."""
        import torch
        dev = xyzq.device
        S = sites.struct.n_sites
        if dG_out is None:
            dG_out = torch.empty(max(S, 1), dtype=torch.float64, device=dev)
        if acc_out is None:
            acc_out = torch.empty(max(S, 1), dtype=torch.uint8, device=dev)
        rc = self.lib.redox_ph_mc_sweep(self.h, C.byref(sites.struct), _ptr(xyzq), _ptr(R), _ptr(pH),
                                        _ptr(E), float(kT), int(seed), int(step), int(kind),
                                        _ptr(state), _ptr(dG_out), _ptr(acc_out), _stream(stream))
        _check(rc, self.h)
        return dG_out[:S], acc_out[:S]

    # -- MD ---------------------------------------------------------------------------
    def md_init(self, st: MDState, stream=None):
        _check(self.lib.gb_md_init(self.h, C.byref(st), _stream(stream)), self.h)

    def set_profiling(self, on: bool):
        _check(self.lib.gb_set_profiling(self.h, 1 if on else 0), self.h)

    def pass_times(self):
        """Mean ms of the Born, energy and chain passes over the last MD block."""
        arr = (C.c_double * 3)()
        _check(self.lib.gb_pass_times(self.h, arr), self.h)
        return [float(v) for v in arr]

    def set_persistent(self, on: bool):
        _check(self.lib.gb_set_persistent(self.h, 1 if on else 0), self.h)

    def autotune_md(self, st: MDState, sites: Optional[SiteTables], trial_steps: int = 100, stream=None):
        """Register caps tuned on MD segments of trial_steps steps (state restored)."""
        sp = C.byref(sites.struct) if sites is not None else None
        _check(self.lib.gb_autotune_md(self.h, C.byref(st), sp, int(trial_steps), _stream(stream)), self.h)
        return self.reg_caps()

    def set_wait_limit(self, polls: int):
        """Polls before a persistent-kernel dependency wait gives up (0: default)."""
        _check(self.lib.gb_set_wait_limit(self.h, int(polls)), self.h)

    def persist_times(self):
        """(ms per MD step, ms per launch, steps per launch) of the persistent
        launches of the last MD block (profiling on)."""
        arr = (C.c_double * 3)()
        _check(self.lib.gb_persist_times(self.h, arr), self.h)
        return [float(v) for v in arr]

    def md_segment(self, st: MDState, sites: Optional[SiteTables], nsteps: int, stream=None):
        sp = C.byref(sites.struct) if sites is not None else None
        _check(self.lib.gb_md_segment(self.h, C.byref(st), sp, int(nsteps), _stream(stream)), self.h)

    def md_segment_host(self, st: MDState, sites: Optional[SiteTables], nsteps: int, host: dict,
                        stream=None):
        """gb_md_segment_host: host tensors (CPU, ideally pinned) keyed by
        xyzq, vel, force, state, pH, E, grid are copied to st's device
        buffers, nsteps MD steps run, and the new state is copied back into
        them before the call returns."""
        h = MDHost()
        for k in ("xyzq", "vel", "force", "state", "pH", "E", "grid"):
            t = host.get(k)
            if t is not None:
                if t.is_cuda or not t.is_contiguous():
                    raise ValueError(f"{k}: a contiguous host tensor is required")
                setattr(h, k, t.data_ptr())
        if host.get("state") is not None:
            h.n_sites = int(host["state"].numel())
        sp = C.byref(sites.struct) if sites is not None else None
        _check(self.lib.gb_md_segment_host(self.h, C.byref(st), sp, int(nsteps), C.byref(h), _stream(stream)),
               self.h)


class Simulation:
    """Batched C(pH,E)-REMD MD driver: the device state of a batch and the
    gb_md_state that points at it.  run(n) advances n BAOAB MD steps, with the
    Monte Carlo attempts and exchanges they contain, through gb_md_segment
    (one captured graph per block of steps).

    xyzq float32 [N, 4] (x, y, z, q) and rad_screen float32 [N, 2] (rho, S)
    are copied to the device.  sites: a site table dict (the layout
    SiteTables takes) or None.  pH, E: float64 [M] per replica.  E_ladder,
    pH_ladder: the exchange grid's ladders, replica p * n_E + e starting at pH
    row p and E column e; exchanges run when n_E * n_pH == M > 1, along E
    (ex_dim 0), pH (1) or alternating (2, the default on a 2-D grid).
    Attributes xyzq, vel, force, R, state, pH, E, grid and ex_count (the
    exchange counters of gb_md_state) are the live device tensors.
    occupancy=True adds occ (int64 [M, states per replica]), the state
    occupancy counts of gb_md_state.occ_count: per grid slot (per replica
    without exchanges), how many Monte Carlo halts found a site in each
    state; occupancy() turns them into fractions.  rep_base:
    global index of replica 0 in the random-number counters (a part of an
    ensemble split over processes; shard.ShardedSimulation sets it)."""

    def __init__(self, atom_off, xyzq, rad_screen, params: Optional[Params] = None, sites=None, pH=None,
                 E=None, E_ladder=None, pH_ladder=None, *, dt=0.002, friction=10.0, mass=12.0,
                 temperature=300.0, bond_k=300.0, bond_r0=1.5, seed=0, mc_every=10, ex_every=100,
                 ex_dim=None, wrap=True, mc_mode=0, device=0, rep_base=0, occupancy=False):
        import torch
        dev = torch.device("cuda", device)
        self.ctx = Context(atom_off, params, device)
        M, N = self.ctx.M, self.ctx.N
        f32 = dict(dtype=torch.float32, device=dev)
        f64 = dict(dtype=torch.float64, device=dev)
        self.xyzq = torch.as_tensor(xyzq, **f32).reshape(N, 4).clone()
        self.rad = torch.as_tensor(rad_screen, **f32).reshape(N, 2).clone()
        self.vel = torch.zeros((N, 4), **f32)
        self.force = torch.zeros((N, 4), **f32)
        self.R = torch.zeros(N, **f32)
        self.pH = torch.as_tensor(np.full(M, 7.0) if pH is None else pH, **f64).clone()
        self.E = torch.as_tensor(np.zeros(M) if E is None else E, **f64).clone()
        E_lad = np.asarray(self.E.cpu().numpy()[:1] if E_ladder is None else E_ladder, np.float64)
        pH_lad = np.asarray(self.pH.cpu().numpy()[:1] if pH_ladder is None else pH_ladder, np.float64)
        self.E_ladder = torch.as_tensor(E_lad, **f64)
        self.pH_ladder = torch.as_tensor(pH_lad, **f64)
        self.grid = torch.arange(M, dtype=torch.int32, device=dev)
        self.ex_count = torch.zeros((2, 2, M), dtype=torch.int64, device=dev)
        self.sites = SiteTables(sites, M, dev) if sites is not None else None
        n_sites = int(sites["n_sites"]) if sites is not None else 0
        self.state = torch.zeros(max(n_sites, 1), dtype=torch.int32, device=dev)
        n_E, n_pH = len(E_lad), len(pH_lad)
        ladder = n_E * n_pH == M and M > 1
        st = MDState()
        st.xyzq, st.vel, st.force = self.xyzq.data_ptr(), self.vel.data_ptr(), self.force.data_ptr()
        st.rad_screen, st.R = self.rad.data_ptr(), self.R.data_ptr()
        st.state, st.pH, st.E = self.state.data_ptr(), self.pH.data_ptr(), self.E.data_ptr()
        st.grid, st.E_ladder, st.pH_ladder = self.grid.data_ptr(), self.E_ladder.data_ptr(), self.pH_ladder.data_ptr()
        st.n_E, st.n_pH = (n_E, n_pH) if ladder else (M, 1)
        st.dt, st.friction, st.mass, st.kT = dt, friction, mass, KB * temperature
        st.bond_k, st.bond_r0 = bond_k, bond_r0
        st.seed, st.step, st.attempt = seed, 0, 0
        st.mc_every = mc_every if self.sites is not None else 0
        st.ex_every = ex_every if (ladder and self.sites is not None) else 0
        st.ex_dim = (2 if n_pH > 1 else 0) if ex_dim is None else ex_dim
        st.wrap, st.mc_mode = 1 if wrap else 0, mc_mode
        st.ex_count = self.ex_count.data_ptr()
        st.rep_base = int(rep_base)
        self.occ = None
        if occupancy:
            if sites is None:
                raise ValueError("occupancy counts need site tables")
            so, sso = np.asarray(sites["site_off"]), np.asarray(sites["site_state_off"])
            per = np.diff(sso[so])
            if len(set(per.tolist())) != 1:
                raise ValueError("occupancy counts need one site layout in every replica")
            self.occ = torch.zeros((M, int(per[0])), dtype=torch.int64, device=dev)
            st.occ_count, st.occ_stride = self.occ.data_ptr(), int(per[0])
        self.st = st
        self.ctx.md_init(st)

    @property
    def step(self) -> int:
        return int(self.st.step)

    def run(self, nsteps: int, stream=None) -> "Simulation":
        self.ctx.md_segment(self.st, self.sites, int(nsteps), stream)
        return self

    def sync(self, stream=None):
        """Waits for the work enqueued so far; raises on a recorded device error."""
        self.ctx.sync_status(stream)

    def energies(self):
        """[M, 3] float64 (GB, Coulomb, soft repulsion) at the current coordinates."""
        return self.ctx.energy_forces(self.xyzq, self.rad, want=("E",))["E"]

    def occupancy(self) -> np.ndarray:
        """Fraction of the Monte Carlo halts so far that found each site state,
        per grid slot: float64 [M, states per replica], columns in the order
        of the replica's site states (site_state_off); NaN before the first
        halt.  With one site per kind this is the reduced / protonated fraction
        at each slot's E and pH (Eq. 3, Eq. 9)."""
        if self.occ is None:
            raise ValueError("the simulation was created without occupancy=True")
        occ = self.occ.cpu().numpy().astype(np.float64)
        so = self.sites.site_off_host
        n_site = int(so[1] - so[0])
        halts = occ.sum(axis=1, keepdims=True) / max(n_site, 1)
        with np.errstate(invalid="ignore", divide="ignore"):
            return occ / halts

    # -- checkpoint / resume ------------------------------------------------------------
    CHECKPOINT_ARRAYS = ("xyzq", "vel", "state", "grid", "pH", "E", "ex_count", "occ")

    def checkpoint(self, stream=None) -> dict:
        """Host copy of the dynamic state: coordinates and charges, velocities,
        site states, the exchange grid, per-replica pH and E, and the step,
        attempt and seed counters.  Every random number of the driver is
        drawn from Philox with counters (replica, step or attempt, purpose),
        and gb_md_init recomputes the forces at the saved coordinates with the
        same kernels a step ends with, so restore() followed by run(n) gives
        bit for bit what this simulation would have given by running on."""
        import torch
        if stream is not None:
            stream.synchronize()
        torch.cuda.synchronize(self.xyzq.device)
        ck = {k: getattr(self, k).cpu().numpy().copy() for k in self.CHECKPOINT_ARRAYS
              if getattr(self, k) is not None}
        ck["step"] = int(self.st.step)
        ck["attempt"] = int(self.st.attempt)
        ck["seed"] = int(self.st.seed)
        return ck

    def restore(self, ck: dict, stream=None) -> "Simulation":
        """Loads a checkpoint() of a simulation built with the same arguments
        (batch layout, parameters, sites, ladders) and re-initialises the
        forces (gb_md_init)."""
        import torch
        for k in self.CHECKPOINT_ARRAYS:
            dst = getattr(self, k)
            if dst is None:
                continue
            src = np.asarray(ck[k])
            if tuple(src.shape) != tuple(dst.shape):
                raise ValueError(f"checkpoint {k} has shape {src.shape}, the simulation {tuple(dst.shape)}")
            dst.copy_(torch.as_tensor(src, dtype=dst.dtype))
        self.st.step = int(ck["step"])
        self.st.attempt = int(ck["attempt"])
        self.st.seed = int(ck["seed"])
        self.ctx.md_init(self.st, stream)
        return self


    # -- metrics -------------------------------------------------------------------------
    def exchange_stats(self) -> dict:
        """Attempts, acceptances and acceptance ratio of every neighbour pair
        of the exchange grid so far.  Keys "E" and "pH": arrays
        [n_pH, n_E] indexed by the pair's first slot (pH row, E column); the
        pair is (column e, e + 1) along E and (row p, p + 1) along pH, the
        wrap pair sitting at the last column (row).  Ratios are NaN where
        nothing was attempted."""
        return exchange_ratios(self.ex_count.cpu().numpy(), int(self.st.n_pH), int(self.st.n_E))

    def metrics(self) -> dict:
        """One record of the run's observables at the current step (host
        values, JSON-serialisable): step and exchange attempt, per replica its
        E, pH, energies (GB, Coulomb, soft repulsion) and the states of its
        sites, the exchange grid, and the exchange counters."""
        import torch
        E_tot = self.energies()
        torch.cuda.synchronize(self.xyzq.device)
        M = self.ctx.M
        rec = {"step": self.step, "attempt": int(self.st.attempt),
               "E": self.E.cpu().tolist(), "pH": self.pH.cpu().tolist(),
               "energies": E_tot.cpu().tolist(), "grid": self.grid.cpu().tolist(),
               "ex_attempts": self.ex_count[:, 0].cpu().tolist(),
               "ex_accepted": self.ex_count[:, 1].cpu().tolist()}
        if self.sites is not None:
            off = self.sites.site_off_host
            st = self.state.cpu().numpy()
            rec["states"] = [st[off[r]:off[r + 1]].tolist() for r in range(M)]
        return rec

    def log_metrics(self, path: str) -> dict:
        """Appends metrics() to a JSON-lines file and returns the record."""
        import json
        rec = self.metrics()
        with open(path, "a") as f:
            f.write(json.dumps(rec) + "\n")
        return rec


def exchange_ratios(ex_count, n_pH: int, n_E: int) -> dict:
    """Host view of gb_md_state.ex_count (int64 [2][2][n_pH * n_E]): for
    "E" (direction 0) and "pH" (direction 1) the attempts, acceptances and
    acceptance ratio (NaN where nothing was attempted) of every neighbour
    pair, as [n_pH, n_E] arrays indexed by the pair's first slot."""
    c = np.asarray(ex_count).reshape(2, 2, n_pH * n_E)
    out = {}
    for d, name in ((0, "E"), (1, "pH")):
        att = c[d, 0].reshape(n_pH, n_E)
        acc = c[d, 1].reshape(n_pH, n_E)
        ratio = np.full(att.shape, np.nan)
        np.divide(acc, att, out=ratio, where=att > 0)
        out[name] = {"attempts": att, "accepted": acc, "ratio": ratio}
    return out


def save_checkpoint(path: str, ck: dict) -> None:
    """Writes a Simulation.checkpoint() to an .npz file (no pickled objects)."""
    arrays = {k: np.asarray(v) for k, v in ck.items()}
    np.savez(path, **arrays)


def load_checkpoint(path: str) -> dict:
    """Reads a file written by save_checkpoint."""
    with np.load(path, allow_pickle=False) as f:
        ck = {k: f[k].copy() for k in f.files}
    for k in ("step", "attempt", "seed"):
        ck[k] = int(ck[k])
    return ck


def eremd_exchange(values, rep_at_slot, n_count, dim, attempt, seed, kT, wrap=True,
                   n_ladders=1, ladder_len=None, ladder_stride=None, slot_stride=1,
                   value_of_rep=None, delta_out=None, acc_out=None, stream=None):
    import torch
    lib = load()
    ladder_len = ladder_len or int(values.numel())
    ladder_stride = ladder_len if ladder_stride is None else ladder_stride
    dev = values.device
    if delta_out is None:
        delta_out = torch.empty(n_ladders * ladder_len, dtype=torch.float64, device=dev)
    if acc_out is None:
        acc_out = torch.empty(n_ladders * ladder_len, dtype=torch.uint8, device=dev)
    rc = lib.eremd_exchange(n_ladders, ladder_len, ladder_stride, slot_stride, _ptr(values),
                            _ptr(rep_at_slot), _ptr(n_count), int(dim), int(attempt), int(seed),
                            float(kT), int(wrap), _ptr(value_of_rep), _ptr(delta_out),
                            _ptr(acc_out), _stream(stream))
    _check(rc, None)
    return delta_out, acc_out


def count_bound(sites: SiteTables, state, kind, out=None, stream=None):
    import torch
    if out is None:
        out = torch.empty(sites.struct.n_rep, dtype=torch.int32, device=state.device)
    _check(load().gb_count_bound(C.byref(sites.struct), _ptr(state), int(kind), _ptr(out),
                                 _stream(stream)), None)
    return out


class GBEnergy:
    """torch.autograd.Function over gb_energy_forces: E[M] = E_GB + E_Coul per
    replica from (xyzq) with backward dE/dx = -F and dE/dq = phi."""

    @staticmethod
    def apply(ctx_obj: "Context", xyzq, rad):
        return _GBEnergyFn.apply(xyzq, rad, ctx_obj)


def _make_fn():
    import torch

    class Fn(torch.autograd.Function):
        @staticmethod
        def forward(fctx, xyzq, rad, gctx):
            out = gctx.energy_forces(xyzq.detach().contiguous(), rad.contiguous(),
                                     want=("F", "E", "dEdq"))
            fctx.save_for_backward(out["F"], out["dEdq"])
            fctx.atom_off = torch.as_tensor(gctx.atom_off, device=xyzq.device)
            return (out["E"][:, 0] + out["E"][:, 1])

        @staticmethod
        def backward(fctx, g):
            F, phi = fctx.saved_tensors
            off = fctx.atom_off
            counts = (off[1:] - off[:-1])
            g_atom = torch.repeat_interleave(g.to(torch.float64), counts)
            grad = torch.zeros((F.shape[0], 4), dtype=torch.float32, device=F.device)
            grad[:, :3] = (-F.double() * g_atom[:, None]).float()
            grad[:, 3] = (phi * g_atom).float()
            return grad, None, None

    return Fn


class _Lazy:
    _fn = None

    def __getattr__(self, k):
        if _Lazy._fn is None:
            _Lazy._fn = _make_fn()
        return getattr(_Lazy._fn, k)


_GBEnergyFn = _Lazy()
