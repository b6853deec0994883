"""Seeded synthetic inputs for the GB / constant-(pH,E) / E-REMD hot path.

This module only draws numbers: chain coordinates, charges, radii, titratable
site tables, potential ladders.  It contains none of the method's arithmetic
(no Born radii, no energies, no Monte Carlo), so both the FP64 oracle and the
CUDA path may consume it.

The paper's own test system (NAcMP8 with a histidine peptide, Sec. III.C) is
not available, so every workload here is a synthetic stand-in with the same
ingredients: one redox-active site (2 states, oxidation adds +1 e over the
site atoms), pH-active sites (deprotonated state 0, protonated states with
+1 e), the OBC GB model of Sec. III.D, E ladders for E-REMD (Sec. II.C, III.B).

All arrays are FP32-representable: floating values are rounded to float32 once
here, and both sides read exactly those numbers.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# Intrinsic radii (Angstrom) the synthetic atoms are drawn from, and the
# common screening factor.
RADIUS_SET = (1.2, 1.5, 1.7, 1.8, 2.0)
SCREEN = 0.8
# Reference potentials: E0_ref of the heme (-203 mV, Sec. III.C) and the two
# reference pKa values quoted for propionic acid / glutamate (Sec. III.C).
E0_REF_V = -0.203
PKA_REF_SET = (4.4, 4.85)


@dataclasses.dataclass
class Site:
    """One titratable residue: a contiguous block of atoms with per-state charges."""
    kind: int                 # 0 = pH-active, 1 = redox-active
    atoms: np.ndarray         # int32, replica-local atom indices
    q_state: np.ndarray       # float32 [n_states, n_atoms] absolute charges
    n_H: np.ndarray           # int32 [n_states] protons bound in each state
    n_e: np.ndarray           # int32 [n_states] electrons bound in each state
    pKa_ref: float            # pH sites
    E0_ref: float             # redox sites (V)

    @property
    def n_states(self) -> int:
        return int(self.q_state.shape[0])


@dataclasses.dataclass
class Replica:
    xyz: np.ndarray           # float32 [n, 3]
    q: np.ndarray             # float32 [n]   charges of the state-0 assignment
    rho: np.ndarray           # float32 [n]   intrinsic radii
    screen: np.ndarray        # float32 [n]
    sites: List[Site]

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])


@dataclasses.dataclass
class Batch:
    """Several replicas packed back to back (the layout every call consumes)."""
    replicas: List[Replica]
    pH: np.ndarray            # float64 [M]
    E: np.ndarray             # float64 [M] (V)
    name: str = ""
    # ladders used by E-REMD / pH-REMD (slot values) and the replica grid
    E_ladder: Optional[np.ndarray] = None
    pH_ladder: Optional[np.ndarray] = None

    @property
    def n_rep(self) -> int:
        return len(self.replicas)

    @property
    def atom_off(self) -> np.ndarray:
        off = np.zeros(self.n_rep + 1, dtype=np.int64)
        off[1:] = np.cumsum([r.n for r in self.replicas])
        return off

    @property
    def n_atoms(self) -> int:
        return int(self.atom_off[-1])

    def xyzq(self) -> np.ndarray:
        out = np.zeros((self.n_atoms, 4), dtype=np.float32)
        off = self.atom_off
        for k, r in enumerate(self.replicas):
            out[off[k]:off[k + 1], :3] = r.xyz
            out[off[k]:off[k + 1], 3] = r.q
        return out

    def rad_screen(self) -> np.ndarray:
        out = np.zeros((self.n_atoms, 2), dtype=np.float32)
        off = self.atom_off
        for k, r in enumerate(self.replicas):
            out[off[k]:off[k + 1], 0] = r.rho
            out[off[k]:off[k + 1], 1] = r.screen
        return out

    def pairs_per_eval(self) -> int:
        return int(sum(r.n * (r.n - 1) // 2 for r in self.replicas))

    def site_tables(self, G_ref: Optional[np.ndarray] = None) -> dict:
        """Flatten the site lists into the index/offset arrays both sides read.

        Layout (all int32 unless noted):
          site_off[M+1]          sites of replica r are [site_off[r], site_off[r+1])
          site_kind[S]           0 pH, 1 redox
          site_nstates[S]
          site_atom_off[S+1]     atoms of site s: site_atom_idx[site_atom_off[s]:...]
          site_atom_idx[...]     replica-local atom index
          site_state_off[S+1]    per-state arrays (n_H, n_e, G_ref) of site s start here
          site_q_off[S+1]        q_state of site s, state k, atom a at
                                 site_q_off[s] + k * n_atoms(s) + a   (float32)
          n_H, n_e               per state
          G_ref (float64)        per state (zeros unless given)
          pKa_ref, E0_ref        per site (float64)
        """
        site_off = [0]
        kind, nst, aoff, aidx, soff, qoff = [], [], [0], [], [0], [0]
        qs, nH, ne, pka, e0 = [], [], [], [], []
        for r in self.replicas:
            for s in r.sites:
                kind.append(s.kind)
                nst.append(s.n_states)
                aidx.extend(int(a) for a in s.atoms)
                aoff.append(len(aidx))
                nH.extend(int(v) for v in s.n_H)
                ne.extend(int(v) for v in s.n_e)
                soff.append(len(nH))
                qs.append(s.q_state.reshape(-1).astype(np.float32))
                qoff.append(qoff[-1] + s.q_state.size)
                pka.append(s.pKa_ref)
                e0.append(s.E0_ref)
            site_off.append(len(kind))
        n_states_total = soff[-1]
        if G_ref is None:
            G_ref = np.zeros(n_states_total, dtype=np.float64)
        i32 = lambda v: np.asarray(v, dtype=np.int32)
        return dict(
            n_sites=len(kind),
            site_off=i32(site_off), site_kind=i32(kind), site_nstates=i32(nst),
            site_atom_off=i32(aoff), site_atom_idx=i32(aidx),
            site_state_off=i32(soff), site_q_off=i32(qoff),
            q_state=(np.concatenate(qs) if qs else np.zeros(0, np.float32)),
            n_H=i32(nH), n_e=i32(ne),
            G_ref=np.asarray(G_ref, dtype=np.float64),
            pKa_ref=np.asarray(pka, dtype=np.float64),
            E0_ref=np.asarray(e0, dtype=np.float64),
        )

    def initial_states(self) -> np.ndarray:
        return np.zeros(sum(len(r.sites) for r in self.replicas), dtype=np.int32)


# ---------------------------------------------------------------------------
# Compact self-avoiding chain
# ---------------------------------------------------------------------------

def compact_chain(n: int, seed: int, step: float = 1.5, clash: float = 1.2,
                  density: float = 0.05, batch: int = 64) -> np.ndarray:
    """Random walk with fixed step length confined to a sphere.

    A proposed position is rejected when it lies within `clash` of any earlier
    atom or outside the sphere that holds `n` atoms at number density
    `density`.  After 1000 rejected proposals the walk backs up one atom.
    Returns float32 [n, 3].
    """
    if n <= 0:
        return np.zeros((0, 3), dtype=np.float32)
    rng = np.random.default_rng(seed)
    r_sph = (3.0 * n / (4.0 * math.pi * density)) ** (1.0 / 3.0)
    cell = step + clash
    grid: dict = {}
    pos = np.zeros((n, 3), dtype=np.float64)

    def key(p):
        return (int(math.floor(p[0] / cell)), int(math.floor(p[1] / cell)),
                int(math.floor(p[2] / cell)))

    def add(idx):
        grid.setdefault(key(pos[idx]), []).append(idx)

    def remove(idx):
        grid[key(pos[idx])].remove(idx)

    add(0)
    m = 1
    fails = 0
    while m < n:
        cur = pos[m - 1]
        cx, cy, cz = key(cur)
        near = []
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    near.extend(grid.get((cx + dx, cy + dy, cz + dz), ()))
        near_pos = pos[near] if near else np.zeros((0, 3))
        placed = False
        for _ in range(1000 // batch + 1):
            d = rng.normal(size=(batch, 3))
            d *= step / np.linalg.norm(d, axis=1, keepdims=True)
            cand = cur + d
            ok = np.einsum("ij,ij->i", cand, cand) <= r_sph * r_sph
            if near_pos.shape[0]:
                dd = cand[:, None, :] - near_pos[None, :, :]
                dmin = np.sqrt(np.einsum("ijk,ijk->ij", dd, dd)).min(axis=1)
                # the current atom is the new atom's bonded neighbour, exactly
                # `step` away, so it never trips the clash test
                ok &= dmin >= clash - 1e-9
            idx = np.flatnonzero(ok)
            if idx.size:
                pos[m] = cand[idx[0]]
                add(m)
                m += 1
                placed = True
                fails = 0
                break
        if not placed:
            fails += 1
            if m > 1:
                m -= 1
                remove(m)
            if fails > 10 * n:
                raise RuntimeError("chain generator stuck")
    return pos.astype(np.float32)


def _place_blocks(rng, n_atoms: int, sizes: List[int]) -> List[int]:
    """Non-overlapping contiguous blocks of the given sizes at random offsets."""
    free = n_atoms - sum(sizes)
    if free < 0:
        raise ValueError("sites do not fit in the chain")
    k = len(sizes)
    cuts = np.sort(rng.integers(0, free + 1, size=k))
    gaps = np.diff(np.concatenate([[0], cuts]))
    order = rng.permutation(k)
    starts = [0] * k
    at = 0
    for slot, site in enumerate(order):
        at += int(gaps[slot])
        starts[site] = at
        at += sizes[site]
    return starts


def _charge_set(rng, base: np.ndarray, n_states: int, offsets: List[int]) -> np.ndarray:
    """State 0 keeps the base charges; state k adds dq ~ N(0, 0.1) summing to offsets[k]."""
    out = np.zeros((n_states, base.size), dtype=np.float64)
    out[0] = base
    for k in range(1, n_states):
        dq = rng.normal(0.0, 0.1, size=base.size)
        dq += (offsets[k] - dq.sum()) / base.size
        out[k] = base + dq
    return out.astype(np.float32)


def make_replica(n: int, seed: int, site_specs: List[tuple]) -> Replica:
    """One synthetic molecule.

    site_specs: list of (kind, n_site_atoms, n_states).  Redox sites have two
    states (0 reduced, 1 oxidized = +1 e, one electron fewer); pH sites have
    state 0 deprotonated and states 1.. protonated tautomers (+1 e, one proton).
    """
    xyz = compact_chain(n, seed)
    rng = np.random.default_rng(seed + 1_000_003)
    q = rng.normal(0.0, 0.3, size=n)
    if n > 1:
        q -= q.mean()
    q = q.astype(np.float32)
    rho = np.asarray(RADIUS_SET, dtype=np.float32)[rng.integers(0, len(RADIUS_SET), size=n)]
    screen = np.full(n, SCREEN, dtype=np.float32)
    starts = _place_blocks(rng, n, [s[1] for s in site_specs])
    sites = []
    for (kind, na, ns), st in zip(site_specs, starts):
        atoms = np.arange(st, st + na, dtype=np.int32)
        if kind == 1:
            ns = 2
            qs = _charge_set(rng, q[atoms].astype(np.float64), 2, [0, 1])
            sites.append(Site(1, atoms, qs, np.zeros(2, np.int32),
                              np.asarray([1, 0], np.int32), 0.0, E0_REF_V))
        else:
            qs = _charge_set(rng, q[atoms].astype(np.float64), ns, [0] + [1] * (ns - 1))
            nH = np.asarray([0] + [1] * (ns - 1), np.int32)
            pka = float(PKA_REF_SET[int(rng.integers(0, len(PKA_REF_SET)))])
            sites.append(Site(0, atoms, qs, nH, np.zeros(ns, np.int32), pka, 0.0))
    # the starting charges are those of state 0 of every site
    for s in sites:
        q[s.atoms] = s.q_state[0]
    return Replica(xyz=xyz, q=q, rho=rho, screen=screen, sites=sites)


def e_ladder(n: int, center: float = E0_REF_V, half_width: float = 0.2) -> np.ndarray:
    """n potentials evenly spanning center +- half_width (V)."""
    if n == 1:
        return np.asarray([center])
    return center - half_width + 2.0 * half_width * np.arange(n) / (n - 1)


# ---------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------

def config_plain(n: int = 256, seed: int = 0) -> Batch:
    """One replica: 256-atom chain, one redox site (20 atoms), one pH site (12 atoms).
    E = E0 and pH = pKa of the pH site."""
    rep = make_replica(n, seed, [(1, 20, 2), (0, 12, 2)])
    pka = rep.sites[1].pKa_ref
    return Batch([rep], pH=np.asarray([pka]), E=np.asarray([E0_REF_V]), name=f"plain_1x{n}")


def config_eremd(n_rep: int = 8, n: int = 2048, seed: int = 0) -> Batch:
    """E-REMD: identical chains, one redox + three pH sites, E ladder E0 +- 0.2 V."""
    rep = make_replica(n, seed, [(1, 20, 2), (0, 12, 2), (0, 12, 2), (0, 12, 2)])
    lad = e_ladder(n_rep)
    reps = [rep] * n_rep
    return Batch(reps, pH=np.full(n_rep, 4.85), E=lad.copy(), name=f"eremd_{n_rep}x{n}",
                 E_ladder=lad)


def config_diff(n_rep: int = 16, n: int = 4096, seed: int = 0) -> Batch:
    """Differentiation check workload: identical chains, same sites as E-REMD."""
    b = config_eremd(n_rep, n, seed)
    b.name = f"diff_{n_rep}x{n}"
    return b


def config_uneven(n_rep: int = 64, seed: int = 3, n_min: int = 500, n_max: int = 20000) -> Batch:
    """Uneven batch: atom counts log-uniform on [n_min, n_max], 4-12 sites each."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=n_rep)).astype(int)
    reps, pH, E = [], [], []
    for k, n in enumerate(ns):
        n_sites = int(rng.integers(4, 13))
        specs = []
        for _ in range(n_sites):
            kind = 1 if rng.random() < 0.25 else 0
            na = int(rng.integers(8, 31))
            st = 2 if kind == 1 else int(rng.integers(2, 6))
            specs.append((kind, na, st))
        reps.append(make_replica(int(n), seed * 100_003 + k, specs))
        pH.append(4.85)
        E.append(E0_REF_V)
    return Batch(reps, pH=np.asarray(pH), E=np.asarray(E), name=f"uneven_{n_rep}")


def config_grid(n_pH: int = 6, n_E: int = 8, n: int = 25000, seed: int = 0) -> Batch:
    """2-D C(pH,E) grid of identical chains with 40 sites (8 redox, 32 pH)."""
    rng = np.random.default_rng(seed + 77)
    specs = [(1, int(rng.integers(8, 31)), 2) for _ in range(8)]
    specs += [(0, int(rng.integers(8, 31)), int(rng.integers(2, 5))) for _ in range(32)]
    rep = make_replica(n, seed, specs)
    pH_l = 3.5 + 0.5 * np.arange(n_pH)
    E_l = e_ladder(n_E)
    reps = [rep] * (n_pH * n_E)
    # replica index = p * n_E + e  (pH row p, E column e)
    pH = np.repeat(pH_l, n_E)
    E = np.tile(E_l, n_pH)
    return Batch(reps, pH=pH, E=E, name=f"grid_{n_pH}x{n_E}x{n}", E_ladder=E_l, pH_ladder=pH_l)


def config_cutoff(n: int = 100000, seed: int = 0) -> Batch:
    """One large chain (default 100,000 atoms) with the grid's 40-site mix, for
    GB with cutoffs: a single replica at pH 4.6 and E = E0."""
    rng = np.random.default_rng(seed + 77)
    specs = [(1, int(rng.integers(8, 31)), 2) for _ in range(8)]
    specs += [(0, int(rng.integers(8, 31)), int(rng.integers(2, 5))) for _ in range(32)]
    rep = make_replica(n, seed, specs)
    return Batch([rep], pH=np.array([4.6]), E=np.array([E0_REF_V]), name=f"cutoff_1x{n}")


def pairs_within(batch: Batch, cut: float) -> int:
    """Unordered pairs closer than `cut` in every replica (the pair terms a
    cutoff keeps), counted with a k-d tree."""
    from scipy.spatial import cKDTree
    total = 0
    for rep in batch.replicas:
        if rep.n < 2:
            continue
        t = cKDTree(rep.xyz.astype(np.float64))
        total += (int(t.count_neighbors(t, cut)) - rep.n) // 2
    return total


def random_batch(sizes: List[int], seed: int, sites: bool = True) -> Batch:
    """Small uneven batches for parity tests (ragged tails, tiny replicas)."""
    reps = []
    for k, n in enumerate(sizes):
        specs = []
        if sites and n >= 40:
            specs = [(1, min(20, n // 4), 2), (0, min(12, n // 5), 3)]
        reps.append(make_replica(int(n), seed * 1000 + k, specs))
    m = len(reps)
    return Batch(reps, pH=np.full(m, 4.85), E=np.full(m, E0_REF_V), name=f"random_{seed}")
