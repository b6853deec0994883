// O(N) and O(sites x N) kernels: Born-radius transform, self terms and
// readout of the fixed-point accumulators, BAOAB half steps, Monte Carlo state
// changes (Eq. 8, 9), replica exchange (Eq. 14, 15).
#include <cmath>

#include "atoms_impl.cuh"

namespace gbk {

__device__ __forceinline__ double block_sum_d(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
    return t;  // valid in thread 0
}

// --- Born radii: I -> psi -> R (OBC), see born_finalize_atom ----------------------
__global__ void k_born_finalize(AtomArgs A, float* R_out) {
    pdl_enter();
    const int r = blockIdx.y;
    const int64_t base = A.atom_off[r];
    const int n = (int)(A.atom_off[r + 1] - base);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    born_finalize_atom(A, base + i, R_out);
}

// --- self terms, dE/dR -> chain factor, dE/dq readout ----------------------------
// With bond_k != 0 (MD) the chain-bond forces k (r - r0)^2 join the force
// accumulators here, while the positions are fixed between the passes.
__global__ void k_energy_finalize(AtomArgs A, int want_energy, double* phi_out, float bond_k, float bond_r0) {
    pdl_enter();
    __shared__ double sh[32];
    const int r = blockIdx.y;
    const int64_t base = A.atom_off[r];
    const int n = (int)(A.atom_off[r + 1] - base);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double eself = 0.0;
    if (i < n) {
        const int64_t g = base + i;
        double R;
        const double q = chain_factor_atom(A, g, &R);
        const double tE = gb_screen(A.kc, A.ke_out, A.kappa, R).x;
        eself = -0.5 * tE * q * q / R;
        if (phi_out) {
            phi_out[g] = unfix(A.phi_acc[g]) - tE * q / R;
            A.phi_acc[g] = 0;
        }
        if (bond_k != 0.0f) {
            const float3 fb = bond_force_kr(bond_k, bond_r0, A.xyzq, base, i, n);
            A.F_acc[g] = __ldcg(&A.F_acc[g]) + (u64)fix(fb.x);
            A.F_acc[A.N + g] = __ldcg(&A.F_acc[A.N + g]) + (u64)fix(fb.y);
            A.F_acc[2 * A.N + g] = __ldcg(&A.F_acc[2 * A.N + g]) + (u64)fix(fb.z);
        }
    }
    if (want_energy) {
        if (blockIdx.x * blockDim.x >= (unsigned)n) return;
        const double t = block_sum_d(eself, sh);
        if (threadIdx.x == 0) red_add(&A.E_acc[4 * r + 0], fix_d(t));
    }
}

// --- readout: int64 forces -> outputs; energies -> FP64; clear accumulators -------
__global__ void k_forces_out(AtomArgs A, int64_t* F_fixed, float* F_out, double* E_out) {
    pdl_enter();
    const int r = blockIdx.y;
    const int64_t base = A.atom_off[r];
    const int n = (int)(A.atom_off[r + 1] - base);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x < 3) {
        if (E_out) E_out[3 * r + threadIdx.x] = unfix(A.E_acc[4 * r + threadIdx.x]);
        A.E_acc[4 * r + threadIdx.x] = 0;
    }
    if (i >= n) return;
    const int64_t g = base + i;
    const u64 fx = A.F_acc[g], fy = A.F_acc[A.N + g], fz = A.F_acc[2 * A.N + g];
    A.F_acc[g] = 0;
    A.F_acc[A.N + g] = 0;
    A.F_acc[2 * A.N + g] = 0;
    if (F_fixed) {
        F_fixed[g] = (long long)fx;
        F_fixed[A.N + g] = (long long)fy;
        F_fixed[2 * A.N + g] = (long long)fz;
    }
    if (F_out) {
        F_out[3 * g + 0] = (float)unfix(fx);
        F_out[3 * g + 1] = (float)unfix(fy);
        F_out[3 * g + 2] = (float)unfix(fz);
    }
}

// --- Langevin BAOAB ---------------------------------------------------------------
// One launch between two force evaluations.  MD_CLOSE: the total force of the
// evaluation just finished (pair accumulators, bonds included; cleared here)
// becomes the stored force, and with MD_KICK the closing half kick B is
// applied.  MD_OPEN: B A O A of the next step (step counter base + step_in_block
// + 1) with the stored or just-closed force, then the bounding boxes of the
// tiles at the new positions for the far-block test of the pair passes.
__global__ void k_md_step(AtomArgs A, MDArgs m, float4* boxes, const int* tile_off, int step_in_block, int mode) {
    pdl_enter();
    const int r = blockIdx.y;
    const int64_t base = A.atom_off[r];
    const int n = (int)(A.atom_off[r + 1] - base);
    if ((int)(blockIdx.x * blockDim.x) >= n) return;      // whole block past this replica
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    float4 x = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (valid) {
        const int64_t g = base + i;
        float4 v = m.vel[g];
        float4 f;
        if (mode & MD_CLOSE) {
            f = make_float4((float)unfix(__ldcg(&A.F_acc[g])), (float)unfix(__ldcg(&A.F_acc[A.N + g])),
                            (float)unfix(__ldcg(&A.F_acc[2 * A.N + g])), 0.0f);
            A.F_acc[g] = 0;
            A.F_acc[A.N + g] = 0;
            A.F_acc[2 * A.N + g] = 0;
            m.force[g] = f;
            if (mode & MD_KICK) {
                v.x = fmaf(m.h * m.inv_m, f.x, v.x);
                v.y = fmaf(m.h * m.inv_m, f.y, v.y);
                v.z = fmaf(m.h * m.inv_m, f.z, v.z);
            }
        } else {
            f = m.force[g];
        }
        if (mode & MD_OPEN) {
            const u64 step = m.ctr[0] + (u64)step_in_block + 1;
            x = m.xyzq[g];
            baoab_first(m, x, v, f, md_normals(m.seed, m.rep_base + (u64)r, step, (u64)i));
            m.xyzq[g] = x;
        }
        m.vel[g] = v;
    }
    if ((mode & MD_OPEN) && boxes) {
        const int t = i >> 5;                              // warp-uniform tile of the replica
        if (32 * t < n) {
            float a = 0.0f, sc = 0.0f;
            if (valid) {
                const float2 rs = A.rad[base + i];
                a = rs.x - A.offset;
                sc = rs.y * a;
            }
            tile_box_store(boxes, (int64_t)tile_off[r] + t, valid, x.x, x.y, x.z, a, sc, x.w, A.err);
        }
    }
}

__global__ void k_set_counters(u64* ctr, u64 step, u64 attempt) {
    pdl_enter();
    ctr[0] = step;
    ctr[1] = attempt;
}

__global__ void k_advance_counters(u64* ctr, u64 steps, u64 attempts) {
    pdl_enter();
    ctr[0] += steps;
    ctr[1] += attempts;
}

// --- Monte Carlo state change at fixed Born radii (Eq. 8, Eq. 9) -------------------
// The energy change of a site's charge change dq is, exactly (E is quadratic
// in q at fixed R),
//   dE = sum_k dq_k phi_k + 1/2 sum_{k,l} dq_k dq_l A_kl
// with the site rows
//   phi_k = sum_{j != k} q_j (k_c / r_kj - tau k_e / f_kj) - tau k_e q_k / R_k
// and the site-site block A_kl = k_c / r_kl - tau k_e / f_kl (k != l),
// A_kk = -tau k_e / R_k.  Terms in FP32, sums and the decision in FP64.
// Stage 1 (k_mc_rows) splits each replica's atoms into MC_CHUNK-atom slices,
// one block per (slice, replica), and stores per-slice partial rows; stage 2
// (k_mc_decide) adds the slices in a fixed order, adds the site block, and
// takes the Metropolis decision -- deterministic, and wide enough to fill the
// GPU for a handful of replicas.

struct MCPick {
    int site, cur, nxt;
    u64 w2;
};

// Site and state proposal of replica r (Sec. III.A, III.A.1).
__device__ __forceinline__ MCPick mc_pick(const MCArgs& A, int r) {
    const u64 step = (A.ctr ? A.ctr[0] : 0) + A.step;
    const Philox4 w = philox4x64(A.rep_base + (u64)r, step, 1 + (u64)A.kind, 0, A.seed, 0);
    MCPick pk;
    pk.site = -1;
    pk.cur = pk.nxt = 0;
    pk.w2 = w.w[2];
    int n_kind = 0;
    for (int s = A.site_off[r]; s < A.site_off[r + 1]; ++s) n_kind += (A.site_kind[s] == A.kind);
    if (n_kind == 0) return pk;
    const int want = pick_int(w.w[0], n_kind);
    for (int s = A.site_off[r], c = 0; s < A.site_off[r + 1]; ++s)
        if (A.site_kind[s] == A.kind) {
            if (c == want) { pk.site = s; break; }
            ++c;
        }
    pk.cur = A.state[pk.site];
    const int k = pick_int(w.w[1], A.site_nstates[pk.site] - 1);
    pk.nxt = (k < pk.cur) ? k : k + 1;
    return pk;
}

// Site table checks of an attempt, by the whole block before any access
// through the table: every atom index of the site inside the replica
// (0 <= idx < n), at least two states, the current state among them.  On a
// violation the attempt is skipped and GB_ERR_INVALID_ARG recorded.
__device__ bool mc_site_ok(const MCArgs& A, const MCPick& pk, int a0, int na, int n) {
    bool bad = false;
    for (int k = threadIdx.x; k < na; k += blockDim.x) {
        const int idx = A.site_atom_idx[a0 + k];
        bad |= idx < 0 || idx >= n;
    }
    if (threadIdx.x == 0) {
        const int ns = A.site_nstates[pk.site];
        bad |= ns < 2 || pk.cur < 0 || pk.cur >= ns;
    }
    bad = __syncthreads_or(bad);
    if (bad && threadIdx.x == 0 && A.err) atomicCAS(A.err, 0, GB_ERR_INVALID_ARG);
    return !bad;
}

// (R, 1/(2R)) of atom g, from whichever radius buffer the caller gave.
__device__ __forceinline__ float2 mc_Rh(const MCArgs& A, int64_t g) {
    if (A.R) {
        const float R = A.R[g];
        return make_float2(R, 0.5f * __frcp_rn(R));
    }
    return A.Rh[g];
}

// A_kj = k_c / r - tE(f) / f, tE the (screened) solvent factor of gb_screen;
// 0 beyond the pair cutoff (cut2 = cut^2 > 0), as in the energy pass.
__device__ __forceinline__ float mc_pair_term(float4 xk, float2 Rk, float4 xj, float2 Rj, float tke, float kc,
                                              float ke_out, float kappa, float cut2) {
    const float dx = xj.x - xk.x, dy = xj.y - xk.y, dz = xj.z - xk.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (cut2 > 0.0f && r2 > cut2) return 0.0f;
    const float e = __expf(-r2 * (Rk.y * Rj.y));          // exp(-r^2 / (4 R_k R_j))
    const float f2 = fmaf(Rk.x * Rj.x, e, r2);
    const float finv = rsqrtf(f2);
    const float t = (kappa == 0.0f) ? tke : kc - ke_out * __expf(-kappa * f2 * finv);
    return kc * rsqrtf(r2) - t * finv;
}
// A_kk = -tE(R_k) / R_k
__device__ __forceinline__ float mc_self_term(float Rk, float tke, float kc, float ke_out, float kappa) {
    const float t = (kappa == 0.0f) ? tke : kc - ke_out * __expf(-kappa * Rk);
    return -t / Rk;
}

__global__ void __launch_bounds__(256) k_mc_rows(MCArgs A) {
    pdl_enter();
    __shared__ MCPick s_pick;
    const int r = blockIdx.y, part = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    if (tid == 0) s_pick = mc_pick(A, r);
    __syncthreads();
    const int site = s_pick.site;
    if (site < 0) return;
    const int a0 = A.site_atom_off[site];
    const int na = A.site_atom_off[site + 1] - a0;
    if (na > MC_MAX_SITE_ATOMS || na < 1) return;
    const int64_t base = A.atom_off[r];
    const int n = (int)(A.atom_off[r + 1] - base);
    if (!mc_site_ok(A, s_pick, a0, na, n)) return;
    const int j0 = part * MC_CHUNK, j1 = min(n, j0 + MC_CHUNK);
    const float tke = (float)A.tau_ke, kc = (float)A.kc, keo = (float)A.ke_out, kap = (float)A.kappa;
    double* out = A.phi_part + ((size_t)r * A.n_parts + part) * MC_MAX_SITE_ATOMS;
    for (int k = wid; k < na; k += nw) {
        const int lk = A.site_atom_idx[a0 + k];
        const int64_t gk = base + lk;
        const float4 xk = A.xyzq[gk];
        const float2 Rk = mc_Rh(A, gk);
        double acc = 0.0;
        for (int j = j0 + lane; j < j1; j += 32) {
            const int64_t gj = base + j;
            const float4 xj = A.xyzq[gj];
            const float term = (j == lk) ? mc_self_term(Rk.x, tke, kc, keo, kap) : mc_pair_term(xk, Rk, xj, mc_Rh(A, gj), tke, kc, keo, kap, A.cut2);
            acc += (double)(xj.w * term);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) out[k] = acc;
    }
}

__global__ void __launch_bounds__(256) k_mc_decide(MCArgs A) {
    pdl_enter();
    __shared__ MCPick s_pick;
    __shared__ double s_phi[MC_MAX_SITE_ATOMS];
    __shared__ double s_dq[MC_MAX_SITE_ATOMS];
    __shared__ double sh[32];
    __shared__ int s_acc;
    const int r = blockIdx.x;
    const int tid = threadIdx.x;
    if (tid == 0) s_pick = mc_pick(A, r);
    __syncthreads();
    const int site = s_pick.site;
    const int a0 = site >= 0 ? A.site_atom_off[site] : 0;
    const int na = site >= 0 ? A.site_atom_off[site + 1] - a0 : 0;
    const int64_t base = A.atom_off[r];
    const int n = (int)(A.atom_off[r + 1] - base);
    bool usable = site >= 0 && na <= MC_MAX_SITE_ATOMS && na >= 1;
    if (usable) usable = mc_site_ok(A, s_pick, a0, na, n);
    if (!usable) {
        if (tid == 0) {
            if (A.dG_out) A.dG_out[r] = site < 0 ? 0.0 : __longlong_as_double(0x7ff8000000000000LL);
            if (A.acc_out) A.acc_out[r] = 0;
            if (site >= 0 && (na > MC_MAX_SITE_ATOMS || na < 1) && A.err) atomicCAS(A.err, 0, GB_ERR_INVALID_ARG);
        }
        return;
    }
    const int n_parts_r = (n + MC_CHUNK - 1) / MC_CHUNK;
    const int qo = A.site_q_off[site] + s_pick.nxt * na;
    for (int k = tid; k < na; k += blockDim.x) {
        const int64_t gk = base + A.site_atom_idx[a0 + k];
        s_dq[k] = (double)A.q_state[qo + k] - (double)A.xyzq[gk].w;
        double phi = 0.0;
        for (int p = 0; p < n_parts_r; ++p)
            phi += A.phi_part[((size_t)r * A.n_parts + p) * MC_MAX_SITE_ATOMS + k];
        s_phi[k] = phi;
    }
    __syncthreads();
    const float tke = (float)A.tau_ke, kc = (float)A.kc, keo = (float)A.ke_out, kap = (float)A.kappa;
    double part = 0.0;
    for (int t = tid; t < na * na; t += blockDim.x) {
        const int k = t / na, l = t % na;
        const int64_t gk = base + A.site_atom_idx[a0 + k];
        const float2 Rk = mc_Rh(A, gk);
        float Akl;
        if (k == l) {
            Akl = mc_self_term(Rk.x, tke, kc, keo, kap);
            part += s_dq[k] * s_phi[k];
        } else {
            const int64_t gl = base + A.site_atom_idx[a0 + l];
            Akl = mc_pair_term(A.xyzq[gk], Rk, A.xyzq[gl], mc_Rh(A, gl), tke, kc, keo, kap, A.cut2);
        }
        part += 0.5 * s_dq[k] * s_dq[l] * (double)Akl;
    }
    const double dE = block_sum_d(part, sh);
    if (tid == 0) {
        const int so = A.site_state_off[site];
        const int cur = s_pick.cur, nxt = s_pick.nxt;
        double dG = dE - (A.G_ref[so + nxt] - A.G_ref[so + cur]);
        dG += FARADAY * (A.E[r] - A.E0_ref[site]) * (double)(A.n_e[so + nxt] - A.n_e[so + cur]);
        dG += A.kT * LN10 * (A.pH[r] - A.pKa_ref[site]) * (double)(A.n_H[so + nxt] - A.n_H[so + cur]);
        const double u = unif53(s_pick.w2);
        const int acc = (dG <= 0.0) || (u < exp(-dG / A.kT));
        if (A.dG_out) A.dG_out[r] = dG;
        if (A.acc_out) A.acc_out[r] = (uint8_t)acc;
        if (acc) A.state[site] = nxt;
        s_acc = acc;
    }
    __syncthreads();
    if (s_acc)
        for (int k = tid; k < na; k += blockDim.x) {
            const int64_t gk = base + A.site_atom_idx[a0 + k];
            A.xyzq[gk].w = A.q_state[qo + k];
        }
}

// --- per-residue sweep (Sec. III.A.2) ---------------------------------------------
// Every site of the requested kind gets one attempt, the sites taken in a
// uniformly random order; each attempt is the one above, with the charges
// left by the attempts before it.  Visit i of replica r draws Philox4x64-10,
// key (seed, 0), counter (r, step, 5 + kind, i): word 0 picks the next site
// among those not yet visited (a Fisher-Yates step over the sites of the kind
// in index order), word 1 the new state, word 2 gives u.  The site rows are
// computed once for all site atoms of the kind (k_sweep_rows, per slice as in
// k_mc_rows); after an accepted move the rows of every listed atom m change
// by sum_a dq_a A_ma, which k_sweep_decide adds before the next visit.

struct SweepList {
    int n_sites, n_atoms;
    int site[SWEEP_MAX_SITES];           // global site index, in index order
    int first[SWEEP_MAX_SITES + 1];      // its atoms are atom[first[k] .. first[k+1])
    int atom[SWEEP_MAX_SITE_ATOMS];      // replica-local atom index
};

// Built by the whole block; false (for every thread) when replica r's sites
// of the kind exceed the limits.
__device__ bool sweep_list(const MCArgs& A, int r, SweepList& L) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ns = 0, na = 0, ok = 1;
        for (int s = A.site_off[r]; s < A.site_off[r + 1] && ok; ++s) {
            if (A.site_kind[s] != A.kind) continue;
            const int n_s = A.site_atom_off[s + 1] - A.site_atom_off[s];
            if (ns >= SWEEP_MAX_SITES || na + n_s > SWEEP_MAX_SITE_ATOMS || n_s > MC_MAX_SITE_ATOMS || n_s < 1) {
                ok = 0;
                break;
            }
            L.site[ns] = s;
            L.first[ns] = na;
            ++ns;
            na += n_s;
        }
        L.n_sites = ns;
        L.n_atoms = na;
        L.first[ns] = na;
        s_ok = ok;
        if (!ok && A.err) atomicCAS(A.err, 0, GB_ERR_INVALID_ARG);
    }
    __syncthreads();
    if (!s_ok) return false;
    // the table checks of mc_site_ok for every listed site
    const int n = (int)(A.atom_off[r + 1] - A.atom_off[r]);
    bool bad = false;
    for (int k = 0; k < L.n_sites; ++k) {
        const int a0 = A.site_atom_off[L.site[k]];
        for (int a = threadIdx.x; a < L.first[k + 1] - L.first[k]; a += blockDim.x) {
            const int idx = A.site_atom_idx[a0 + a];
            bad |= idx < 0 || idx >= n;
            L.atom[L.first[k] + a] = idx;
        }
    }
    for (int k = threadIdx.x; k < L.n_sites; k += blockDim.x) {
        const int ns = A.site_nstates[L.site[k]], cur = A.state[L.site[k]];
        bad |= ns < 2 || cur < 0 || cur >= ns;
    }
    bad = __syncthreads_or(bad);
    if (bad) {
        if (threadIdx.x == 0 && A.err) atomicCAS(A.err, 0, GB_ERR_INVALID_ARG);
        return false;
    }
    return true;
}

__global__ void __launch_bounds__(256) k_sweep_rows(MCArgs A) {
    pdl_enter();
    __shared__ SweepList L;
    const int r = blockIdx.y, part = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    if (!sweep_list(A, r, L) || L.n_sites == 0) return;
    const int64_t base = A.atom_off[r];
    const int n = (int)(A.atom_off[r + 1] - base);
    const int j0 = part * MC_CHUNK, j1 = min(n, j0 + MC_CHUNK);
    const float tke = (float)A.tau_ke, kc = (float)A.kc, keo = (float)A.ke_out, kap = (float)A.kappa;
    double* out = A.phi_part + ((size_t)r * A.n_parts + part) * SWEEP_MAX_SITE_ATOMS;
    for (int k = wid; k < L.n_atoms; k += nw) {
        const int lk = L.atom[k];
        const int64_t gk = base + lk;
        const float4 xk = A.xyzq[gk];
        const float2 Rk = mc_Rh(A, gk);
        double acc = 0.0;
        for (int j = j0 + lane; j < j1; j += 32) {
            const int64_t gj = base + j;
            const float4 xj = A.xyzq[gj];
            const float term = (j == lk) ? mc_self_term(Rk.x, tke, kc, keo, kap) : mc_pair_term(xk, Rk, xj, mc_Rh(A, gj), tke, kc, keo, kap, A.cut2);
            acc += (double)(xj.w * term);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) out[k] = acc;
    }
}

__global__ void __launch_bounds__(256) k_sweep_decide(MCArgs A) {
    pdl_enter();
    __shared__ SweepList L;
    __shared__ double s_phi[SWEEP_MAX_SITE_ATOMS];
    __shared__ double s_dq[MC_MAX_SITE_ATOMS];
    __shared__ int s_order[SWEEP_MAX_SITES];
    __shared__ double sh[32];
    __shared__ int s_li, s_site, s_nxt, s_acc;
    const int r = blockIdx.x;
    const int tid = threadIdx.x;
    // every site of the replica starts as "not visited"
    for (int s = A.site_off[r] + tid; s < A.site_off[r + 1]; s += blockDim.x) {
        if (A.dG_out) A.dG_out[s] = 0.0;
        if (A.acc_out) A.acc_out[s] = 2;
    }
    if (!sweep_list(A, r, L) || L.n_sites == 0) return;
    const int64_t base = A.atom_off[r];
    const int n = (int)(A.atom_off[r + 1] - base);
    const int n_parts_r = (n + MC_CHUNK - 1) / MC_CHUNK;
    for (int k = tid; k < L.n_atoms; k += blockDim.x) {
        double phi = 0.0;
        for (int p = 0; p < n_parts_r; ++p)
            phi += A.phi_part[((size_t)r * A.n_parts + p) * SWEEP_MAX_SITE_ATOMS + k];
        s_phi[k] = phi;
    }
    for (int k = tid; k < L.n_sites; k += blockDim.x) s_order[k] = k;
    __syncthreads();
    const u64 step = (A.ctr ? A.ctr[0] : 0) + A.step;
    const float tke = (float)A.tau_ke, kc = (float)A.kc, keo = (float)A.ke_out, kap = (float)A.kappa;
    double u = 0.0;
    int cur = 0;
    for (int i = 0; i < L.n_sites; ++i) {
        if (tid == 0) {
            const Philox4 w = philox4x64(A.rep_base + (u64)r, step, 5 + (u64)A.kind, (u64)i, A.seed, 0);
            const int j = i + pick_int(w.w[0], L.n_sites - i);
            const int t = s_order[i];
            s_order[i] = s_order[j];
            s_order[j] = t;
            s_li = s_order[i];
            s_site = L.site[s_li];
            cur = A.state[s_site];
            const int k = pick_int(w.w[1], A.site_nstates[s_site] - 1);
            s_nxt = (k < cur) ? k : k + 1;
            u = unif53(w.w[2]);
        }
        __syncthreads();
        const int li = s_li, site = s_site, nxt = s_nxt;
        const int a0 = L.first[li], na = L.first[li + 1] - a0;
        const int qo = A.site_q_off[site] + nxt * na;
        for (int a = tid; a < na; a += blockDim.x)
            s_dq[a] = (double)A.q_state[qo + a] - (double)A.xyzq[base + L.atom[a0 + a]].w;
        __syncthreads();
        double part = 0.0;
        for (int t = tid; t < na * na; t += blockDim.x) {
            const int k = t / na, l = t % na;
            const int64_t gk = base + L.atom[a0 + k];
            const float2 Rk = mc_Rh(A, gk);
            float Akl;
            if (k == l) {
                Akl = mc_self_term(Rk.x, tke, kc, keo, kap);
                part += s_dq[k] * s_phi[a0 + k];
            } else {
                const int64_t gl = base + L.atom[a0 + l];
                Akl = mc_pair_term(A.xyzq[gk], Rk, A.xyzq[gl], mc_Rh(A, gl), tke, kc, keo, kap, A.cut2);
            }
            part += 0.5 * s_dq[k] * s_dq[l] * (double)Akl;
        }
        const double dE = block_sum_d(part, sh);
        if (tid == 0) {
            const int so = A.site_state_off[site];
            double dG = dE - (A.G_ref[so + nxt] - A.G_ref[so + cur]);
            dG += FARADAY * (A.E[r] - A.E0_ref[site]) * (double)(A.n_e[so + nxt] - A.n_e[so + cur]);
            dG += A.kT * LN10 * (A.pH[r] - A.pKa_ref[site]) * (double)(A.n_H[so + nxt] - A.n_H[so + cur]);
            const int acc = (dG <= 0.0) || (u < exp(-dG / A.kT));
            if (A.dG_out) A.dG_out[site] = dG;
            if (A.acc_out) A.acc_out[site] = (uint8_t)acc;
            if (acc) A.state[site] = nxt;
            s_acc = acc;
        }
        __syncthreads();
        if (s_acc) {
            // rows of every listed atom: phi_m += sum_a dq_a A_ma (charges still old here)
            for (int m = tid; m < L.n_atoms; m += blockDim.x) {
                const int64_t gm = base + L.atom[m];
                const float4 xm = A.xyzq[gm];
                const float2 Rm = mc_Rh(A, gm);
                double d = 0.0;
                for (int a = 0; a < na; ++a) {
                    const int64_t ga = base + L.atom[a0 + a];
                    const float Ama = (ga == gm) ? mc_self_term(Rm.x, tke, kc, keo, kap) : mc_pair_term(xm, Rm, A.xyzq[ga], mc_Rh(A, ga), tke, kc, keo, kap, A.cut2);
                    d += s_dq[a] * (double)Ama;
                }
                s_phi[m] += d;
            }
            __syncthreads();
            for (int a = tid; a < na; a += blockDim.x) A.xyzq[base + L.atom[a0 + a]].w = A.q_state[qo + a];
        }
        __syncthreads();
    }
}

cudaError_t launch_mc_sweep(const MCArgs& a, int32_t M, cudaStream_t s) {
    if (M == 0) return cudaSuccess;
    if (a.n_parts > 0) {
        const cudaError_t e = launch_pdl(k_sweep_rows, dim3((unsigned)a.n_parts, (unsigned)M), dim3(256), 0, s, a);
        if (e != cudaSuccess) return e;
    }
    return launch_pdl(k_sweep_decide, dim3(M), dim3(256), 0, s, a);
}

// --- replica exchange (Eq. 14, 15; schedule of Sec. III.B) ----------------------------
__device__ __forceinline__ void exchange_pair(int32_t* rep_at_slot, const double* values,
                                              const int32_t* n_count, double c, int l, int len,
                                              int ladder_stride, int slot_stride, int a, int b,
                                              u64 attempt, u64 seed, double* value_of_rep,
                                              double* delta_out, uint8_t* acc_out) {
    int32_t* pa = &rep_at_slot[l * ladder_stride + a * slot_stride];
    int32_t* pb = &rep_at_slot[l * ladder_stride + b * slot_stride];
    const int i = *pa, j = *pb;
    const double delta = c * (values[b] - values[a]) * (double)(n_count[i] - n_count[j]);
    const Philox4 w = philox4x64((u64)(l * len + a), attempt, 3, 0, seed, 0);
    const double u = unif53(w.w[0]);
    const int acc = (delta <= 0.0) || (u < exp(-delta));
    if (delta_out) delta_out[l * len + a] = delta;
    if (acc_out) acc_out[l * len + a] = (uint8_t)acc;
    if (acc) { *pa = j; *pb = i; }
    if (value_of_rep) {
        value_of_rep[*pa] = values[a];
        value_of_rep[*pb] = values[b];
    }
}

// the partner of slot a in attempt `attempt`, or -1
__device__ __forceinline__ int partner(int a, int len, u64 attempt, int wrap) {
    if ((a & 1) != (int)(attempt & 1)) return -1;
    int b = a + 1;
    if (b == len) {
        if (!(wrap && (attempt & 1) && (len % 2 == 0))) return -1;
        b = 0;
    }
    return b;
}

__global__ void k_exchange(ExArgs A) {
    pdl_enter();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= A.n_ladders * A.len) return;
    const int l = t / A.len, a = t % A.len;
    const u64 attempt = (A.ctr ? A.ctr[1] : 0) + A.attempt;
    if (A.delta_out) A.delta_out[t] = __longlong_as_double(0x7ff8000000000000LL);
    if (A.acc_out) A.acc_out[t] = 0;
    const int b = partner(a, A.len, attempt, A.wrap);
    if (b < 0) return;
    const double c = (A.dim == 0) ? FARADAY / A.kT : LN10;
    exchange_pair(A.rep_at_slot, A.values, A.n_count, c, l, A.len, A.ladder_stride, A.slot_stride,
                  a, b, attempt, A.seed, A.value_of_rep, A.delta_out, A.acc_out);
}

// Bound electrons (kind 1) or protons (kind 0) of replica rep; -1 when a
// site of that kind has a state outside [0, nstates).
__device__ __forceinline__ int bound_count(const int32_t* site_off, const int32_t* site_kind,
                                           const int32_t* site_nstates, const int32_t* site_state_off,
                                           const int32_t* n_H, const int32_t* n_e, const int32_t* state,
                                           int rep, int kind) {
    int c = 0;
    for (int s = site_off[rep]; s < site_off[rep + 1]; ++s) {
        if (site_kind[s] != kind) continue;
        const int st = state[s];
        if (st < 0 || st >= site_nstates[s]) return -1;
        const int so = site_state_off[s] + st;
        c += kind ? n_e[so] : n_H[so];
    }
    return c;
}

__global__ void k_grid_exchange(GridExArgs A) {
    pdl_enter();
    const u64 attempt = A.ctr[1];
    const int dimE = (A.ex_dim == 0) || (A.ex_dim == 2 && ((attempt >> 1) & 1) == 0);
    const int n_lad = dimE ? A.n_pH : A.n_E;
    const int len = dimE ? A.n_E : A.n_pH;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_lad * len) return;
    const int l = t / len, a = t % len;
    const int b = partner(a, len, attempt, A.wrap);
    if (b < 0) return;
    const int ladder_stride = dimE ? A.n_E : 1;
    const int slot_stride = dimE ? 1 : A.n_E;
    int32_t* pa = &A.grid[l * ladder_stride + a * slot_stride];
    int32_t* pb = &A.grid[l * ladder_stride + b * slot_stride];
    const int i = *pa, j = *pb;
    const int kind = dimE ? 1 : 0;
    const double* values = dimE ? A.E_ladder : A.pH_ladder;
    const double c = dimE ? FARADAY / A.kT : LN10;
    const int ci = bound_count(A.site_off, A.site_kind, A.site_nstates, A.site_state_off, A.n_H, A.n_e, A.state, i, kind);
    const int cj = bound_count(A.site_off, A.site_kind, A.site_nstates, A.site_state_off, A.n_H, A.n_e, A.state, j, kind);
    if (ci < 0 || cj < 0) {                 // corrupt state: no exchange for this pair
        if (A.err) atomicCAS(A.err, 0, GB_ERR_INVALID_ARG);
        return;
    }
    const double delta = c * (values[b] - values[a]) * (double)(ci - cj);
    const Philox4 w = philox4x64((u64)(l * len + a), attempt, 3, 0, A.seed, 0);
    const int acc = (delta <= 0.0) || (unif53(w.w[0]) < exp(-delta));
    if (acc) { *pa = j; *pb = i; }
    if (A.ex_count) {
        const int ng = A.n_pH * A.n_E;
        u64* cnt = A.ex_count + (size_t)(dimE ? 0 : 2) * ng + (l * ladder_stride + a * slot_stride);
        atomicAdd(cnt, 1ull);
        if (acc) atomicAdd(cnt + ng, 1ull);
    }
    double* vr = dimE ? A.E_rep : A.pH_rep;
    vr[*pa] = values[a];
    vr[*pb] = values[b];
}

__global__ void k_occupancy(OccArgs A) {
    pdl_enter();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= A.n_sites) return;
    int lo = 0, hi = A.M;                       // replica r with site_off[r] <= s < site_off[r+1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (A.site_off[mid] <= s) lo = mid;
        else hi = mid;
    }
    const int r = lo;
    const int base = A.site_state_off[A.site_off[r]];
    const int st = A.state[s];
    if (A.site_state_off[A.site_off[r + 1]] - base != A.stride || st < 0 || st >= A.site_nstates[s]) {
        atomicCAS(A.err, 0, GB_ERR_INVALID_ARG);
        return;
    }
    int g = r;
    if (A.grid)
        for (int k = 0; k < A.M; ++k)
            if (A.grid[k] == r) { g = k; break; }
    atomicAdd(&A.occ[(size_t)g * A.stride + (A.site_state_off[s] - base) + st], 1ull);
}

__global__ void k_count(const int32_t* site_off, const int32_t* site_kind, const int32_t* site_nstates,
                        const int32_t* site_state_off, const int32_t* n_H, const int32_t* n_e,
                        const int32_t* state, int32_t kind, int32_t M, int32_t* out) {
    pdl_enter();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= M) return;
    out[r] = bound_count(site_off, site_kind, site_nstates, site_state_off, n_H, n_e, state, r, kind);
}

// --- launchers -----------------------------------------------------------------------
static dim3 atom_grid(const AtomArgs& a) {
    return dim3((unsigned)((a.max_n + 255) / 256 > 0 ? (a.max_n + 255) / 256 : 1), (unsigned)a.M);
}

cudaError_t launch_born_finalize(const AtomArgs& a, float* R_out, cudaStream_t s) {
    return launch_pdl(k_born_finalize, atom_grid(a), dim3(256), 0, s, a, R_out);
}

cudaError_t launch_energy_finalize(const AtomArgs& a, int want_energy, double* phi_out, cudaStream_t s,
                                   float bond_k, float bond_r0) {
    return launch_pdl(k_energy_finalize, atom_grid(a), dim3(256), 0, s, a, want_energy, phi_out, bond_k, bond_r0);
}

cudaError_t launch_forces_out(const AtomArgs& a, int64_t* F_fixed, float* F_out, double* E_out,
                              cudaStream_t s) {
    return launch_pdl(k_forces_out, atom_grid(a), dim3(256), 0, s, a, F_fixed, F_out, E_out);
}

cudaError_t launch_md_step(const AtomArgs& a, const MDArgs& m, float4* boxes, const int* tile_off,
                           int step_in_block, int mode, cudaStream_t s) {
    return launch_pdl(k_md_step, atom_grid(a), dim3(256), 0, s, a, m, boxes, tile_off, step_in_block, mode);
}

cudaError_t launch_set_counters(u64* ctr, u64 step, u64 attempt, cudaStream_t s) {
    return launch_pdl(k_set_counters, dim3(1), dim3(1), 0, s, ctr, step, attempt);
}

cudaError_t launch_advance_counters(u64* ctr, u64 steps, u64 attempts, cudaStream_t s) {
    return launch_pdl(k_advance_counters, dim3(1), dim3(1), 0, s, ctr, steps, attempts);
}

cudaError_t launch_mc(const MCArgs& a, int32_t M, cudaStream_t s) {
    if (M == 0) return cudaSuccess;
    if (a.n_parts > 0) {
        const cudaError_t e = launch_pdl(k_mc_rows, dim3((unsigned)a.n_parts, (unsigned)M), dim3(256), 0, s, a);
        if (e != cudaSuccess) return e;
    }
    return launch_pdl(k_mc_decide, dim3(M), dim3(256), 0, s, a);
}

cudaError_t launch_exchange(const ExArgs& a, cudaStream_t s) {
    const int n = a.n_ladders * a.len;
    if (n == 0) return cudaSuccess;
    return launch_pdl(k_exchange, dim3((n + 255) / 256), dim3(256), 0, s, a);
}

cudaError_t launch_grid_exchange(const GridExArgs& a, cudaStream_t s) {
    const int n = a.n_pH * a.n_E;
    if (n < 2) return cudaSuccess;
    return launch_pdl(k_grid_exchange, dim3((n + 255) / 256), dim3(256), 0, s, a);
}

cudaError_t launch_occupancy(const OccArgs& a, cudaStream_t s) {
    if (a.n_sites == 0) return cudaSuccess;
    return launch_pdl(k_occupancy, dim3((a.n_sites + 127) / 128), dim3(128), 0, s, a);
}

cudaError_t launch_count(const int32_t* site_off, const int32_t* site_kind, const int32_t* site_nstates,
                         const int32_t* site_state_off, const int32_t* n_H, const int32_t* n_e,
                         const int32_t* state, int32_t kind, int32_t M, int32_t* out,
                         cudaStream_t s) {
    if (M == 0) return cudaSuccess;
    return launch_pdl(k_count, dim3((M + 127) / 128), dim3(128), 0, s, site_off, site_kind, site_nstates,
                      site_state_off, n_H, n_e, state, kind, M, out);
}

}  // namespace gbk
