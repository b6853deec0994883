/*
 * gbremd.h -- C ABI of the GB300 hot path of discrete-state constant redox
 * potential MD (CEMD), coupled constant pH / redox potential MD (C(pH,E)MD)
 * and redox-potential replica exchange (E-REMD) in Generalized Born implicit
 * solvent (Cruzeiro, Amaral, Roitberg, "Redox Potential Replica Exchange
 * Molecular Dynamics at Constant pH in AMBER").
 *
 * Conventions shared by every call
 *  - Units: kcal/mol, Angstrom, elementary charge e, ps, amu, V, K.
 *  - A batch holds M replicas (independent molecules) packed back to back;
 *    replica r owns atoms [atom_off[r], atom_off[r+1]) of every per-atom array.
 *  - Array arguments are DEVICE pointers owned by the caller unless marked
 *    "host".  Per-atom arrays may be NULL when every replica of the batch is
 *    empty (N = 0).  The library owns only what gb_ctx_create allocates (workspace,
 *    work lists, captured graphs) and frees it in gb_ctx_destroy.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Every call only enqueues work on that stream and returns; outputs are
 *    valid once the stream reaches that point.
 *  - Return value: GB_OK (0) or a negative GB_ERR_* code.  Argument and launch
 *    errors are reported synchronously; gb_last_error() has the message.
 *    Errors detected on the device set a device error word that
 *    gb_sync_status() reads and clears (the first one recorded is kept):
 *    GB_ERR_NONFINITE for a non-finite coordinate, charge or Born radius, or
 *    two atoms of a replica at the same position (coincident); GB_ERR_TIMEOUT
 *    for a bounded wait that gave up; GB_ERR_INVALID_ARG for a site table
 *    that fails the checks listed at gb_sites.
 *  - Per-atom layouts:
 *      xyzq        float[N][4]   x, y, z, charge q
 *      rad_screen  float[N][2]   intrinsic radius rho, HCT screening factor S
 *      forces      float[N][3]   F = -dE/dx
 *      fixed forces int64[3][N]  components x, then y, then z; F * 2^32,
 *                                rounded (the accumulators themselves)
 *  - Arithmetic: FP32 pair terms; int64 fixed-point accumulation of forces,
 *    Born integrals, dE/dR and dE/dq; the O(N) Born-radius transform in FP32
 *    written without cancellation; FP64 for the self terms, the per-replica
 *    energy totals, the Monte Carlo energy change and every acceptance test.
 */
#ifndef GBREMD_H
#define GBREMD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GB_OK 0
#define GB_ERR_INVALID_ARG (-1)
#define GB_ERR_CUDA (-2)
#define GB_ERR_TIMEOUT (-3)
#define GB_ERR_NONFINITE (-4)
#define GB_ERR_NOMEM (-5)

typedef struct gb_ctx gb_ctx;

/* Generalized Born model parameters.  The paper runs the OBC model of
 * Onufriev, Bashford and Case ("igb=2", Sec. III.D) for MD and for every
 * state-change energy; alpha, beta, gamma rescale the HCT integral into the
 * effective Born radius, `offset` is subtracted from each intrinsic radius,
 * eps_in / eps_out are the solute and solvent dielectric constants.
 * rep_k, rep_sigma: optional soft repulsion rep_k (rep_sigma - r)^2 for
 * r < rep_sigma between atoms more than one position apart in the chain (0
 * disables it; MD driver only; never cut).  kappa: inverse
 * Debye length of dissolved salt (1/A; 0 = no salt, the paper's setting);
 * the solvent term of every GB pair (and self) term is screened,
 *   (1/eps_in - 1/eps_out) / f  ->  (1/eps_in - exp(-kappa f)/eps_out) / f,
 * in energies, forces, dE/dq and the Monte Carlo energy changes.
 * Optional cutoffs (0 = none, the paper's GB setting; both in A, finite):
 *   rgbmax  Born-radius cutoff: the HCT descreening integral of atom i counts
 *           only the part of each sphere j that lies within rgbmax of atom i
 *           (an integral restricted to that ball, so radii stay continuous
 *           in the coordinates);
 *   cut     pair cutoff: GB and Coulomb pair terms of pairs farther apart
 *           than `cut` are left out (truncation; self terms stay) in
 *           energies, forces, dE/dq and the Monte Carlo energy changes.
 * With a cutoff the pair kernels skip, per 64 x 32-atom block, every block
 * whose atoms' bounding boxes prove all its pairs out of range (a block
 * neighbour list rebuilt from the coordinates of each evaluation). */
typedef struct {
    float alpha, beta, gamma;
    float offset;
    float eps_in, eps_out;
    float rep_k, rep_sigma;
    float kappa;
    float rgbmax, cut;
} gb_params;

/* Create a context for a fixed batch layout.
 *   n_rep     number of replicas M (>= 1)
 *   atom_off  HOST int64[M+1], atom_off[0] = 0, non-decreasing; replicas may
 *             be empty; total atoms N = atom_off[M] < 2^31
 *   params    HOST pointer, copied
 *   device    CUDA device ordinal the context lives on
 * Allocates device workspace proportional to N and M (about 80 bytes per atom).
 * Errors: GB_ERR_INVALID_ARG, GB_ERR_NOMEM, GB_ERR_CUDA. */
int gb_ctx_create(gb_ctx** out, int32_t n_rep, const int64_t* atom_off, const gb_params* params,
                  int32_t device);

/* Release everything the context owns.  NULL is accepted. */
int gb_ctx_destroy(gb_ctx* ctx);

/* Message of the last error reported on this context (or, for ctx == NULL, of
 * the last gb_ctx_create failure in this thread).  Owned by the library. */
const char* gb_last_error(const gb_ctx* ctx);

/* Read and clear the device error word after synchronising `stream`.
 * Returns GB_OK or the GB_ERR_* code a kernel recorded. */
int gb_sync_status(gb_ctx* ctx, void* stream);

/* Tile configuration of the pair kernels: warps per block and blocks (64 x 32
 * atoms) per warp task of the static task list (a pass with a cutoff walks
 * its neighbour list instead, in runs of up to 16 blocks).  gb_autotune times
 * the candidates and register caps pass by pass on the given inputs and
 * keeps the fastest; gb_set_tiles forces one. */
int gb_autotune(gb_ctx* ctx, const float* xyzq, const float* rad_screen, void* stream);
int gb_set_tiles(gb_ctx* ctx, int32_t warps_per_block, int32_t tiles_per_task);
/* Register cap of the pair kernel of one pass (0 Born radii, 1 energy and
 * direct forces, 2 Born chain rule; -1 = all three), as 256-thread blocks
 * per SM: 1 = the compiler's choice, 3 = at most 80 registers per thread,
 * 4 = at most 64 (more resident warps, more spills; a pass with a cutoff
 * runs cap 3 instead).  gb_autotune picks each pass's cap and gb_autotune_md
 * re-tunes them on MD segments; the default is 3.  GB_ERR_INVALID_ARG for
 * other values. */
int gb_set_reg_cap(gb_ctx* ctx, int32_t pass, int32_t min_blocks_per_sm);
/* The three caps in pass order into caps[3] (host memory). */
int gb_get_reg_caps(const gb_ctx* ctx, int32_t* caps);
int gb_get_tiles(const gb_ctx* ctx, int32_t* warps_per_block, int32_t* tiles_per_task);

/* Effective Born radii of every atom (OBC model, Sec. III.D):
 *   a_i = rho_i - offset,  s_j = S_j a_j
 *   I_i = sum_{j != i} H(r_ij; a_i, s_j)    (HCT pairwise descreening integral)
 *   psi_i = a_i I_i
 *   R_i = 1 / (1/a_i - tanh(alpha psi_i - beta psi_i^2 + gamma psi_i^3) / rho_i)
 * in:  xyzq float[N][4], rad_screen float[N][2]
 * out: R_out float[N] */
int gb_born_radii(gb_ctx* ctx, const float* xyzq, const float* rad_screen, float* R_out,
                  void* stream);

/* GB + Coulomb energy, forces and charge derivative of every replica at the
 * Born radii of the given coordinates (the radii are recomputed here because
 * the force needs the chain rule through them):
 *   E_GB   = -1/2 (1/eps_in - 1/eps_out) k_e sum_i sum_j q_i q_j / f_ij
 *   f_ij   = sqrt(r_ij^2 + R_i R_j exp(-r_ij^2 / (4 R_i R_j))),  f_ii = R_i
 *   E_Coul = (k_e / eps_in) sum_{i<j} q_i q_j / r_ij,   k_e = 332.0522173
 * plus the soft repulsion of gb_params when enabled.  All outputs are
 * nullable except that at least one must be given:
 *   R_out      float[N]       Born radii
 *   F_fixed    int64[3][N]    forces in 2^-32 kcal/mol/A units
 *   F_out      float[N][3]    forces
 *   E_out      double[M][3]   E_GB (self terms included), E_Coul, E_repulsion
 *   dEdq_out   double[N]      phi_i = dE/dq_i at fixed Born radii; the state
 *                             change energies of Eq. 8 and 9 are built from it */
int gb_energy_forces(gb_ctx* ctx, const float* xyzq, const float* rad_screen, float* R_out,
                     int64_t* F_fixed, float* F_out, double* E_out, double* dEdq_out,
                     void* stream);

/* Titratable sites (residues whose charge set changes between discrete
 * protonation or redox states, Sec. II.A, II.B).  All DEVICE arrays except
 * site_off_host.  Site s belongs to the replica r with
 * site_off[r] <= s < site_off[r+1].
 *   site_kind[S]        0 = pH-active, 1 = redox-active
 *   site_nstates[S]     number of states (>= 2)
 *   site_atom_off[S+1]  atoms of site s are site_atom_idx[site_atom_off[s] ..]
 *   site_atom_idx[]     replica-local atom index
 *   site_state_off[S+1] per-state entries of site s start here (G_ref, n_H, n_e)
 *   site_q_off[S+1]     charge of site s, state k, site atom a at
 *                       q_state[site_q_off[s] + k * n_atoms(s) + a]
 *   G_ref (double)      Delta G_elec,ref term of Eq. 8 / 9 as a per-state value;
 *                       the change of state k -> k' subtracts G_ref[k'] - G_ref[k]
 *   n_H, n_e            protons / electrons bound in each state
 *   pKa_ref, E0_ref     per site (double; E0_ref in V)
 * The tables stay on the device and are not read on the host.  The kernels
 * check, before any access through them, that the atom indices of every site
 * they touch lie in [0, n) of its replica, that nstates >= 2 and that the
 * current state lies in [0, nstates).  An attempt or exchange that fails a
 * check is skipped, leaves charges and states unchanged and records
 * GB_ERR_INVALID_ARG for gb_sync_status. */
typedef struct {
    int32_t n_rep;
    int32_t n_sites;
    const int32_t* site_off_host;   /* HOST int32[M+1], the values of site_off: checked
                                       on the host (0 first, non-decreasing, n_sites
                                       last; GB_ERR_INVALID_ARG otherwise) */
    const int32_t* site_off;        /* DEVICE copy */
    const int32_t* site_kind;
    const int32_t* site_nstates;
    const int32_t* site_atom_off;
    const int32_t* site_atom_idx;
    const int32_t* site_state_off;
    const int32_t* site_q_off;
    const float* q_state;
    const double* G_ref;
    const int32_t* n_H;
    const int32_t* n_e;
    const double* pKa_ref;
    const double* E0_ref;
} gb_sites;

/* One Monte Carlo state-change attempt per replica at fixed Born radii
 * (implicit-solvent scheme, Sec. III.A.1): a single residue of the requested
 * kind is picked uniformly, a new state is drawn uniformly from its other
 * states (Sec. III.A), and
 *   dG = dE_elec - (G_ref[k'] - G_ref[k])
 *        + F (E - E0_ref) (n_e[k'] - n_e[k])          redox, Eq. 8
 *        + kT ln10 (pH - pKa_ref) (n_H[k'] - n_H[k])  protonation, Eq. 9
 * is accepted iff dG <= 0 or u < exp(-dG/kT).  dE_elec is the exact change of
 * E_GB + E_Coul for the site's new charges with R held fixed, from the
 * site rows phi_k and the site-site block.  Random numbers: Philox4x64-10,
 * key (seed, 0), counter (replica, step, 1 + kind, 0); words 0, 1, 2 choose
 * the site, the state and u.
 *   kind       0 protonation attempt, 1 redox attempt (C(pH,E)MD runs the
 *              protonation attempt first when both fall on a step, Sec. III.A)
 *   xyzq       updated in place: charges of the site atoms on acceptance
 *   R          Born radii of these coordinates (gb_born_radii)
 *   pH, E      double[M] per replica (E in V); kT in kcal/mol
 *   state_inout int32[S] current state of every site, updated on acceptance
 *   dG_out     double[M] (nullable), acc_out uint8[M] (nullable); replicas
 *              without a site of this kind report dG = 0, acc = 0 */
int redox_ph_mc_step(gb_ctx* ctx, const gb_sites* sites, float* xyzq, const float* R,
                     const double* pH, const double* E, double kT, uint64_t seed, uint64_t step,
                     int32_t kind, int32_t* state_inout, double* dG_out, uint8_t* acc_out,
                     void* stream);

/* Per-residue sweep: every site of the requested kind in every replica gets
 * one state-change attempt, the sites of a replica taken in a uniformly
 * random order -- the visiting rule of the explicit-solvent scheme (Sec.
 * III.A.2), here with the same GB energies as redox_ph_mc_step (no solvent
 * stripping or relaxation).  Each attempt is the one of redox_ph_mc_step
 * (uniform new state, dG of Eq. 8 / 9 at fixed R, Metropolis) with the
 * charges left by the attempts before it.  Random numbers: Philox4x64-10, key
 * (seed, 0), counter (replica, step, 5 + kind, i) for visit i: word 0 picks
 * the next site among those not yet visited (a Fisher-Yates step over the
 * replica's sites of the kind in index order), word 1 the state, word 2 u.
 *   arguments as in redox_ph_mc_step, except the outputs, which are per SITE:
 *   dG_out     double[S] (nullable): dG of the site's attempt, 0 if not visited
 *   acc_out    uint8[S]  (nullable): 1 accepted, 0 rejected, 2 not of this kind
 * Limits per replica and kind: 256 sites, 1024 site atoms, 128 atoms per site;
 * a replica over them is skipped and GB_ERR_INVALID_ARG is recorded for
 * gb_sync_status.  The first call on a context allocates its workspace
 * (8 bytes x replicas x ceil(largest replica / 256) x 1024); make it outside
 * stream capture. */
int redox_ph_mc_sweep(gb_ctx* ctx, const gb_sites* sites, float* xyzq, const float* R,
                      const double* pH, const double* E, double kT, uint64_t seed, uint64_t step,
                      int32_t kind, int32_t* state_inout, double* dG_out, uint8_t* acc_out,
                      void* stream);

/* Replica exchange between neighbouring slots of one or more ladders
 * (E-REMD, Eq. 14-15 and Sec. III.B; pH ladders by the same argument with
 * protons, Eq. 12 analogue).  Ladder l, slot k is occupied by replica
 * rep_at_slot[l * ladder_stride + k * slot_stride] at value values[k].
 * Attempt number `attempt` pairs slots (0,1),(2,3),... when even and
 * (1,2),(3,4),... when odd, plus (len-1, 0) for odd attempts when `wrap` is
 * set and len is even.  For replica i in slot a and j in slot b:
 *   Delta = c (values[b] - values[a]) (n_count[i] - n_count[j]),
 *   c = F/kT for dim 0 (E in V, n_count = electrons), ln 10 for dim 1 (pH,
 *   n_count = protons);
 * accepted iff Delta <= 0 or u < exp(-Delta), u from Philox4x64-10 with key
 * (seed, 0) and counter (l*len + a, attempt, 3, 0).  An accepted pair swaps
 * the two replicas' slots; value_of_rep (nullable, double[M]) then receives
 * the new ladder value of both replicas.
 *   delta_out double[n_ladders*len], acc_out uint8[n_ladders*len] (nullable):
 *   written at index l*len + a of each pair's first slot, NaN / 0 elsewhere. */
int eremd_exchange(int32_t n_ladders, int32_t ladder_len, int32_t ladder_stride,
                   int32_t slot_stride, const double* values, int32_t* rep_at_slot,
                   const int32_t* n_count, int32_t dim, uint64_t attempt, uint64_t seed,
                   double kT, int32_t wrap, double* value_of_rep, double* delta_out,
                   uint8_t* acc_out, void* stream);

/* Electrons (kind 1) or protons (kind 0) bound by each replica's sites in
 * the given states: n_count_out int32[M].  A replica with a site of that
 * kind whose state lies outside [0, site_nstates) gets -1, and no table entry
 * past the site's states is read. */
int gb_count_bound(const gb_sites* sites, const int32_t* state, int32_t kind,
                   int32_t* n_count_out, void* stream);

/* Langevin MD driver of a whole batch: BAOAB splitting, every replica, with
 * GB + Coulomb + soft repulsion + harmonic chain bonds k (r - r0)^2 between
 * atoms i, i+1; Monte Carlo attempts every mc_every steps (protonation then
 * redox, Sec. III.A) and neighbour exchanges every ex_every steps (Sec.
 * III.B) along the E ladder (ex_dim 0) or pH ladder (ex_dim 1), alternating
 * between E and pH lines when ex_dim is 2 (two-dimensional grid).  Noise:
 * Philox4x64-10, key (seed, 0), counter (rep_base + replica, step, 4, atom),
 * Box-Muller; the Monte Carlo attempts count replicas from rep_base too.
 * The state buffers are owned by the caller and updated in place. */
typedef struct {
    float* xyzq;            /* float[N][4] positions + current charges */
    float* vel;             /* float[N][4] velocities (A/ps), 4th lane unused */
    float* force;           /* float[N][4] forces at xyzq, kept between calls */
    const float* rad_screen;
    float* R;               /* float[N] Born radii of the last evaluation */
    int32_t* state;         /* int32[S] site states */
    double* pH;             /* double[M] per replica, rewritten by pH exchanges */
    double* E;              /* double[M] per replica (V), rewritten by E exchanges */
    int32_t* grid;          /* int32[n_pH * n_E] replica at (pH row, E column) */
    const double* E_ladder; /* double[n_E] */
    const double* pH_ladder;/* double[n_pH] */
    int32_t n_E, n_pH;
    double dt, friction, mass, kT;   /* ps, 1/ps, amu, kcal/mol; dt = 0 freezes the
                                        coordinates (MC and exchange on a fixed structure) */
    float bond_k, bond_r0;
    uint64_t seed;
    uint64_t step;          /* absolute step counter, advanced by the call */
    uint64_t attempt;       /* exchange attempt counter, advanced by the call */
    int32_t mc_every, ex_every, ex_dim, wrap;
    int32_t mc_mode;        /* 0: one residue per attempt (redox_ph_mc_step, the implicit-
                               solvent scheme); 1: every residue once (redox_ph_mc_sweep) */
    int64_t* ex_count;      /* nullable, int64[2][2][n_pH * n_E], accumulated by every
                               exchange: [d][0][g] attempts and [d][1][g] acceptances of the
                               neighbour pair whose first slot is grid index g (the pair
                               (g, g+1) along E for d = 0, (g, g+n_E) along pH for d = 1;
                               the wrap pair has its first slot at the ladder's end).  An
                               exchange skipped for a corrupt state counts as neither.
                               The caller zeroes it; gb_autotune_md leaves it as it was. */
    int64_t* occ_count;     /* nullable, int64[n_slots][occ_stride]: state occupancy.  After
                               every step with Monte Carlo attempts (and after that step's
                               exchange), each site of each replica adds 1 to the entry of
                               its current state: row = the grid slot the replica holds
                               (the replica itself when grid is NULL or exchanges are off),
                               column = the state's index among the replica's site states
                               (site_state_off relative to the replica's first site).
                               Counts / halts = the fraction of time in each state at each
                               E / pH value (the titration data of Eq. 3 and Eq. 9).  Every
                               replica must hold occ_stride site states (one site layout,
                               as replica-exchange copies do); a replica that does not is
                               skipped and GB_ERR_INVALID_ARG recorded.  The caller zeroes
                               it. */
    int32_t occ_stride;     /* site states per replica (the row length of occ_count) */
    int64_t rep_base;       /* global index of this batch's replica 0 in the Philox counters
                               of the MD noise and the Monte Carlo attempts (>= 0; 0 when the
                               batch is the whole ensemble).  A replica ensemble split over
                               processes gives each part the index of its first replica, so
                               that every replica draws the numbers it would draw in one
                               batch. */
} gb_md_state;

/* Advance the batch by nsteps MD steps.  Step t (1-based, absolute) is
 * followed by MC attempts when t % mc_every == 0 and by an exchange when
 * t % ex_every == 0.  Requires state->force to hold the forces at the
 * incoming coordinates (gb_md_init computes them).  gb_md_init is also the
 * restart point after a device error: it clears the context's accumulators
 * before it evaluates. */
int gb_md_init(gb_ctx* ctx, gb_md_state* state, void* stream);
int gb_md_segment(gb_ctx* ctx, gb_md_state* state, const gb_sites* sites, int64_t nsteps,
                  void* stream);

/* The dynamic MD state of a batch kept in HOST memory, for gb_md_segment_host.
 * Every pointer is a HOST array mirroring the device buffer of the same name
 * in gb_md_state (same layout and length); NULL leaves that buffer on the
 * device untouched.  Pinned memory (cudaHostAlloc / cudaHostRegister) makes
 * the copies asynchronous DMA; pageable memory works, staged by the driver. */
typedef struct {
    float* xyzq;            /* float[N][4] */
    float* vel;             /* float[N][4] */
    float* force;           /* float[N][4] */
    int32_t* state;         /* int32[n_sites] */
    double* pH;             /* double[M] */
    double* E;              /* double[M] */
    int32_t* grid;          /* int32[n_pH * n_E] */
    int32_t n_sites;        /* length of state (0 when state is NULL) */
} gb_md_host;

/* gb_md_segment for a caller whose batch state lives in host memory between
 * segments (the paper's MD advances one replica's coordinates, charges and
 * site states by blocks of steps between halts, Sec. III.A-B; here a whole
 * batch at once).  On `stream`: one cudaMemcpyAsync per non-NULL array of
 * `host` into the device buffer `state` points at, nsteps MD steps exactly as
 * gb_md_segment, one cudaMemcpyAsync per array back into `host`; then waits
 * for the stream, so the host arrays hold the new state when the call
 * returns.  The device buffers of `state` are the caller's working copy.
 * Returns what gb_md_segment returns, then, after the wait, a device-detected
 * error as gb_sync_status does. */
int gb_md_segment_host(gb_ctx* ctx, gb_md_state* state, const gb_sites* sites, int64_t nsteps,
                       const gb_md_host* host, void* stream);

/* The register caps tuned on the MD driver itself: coordinate descent over
 * the three passes' caps, every candidate timed (CUDA events, best of four) on
 * an MD segment of trial_steps steps (gb_md_segment with these sites, as the
 * caller will run it), each starting from a copy of the state.  The state
 * buffers and the state struct are put back as they were before the call
 * returns; the chosen caps stay on the context (gb_get_reg_caps).  Needs
 * forces at the incoming coordinates (after gb_md_init).  Allocates a copy
 * of the state.  GB_ERR_INVALID_ARG for trial_steps outside 1..100000. */
int gb_autotune_md(gb_ctx* ctx, gb_md_state* state, const gb_sites* sites, int64_t trial_steps, void* stream);

/* Allocation-free energy / force evaluation of ONE molecule.
 *
 * The paper has no counterpart: this is a service for callers that cannot
 * call cudaMalloc -- code whose device memory all belongs to an arena or pool
 * allocator, plugins inside a host program that forbids allocations after
 * start-up, real-time loops where an allocation could stall.  Such callers
 * cannot create a gb_ctx, so this call keeps its workspace in a fixed array
 * of device memory that the library declares statically (about 0.7 MB, held by
 * every GPU that loads the library until the process exits).
 *
 * Same inputs and outputs as gb_energy_forces for a batch of one replica of
 * n_atoms atoms (1 <= n_atoms <= GB_STATIC_MAX_ATOMS); E_out is double[3].
 * The arithmetic differs in one respect: this path builds no tile bounding
 * boxes, so no block is proven far and every block takes the exact
 * near-field path (with cutoffs, every block is tested pair by pair and none
 * is skipped).  Results therefore agree with gb_energy_forces within the
 * parity tolerances (energy 1e-6 relative, forces 1e-3 kcal/mol/A), not bit
 * for bit, and the call is slower than a context's.  Works on the current
 * device.  It allocates nothing: no cudaMalloc, no cudaFree, no allocating
 * library routine.
 *  - A call outside stream capture looks up the array's device address with
 *    the device current (this allocates nothing).  A call on a capturing
 *    stream reuses the address of the last call on that device outside
 *    capture, so make one call outside capture first (again after a
 *    cudaDeviceReset); otherwise it returns GB_ERR_INVALID_ARG.
 *  - Every call on a device shares the one array and clears its accumulators
 *    first; calls that overlap on the GPU (other streams, other host threads)
 *    race on it and must be serialised by the caller.
 *  - Returns GB_ERR_INVALID_ARG when n_atoms is outside 1..GB_STATIC_MAX_ATOMS
 *    or an argument is NULL / misaligned, GB_ERR_CUDA on a launch error.
 *    Device-side non-finite results are not reported (there is no context to
 *    hold the error word, so GB_ERR_NONFINITE never comes back); they show up
 *    as NaN in the outputs. */
#define GB_STATIC_MAX_ATOMS 8192
int gb_energy_forces_static(int32_t n_atoms, const gb_params* params, const float* xyzq,
                            const float* rad_screen, float* R_out, int64_t* F_fixed,
                            float* F_out, double* E_out, double* dEdq_out, void* stream);

/* Kernel timing inside the MD driver.  When enabled, CUDA events are recorded
 * around the three pair passes of every MD step (inside a captured graph they
 * become event nodes of the graph).  gb_pass_times waits for the events of the
 * last enqueued block of steps and returns the mean duration (ms) of each pass:
 * mean_ms[0] Born integrals, [1] energy / direct forces, [2] chain rule. */
int gb_set_profiling(gb_ctx* ctx, int32_t enable);
int gb_pass_times(gb_ctx* ctx, double* mean_ms);

/* MD driver kernel choice.  Enabled (off by default): every run of MD steps
 * up to the next Monte Carlo or exchange point is ONE launch of a persistent
 * kernel whose warps take the work of those steps -- BAOAB halves, the three
 * pair passes, the O(N) transforms, replica by replica -- from a queue, each
 * item waiting only for the items of the same replica it depends on, so the
 * passes of different replicas overlap.  A wait that takes too long records
 * GB_ERR_TIMEOUT (see gb_sync_status) instead of hanging.  Disabled: six
 * launches per step (the close-and-open BAOAB step with the tile bounding
 * boxes, then the three pair passes and their two O(N) transforms), eight
 * with a cutoff (the neighbour list's reset and build).  With profiling on, gb_persist_times returns
 * out[0] the mean ms per MD step inside the persistent launches of the last
 * block, out[1] the mean ms per launch and out[2] the mean steps per launch. */
int gb_set_persistent(gb_ctx* ctx, int32_t enable);
/* Bound of every dependency wait inside the persistent MD kernel, in polls of
 * about 64 ns (0 restores the default 2^22, about a quarter of a second).  A
 * wait that runs out records GB_ERR_TIMEOUT in the context's error word
 * (gb_sync_status); the other warps then stop too and the launch ends, with
 * the MD state of that segment left undefined and the context usable (call
 * gb_md_init again).  GB_ERR_INVALID_ARG for a negative or too large value. */
int gb_set_wait_limit(gb_ctx* ctx, int64_t polls);
int gb_persist_times(gb_ctx* ctx, double* out);

#ifdef __cplusplus
}
#endif

#endif /* GBREMD_H */
