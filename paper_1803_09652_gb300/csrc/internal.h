// Internal interfaces between the host library and the kernel translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gbremd.h"

namespace gbk {

typedef unsigned long long u64;

// Everything the O(N^2) pair passes read and write.
struct PairArgs {
    const int64_t* atom_off;   // [M+1]
    const float4* xyzq;        // x, y, z, q
    const float2* rad;         // rho, S
    const float2* Rh;          // R, 1/(2R)          (pass 2)
    const float* cc;           // chain factor c_i   (pass 3)
    float offset;
    float tau_ke;              // (1/eps_in - 1/eps_out) k_e
    float ke_out, kappa;       // k_e / eps_out and the salt's inverse Debye length (EF_SALT)
    float kc;                  // k_e / eps_in
    float rep_k, rep_sigma;    // soft repulsion (rep_k == 0: off)
    float rgbmax;              // Born-radius cutoff (EF_CUT kernels of the Born and chain passes)
    float cut2;                // pair cutoff squared (EF_CUT kernels of the energy pass)
    float e_range2;            // energy-pass block range squared: max(cut, rep_sigma)^2
    u64* I_acc;                // [N]   Born integrals, 2^40 fixed point
    u64* dR_acc;               // [N]   R dE/dR pair part, 2^32
    u64* phi_acc;              // [N]   dE/dq pair part, 2^32
    u64* F_acc;                // [3N]  forces x | y | z, 2^32
    u64* E_acc;                // [M*4] E_GB, E_Coul, E_rep, spare, 2^32
    int64_t N;
    float4* boxes;             // [2 * tiles] bounding boxes of 32-atom tiles (nullable)
    const int* tile_off;       // [M+1] first tile of each replica
    int* err;                  // device error word (non-finite input, nullable)
};

// One warp task: replica, super-row K (atoms 64K .. 64K+63), first tile J
// (atoms 32J .. 32J+31, J >= 2K) and number of tiles; the walk continues
// along the super-row, then into the next super-rows and replicas.
struct TaskList {
    int4* d_tasks = nullptr;
    int n_tasks = 0;
    // register cap of each pass's kernel (Born, energy, chain), as 256-thread
    // blocks per SM: 1 (compiler's choice), 3 (80 registers) or 4 (64)
    int cap[3] = {1, 1, 1};
};

enum PassKind { PASS_BORN = 0, PASS_ENERGY = 1, PASS_CHAIN = 2 };

// flags for the energy pass; EF_CUT for any pass: the kernel applies the
// pass's cutoff (Born and chain passes: rgbmax; energy pass: cut) to a task
// list of in-range blocks (launch_pairs_list).  EF_STRADDLE is internal to
// the walker: the block has pairs on both sides of the cutoff and tests each
// pair.
enum { EF_ENERGY = 1, EF_PHI = 2, EF_REP = 4, EF_SALT = 8, EF_CUT = 16, EF_STRADDLE = 32 };

cudaError_t launch_pairs(int pass, int flags, const PairArgs& a, const TaskList& t,
                         int warps_per_block, cudaStream_t s);
// Cutoff passes (pairs_cut.cu).  launch_block_list clears the LIST_CTRS
// counters and builds the block neighbour lists from the tile boxes: list_b
// (Born-radius cutoff, when want_b) and list_e (pair cutoff, when want_e),
// each with room for every block of the batch; win_off [M+1] holds the first
// list-building warp of each replica (ceil(nb/2) * ceil(nb/32) warps per
// replica of nb tiles).  launch_pairs_list runs pass `pass` with EF_CUT over
// a device-built task list whose length is ctr[0] (Born, chain) or ctr[1]
// (energy), taking tasks from the queue head ctr[2 + pass].
constexpr int LIST_CTRS = 5;
cudaError_t launch_block_list(const PairArgs& a, const int* win_off, int M, int total_warps, int4* list_b,
                              int4* list_e, int* ctr, int want_b, int want_e, cudaStream_t s);
cudaError_t launch_pairs_list(int pass, int flags, const PairArgs& a, const int4* list, int* ctr, int cap,
                              int warps_per_block, cudaStream_t s);

// Cutoff fields of the pair arguments, and the EF_CUT flag of each pass.
inline void set_cutoffs(PairArgs& a, const gb_params& p) {
    a.rgbmax = p.rgbmax;
    a.cut2 = p.cut * p.cut;
    const float er = (p.rep_k != 0.0f && p.rep_sigma > p.cut) ? p.rep_sigma : p.cut;
    a.e_range2 = er * er;
}
inline int cut_flag(int pass, const gb_params& p) {
    return (pass == PASS_ENERGY ? p.cut > 0.0f : p.rgbmax > 0.0f) ? EF_CUT : 0;
}
// Parameter checks shared by every entry point that takes gb_params.
inline bool params_ok(const gb_params& p) {
    return p.offset >= 0.0f && p.eps_in > 0.0f && p.eps_out > 0.0f && p.rep_k >= 0.0f &&
           p.rep_sigma >= 0.0f && p.kappa >= 0.0f && p.kappa < 1.0e3f && p.rgbmax >= 0.0f &&
           p.rgbmax < 1.0e6f && p.cut >= 0.0f && p.cut < 1.0e6f;
}

// Work units (32-atom tiles against 64-atom super-rows) of an n-atom replica.
int64_t pair_units(int64_t n);
// Bounding boxes of all tiles (PairArgs::boxes, tile_off); no-op when boxes is null.
cudaError_t launch_tile_boxes(const PairArgs& a, int M, int total_tiles, cudaStream_t s);

// O(N) kernels --------------------------------------------------------------

struct AtomArgs {
    const int64_t* atom_off;
    int32_t M;
    int32_t max_n;             // largest replica
    const float4* xyzq;
    const float2* rad;
    float alpha, beta, gamma, offset;
    double tau_ke;
    double kc, ke_out, kappa;  // k_e / eps_in, k_e / eps_out, salt (self terms)
    u64* I_acc;
    u64* dR_acc;
    u64* phi_acc;
    u64* F_acc;
    u64* E_acc;
    float2* Rh;
    float* cfac;               // a_i dR_i/dpsi_i
    float* cc;                 // c_i = dE/dR_i * cfac_i
    int* err;
    int64_t N;
};

cudaError_t launch_born_finalize(const AtomArgs& a, float* R_out, cudaStream_t s);
// bond_k != 0 adds the chain-bond forces (MD) to the force accumulators.
cudaError_t launch_energy_finalize(const AtomArgs& a, int want_energy, double* phi_out, cudaStream_t s,
                                   float bond_k = 0.0f, float bond_r0 = 0.0f);
cudaError_t launch_forces_out(const AtomArgs& a, int64_t* F_fixed, float* F_out, double* E_out,
                              cudaStream_t s);

struct MDArgs {
    float4* xyzq;
    float4* vel;
    float4* force;
    const u64* ctr;            // [0] step base, [1] exchange attempt base
    float h;                   // dt / 2
    float inv_m;               // ACCEL / mass
    float c1, c2;              // exp(-gamma dt), sqrt((1 - c1^2) kT ACCEL / m)
    float bond_k, bond_r0;
    u64 seed;
    u64 rep_base;              // global index of replica 0 in the Philox counters
};

// MD half steps between force evaluations (k_md_step): MD_CLOSE stores the
// evaluated force (MD_KICK: and applies the closing half kick), MD_OPEN runs
// B A O A of the next step and rebuilds the tile boxes (boxes may be null).
enum { MD_CLOSE = 1, MD_KICK = 2, MD_OPEN = 4 };
cudaError_t launch_md_step(const AtomArgs& a, const MDArgs& m, float4* boxes, const int* tile_off,
                           int step_in_block, int mode, cudaStream_t s);
cudaError_t launch_set_counters(u64* ctr, u64 step, u64 attempt, cudaStream_t s);
cudaError_t launch_advance_counters(u64* ctr, u64 steps, u64 attempts, cudaStream_t s);

// Monte Carlo: site rows are summed over MC_CHUNK-atom slices of a replica.
constexpr int MC_MAX_SITE_ATOMS = 128;
constexpr int MC_CHUNK = 256;

struct MCArgs {
    const int64_t* atom_off;
    const int32_t* site_off;
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
    float4* xyzq;
    const float* R;            // Born radii (stride 1) ...
    const float2* Rh;          // ... or (R, 1/(2R)) pairs when R == nullptr
    const double* pH;
    const double* E;
    double kT;
    double tau_ke, kc;
    double ke_out, kappa;      // salt screening of the solvent term (kappa 0: none)
    float cut2;                // pair cutoff squared (0: none)
    u64 seed;
    u64 step;
    u64 rep_base;              // global index of replica 0 in the Philox counters
    const u64* ctr;            // when non-null the step is ctr[0] + step
    int32_t kind;
    int32_t* state;
    double* dG_out;
    uint8_t* acc_out;
    double* phi_part;          // [M][n_parts][MC_MAX_SITE_ATOMS] slice partials (workspace;
                               // [M][n_parts][SWEEP_MAX_SITE_ATOMS] for sweeps)
    int32_t n_parts;           // slices of the largest replica
    int* err;                  // device error word (sweeps over their limits)
};

// Per-residue sweeps (Sec. III.A.2): limits per replica and kind.
constexpr int SWEEP_MAX_SITE_ATOMS = 1024;
constexpr int SWEEP_MAX_SITES = 256;
cudaError_t launch_mc_sweep(const MCArgs& a, int32_t M, cudaStream_t s);

cudaError_t launch_mc(const MCArgs& a, int32_t M, cudaStream_t s);

struct ExArgs {
    int32_t n_ladders, len, ladder_stride, slot_stride;
    const double* values;
    int32_t* rep_at_slot;
    const int32_t* n_count;
    int32_t dim;
    u64 attempt;
    const u64* ctr;            // when non-null the attempt is ctr[1] + attempt
    u64 seed;
    double kT;
    int32_t wrap;
    double* value_of_rep;
    double* delta_out;
    uint8_t* acc_out;
};

cudaError_t launch_exchange(const ExArgs& a, cudaStream_t s);

// Two-dimensional grid exchange used by the MD driver: the dimension of
// attempt k is E when (k / 2) is even and pH otherwise (or fixed by ex_dim).
struct GridExArgs {
    int32_t n_pH, n_E;
    const double* E_ladder;
    const double* pH_ladder;
    int32_t* grid;
    const int32_t* site_off;
    const int32_t* site_kind;
    const int32_t* site_nstates;
    const int32_t* site_state_off;
    const int32_t* n_H;
    const int32_t* n_e;
    const int32_t* state;
    const u64* ctr;
    int* err;                  // GB_ERR_INVALID_ARG on a state outside its site's range
    u64* ex_count;             // nullable [2 dims][attempts, acceptances][n_pH * n_E]
    int32_t ex_dim;            // 0 E only, 1 pH only, 2 alternate
    int32_t wrap;
    u64 seed;
    double kT;
    double* E_rep;
    double* pH_rep;
};

cudaError_t launch_grid_exchange(const GridExArgs& a, cudaStream_t s);

// State occupancy counts after a Monte Carlo halt: for every site of replica
// r, occ[g * stride + (local index of its current state)] += 1, with g the
// grid slot holding r (r itself without a grid).
struct OccArgs {
    const int32_t* site_off;
    const int32_t* site_nstates;
    const int32_t* site_state_off;
    const int32_t* state;
    const int32_t* grid;       // nullable: slot -> replica
    int32_t M, n_sites, stride;
    u64* occ;
    int* err;                  // GB_ERR_INVALID_ARG: a replica's layout or a state out of range
};
cudaError_t launch_occupancy(const OccArgs& a, cudaStream_t s);

// Persistent MD kernel (persist.cu): nsteps MD steps of the whole batch in one
// launch, as a queue of warp items with per-(phase, replica) completion counts.
struct PersistArgs {
    PairArgs pa;
    AtomArgs aa;
    MDArgs md;
    const int4* tasks;         // pair tasks of every replica, replica after replica
    const int* task_off;       // [M+1] first task of each replica
    const int* phase_off;      // [6][M+1] first item of each replica within a phase
    const int* count;          // [6][M] items of each replica per phase
    int phase_base[7];         // first item of each phase within a step; [6] = items per step
    int M;
    int nsteps;                // MD steps in this launch
    int step0;                 // index of the first of them in the enqueued block
    float* R_out;              // Born radii of the last step (nullable)
    unsigned* head;            // queue head, followed by the 6 x M completion counters
    unsigned* done;
    int* err;
    unsigned spin_limit;       // polls before a dependency wait gives up (GB_ERR_TIMEOUT)
};
size_t persist_smem();
cudaError_t persist_occupancy(int rep, int* blocks_per_sm);
cudaError_t launch_persist(const PersistArgs& a, int rep, int grid, cudaStream_t s);

cudaError_t launch_count(const int32_t* site_off, const int32_t* site_kind, const int32_t* site_nstates,
                         const int32_t* site_state_off, const int32_t* n_H,
                         const int32_t* n_e, const int32_t* state, int32_t kind, int32_t M,
                         int32_t* out, cudaStream_t s);

}  // namespace gbk
