// Persistent MD kernel: several BAOAB steps of the whole batch in one launch,
// scheduled as a stream of warp-sized work items with per-replica
// dependencies instead of global barriers.
//
// Each MD step s of replica r runs six phases:
//   0  close step s-1 (total force -> kick), open step s (B A O A), rebuild
//      the tile's bounding box                              [item: 32-atom tile]
//   1  Born integrals                                       [item: pair task]
//   2  Born radii                                           [item: 32 atoms]
//   3  GB + Coulomb forces, dE/dR, soft repulsion           [item: pair task]
//   4  chain factors, chain bonds                           [item: 32 atoms]
//   5  Born chain-rule forces                               [item: pair task]
// and the launch ends with phase 0 of step nsteps (kick only; the forces are
// stored for the next launch).  Items are numbered step-major, then
// phase-major, then replica-major, and warps take them in that order from a
// global counter.  Phase p > 0 of (s, r) waits until all phase p-1 items of
// (s, r) are done, phase 0 of (s, r) until all phase 5 items of (s-1, r) are
// done.  Every wait is on items that come earlier in the order, which some
// running warp has already taken and will finish, so the schedule cannot
// deadlock and needs no co-residency.  While the last replica of a pass is
// still finishing, other warps already work on the next pass of the first
// replicas: the pass tails of a small batch overlap.
//
// Waits are bounded: after P.spin_limit polls (2^22 by default, about a
// quarter of a second; gb_set_wait_limit) the warp records GB_ERR_TIMEOUT and
// stops taking work; the others then see the error word, or time out on it,
// and stop too, so the launch always ends and the context stays usable.
#include "atoms_impl.cuh"
#include "pairs_impl.cuh"

namespace gbk {

constexpr int PERSIST_THREADS = 128;
constexpr int PERSIST_NQ = Energy::NQ;   // largest i-side accumulator slot of the three passes

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Lane 0 waits until *ctr >= target; returns false when the wait gave up or
// another warp reported an error.
__device__ __forceinline__ bool wait_count(const unsigned* ctr, unsigned target, int* err, unsigned limit,
                                           int lane) {
    int ok = 1;
    if (lane == 0) {
        unsigned it = 0;
        while (ld_acquire(ctr) < target) {
            if (*(volatile int*)err != 0) { ok = 0; break; }
            if (++it > limit) {
                atomicCAS(err, 0, GB_ERR_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok != 0;
}

// Phase 0 on tile u of replica r.  second: close the previous step (force
// from the accumulators, kick).  first: open step `step` (B A O A with the
// same force) and rebuild the tile's box; otherwise store the force.
__device__ __forceinline__ void tile_halfsteps(const PersistArgs& P, int r, int u, int lane, bool second,
                                               bool first, u64 step) {
    const MDArgs& m = P.md;
    const int64_t N = P.pa.N;
    const int64_t base = P.pa.atom_off[r];
    const int n = (int)(P.pa.atom_off[r + 1] - base);
    const int i = 32 * u + lane;
    if (i < n) {
        const int64_t g = base + i;
        float4 v = __ldcg(&m.vel[g]);
        float4 f;
        if (second) {
            f = make_float4((float)unfix(__ldcg(&P.aa.F_acc[g])), (float)unfix(__ldcg(&P.aa.F_acc[N + g])),
                            (float)unfix(__ldcg(&P.aa.F_acc[2 * N + g])), 0.0f);
            P.aa.F_acc[g] = 0;
            P.aa.F_acc[N + g] = 0;
            P.aa.F_acc[2 * N + g] = 0;
            v.x = fmaf(m.h * m.inv_m, f.x, v.x);
            v.y = fmaf(m.h * m.inv_m, f.y, v.y);
            v.z = fmaf(m.h * m.inv_m, f.z, v.z);
        } else {
            f = __ldcg(&m.force[g]);
        }
        if (first) {
            float4 x = __ldcg(&m.xyzq[g]);
            baoab_first(m, x, v, f, md_normals(m.seed, m.rep_base + (u64)r, step, (u64)i));
            m.xyzq[g] = x;
        } else {
            m.force[g] = f;
        }
        m.vel[g] = v;
    }
    if (first) tile_box_warp(P.pa, P.M, P.pa.tile_off[r] + u, lane);
}

// Phase 4 on atoms 32u .. 32u+31 of replica r: chain factor, chain bonds.
__device__ __forceinline__ void atoms_chain_bonds(const PersistArgs& P, int r, int u, int lane) {
    const int64_t N = P.pa.N;
    const int64_t base = P.pa.atom_off[r];
    const int n = (int)(P.pa.atom_off[r + 1] - base);
    const int i = 32 * u + lane;
    if (i >= n) return;
    const int64_t g = base + i;
    double R;
    chain_factor_atom(P.aa, g, &R);
    const float3 fb = bond_force(P.md, P.md.xyzq, base, i, n);
    P.aa.F_acc[g] = __ldcg(&P.aa.F_acc[g]) + (u64)fix(fb.x);
    P.aa.F_acc[N + g] = __ldcg(&P.aa.F_acc[N + g]) + (u64)fix(fb.y);
    P.aa.F_acc[2 * N + g] = __ldcg(&P.aa.F_acc[2 * N + g]) + (u64)fix(fb.z);
}

template <int REP>
__global__ void __launch_bounds__(PERSIST_THREADS, 6) k_md_persist(PersistArgs P) {
    extern __shared__ long long s_acc[];
    constexpr int EFL = REP ? EF_REP : 0;
    const int lane = threadIdx.x & 31;
    long long* sa = s_acc + (threadIdx.x >> 5) * PERSIST_NQ * 64;
    const unsigned per_step = (unsigned)P.phase_base[6];
    const unsigned total = per_step * (unsigned)P.nsteps + (unsigned)P.phase_base[1];
    const u64 step0 = __ldcg(&P.md.ctr[0]) + (u64)P.step0;
    for (;;) {
        unsigned item = 0;
        if (lane == 0) item = atomicAdd(P.head, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= total) break;
        const int s = (int)(item / per_step);
        const unsigned rem = item - (unsigned)s * per_step;
        int p = 0;
        while (p < 5 && rem >= (unsigned)P.phase_base[p + 1]) ++p;
        const int* off = P.phase_off + p * (P.M + 1);
        const int x = (int)(rem - (unsigned)P.phase_base[p]);
        int lo = 0, hi = P.M;                  // replica with off[lo] <= x < off[lo + 1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (off[mid] <= x) lo = mid;
            else hi = mid;
        }
        const int r = lo, u = x - off[r];
        // dependency: the previous phase of (s, r) -- or phase 5 of (s-1, r)
        bool ok = true;
        if (p > 0) {
            ok = wait_count(&P.done[(p - 1) * P.M + r], (unsigned)(s + 1) * (unsigned)P.count[(p - 1) * P.M + r],
                            P.err, P.spin_limit, lane);
        } else if (s > 0) {
            ok = wait_count(&P.done[5 * P.M + r], (unsigned)s * (unsigned)P.count[5 * P.M + r], P.err,
                            P.spin_limit, lane);
        }
        if (!ok) break;
        switch (p) {
            case 0: tile_halfsteps(P, r, u, lane, s > 0, s < P.nsteps, step0 + (u64)s + 1); break;
            case 1: walk_task<Born, 0>(P.pa, P.tasks[P.task_off[r] + u], sa, lane); break;
            case 2: {
                const int64_t base = P.pa.atom_off[r];
                const int i = 32 * u + lane;
                if (i < (int)(P.pa.atom_off[r + 1] - base)) born_finalize_atom(P.aa, base + i, P.R_out);
                break;
            }
            case 3: walk_task<EnergyF<EFL>, EFL>(P.pa, P.tasks[P.task_off[r] + u], sa, lane); break;
            case 4: atoms_chain_bonds(P, r, u, lane); break;
            default: walk_task<Chain, 0>(P.pa, P.tasks[P.task_off[r] + u], sa, lane); break;
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) atomicAdd(&P.done[p * P.M + r], 1u);
    }
}

size_t persist_smem() { return (size_t)(PERSIST_THREADS / 32) * PERSIST_NQ * 64 * sizeof(long long); }

cudaError_t persist_occupancy(int rep, int* blocks_per_sm) {
    const size_t smem = persist_smem();
    if (rep) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_md_persist<1>, PERSIST_THREADS, smem);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_md_persist<0>, PERSIST_THREADS, smem);
}

cudaError_t launch_persist(const PersistArgs& a, int rep, int grid, cudaStream_t s) {
    // queue head and the per-(phase, replica) completion counters start at zero
    cudaError_t e = cudaMemsetAsync(a.head, 0, sizeof(unsigned) * (1 + 6 * (size_t)a.M), s);
    if (e != cudaSuccess) return e;
    const size_t smem = persist_smem();
    if (rep) k_md_persist<1><<<grid, PERSIST_THREADS, smem, s>>>(a);
    else k_md_persist<0><<<grid, PERSIST_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gbk
