// Persistent MD kernel: all phases of several BAOAB steps of the whole batch in
// one cooperative launch, separated by grid-wide barriers.
//
// The three pair passes of a small batch (8 x 2048 atoms: ~40 us each) lose a
// large share of their time to launch, ramp-up and tail; here every block
// stays resident for the whole launch and the phases of a step are
//   A  second half of the previous step (total force -> kick), first half of
//      this step (B A O A), bounding boxes of the moved tiles   [warp per tile]
//   1  Born integrals                                          [warp tasks]
//   2  Born radii                                              [thread per atom]
//   3  GB + Coulomb forces, dE/dR, soft repulsion              [warp tasks]
//   4  chain factors, chain bonds                              [thread per atom]
//   5  Born chain-rule forces                                  [warp tasks]
// with a barrier after each.  The last step ends with the second half only
// and stores the forces for the next launch.  Monte Carlo attempts and
// exchanges run between launches.
//
// Barrier: one arrival counter and one release word, both cleared before the
// launch.  Waits are bounded: after SPIN_LIMIT polls a block records
// GB_ERR_TIMEOUT and every block leaves the kernel at its next barrier.  The
// launch is cooperative, so all blocks are co-resident and the limit is never
// reached in correct operation.
#include "atoms_impl.cuh"
#include "pairs_impl.cuh"

namespace gbk {

constexpr unsigned SPIN_LIMIT = 1u << 22;
constexpr int PERSIST_THREADS = 128;
constexpr int PERSIST_NQ = Energy::NQ;   // largest i-side accumulator slot of the three passes

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Returns false (in every thread of the block) when the kernel must stop.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned& epoch, int* err) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ++epoch;
        __threadfence();
        const unsigned arrived = atomicAdd(&bar[0], 1u) + 1u;
        int ok = 1;
        if (arrived == gridDim.x * epoch) {
            __threadfence();
            atomicExch(&bar[1], epoch);
        } else {
            unsigned it = 0;
            while (ld_acquire(&bar[1]) < epoch) {
                if (++it > SPIN_LIMIT) {
                    atomicCAS(err, 0, GB_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        s_ok = ok && (*(volatile int*)err == 0);
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ int replica_of_tile(const PairArgs& A, int M, int t) {
    int lo = 0, hi = M;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (A.tile_off[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int replica_of_atom(const AtomArgs& A, int M, int64_t g) {
    int lo = 0, hi = M;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (A.atom_off[mid] <= g) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Phase A over the tiles owned by this warp.  second: close the previous step
// (force from the accumulators, kick).  s_first >= 0: open step s_first
// (B A O A with the same force) and rebuild the tile's box; otherwise store
// the force for the next launch.
__device__ __forceinline__ void phase_halfsteps(const PersistArgs& P, int gw, int W, int lane, bool second,
                                                int s_first) {
    const MDArgs& m = P.md;
    const int64_t N = P.pa.N;
    for (int t = gw; t < P.total_tiles; t += W) {
        const int r = replica_of_tile(P.pa, P.M, t);
        const int64_t base = P.pa.atom_off[r];
        const int n = (int)(P.pa.atom_off[r + 1] - base);
        const int i = 32 * (t - P.pa.tile_off[r]) + lane;
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
            if (s_first >= 0) {
                float4 x = __ldcg(&m.xyzq[g]);
                const u64 step = __ldcg(&m.ctr[0]) + (u64)(P.step0 + s_first) + 1;
                baoab_first(m, x, v, f, md_normals(m.seed, (u64)r, step, (u64)i));
                m.xyzq[g] = x;
            } else {
                m.force[g] = f;
            }
            m.vel[g] = v;
        }
        if (s_first >= 0) tile_box_warp(P.pa, P.M, t, lane);
    }
}

template <int REP>
__global__ void __launch_bounds__(PERSIST_THREADS, 6) k_md_persist(PersistArgs P) {
    extern __shared__ long long s_acc[];
    constexpr int EFL = REP ? EF_REP : 0;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
    const int W = gridDim.x * (blockDim.x >> 5);
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    long long* sa = s_acc + wib * PERSIST_NQ * 64;
    const int64_t N = P.pa.N;
    unsigned epoch = 0;

    phase_halfsteps(P, gw, W, lane, false, 0);
    for (int s = 0; s < P.nsteps; ++s) {
        if (!grid_barrier(P.bar, epoch, P.err)) return;
        for (int t = gw; t < P.n_tasks; t += W) walk_task<Born, 0>(P.pa, P.tasks[t], sa, lane);
        if (!grid_barrier(P.bar, epoch, P.err)) return;
        for (int64_t g = gt; g < N; g += T) born_finalize_atom(P.aa, g, P.R_out);
        if (!grid_barrier(P.bar, epoch, P.err)) return;
        for (int t = gw; t < P.n_tasks; t += W) walk_task<EnergyF<EFL>, EFL>(P.pa, P.tasks[t], sa, lane);
        if (!grid_barrier(P.bar, epoch, P.err)) return;
        for (int64_t g = gt; g < N; g += T) {
            double R;
            chain_factor_atom(P.aa, g, &R);
            const int r = replica_of_atom(P.aa, P.M, g);
            const int64_t base = P.aa.atom_off[r];
            const int n = (int)(P.aa.atom_off[r + 1] - base);
            const float3 fb = bond_force(P.md, P.md.xyzq, base, (int)(g - base), n);
            P.aa.F_acc[g] = __ldcg(&P.aa.F_acc[g]) + (u64)fix(fb.x);
            P.aa.F_acc[N + g] = __ldcg(&P.aa.F_acc[N + g]) + (u64)fix(fb.y);
            P.aa.F_acc[2 * N + g] = __ldcg(&P.aa.F_acc[2 * N + g]) + (u64)fix(fb.z);
        }
        if (!grid_barrier(P.bar, epoch, P.err)) return;
        for (int t = gw; t < P.n_tasks; t += W) walk_task<Chain, 0>(P.pa, P.tasks[t], sa, lane);
        if (!grid_barrier(P.bar, epoch, P.err)) return;
        phase_halfsteps(P, gw, W, lane, true, s + 1 < P.nsteps ? s + 1 : -1);
    }
}

size_t persist_smem() { return (size_t)(PERSIST_THREADS / 32) * PERSIST_NQ * 64 * sizeof(long long); }

cudaError_t persist_occupancy(int rep, int* blocks_per_sm) {
    const size_t smem = persist_smem();
    if (rep) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_md_persist<1>, PERSIST_THREADS, smem);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_md_persist<0>, PERSIST_THREADS, smem);
}

cudaError_t launch_persist(const PersistArgs& a, int rep, int grid, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(PERSIST_THREADS);
    cfg.dynamicSmemBytes = persist_smem();
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (rep) return cudaLaunchKernelEx(&cfg, k_md_persist<1>, a);
    return cudaLaunchKernelEx(&cfg, k_md_persist<0>, a);
}

}  // namespace gbk
