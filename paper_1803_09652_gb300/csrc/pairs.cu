// Launchers of the O(N^2) pair passes; the pass arithmetic and the warp walk
// are in pairs_impl.cuh (shared with the persistent MD kernel).
#include "pairs_impl.cuh"

namespace gbk {

// MINB = 1 leaves the register count to the compiler; MINB = 3 or 4 caps it so
// that three or four 256-thread blocks fit on an SM (more warps, some spills).
template <class P, int FLAGS, int MINB>
__global__ void __launch_bounds__(256, MINB) k_pairs(PairArgs A, const int4* __restrict__ tasks, int n_tasks) {
    pdl_enter();
    extern __shared__ long long s_acc[];
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= n_tasks) return;
    walk_task<P, FLAGS>(A, tasks[w], s_acc + (threadIdx.x >> 5) * P::NQ * 64, lane);
}

__global__ void k_tile_boxes(PairArgs A, int M, int total_tiles) {
    pdl_enter();
    const int lane = threadIdx.x & 31;
    const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (t >= total_tiles) return;
    tile_box_warp(A, M, t, lane);
}

cudaError_t launch_tile_boxes(const PairArgs& a, int M, int total_tiles, cudaStream_t s) {
    if (!a.boxes || total_tiles == 0) return cudaSuccess;
    return launch_pdl(k_tile_boxes, dim3((total_tiles + 7) / 8), dim3(256), 0, s, a, M, total_tiles);
}

template <class P, int FLAGS>
static cudaError_t go(const PairArgs& a, const TaskList& t, int cap, int wpb, cudaStream_t s) {
    if (t.n_tasks == 0) return cudaSuccess;
    const int blocks = (t.n_tasks + wpb - 1) / wpb;
    const size_t smem = (size_t)wpb * P::NQ * 64 * sizeof(long long);
    const dim3 g(blocks), b(32 * wpb);
    if (cap >= 4) return launch_pdl(k_pairs<P, FLAGS, 4>, g, b, smem, s, a, t.d_tasks, t.n_tasks);
    if (cap == 3) return launch_pdl(k_pairs<P, FLAGS, 3>, g, b, smem, s, a, t.d_tasks, t.n_tasks);
    return launch_pdl(k_pairs<P, FLAGS, 1>, g, b, smem, s, a, t.d_tasks, t.n_tasks);
}

cudaError_t launch_pairs(int pass, int flags, const PairArgs& a, const TaskList& t, int wpb,
                         cudaStream_t s) {
    const int cap = t.cap[pass];
    if (pass == PASS_BORN) return go<Born, 0>(a, t, cap, wpb, s);
    if (pass == PASS_CHAIN) return go<Chain, 0>(a, t, cap, wpb, s);
    switch (flags & 15) {
        case 0: return go<EnergyF<0>, 0>(a, t, cap, wpb, s);
        case 1: return go<EnergyF<1>, 1>(a, t, cap, wpb, s);
        case 2: return go<EnergyF<2>, 2>(a, t, cap, wpb, s);
        case 3: return go<EnergyF<3>, 3>(a, t, cap, wpb, s);
        case 4: return go<EnergyF<4>, 4>(a, t, cap, wpb, s);
        case 5: return go<EnergyF<5>, 5>(a, t, cap, wpb, s);
        case 6: return go<EnergyF<6>, 6>(a, t, cap, wpb, s);
        case 7: return go<EnergyF<7>, 7>(a, t, cap, wpb, s);
        case 8: return go<EnergyF<8>, 8>(a, t, cap, wpb, s);
        case 9: return go<EnergyF<9>, 9>(a, t, cap, wpb, s);
        case 10: return go<EnergyF<10>, 10>(a, t, cap, wpb, s);
        case 11: return go<EnergyF<11>, 11>(a, t, cap, wpb, s);
        case 12: return go<EnergyF<12>, 12>(a, t, cap, wpb, s);
        case 13: return go<EnergyF<13>, 13>(a, t, cap, wpb, s);
        case 14: return go<EnergyF<14>, 14>(a, t, cap, wpb, s);
        default: return go<EnergyF<15>, 15>(a, t, cap, wpb, s);
    }
}

// Work units (tiles) of one replica of n atoms in the walk above.
int64_t pair_units(int64_t n) {
    const int64_t nb = (n + 31) / 32, nk = (nb + 1) / 2;
    return nk * nb - nk * (nk - 1);
}

}  // namespace gbk
