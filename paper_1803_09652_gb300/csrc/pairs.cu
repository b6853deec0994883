// Launchers of the O(N^2) pair passes without cutoffs (the block neighbour
// list and the passes with a cutoff are in pairs_cut.cu); the pass
// arithmetic, the warp walk and the kernel templates are in pairs_impl.cuh
// (shared with the persistent MD kernel).
#include "pairs_impl.cuh"

namespace gbk {

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

cudaError_t launch_pairs(int pass, int flags, const PairArgs& a, const TaskList& t, int wpb,
                         cudaStream_t s) {
    if (flags & EF_CUT) return cudaErrorInvalidValue;     // cutoff passes: launch_pairs_list
    const int cap = t.cap[pass];
    if (pass == PASS_BORN) return launch_pass<Born, 0>(a, t, cap, wpb, s);
    if (pass == PASS_CHAIN) return launch_pass<Chain, 0>(a, t, cap, wpb, s);
    switch (flags & 15) {
        case 0: return launch_pass<EnergyF<0>, 0>(a, t, cap, wpb, s);
        case 1: return launch_pass<EnergyF<1>, 1>(a, t, cap, wpb, s);
        case 2: return launch_pass<EnergyF<2>, 2>(a, t, cap, wpb, s);
        case 3: return launch_pass<EnergyF<3>, 3>(a, t, cap, wpb, s);
        case 4: return launch_pass<EnergyF<4>, 4>(a, t, cap, wpb, s);
        case 5: return launch_pass<EnergyF<5>, 5>(a, t, cap, wpb, s);
        case 6: return launch_pass<EnergyF<6>, 6>(a, t, cap, wpb, s);
        case 7: return launch_pass<EnergyF<7>, 7>(a, t, cap, wpb, s);
        case 8: return launch_pass<EnergyF<8>, 8>(a, t, cap, wpb, s);
        case 9: return launch_pass<EnergyF<9>, 9>(a, t, cap, wpb, s);
        case 10: return launch_pass<EnergyF<10>, 10>(a, t, cap, wpb, s);
        case 11: return launch_pass<EnergyF<11>, 11>(a, t, cap, wpb, s);
        case 12: return launch_pass<EnergyF<12>, 12>(a, t, cap, wpb, s);
        case 13: return launch_pass<EnergyF<13>, 13>(a, t, cap, wpb, s);
        case 14: return launch_pass<EnergyF<14>, 14>(a, t, cap, wpb, s);
        default: return launch_pass<EnergyF<15>, 15>(a, t, cap, wpb, s);
    }
}

// Work units (tiles) of one replica of n atoms in the walk above.
int64_t pair_units(int64_t n) {
    const int64_t nb = (n + 31) / 32, nk = (nb + 1) / 2;
    return nk * nb - nk * (nk - 1);
}

}  // namespace gbk
