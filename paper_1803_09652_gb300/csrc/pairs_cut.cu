// GB with cutoffs: the block neighbour list and the pair passes that walk it.
//
// Every evaluation rebuilds the list from the tile bounding boxes of that
// evaluation (k_tile_boxes, or k_md_step in the MD driver).  One warp covers
// 32 consecutive blocks (K, J0 .. J0+31) of a super-row: lane l classifies
// block (K, J0 + l) with cut_class, a ballot gives the warp the in-range bits,
// and every run of consecutive in-range blocks (cut at 16 blocks) becomes one
// task (replica, K, first J, length) of a compacted list, placed with one
// atomic per warp.  Two lists: the Born-radius cutoff's (Born and chain
// passes) and the pair cutoff's (energy pass).  The passes then take the
// tasks from a queue (k_pairs_dyn): blocks out of range cost nothing, and
// the warps' work evens out whatever the list's order.
//
// Counters (one int each): [0] Born-list length, [1] energy-list length,
// [2] [3] [4] queue heads of the Born, energy and chain passes.  The cutoff
// kernels come with register caps 1 and 3 (a request for 4 takes 3).
#include "pairs_impl.cuh"

namespace gbk {

namespace {

__global__ void k_list_reset(int* ctr) {
    pdl_enter();
    if (threadIdx.x < LIST_CTRS) ctr[threadIdx.x] = 0;
}

// Appends the runs of set bits of m (lanes = blocks J0 ..) to a list.
__device__ __forceinline__ void emit_runs(unsigned m, int lane, int r, int K, int J0, int4* list, int* counter) {
    const bool on = (m >> lane) & 1u;
    const bool prev = lane > 0 && ((m >> (lane - 1)) & 1u);
    const bool start = on && (!prev || (lane & 15) == 0);
    const unsigned sm = __ballot_sync(0xffffffffu, start);
    if (!sm) return;
    int base = 0;
    if (lane == 0) base = atomicAdd(counter, __popc(sm));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (start) {
        const unsigned rest = ~(m >> lane);          // the run ends at the first zero
        int len = rest ? __ffs(rest) - 1 : 32 - lane;
        len = min(len, 16 - (lane & 15));
        list[base + __popc(sm & ((1u << lane) - 1u))] = make_int4(r, K, J0 + lane, len);
    }
}

// win_off[r]: first warp of replica r; a replica has ceil(nb/2) super-rows of
// ceil(nb/32) warps each (warps past the row's last block exit).
__global__ void k_block_list(PairArgs A, const int* __restrict__ win_off, int M, int total, int4* list_b,
                             int4* list_e, int* ctr, int want_b, int want_e) {
    pdl_enter();
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= total) return;
    int lo = 0, hi = M;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (win_off[mid] <= w) lo = mid;
        else hi = mid;
    }
    const int r = lo;
    const int n = (int)(A.atom_off[r + 1] - A.atom_off[r]);
    const int nb = (n + 31) >> 5;
    const int wr = (nb + 31) >> 5;
    const int local = w - win_off[r];
    const int K = local / wr;
    const int J0 = 2 * K + 32 * (local % wr);
    if (J0 >= nb) return;
    const int t0 = A.tile_off[r];
    float4 ih;
    const float4 il = row_box_lo(A, t0, K, nb, &ih);
    const int J = J0 + lane;
    bool in_b = false, in_e = false, st;
    if (J < nb) {
        const BoxPair b = box_pair(il, ih, __ldcg(&A.boxes[2 * (t0 + J)]), __ldcg(&A.boxes[2 * (t0 + J) + 1]));
        if (want_b) cut_class(A, true, b, in_b, st);
        if (want_e) cut_class(A, false, b, in_e, st);
    }
    if (want_b) emit_runs(__ballot_sync(0xffffffffu, in_b), lane, r, K, J0, list_b, &ctr[0]);
    if (want_e) emit_runs(__ballot_sync(0xffffffffu, in_e), lane, r, K, J0, list_e, &ctr[1]);
}

constexpr int MAX_DEVICES = 64;

int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) dev = 0;
    return dev;
}

// Resident blocks per SM of one instantiation at wpb warps per block, cached
// per device (0 = not queried yet; a lost race only repeats the query).
template <class P, int FLAGS, int MINB>
int resident_blocks(int wpb) {
    static int cache[MAX_DEVICES][17] = {};
    if (wpb < 1 || wpb > 16) return 1;
    int& c = cache[current_device()][wpb];
    if (!c) {
        int per_sm = 0;
        const size_t smem = (size_t)wpb * P::NQ * 64 * sizeof(long long);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pairs_dyn<P, FLAGS, MINB>, 32 * wpb, smem) !=
                cudaSuccess || per_sm < 1)
            per_sm = 1;
        c = per_sm;
    }
    return c;
}

int sm_count() {
    static int cache[MAX_DEVICES] = {};
    const int dev = current_device();
    if (!cache[dev]) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
        cache[dev] = sms;
    }
    return cache[dev];
}

template <class P, int FLAGS, int MINB>
cudaError_t dyn_pass_cap(const PairArgs& a, const int4* list, int* ctr, int ci, int hi, int wpb, cudaStream_t s) {
    const size_t smem = (size_t)wpb * P::NQ * 64 * sizeof(long long);
    const int blocks = sm_count() * resident_blocks<P, FLAGS, MINB>(wpb);
    return launch_pdl(k_pairs_dyn<P, FLAGS, MINB>, dim3(blocks), dim3(32 * wpb), smem, s, a, list, ctr, ci, hi);
}

template <class P, int FLAGS>
cudaError_t dyn_pass(const PairArgs& a, const int4* list, int* ctr, int ci, int hi, int cap, int wpb,
                     cudaStream_t s) {
    if (cap >= 3) return dyn_pass_cap<P, FLAGS, 3>(a, list, ctr, ci, hi, wpb, s);
    return dyn_pass_cap<P, FLAGS, 1>(a, list, ctr, ci, hi, wpb, s);
}

template <int F>
cudaError_t energy_dyn(int flags, const PairArgs& a, const int4* list, int* ctr, int ci, int hi, int cap, int wpb,
                       cudaStream_t s) {
    if constexpr (F > 15) {
        return cudaErrorInvalidValue;
    } else {
        if ((flags & 15) == F) return dyn_pass<EnergyF<F | EF_CUT>, F | EF_CUT>(a, list, ctr, ci, hi, cap, wpb, s);
        return energy_dyn<F + 1>(flags, a, list, ctr, ci, hi, cap, wpb, s);
    }
}

}  // namespace

cudaError_t launch_block_list(const PairArgs& a, const int* win_off, int M, int total_warps, int4* list_b,
                              int4* list_e, int* ctr, int want_b, int want_e, cudaStream_t s) {
    cudaError_t e = launch_pdl(k_list_reset, dim3(1), dim3(32), 0, s, ctr);
    if (e != cudaSuccess || total_warps == 0) return e;
    return launch_pdl(k_block_list, dim3((total_warps + 7) / 8), dim3(256), 0, s, a, win_off, M, total_warps,
                      list_b, list_e, ctr, want_b, want_e);
}

cudaError_t launch_pairs_list(int pass, int flags, const PairArgs& a, const int4* list, int* ctr, int cap, int wpb,
                              cudaStream_t s) {
    const int ci = (pass == PASS_ENERGY) ? 1 : 0;
    const int hi = 2 + pass;
    if (pass == PASS_BORN) return dyn_pass<Born, EF_CUT>(a, list, ctr, ci, hi, cap, wpb, s);
    if (pass == PASS_CHAIN) return dyn_pass<Chain, EF_CUT>(a, list, ctr, ci, hi, cap, wpb, s);
    return energy_dyn<0>(flags, a, list, ctr, ci, hi, cap, wpb, s);
}

}  // namespace gbk
