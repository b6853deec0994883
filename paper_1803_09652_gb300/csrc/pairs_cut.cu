// Launchers of the pair passes with a cutoff (EF_CUT): the Born and chain
// passes restricted to the Born-radius cutoff rgbmax, the energy pass to the
// pair cutoff `cut`.  Same walker and pass arithmetic as pairs.cu; the walker
// skips out-of-range blocks and tests the pairs of straddling ones.  Register
// caps 1 and 3 are instantiated (a request for 4 takes 3).
#include "pairs_impl.cuh"

namespace gbk {

namespace {

template <int F>
cudaError_t energy_cut(int flags, const PairArgs& a, const TaskList& t, int cap, int wpb, cudaStream_t s) {
    if constexpr (F > 15) {
        return cudaErrorInvalidValue;
    } else {
        if ((flags & 15) == F) return launch_pass<EnergyF<F | EF_CUT>, F | EF_CUT, 3>(a, t, cap, wpb, s);
        return energy_cut<F + 1>(flags, a, t, cap, wpb, s);
    }
}

}  // namespace

cudaError_t launch_pairs_cut(int pass, int flags, const PairArgs& a, const TaskList& t, int wpb,
                             cudaStream_t s) {
    const int cap = t.cap[pass];
    if (pass == PASS_BORN) return launch_pass<Born, EF_CUT, 3>(a, t, cap, wpb, s);
    if (pass == PASS_CHAIN) return launch_pass<Chain, EF_CUT, 3>(a, t, cap, wpb, s);
    return energy_cut<0>(flags, a, t, cap, wpb, s);
}

}  // namespace gbk
