// gb_energy_forces_static: the energy / force evaluation of one molecule
// without any device allocation.
//
// Who needs it: callers that may not call cudaMalloc -- code running inside a
// memory-pool or arena allocator that owns all device memory, plugins loaded
// into a host program that forbids allocations after start-up, and real-time
// loops where an allocation could block.  Such a caller cannot create a
// gb_ctx (gb_ctx_create allocates its workspace), so this entry point keeps
// its workspace in one file-scope __device__ array instead.
//
// The array holds the fixed-point accumulators, Born radii, chain factors and
// the tile work list for one molecule of at most GB_STATIC_MAX_ATOMS atoms
// (about 0.7 MB).  Every GPU that loads the library keeps it until the
// process exits.  It is shared by all calls on a device: calls that overlap
// on the GPU (two streams, or two host threads) race on it and must be
// serialised by the caller.
#include <cstdint>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int kMaxAtoms = GB_STATIC_MAX_ATOMS;
constexpr int kTilesPerTask = 4;
constexpr int kMaxTiles = (kMaxAtoms / 32) * (kMaxAtoms / 32 + 1) / 2;
constexpr int kMaxTasks = (kMaxTiles + kTilesPerTask - 1) / kTilesPerTask;

constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Byte offsets of the sub-buffers inside the scratch array.
constexpr size_t kOffI = 0;                                                   // u64[max]
constexpr size_t kOffDR = kOffI + align256(8ull * kMaxAtoms);                  // u64[max]
constexpr size_t kOffPhi = kOffDR + align256(8ull * kMaxAtoms);                // u64[max]
constexpr size_t kOffF = kOffPhi + align256(8ull * kMaxAtoms);                 // u64[3 max]
constexpr size_t kOffE = kOffF + align256(24ull * kMaxAtoms);                  // u64[4]
constexpr size_t kAccEnd = kOffE + 256;                                        // accumulators end here
constexpr size_t kOffRh = kAccEnd;                                             // float2[max]
constexpr size_t kOffCfac = kOffRh + align256(8ull * kMaxAtoms);               // float[max]
constexpr size_t kOffCc = kOffCfac + align256(4ull * kMaxAtoms);               // float[max]
constexpr size_t kOffOff = kOffCc + align256(4ull * kMaxAtoms);                // int64[2]
constexpr size_t kOffErr = kOffOff + 256;                                      // int
constexpr size_t kOffCtr = kOffErr + 256;                                      // int[LIST_CTRS]
constexpr size_t kOffTasks = kOffCtr + 256;                                    // int4[max tasks]
constexpr size_t kBytes = kOffTasks + align256(16ull * kMaxTasks);

__device__ __align__(256) unsigned char gb_static_scratch[kBytes];

// Device address of gb_static_scratch.  The host-side symbol is only a
// stand-in, so the address is looked up with the device current.  A call
// outside stream capture looks it up afresh every time: the lookup allocates
// nothing, and after cudaDeviceReset the module (and with it the array) may
// come back at another address.  A call on a capturing stream cannot make
// API calls that might load a module, so it uses the address of the last
// call on that device outside capture, cached per device ordinal.
constexpr int kMaxDevices = 64;
unsigned char* g_scratch[kMaxDevices] = {};
std::mutex g_scratch_mu;

int scratch_for_current_device(cudaStream_t s, unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GB_ERR_CUDA;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return GB_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, gb_static_scratch) != cudaSuccess || !p) return GB_ERR_CUDA;
        g_scratch[dev] = (unsigned char*)p;
    }
    if (!g_scratch[dev]) return GB_ERR_INVALID_ARG;   // first call on this device is inside a capture
    *out = g_scratch[dev];
    return GB_OK;
}

// Work list of one molecule: run w covers work units [w*tpt, (w+1)*tpt) of the
// pair walk (super-rows K of 64 atoms against tiles J = 2K .. nb-1).  Also
// writes atom_off = {0, n}.
__global__ void k_static_tasks(int n, int nb, int tpt, int n_tasks, int64_t total, int4* tasks,
                               int64_t* atom_off, int* ctr) {
    gbk::pdl_enter();
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w == 0) {
        atom_off[0] = 0;
        atom_off[1] = n;
        // the cutoff passes walk this list from a queue: lengths, cleared heads
        ctr[0] = ctr[1] = n_tasks;
        ctr[2] = ctr[3] = ctr[4] = 0;
    }
    if (w >= n_tasks) return;
    int64_t p = (int64_t)w * tpt;
    const int nk = (nb + 1) / 2;
    int K = 0;
    while (K < nk && p >= nb - 2 * K) {
        p -= nb - 2 * K;
        ++K;
    }
    const int64_t left = total - (int64_t)w * tpt;
    tasks[w] = make_int4(0, K, 2 * K + (int)p, (int)(left < tpt ? left : tpt));
}

}  // namespace

extern "C" int gb_energy_forces_static(int32_t n_atoms, const gb_params* params, const float* xyzq,
                                       const float* rad_screen, float* R_out, int64_t* F_fixed,
                                       float* F_out, double* E_out, double* dEdq_out, void* stream) {
    if (n_atoms < 1 || n_atoms > kMaxAtoms) return GB_ERR_INVALID_ARG;
    if (!params || !xyzq || !rad_screen) return GB_ERR_INVALID_ARG;
    if (!R_out && !F_fixed && !F_out && !E_out && !dEdq_out) return GB_ERR_INVALID_ARG;
    if (((uintptr_t)xyzq % 16) || ((uintptr_t)rad_screen % 8)) return GB_ERR_INVALID_ARG;
    if (!gbk::params_ok(*params)) return GB_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* base = nullptr;
    int rc = scratch_for_current_device(s, &base);
    if (rc) return rc;
    const int n = n_atoms;
    const int nb = (n + 31) / 32;
    const int64_t total = gbk::pair_units(n);
    const int n_tasks = (int)((total + kTilesPerTask - 1) / kTilesPerTask);

    gbk::u64* I_acc = (gbk::u64*)(base + kOffI);
    gbk::u64* dR_acc = (gbk::u64*)(base + kOffDR);
    gbk::u64* phi_acc = (gbk::u64*)(base + kOffPhi);
    gbk::u64* F_acc = (gbk::u64*)(base + kOffF);
    gbk::u64* E_acc = (gbk::u64*)(base + kOffE);
    float2* Rh = (float2*)(base + kOffRh);
    float* cfac = (float*)(base + kOffCfac);
    float* cc = (float*)(base + kOffCc);
    int64_t* atom_off = (int64_t*)(base + kOffOff);
    int* err = (int*)(base + kOffErr);
    int* ctr = (int*)(base + kOffCtr);
    int4* tasks = (int4*)(base + kOffTasks);

    // the accumulators keep the last call's contents: start from zero
    if (cudaMemsetAsync(base, 0, kAccEnd, s) != cudaSuccess) return GB_ERR_CUDA;
    if (gbk::launch_pdl(k_static_tasks, dim3((n_tasks + 255) / 256), dim3(256), 0, s, n, nb, kTilesPerTask, n_tasks,
                        total, tasks, atom_off, ctr) != cudaSuccess)
        return GB_ERR_CUDA;

    gbk::PairArgs pa{};
    pa.atom_off = atom_off;
    pa.xyzq = (const float4*)xyzq;
    pa.rad = (const float2*)rad_screen;
    pa.Rh = Rh;
    pa.cc = cc;
    pa.offset = params->offset;
    pa.tau_ke = (float)((1.0 / params->eps_in - 1.0 / params->eps_out) * gbk::KE);
    pa.kc = (float)(gbk::KE / params->eps_in);
    pa.ke_out = (float)(gbk::KE / params->eps_out);
    pa.kappa = params->kappa;
    pa.rep_k = params->rep_k;
    pa.rep_sigma = params->rep_sigma;
    gbk::set_cutoffs(pa, *params);
    pa.I_acc = I_acc;
    pa.dR_acc = dR_acc;
    pa.phi_acc = phi_acc;
    pa.F_acc = F_acc;
    pa.E_acc = E_acc;
    pa.N = n;

    gbk::AtomArgs aa{};
    aa.atom_off = atom_off;
    aa.M = 1;
    aa.max_n = n;
    aa.xyzq = (const float4*)xyzq;
    aa.rad = (const float2*)rad_screen;
    aa.alpha = params->alpha;
    aa.beta = params->beta;
    aa.gamma = params->gamma;
    aa.offset = params->offset;
    aa.tau_ke = (1.0 / params->eps_in - 1.0 / params->eps_out) * gbk::KE;
    aa.kc = gbk::KE / params->eps_in;
    aa.ke_out = gbk::KE / params->eps_out;
    aa.kappa = params->kappa;
    aa.I_acc = I_acc;
    aa.dR_acc = dR_acc;
    aa.phi_acc = phi_acc;
    aa.F_acc = F_acc;
    aa.E_acc = E_acc;
    aa.Rh = Rh;
    aa.cfac = cfac;
    aa.cc = cc;
    aa.err = err;
    aa.N = n;

    gbk::TaskList tl;
    tl.d_tasks = tasks;
    tl.n_tasks = n_tasks;
    const int flags = (E_out ? gbk::EF_ENERGY : 0) | (dEdq_out ? gbk::EF_PHI : 0) |
                      (params->rep_k != 0.0f ? gbk::EF_REP : 0) | (params->kappa != 0.0f ? gbk::EF_SALT : 0);
    const int wpb = 8;
    // with a cutoff a pass walks the same task list from a queue, testing
    // every pair (no boxes here, so no block is proven in or out of range)
    const gb_params& P = *params;
    auto pass = [&](int which, int f) {
        if (gbk::cut_flag(which, P))
            return gbk::launch_pairs_list(which, f | gbk::EF_CUT, pa, tasks, ctr, 3, wpb, s);
        return gbk::launch_pairs(which, f, pa, tl, wpb, s);
    };
    if (pass(gbk::PASS_BORN, 0) != cudaSuccess) return GB_ERR_CUDA;
    if (gbk::launch_born_finalize(aa, R_out, s) != cudaSuccess) return GB_ERR_CUDA;
    if (pass(gbk::PASS_ENERGY, flags) != cudaSuccess) return GB_ERR_CUDA;
    if (gbk::launch_energy_finalize(aa, E_out ? 1 : 0, dEdq_out, s) != cudaSuccess) return GB_ERR_CUDA;
    if (pass(gbk::PASS_CHAIN, 0) != cudaSuccess) return GB_ERR_CUDA;
    if (gbk::launch_forces_out(aa, F_fixed, F_out, E_out, s) != cudaSuccess) return GB_ERR_CUDA;
    return GB_OK;
}
