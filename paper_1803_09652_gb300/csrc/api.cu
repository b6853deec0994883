// Host side of libgbremd: context, work lists, argument checks, the C ABI.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

using gbk::u64;

struct gb_ctx {
    int device = 0;
    int32_t M = 0;
    int64_t N = 0;
    int32_t max_n = 0;
    std::vector<int64_t> off_h;
    gb_params p{};
    int64_t* off_d = nullptr;
    u64* I_acc = nullptr;
    u64* dR_acc = nullptr;
    u64* phi_acc = nullptr;
    u64* F_acc = nullptr;
    u64* E_acc = nullptr;
    u64* ctr = nullptr;
    float2* Rh = nullptr;
    float* cfac = nullptr;
    float* cc = nullptr;
    int* err = nullptr;
    double* mc_part = nullptr;          // MC site-row slice partials
    double* sweep_part = nullptr;       // the same for per-residue sweeps (allocated on first use)
    float4* boxes = nullptr;            // tile bounding boxes
    int* tile_off = nullptr;
    // block neighbour lists of the cutoffs (allocated only with a cutoff)
    int4* list_b = nullptr;             // Born-radius cutoff: Born and chain passes
    int4* list_e = nullptr;             // pair cutoff: energy pass
    int* list_ctr = nullptr;            // [gbk::LIST_CTRS] lengths and queue heads
    int* win_off = nullptr;             // [M+1] first list-building warp of each replica
    int list_warps = 0;
    int n_tiles32 = 0;
    int32_t mc_parts = 0;
    gbk::TaskList tasks;
    int wpb = 4;
    int tpt = 0;
    int64_t total_tiles = 0;
    std::string msg;
    cudaStream_t cs = nullptr;          // private stream for graph capture
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // per-pass timing events inside the MD driver (2 per pass per step)
    bool prof = false;
    std::vector<cudaEvent_t> prof_ev;
    int64_t prof_steps = 0;
    bool capturing = false;
    // persistent MD kernel: grid (0 = unavailable), its task list, barrier words
    int persist_grid = 0;
    bool use_persist = false;
    gbk::TaskList ptasks;
    int* ptask_off = nullptr;           // [M+1]
    int* phase_off = nullptr;           // [6][M+1]
    int* phase_count = nullptr;         // [6][M]
    int phase_base[7] = {0};
    unsigned* qwords = nullptr;         // queue head + 6 x M completion counters
    unsigned spin_limit = 1u << 22;     // polls before a persistent-kernel wait gives up
    std::vector<int> prof_steps_per_launch;
    // cached MD graph
    cudaGraphExec_t md_exec = nullptr;
    std::vector<uint8_t> md_key;
    int64_t md_len = 0;
};

static thread_local std::string g_create_error;

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

int fail(gb_ctx* c, int code, const std::string& m) {
    if (c) c->msg = m;
    else g_create_error = m;
    return code;
}

int cuda_fail(gb_ctx* c, cudaError_t e, const char* where) {
    return fail(c, GB_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define GB_CHECK(c, call)                                                  \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return cuda_fail((c), e_, #call);           \
    } while (0)

template <class T>
cudaError_t zalloc(T** p, size_t n) {
    cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    return cudaMemset(*p, 0, std::max<size_t>(n, 1) * sizeof(T));
}

// Cut the work of all replicas (super-rows of 64 atoms against 32-atom tiles
// J >= 2K, replicas in order) into runs of `tpt` tiles, one warp task each.
int build_tasks_into(gb_ctx* c, int tpt, gbk::TaskList& out) {
    std::vector<int4> t;
    t.reserve((size_t)(c->total_tiles / tpt + 1));
    int64_t left_total = c->total_tiles;
    int r = 0, K = 0, J = 0;
    auto nb_of = [&](int rr) { return (int)((c->off_h[rr + 1] - c->off_h[rr] + 31) / 32); };
    while (r < c->M && nb_of(r) == 0) ++r;
    while (left_total > 0) {
        const int cnt = (int)std::min<int64_t>(tpt, left_total);
        t.push_back(make_int4(r, K, J, cnt));
        left_total -= cnt;
        int64_t k = cnt;
        while (k > 0 && r < c->M) {
            const int nb = nb_of(r);
            const int rowleft = nb - J;
            if (k < rowleft) {
                J += (int)k;
                k = 0;
            } else {
                k -= rowleft;
                ++K;
                if (K == (nb + 1) / 2) {
                    ++r;
                    while (r < c->M && nb_of(r) == 0) ++r;
                    K = 0;
                }
                J = 2 * K;
            }
        }
    }
    // Costly blocks first: those at and next to a super-row's diagonal hold the
    // chain's near pairs (closed forms, no far-block shortcut), so starting
    // them early leaves the cheap far blocks for the end of the pass, where
    // they even out the finishing times of the SMs.  Any order gives the same
    // fixed-point sums.
    std::stable_sort(t.begin(), t.end(), [](const int4& a, const int4& b) {
        return a.z - 2 * a.y < b.z - 2 * b.y;
    });
    if (out.d_tasks) cudaFree(out.d_tasks);
    out.d_tasks = nullptr;
    out.n_tasks = (int)t.size();
    GB_CHECK(c, zalloc(&out.d_tasks, t.size()));
    if (!t.empty())
        GB_CHECK(c, cudaMemcpy(out.d_tasks, t.data(), t.size() * sizeof(int4), cudaMemcpyHostToDevice));
    return GB_OK;
}

int build_tasks(gb_ctx* c) { return build_tasks_into(c, c->tpt, c->tasks); }

// Tables of the persistent MD kernel: per-replica pair tasks (runs of `tpt`
// tiles that never leave their replica), item offsets and counts of the six
// phases.  The grid is sized to the resident capacity of the device.
int setup_persist(gb_ctx* c) {
    int dev = 0, sms = 0, per_sm = 0;
    GB_CHECK(c, cudaGetDevice(&dev));
    GB_CHECK(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    GB_CHECK(c, gbk::persist_occupancy(c->p.rep_k != 0.0f ? 1 : 0, &per_sm));
    if (per_sm < 1 || c->total_tiles == 0) {
        c->persist_grid = 0;
        return GB_OK;
    }
    c->persist_grid = sms * per_sm;
    const int64_t warps = (int64_t)c->persist_grid * 4;
    // about four pair items per resident warp and pass
    const int tpt = (int)std::max<int64_t>(1, c->total_tiles / (4 * warps));
    const int M = c->M;
    std::vector<int4> t;
    std::vector<int> toff(M + 1, 0), cnt(6 * M, 0), poff(6 * (M + 1), 0);
    for (int r = 0; r < M; ++r) {
        const int64_t n = c->off_h[r + 1] - c->off_h[r];
        const int nb = (int)((n + 31) / 32), nk = (nb + 1) / 2;
        int64_t left = gbk::pair_units(n);
        int K = 0, J = 0;
        while (left > 0) {
            const int run = (int)std::min<int64_t>(tpt, left);
            t.push_back(make_int4(r, K, J, run));
            left -= run;
            int64_t k = run;
            while (k > 0 && K < nk) {
                const int rowleft = nb - J;
                if (k < rowleft) { J += (int)k; k = 0; }
                else { k -= rowleft; ++K; J = 2 * K; }
            }
        }
        toff[r + 1] = (int)t.size();
        const int tasks_r = toff[r + 1] - toff[r];
        const int per_phase[6] = {nb, tasks_r, nb, tasks_r, nb, tasks_r};
        for (int p = 0; p < 6; ++p) cnt[p * M + r] = per_phase[p];
    }
    c->phase_base[0] = 0;
    for (int p = 0; p < 6; ++p) {
        for (int r = 0; r < M; ++r) poff[p * (M + 1) + r + 1] = poff[p * (M + 1) + r] + cnt[p * M + r];
        c->phase_base[p + 1] = c->phase_base[p] + poff[p * (M + 1) + M];
    }
    if (c->ptasks.d_tasks) cudaFree(c->ptasks.d_tasks);
    c->ptasks.n_tasks = (int)t.size();
    GB_CHECK(c, zalloc(&c->ptasks.d_tasks, t.size()));
    GB_CHECK(c, cudaMemcpy(c->ptasks.d_tasks, t.data(), t.size() * sizeof(int4), cudaMemcpyHostToDevice));
    GB_CHECK(c, zalloc(&c->ptask_off, M + 1));
    GB_CHECK(c, cudaMemcpy(c->ptask_off, toff.data(), sizeof(int) * (M + 1), cudaMemcpyHostToDevice));
    GB_CHECK(c, zalloc(&c->phase_count, 6 * (size_t)M));
    GB_CHECK(c, cudaMemcpy(c->phase_count, cnt.data(), sizeof(int) * 6 * M, cudaMemcpyHostToDevice));
    GB_CHECK(c, zalloc(&c->phase_off, 6 * (size_t)(M + 1)));
    GB_CHECK(c, cudaMemcpy(c->phase_off, poff.data(), sizeof(int) * 6 * (M + 1), cudaMemcpyHostToDevice));
    GB_CHECK(c, zalloc(&c->qwords, 1 + 6 * (size_t)M));
    return GB_OK;
}

int default_tpt(const gb_ctx* c) {
    // about four warp tasks per resident warp slot of 152 SMs x 32 warps; with
    // a cutoff most blocks are skipped and the rest cluster along the diagonal,
    // so tasks eight times shorter even out the warps' work
    const int64_t slots = 152LL * 32 * 4;
    int64_t t = (c->total_tiles + slots - 1) / slots;
    if (c->p.rgbmax > 0.0f || c->p.cut > 0.0f) t = (t + 7) / 8;
    return (int)std::max<int64_t>(1, std::min<int64_t>(t, 256));
}

gbk::PairArgs pair_args(const gb_ctx* c, const float* xyzq, const float* rad) {
    gbk::PairArgs a{};
    a.atom_off = c->off_d;
    a.xyzq = (const float4*)xyzq;
    a.rad = (const float2*)rad;
    a.Rh = c->Rh;
    a.cc = c->cc;
    a.offset = c->p.offset;
    a.tau_ke = (float)((1.0 / c->p.eps_in - 1.0 / c->p.eps_out) * gbk::KE);
    a.kc = (float)(gbk::KE / c->p.eps_in);
    a.ke_out = (float)(gbk::KE / c->p.eps_out);
    a.kappa = c->p.kappa;
    a.rep_k = c->p.rep_k;
    a.rep_sigma = c->p.rep_sigma;
    gbk::set_cutoffs(a, c->p);
    a.I_acc = c->I_acc;
    a.dR_acc = c->dR_acc;
    a.phi_acc = c->phi_acc;
    a.F_acc = c->F_acc;
    a.E_acc = c->E_acc;
    a.N = c->N;
    a.boxes = c->boxes;
    a.tile_off = c->tile_off;
    a.err = c->err;
    return a;
}

gbk::AtomArgs atom_args(const gb_ctx* c, const float* xyzq, const float* rad) {
    gbk::AtomArgs a{};
    a.atom_off = c->off_d;
    a.M = c->M;
    a.max_n = c->max_n;
    a.xyzq = (const float4*)xyzq;
    a.rad = (const float2*)rad;
    a.alpha = c->p.alpha;
    a.beta = c->p.beta;
    a.gamma = c->p.gamma;
    a.offset = c->p.offset;
    a.tau_ke = (1.0 / c->p.eps_in - 1.0 / c->p.eps_out) * gbk::KE;
    a.kc = gbk::KE / c->p.eps_in;
    a.ke_out = gbk::KE / c->p.eps_out;
    a.kappa = c->p.kappa;
    a.I_acc = c->I_acc;
    a.dR_acc = c->dR_acc;
    a.phi_acc = c->phi_acc;
    a.F_acc = c->F_acc;
    a.E_acc = c->E_acc;
    a.Rh = c->Rh;
    a.cfac = c->cfac;
    a.cc = c->cc;
    a.err = c->err;
    a.N = c->N;
    return a;
}

// The three passes of one energy/force evaluation.  flags: gbk::EF_*.
cudaError_t mark(gb_ctx* c, cudaEvent_t e, cudaStream_t s) {
    return c->capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) : cudaEventRecord(e, s);
}

// One pair pass: over the static task list, or with the pass's cutoff over
// its block neighbour list (built by launch_block_list for this evaluation).
cudaError_t pass(const gb_ctx* c, int which, int flags, const gbk::PairArgs& pa, cudaStream_t s) {
    const int4* list = (which == gbk::PASS_ENERGY) ? c->list_e : c->list_b;
    if (list) return gbk::launch_pairs_list(which, flags | gbk::EF_CUT, pa, list, c->list_ctr, c->tasks.cap[which],
                                            c->wpb, s);
    return gbk::launch_pairs(which, flags, pa, c->tasks, c->wpb, s);
}

// md != null: an MD step; the chain-bond forces join the force accumulators
// and the tile boxes were already built by k_md_step (build_boxes false).
int evaluate(gb_ctx* c, const float* xyzq, const float* rad, float* R_out, int flags,
             double* phi_out, cudaStream_t s, const cudaEvent_t* ev = nullptr,
             const gbk::MDArgs* md = nullptr, bool build_boxes = true) {
    if (c->p.kappa != 0.0f) flags |= gbk::EF_SALT;
    const gbk::PairArgs pa = pair_args(c, xyzq, rad);
    const gbk::AtomArgs aa = atom_args(c, xyzq, rad);
    if (build_boxes) GB_CHECK(c, gbk::launch_tile_boxes(pa, c->M, c->n_tiles32, s));
    if (c->list_ctr)
        GB_CHECK(c, gbk::launch_block_list(pa, c->win_off, c->M, c->list_warps, c->list_b, c->list_e, c->list_ctr,
                                           c->list_b ? 1 : 0, c->list_e ? 1 : 0, s));
    if (ev) GB_CHECK(c, mark(c, ev[0], s));
    GB_CHECK(c, pass(c, gbk::PASS_BORN, 0, pa, s));
    if (ev) GB_CHECK(c, mark(c, ev[1], s));
    GB_CHECK(c, gbk::launch_born_finalize(aa, R_out, s));
    if (ev) GB_CHECK(c, mark(c, ev[2], s));
    GB_CHECK(c, pass(c, gbk::PASS_ENERGY, flags, pa, s));
    if (ev) GB_CHECK(c, mark(c, ev[3], s));
    GB_CHECK(c, gbk::launch_energy_finalize(aa, (flags & gbk::EF_ENERGY) ? 1 : 0, phi_out, s,
                                            md ? md->bond_k : 0.0f, md ? md->bond_r0 : 0.0f));
    if (ev) GB_CHECK(c, mark(c, ev[4], s));
    GB_CHECK(c, pass(c, gbk::PASS_CHAIN, 0, pa, s));
    if (ev) GB_CHECK(c, mark(c, ev[5], s));
    return GB_OK;
}

int ensure_prof_events(gb_ctx* c, int64_t steps) {
    while ((int64_t)c->prof_ev.size() < 6 * steps) {
        cudaEvent_t e;
        GB_CHECK(c, cudaEventCreate(&e));
        c->prof_ev.push_back(e);
    }
    return GB_OK;
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

// The replica -> site ranges, checked on the host copy: the kernels walk
// site_off[r] .. site_off[r+1] and index the per-site tables with it.
const char* site_off_error(const gb_sites* s) {
    if (s->n_sites < 0) return "sites->n_sites < 0";
    if (!s->site_off_host) return "sites->site_off_host is NULL";
    if (s->site_off_host[0] != 0) return "site_off_host[0] must be 0";
    for (int r = 0; r < s->n_rep; ++r)
        if (s->site_off_host[r + 1] < s->site_off_host[r]) return "site_off_host must be non-decreasing";
    if (s->site_off_host[s->n_rep] != s->n_sites) return "site_off_host[n_rep] must equal n_sites";
    return nullptr;
}

int check_sites(gb_ctx* c, const gb_sites* s) {
    if (!s) return fail(c, GB_ERR_INVALID_ARG, "sites is NULL");
    if (s->n_rep != c->M) return fail(c, GB_ERR_INVALID_ARG, "sites->n_rep differs from the context's replica count");
    if (const char* e = site_off_error(s)) return fail(c, GB_ERR_INVALID_ARG, e);
    if (s->n_sites > 0 && (!s->site_off || !s->site_kind || !s->site_nstates || !s->site_atom_off ||
                           !s->site_atom_idx || !s->site_state_off || !s->site_q_off || !s->q_state ||
                           !s->G_ref || !s->n_H || !s->n_e || !s->pKa_ref || !s->E0_ref))
        return fail(c, GB_ERR_INVALID_ARG, "a site table pointer is NULL");
    if (!s->site_off) return fail(c, GB_ERR_INVALID_ARG, "sites->site_off is NULL");
    return GB_OK;
}

}  // namespace

// ----------------------------------------------------------------------------------

extern "C" int gb_ctx_create(gb_ctx** out, int32_t n_rep, const int64_t* atom_off,
                             const gb_params* params, int32_t device) {
    if (!out || !atom_off || !params) return fail(nullptr, GB_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (n_rep < 1) return fail(nullptr, GB_ERR_INVALID_ARG, "n_rep must be >= 1");
    if (atom_off[0] != 0) return fail(nullptr, GB_ERR_INVALID_ARG, "atom_off[0] must be 0");
    for (int r = 0; r < n_rep; ++r)
        if (atom_off[r + 1] < atom_off[r]) return fail(nullptr, GB_ERR_INVALID_ARG, "atom_off must be non-decreasing");
    if (atom_off[n_rep] >= (1LL << 31)) return fail(nullptr, GB_ERR_INVALID_ARG, "too many atoms");
    if (!gbk::params_ok(*params)) return fail(nullptr, GB_ERR_INVALID_ARG, "invalid GB parameters");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(nullptr, GB_ERR_CUDA, "no such CUDA device");
    DeviceGuard g(device);
    gb_ctx* c = new gb_ctx();
    c->device = device;
    c->M = n_rep;
    c->off_h.assign(atom_off, atom_off + n_rep + 1);
    c->N = atom_off[n_rep];
    c->p = *params;
    for (int r = 0; r < n_rep; ++r) {
        const int64_t n = atom_off[r + 1] - atom_off[r];
        c->max_n = (int32_t)std::max<int64_t>(c->max_n, n);
        c->total_tiles += gbk::pair_units(n);
    }
    const size_t N = (size_t)c->N;
    cudaError_t e = cudaSuccess;
    auto step = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    step(zalloc(&c->off_d, n_rep + 1));
    step(cudaMemcpy(c->off_d, atom_off, sizeof(int64_t) * (n_rep + 1), cudaMemcpyHostToDevice));
    step(zalloc(&c->I_acc, N));
    step(zalloc(&c->dR_acc, N));
    step(zalloc(&c->phi_acc, N));
    step(zalloc(&c->F_acc, 3 * N));
    step(zalloc(&c->E_acc, 4 * (size_t)n_rep));
    step(zalloc(&c->ctr, 2));
    step(zalloc(&c->Rh, N));
    step(zalloc(&c->cfac, N));
    step(zalloc(&c->cc, N));
    step(zalloc(&c->err, 1));

    c->mc_parts = (c->max_n + gbk::MC_CHUNK - 1) / gbk::MC_CHUNK;
    {
        std::vector<int> toff(n_rep + 1, 0);
        for (int r = 0; r < n_rep; ++r) toff[r + 1] = toff[r] + (int)((atom_off[r + 1] - atom_off[r] + 31) / 32);
        c->n_tiles32 = toff[n_rep];
        step(zalloc(&c->tile_off, n_rep + 1));
        if (e == cudaSuccess)
            e = cudaMemcpy(c->tile_off, toff.data(), sizeof(int) * (n_rep + 1), cudaMemcpyHostToDevice);
        step(zalloc(&c->boxes, 2 * (size_t)std::max(c->n_tiles32, 1)));
        if (params->rgbmax > 0.0f || params->cut > 0.0f) {
            // every block of the batch may be in range: one task of one block each
            std::vector<int> woff(n_rep + 1, 0);
            for (int r = 0; r < n_rep; ++r) {
                const int64_t nb = (atom_off[r + 1] - atom_off[r] + 31) / 32;
                woff[r + 1] = woff[r] + (int)(((nb + 1) / 2) * ((nb + 31) / 32));
            }
            c->list_warps = woff[n_rep];
            const size_t cap = (size_t)std::max<int64_t>(c->total_tiles, 1);
            if (params->rgbmax > 0.0f) step(zalloc(&c->list_b, cap));
            if (params->cut > 0.0f) step(zalloc(&c->list_e, cap));
            step(zalloc(&c->list_ctr, gbk::LIST_CTRS));
            step(zalloc(&c->win_off, n_rep + 1));
            if (e == cudaSuccess)
                e = cudaMemcpy(c->win_off, woff.data(), sizeof(int) * (n_rep + 1), cudaMemcpyHostToDevice);
        }
    }
    step(zalloc(&c->mc_part, (size_t)n_rep * std::max(c->mc_parts, 1) * gbk::MC_MAX_SITE_ATOMS));
    step(cudaStreamCreateWithFlags(&c->cs, cudaStreamNonBlocking));
    step(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
    step(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
    if (e != cudaSuccess) {
        int code = (e == cudaErrorMemoryAllocation) ? GB_ERR_NOMEM : GB_ERR_CUDA;
        fail(nullptr, code, std::string("context allocation: ") + cudaGetErrorString(e));
        gb_ctx_destroy(c);
        return code;
    }
    c->tpt = default_tpt(c);
    for (int k = 0; k < 3; ++k) c->tasks.cap[k] = 3;
    int rc = build_tasks(c);
    if (rc == GB_OK) rc = setup_persist(c);
    if (rc != GB_OK) {
        g_create_error = c->msg;
        gb_ctx_destroy(c);
        return rc;
    }
    *out = c;
    return GB_OK;
}

extern "C" int gb_ctx_destroy(gb_ctx* c) {
    if (!c) return GB_OK;
    DeviceGuard g(c->device);
    if (c->md_exec) cudaGraphExecDestroy(c->md_exec);
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    cudaFree(c->tasks.d_tasks);
    cudaFree(c->ptasks.d_tasks);
    cudaFree(c->ptask_off);
    cudaFree(c->phase_off);
    cudaFree(c->phase_count);
    cudaFree(c->qwords);
    cudaFree(c->off_d);
    cudaFree(c->I_acc);
    cudaFree(c->dR_acc);
    cudaFree(c->phi_acc);
    cudaFree(c->F_acc);
    cudaFree(c->E_acc);
    cudaFree(c->ctr);
    cudaFree(c->Rh);
    cudaFree(c->cfac);
    cudaFree(c->cc);
    cudaFree(c->err);
    cudaFree(c->mc_part);
    cudaFree(c->sweep_part);
    cudaFree(c->boxes);
    cudaFree(c->list_b);
    cudaFree(c->list_e);
    cudaFree(c->list_ctr);
    cudaFree(c->win_off);
    cudaFree(c->tile_off);
    if (c->cs) cudaStreamDestroy(c->cs);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    delete c;
    return GB_OK;
}

extern "C" const char* gb_last_error(const gb_ctx* c) {
    return c ? c->msg.c_str() : g_create_error.c_str();
}

extern "C" int gb_sync_status(gb_ctx* c, void* stream) {
    if (!c) return fail(nullptr, GB_ERR_INVALID_ARG, "NULL context");
    DeviceGuard g(c->device);
    GB_CHECK(c, cudaStreamSynchronize((cudaStream_t)stream));
    int h = 0;
    GB_CHECK(c, cudaMemcpy(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost));
    GB_CHECK(c, cudaMemset(c->err, 0, sizeof(int)));
    if (h != 0) return fail(c, h, "error recorded on the device");
    return GB_OK;
}

extern "C" int gb_set_tiles(gb_ctx* c, int32_t wpb, int32_t tpt) {
    if (!c) return fail(nullptr, GB_ERR_INVALID_ARG, "NULL context");
    if (wpb < 1 || wpb > 8 || tpt < 1 || tpt > (1 << 20))
        return fail(c, GB_ERR_INVALID_ARG, "warps_per_block must be 1..8, tiles_per_task 1..2^20");
    DeviceGuard g(c->device);
    c->wpb = wpb;
    if (tpt != c->tpt) {
        GB_CHECK(c, cudaDeviceSynchronize());
        c->tpt = tpt;
        int rc = build_tasks(c);
        if (rc) return rc;
        if (c->md_exec) { cudaGraphExecDestroy(c->md_exec); c->md_exec = nullptr; c->md_key.clear(); }
    }
    return GB_OK;
}

extern "C" int gb_set_reg_cap(gb_ctx* c, int32_t pass, int32_t min_blocks) {
    if (!c) return fail(nullptr, GB_ERR_INVALID_ARG, "NULL context");
    if (pass < -1 || pass > 2) return fail(c, GB_ERR_INVALID_ARG, "pass must be -1, 0, 1 or 2");
    if (min_blocks != 1 && min_blocks != 3 && min_blocks != 4)
        return fail(c, GB_ERR_INVALID_ARG, "min_blocks must be 1, 3 or 4");
    for (int k = 0; k < 3; ++k)
        if (pass < 0 || pass == k) c->tasks.cap[k] = min_blocks;
    if (c->md_exec) { cudaGraphExecDestroy(c->md_exec); c->md_exec = nullptr; c->md_key.clear(); }
    return GB_OK;
}

extern "C" int gb_get_reg_caps(const gb_ctx* c, int32_t* caps) {
    if (!c || !caps) return GB_ERR_INVALID_ARG;
    for (int k = 0; k < 3; ++k) caps[k] = c->tasks.cap[k];
    return GB_OK;
}

extern "C" int gb_get_tiles(const gb_ctx* c, int32_t* wpb, int32_t* tpt) {
    if (!c || !wpb || !tpt) return GB_ERR_INVALID_ARG;
    *wpb = c->wpb;
    *tpt = c->tpt;
    return GB_OK;
}

static int check_inputs(gb_ctx* c, const float* xyzq, const float* rad) {
    if (!c) return fail(nullptr, GB_ERR_INVALID_ARG, "NULL context");
    if (c->N == 0) return GB_OK;               // every replica empty: nothing is read
    if (!xyzq || !rad) return fail(c, GB_ERR_INVALID_ARG, "xyzq / rad_screen is NULL");
    if (!aligned(xyzq, 16) || !aligned(rad, 8))
        return fail(c, GB_ERR_INVALID_ARG, "xyzq must be 16-byte and rad_screen 8-byte aligned");
    return GB_OK;
}

extern "C" int gb_born_radii(gb_ctx* c, const float* xyzq, const float* rad, float* R_out, void* stream) {
    int rc = check_inputs(c, xyzq, rad);
    if (rc) return rc;
    if (!R_out && c->N > 0) return fail(c, GB_ERR_INVALID_ARG, "R_out is NULL");
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    const gbk::PairArgs pa = pair_args(c, xyzq, rad);
    const gbk::AtomArgs aa = atom_args(c, xyzq, rad);
    GB_CHECK(c, gbk::launch_tile_boxes(pa, c->M, c->n_tiles32, s));
    if (c->list_b)
        GB_CHECK(c, gbk::launch_block_list(pa, c->win_off, c->M, c->list_warps, c->list_b, nullptr, c->list_ctr, 1, 0,
                                           s));
    GB_CHECK(c, pass(c, gbk::PASS_BORN, 0, pa, s));
    GB_CHECK(c, gbk::launch_born_finalize(aa, R_out, s));
    return GB_OK;
}

extern "C" int gb_energy_forces(gb_ctx* c, const float* xyzq, const float* rad, float* R_out,
                                int64_t* F_fixed, float* F_out, double* E_out, double* dEdq_out,
                                void* stream) {
    int rc = check_inputs(c, xyzq, rad);
    if (rc) return rc;
    if (!R_out && !F_fixed && !F_out && !E_out && !dEdq_out)
        return fail(c, GB_ERR_INVALID_ARG, "no output requested");
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    int flags = (E_out ? gbk::EF_ENERGY : 0) | (dEdq_out ? gbk::EF_PHI : 0) |
                (c->p.rep_k != 0.0f ? gbk::EF_REP : 0);
    rc = evaluate(c, xyzq, rad, R_out, flags, dEdq_out, s);
    if (rc) return rc;
    GB_CHECK(c, gbk::launch_forces_out(atom_args(c, xyzq, rad), F_fixed, F_out, E_out, s));
    return GB_OK;
}

static gbk::MCArgs mc_args(const gb_ctx* c, const gb_sites* sites, float* xyzq, const float* R,
                           const double* pH, const double* E, double kT, uint64_t seed, uint64_t step,
                           int32_t kind, int32_t* state, double* dG_out, uint8_t* acc_out) {
    gbk::MCArgs a{};
    a.atom_off = c->off_d;
    a.site_off = sites->site_off;
    a.site_kind = sites->site_kind;
    a.site_nstates = sites->site_nstates;
    a.site_atom_off = sites->site_atom_off;
    a.site_atom_idx = sites->site_atom_idx;
    a.site_state_off = sites->site_state_off;
    a.site_q_off = sites->site_q_off;
    a.q_state = sites->q_state;
    a.G_ref = sites->G_ref;
    a.n_H = sites->n_H;
    a.n_e = sites->n_e;
    a.pKa_ref = sites->pKa_ref;
    a.E0_ref = sites->E0_ref;
    a.xyzq = (float4*)xyzq;
    a.R = R;
    a.pH = pH;
    a.E = E;
    a.kT = kT;
    a.tau_ke = (1.0 / c->p.eps_in - 1.0 / c->p.eps_out) * gbk::KE;
    a.kc = gbk::KE / c->p.eps_in;
    a.ke_out = gbk::KE / c->p.eps_out;
    a.kappa = c->p.kappa;
    a.cut2 = c->p.cut * c->p.cut;
    a.seed = seed;
    a.step = step;
    a.ctr = nullptr;
    a.kind = kind;
    a.state = state;
    a.dG_out = dG_out;
    a.acc_out = acc_out;
    a.n_parts = c->mc_parts;
    a.err = c->err;
    return a;
}

// Workspace of per-residue sweeps, allocated on first use (outside capture).
static int ensure_sweep_part(gb_ctx* c) {
    if (c->sweep_part) return GB_OK;
    const size_t n = (size_t)c->M * std::max(c->mc_parts, 1) * gbk::SWEEP_MAX_SITE_ATOMS;
    cudaError_t e = cudaMalloc((void**)&c->sweep_part, n * sizeof(double));
    if (e != cudaSuccess) {
        c->sweep_part = nullptr;
        return cuda_fail(c, e, "sweep workspace");
    }
    return GB_OK;
}

static int check_mc(gb_ctx* c, const gb_sites* sites, float* xyzq, const float* R, const double* pH,
                    const double* E, double kT, int32_t kind, int32_t* state) {
    if (!c) return fail(nullptr, GB_ERR_INVALID_ARG, "NULL context");
    int rc = check_sites(c, sites);
    if (rc) return rc;
    if (!xyzq || !R || !pH || !E || !state) return fail(c, GB_ERR_INVALID_ARG, "NULL array");
    if (kind != 0 && kind != 1) return fail(c, GB_ERR_INVALID_ARG, "kind must be 0 (pH) or 1 (redox)");
    if (!(kT > 0.0)) return fail(c, GB_ERR_INVALID_ARG, "kT must be positive");
    if (!aligned(xyzq, 16)) return fail(c, GB_ERR_INVALID_ARG, "xyzq must be 16-byte aligned");
    return GB_OK;
}

extern "C" int redox_ph_mc_step(gb_ctx* c, const gb_sites* sites, float* xyzq, const float* R,
                                const double* pH, const double* E, double kT, uint64_t seed,
                                uint64_t step, int32_t kind, int32_t* state, double* dG_out,
                                uint8_t* acc_out, void* stream) {
    int rc = check_mc(c, sites, xyzq, R, pH, E, kT, kind, state);
    if (rc) return rc;
    DeviceGuard g(c->device);
    gbk::MCArgs a = mc_args(c, sites, xyzq, R, pH, E, kT, seed, step, kind, state, dG_out, acc_out);
    a.phi_part = c->mc_part;
    GB_CHECK(c, gbk::launch_mc(a, c->M, (cudaStream_t)stream));
    return GB_OK;
}

extern "C" int redox_ph_mc_sweep(gb_ctx* c, const gb_sites* sites, float* xyzq, const float* R,
                                 const double* pH, const double* E, double kT, uint64_t seed,
                                 uint64_t step, int32_t kind, int32_t* state, double* dG_out,
                                 uint8_t* acc_out, void* stream) {
    int rc = check_mc(c, sites, xyzq, R, pH, E, kT, kind, state);
    if (rc) return rc;
    DeviceGuard g(c->device);
    rc = ensure_sweep_part(c);
    if (rc) return rc;
    gbk::MCArgs a = mc_args(c, sites, xyzq, R, pH, E, kT, seed, step, kind, state, dG_out, acc_out);
    a.phi_part = c->sweep_part;
    GB_CHECK(c, gbk::launch_mc_sweep(a, c->M, (cudaStream_t)stream));
    return GB_OK;
}

extern "C" int eremd_exchange(int32_t n_ladders, int32_t len, int32_t ladder_stride,
                              int32_t slot_stride, const double* values, int32_t* rep_at_slot,
                              const int32_t* n_count, int32_t dim, uint64_t attempt, uint64_t seed,
                              double kT, int32_t wrap, double* value_of_rep, double* delta_out,
                              uint8_t* acc_out, void* stream) {
    if (n_ladders < 0 || len < 0 || !values || !rep_at_slot || !n_count)
        return fail(nullptr, GB_ERR_INVALID_ARG, "invalid exchange arguments");
    if (dim != 0 && dim != 1) return fail(nullptr, GB_ERR_INVALID_ARG, "dim must be 0 (E) or 1 (pH)");
    if (!(kT > 0.0)) return fail(nullptr, GB_ERR_INVALID_ARG, "kT must be positive");
    gbk::ExArgs a{};
    a.n_ladders = n_ladders;
    a.len = len;
    a.ladder_stride = ladder_stride;
    a.slot_stride = slot_stride;
    a.values = values;
    a.rep_at_slot = rep_at_slot;
    a.n_count = n_count;
    a.dim = dim;
    a.attempt = attempt;
    a.ctr = nullptr;
    a.seed = seed;
    a.kT = kT;
    a.wrap = wrap;
    a.value_of_rep = value_of_rep;
    a.delta_out = delta_out;
    a.acc_out = acc_out;
    cudaError_t e = gbk::launch_exchange(a, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(nullptr, GB_ERR_CUDA, cudaGetErrorString(e));
    return GB_OK;
}

extern "C" int gb_count_bound(const gb_sites* s, const int32_t* state, int32_t kind,
                              int32_t* out, void* stream) {
    if (!s || !state || !out || !s->site_off) return fail(nullptr, GB_ERR_INVALID_ARG, "NULL argument");
    if (s->n_rep < 1) return fail(nullptr, GB_ERR_INVALID_ARG, "sites->n_rep must be >= 1");
    if (const char* e = site_off_error(s)) return fail(nullptr, GB_ERR_INVALID_ARG, e);
    if (s->n_sites > 0 && (!s->site_kind || !s->site_nstates || !s->site_state_off || !s->n_H || !s->n_e))
        return fail(nullptr, GB_ERR_INVALID_ARG, "a site table pointer is NULL");
    cudaError_t e = gbk::launch_count(s->site_off, s->site_kind, s->site_nstates, s->site_state_off, s->n_H, s->n_e,
                                      state, kind, s->n_rep, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(nullptr, GB_ERR_CUDA, cudaGetErrorString(e));
    return GB_OK;
}

// ---------------------------------------------------------------------------------
// MD driver

namespace {

gbk::MDArgs md_args(const gb_ctx* c, const gb_md_state* st) {
    gbk::MDArgs m{};
    m.xyzq = (float4*)st->xyzq;
    m.vel = (float4*)st->vel;
    m.force = (float4*)st->force;
    m.ctr = c->ctr;
    m.h = (float)(0.5 * st->dt);
    m.inv_m = (float)(gbk::ACCEL / st->mass);
    const double c1 = std::exp(-st->friction * st->dt);
    m.c1 = (float)c1;
    m.c2 = (float)std::sqrt((1.0 - c1 * c1) * st->kT * gbk::ACCEL / st->mass);
    m.bond_k = st->bond_k;
    m.bond_r0 = st->bond_r0;
    m.seed = st->seed;
    m.rep_base = (u64)st->rep_base;
    return m;
}

int check_md(gb_ctx* c, const gb_md_state* st) {
    if (!c) return fail(nullptr, GB_ERR_INVALID_ARG, "NULL context");
    if (!st) return fail(c, GB_ERR_INVALID_ARG, "MD state is NULL");
    if (c->N > 0 && (!st->xyzq || !st->vel || !st->force || !st->rad_screen))
        return fail(c, GB_ERR_INVALID_ARG, "MD state buffer is NULL");
    if (!aligned(st->xyzq, 16) || !aligned(st->vel, 16) || !aligned(st->force, 16))
        return fail(c, GB_ERR_INVALID_ARG, "MD buffers must be 16-byte aligned");
    if (!(st->dt >= 0) || !(st->mass > 0) || !(st->kT > 0) || !(st->friction >= 0))
        return fail(c, GB_ERR_INVALID_ARG, "invalid MD constants");
    if (st->mc_mode != 0 && st->mc_mode != 1) return fail(c, GB_ERR_INVALID_ARG, "mc_mode must be 0 or 1");
    if (st->rep_base < 0) return fail(c, GB_ERR_INVALID_ARG, "rep_base < 0");
    return GB_OK;
}

// Monte Carlo attempts (protonation, then redox) after block step k (1-based):
// the Philox step is the device counter ctr[0] + k.
int enqueue_mc(gb_ctx* c, gb_md_state* st, const gb_sites* sites, int64_t k, cudaStream_t s) {
    for (int kind = 0; kind < 2; ++kind) {
        gbk::MCArgs a{};
        a.atom_off = c->off_d;
        a.site_off = sites->site_off;
        a.site_kind = sites->site_kind;
        a.site_nstates = sites->site_nstates;
        a.site_atom_off = sites->site_atom_off;
        a.site_atom_idx = sites->site_atom_idx;
        a.site_state_off = sites->site_state_off;
        a.site_q_off = sites->site_q_off;
        a.q_state = sites->q_state;
        a.G_ref = sites->G_ref;
        a.n_H = sites->n_H;
        a.n_e = sites->n_e;
        a.pKa_ref = sites->pKa_ref;
        a.E0_ref = sites->E0_ref;
        a.xyzq = (float4*)st->xyzq;
        a.R = nullptr;
        a.Rh = c->Rh;
        a.pH = st->pH;
        a.E = st->E;
        a.kT = st->kT;
        a.tau_ke = (1.0 / c->p.eps_in - 1.0 / c->p.eps_out) * gbk::KE;
        a.kc = gbk::KE / c->p.eps_in;
        a.ke_out = gbk::KE / c->p.eps_out;
        a.kappa = c->p.kappa;
        a.cut2 = c->p.cut * c->p.cut;
        a.seed = st->seed;
        a.step = (u64)k;
        a.rep_base = (u64)st->rep_base;
        a.ctr = c->ctr;
        a.kind = kind;
        a.state = st->state;
        a.dG_out = nullptr;
        a.acc_out = nullptr;
        a.n_parts = c->mc_parts;
        a.err = c->err;
        if (st->mc_mode == 1) {
            a.phi_part = c->sweep_part;
            GB_CHECK(c, gbk::launch_mc_sweep(a, c->M, s));
        } else {
            a.phi_part = c->mc_part;
            GB_CHECK(c, gbk::launch_mc(a, c->M, s));
        }
    }
    return GB_OK;
}


// State occupancy after a step with Monte Carlo attempts (and its exchange).
int enqueue_occupancy(gb_ctx* c, gb_md_state* st, const gb_sites* sites, cudaStream_t s) {
    if (!st->occ_count) return GB_OK;
    gbk::OccArgs a{};
    a.site_off = sites->site_off;
    a.site_nstates = sites->site_nstates;
    a.site_state_off = sites->site_state_off;
    a.state = st->state;
    a.grid = (st->grid && st->ex_every > 0) ? st->grid : nullptr;
    a.M = c->M;
    a.n_sites = sites->n_sites;
    a.stride = st->occ_stride;
    a.occ = (u64*)st->occ_count;
    a.err = c->err;
    GB_CHECK(c, gbk::launch_occupancy(a, s));
    return GB_OK;
}

// Neighbour exchange on the (pH x E) grid; the attempt number is ctr[1], which
// the second kernel advances.
int enqueue_exchange(gb_ctx* c, gb_md_state* st, const gb_sites* sites, cudaStream_t s) {
    gbk::GridExArgs x{};
    x.n_pH = st->n_pH;
    x.n_E = st->n_E;
    x.E_ladder = st->E_ladder;
    x.pH_ladder = st->pH_ladder;
    x.grid = st->grid;
    x.site_off = sites->site_off;
    x.site_kind = sites->site_kind;
    x.site_nstates = sites->site_nstates;
    x.site_state_off = sites->site_state_off;
    x.n_H = sites->n_H;
    x.n_e = sites->n_e;
    x.state = st->state;
    x.ctr = c->ctr;
    x.err = c->err;
    x.ex_count = (gbk::u64*)st->ex_count;
    x.ex_dim = st->ex_dim;
    x.wrap = st->wrap;
    x.seed = st->seed;
    x.kT = st->kT;
    x.E_rep = st->E;
    x.pH_rep = st->pH;
    GB_CHECK(c, gbk::launch_grid_exchange(x, s));
    GB_CHECK(c, gbk::launch_advance_counters(c->ctr, 0, 1, s));
    return GB_OK;
}

// Enqueue `len` MD steps (with their MC attempts and exchanges) on stream s.
// Steps are numbered from the device counter ctr[0]; the last node advances it.
// With the persistent kernel every run of steps up to the next MC / exchange
// point is one launch; otherwise each step is six launches (eight with a
// cutoff: the neighbour list's reset and build).
int enqueue_steps(gb_ctx* c, gb_md_state* st, const gb_sites* sites, int64_t len, cudaStream_t s) {
    const float* xyzq = st->xyzq;
    const float* rad = st->rad_screen;
    const gbk::AtomArgs aa = atom_args(c, xyzq, rad);
    const gbk::MDArgs m = md_args(c, st);
    const int flags = (c->p.rep_k != 0.0f) ? gbk::EF_REP : 0;
    auto mc_due = [&](int64_t t) { return sites && st->mc_every > 0 && t % st->mc_every == 0; };
    auto ex_due = [&](int64_t t) { return sites && st->grid && st->ex_every > 0 && t % st->ex_every == 0; };
    if (c->use_persist && c->persist_grid > 0 && c->p.kappa == 0.0f && c->p.rgbmax == 0.0f && c->p.cut == 0.0f) {
        gbk::PersistArgs a{};
        a.pa = pair_args(c, xyzq, rad);
        a.aa = aa;
        a.md = m;
        a.tasks = c->ptasks.d_tasks;
        a.task_off = c->ptask_off;
        a.phase_off = c->phase_off;
        a.count = c->phase_count;
        for (int p = 0; p < 7; ++p) a.phase_base[p] = c->phase_base[p];
        a.M = c->M;
        a.R_out = st->R;
        a.head = c->qwords;
        a.done = c->qwords + 1;
        a.err = c->err;
        a.spin_limit = c->spin_limit;
        if (c->prof) {
            int rc = ensure_prof_events(c, len);
            if (rc) return rc;
            c->prof_steps_per_launch.clear();
        }
        int64_t k = 0;
        while (k < len) {
            int64_t run = 0;
            for (int64_t kk = k; kk < len; ++kk) {
                ++run;
                const int64_t t = (int64_t)st->step + kk + 1;
                if (mc_due(t) || ex_due(t)) break;
            }
            a.nsteps = (int)run;
            a.step0 = (int)k;
            const size_t pe = 2 * c->prof_steps_per_launch.size();
            if (c->prof) GB_CHECK(c, mark(c, c->prof_ev[pe], s));
            GB_CHECK(c, gbk::launch_persist(a, flags ? 1 : 0, c->persist_grid, s));
            if (c->prof) {
                GB_CHECK(c, mark(c, c->prof_ev[pe + 1], s));
                c->prof_steps_per_launch.push_back((int)run);
            }
            k += run;
            const int64_t t = (int64_t)st->step + k;
            if (mc_due(t)) {
                int rc = enqueue_mc(c, st, sites, k, s);
                if (rc) return rc;
            }
            if (ex_due(t)) {
                int rc = enqueue_exchange(c, st, sites, s);
                if (rc) return rc;
            }
            if (mc_due(t)) {
                int rc = enqueue_occupancy(c, st, sites, s);
                if (rc) return rc;
            }
        }
        GB_CHECK(c, gbk::launch_advance_counters(c->ctr, (u64)len, 0, s));
        return GB_OK;
    }
    if (c->prof) {
        int rc = ensure_prof_events(c, len);
        if (rc) return rc;
        c->prof_steps = len;
        c->prof_steps_per_launch.clear();
    }
    // B A O A of the first step; then per step the evaluation, the MC and
    // exchange attempts due at its end (they read positions, radii and charges,
    // none of which the closing half kick changes), and one launch that closes
    // this step and opens the next.
    GB_CHECK(c, gbk::launch_md_step(aa, m, c->boxes, c->tile_off, 0, gbk::MD_OPEN, s));
    for (int64_t k = 0; k < len; ++k) {
        int rc = evaluate(c, xyzq, rad, st->R, flags, nullptr, s, c->prof ? &c->prof_ev[6 * k] : nullptr, &m,
                          false);
        if (rc) return rc;
        const int64_t t = (int64_t)st->step + k + 1;   // only its residues matter
        if (mc_due(t)) {
            rc = enqueue_mc(c, st, sites, k + 1, s);
            if (rc) return rc;
        }
        if (ex_due(t)) {
            rc = enqueue_exchange(c, st, sites, s);
            if (rc) return rc;
        }
        if (mc_due(t)) {
            rc = enqueue_occupancy(c, st, sites, s);
            if (rc) return rc;
        }
        const int mode = gbk::MD_CLOSE | gbk::MD_KICK | (k + 1 < len ? gbk::MD_OPEN : 0);
        GB_CHECK(c, gbk::launch_md_step(aa, m, c->boxes, c->tile_off, (int)(k + 1), mode, s));
    }
    GB_CHECK(c, gbk::launch_advance_counters(c->ctr, (u64)len, 0, s));
    return GB_OK;
}

}  // namespace

extern "C" int gb_md_init(gb_ctx* c, gb_md_state* st, void* stream) {
    int rc = check_md(c, st);
    if (rc) return rc;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int flags = (c->p.rep_k != 0.0f) ? gbk::EF_REP : 0;
    const gbk::MDArgs m = md_args(c, st);
    // a restart point: a segment that stopped early (a wait that ran out) may
    // have left partial sums in the accumulators, which the kernels otherwise
    // clear as they read them
    const size_t N = (size_t)c->N;
    GB_CHECK(c, cudaMemsetAsync(c->I_acc, 0, sizeof(u64) * N, s));
    GB_CHECK(c, cudaMemsetAsync(c->dR_acc, 0, sizeof(u64) * N, s));
    GB_CHECK(c, cudaMemsetAsync(c->phi_acc, 0, sizeof(u64) * N, s));
    GB_CHECK(c, cudaMemsetAsync(c->F_acc, 0, sizeof(u64) * 3 * N, s));
    GB_CHECK(c, cudaMemsetAsync(c->E_acc, 0, sizeof(u64) * 4 * (size_t)c->M, s));
    rc = evaluate(c, st->xyzq, st->rad_screen, st->R, flags, nullptr, s, nullptr, &m, true);
    if (rc) return rc;
    GB_CHECK(c, gbk::launch_md_step(atom_args(c, st->xyzq, st->rad_screen), m, nullptr, nullptr, 0, gbk::MD_CLOSE, s));
    return GB_OK;
}

extern "C" int gb_md_segment(gb_ctx* c, gb_md_state* st, const gb_sites* sites, int64_t nsteps,
                             void* stream) {
    int rc = check_md(c, st);
    if (rc) return rc;
    if (nsteps < 0) return fail(c, GB_ERR_INVALID_ARG, "nsteps < 0");
    if (sites) {
        rc = check_sites(c, sites);
        if (rc) return rc;
        if (st->mc_every > 0 && !st->state) return fail(c, GB_ERR_INVALID_ARG, "state is NULL");
        if (st->occ_count && st->occ_stride <= 0) return fail(c, GB_ERR_INVALID_ARG, "occ_stride must be > 0");
        if (st->ex_every > 0 && st->grid &&
            (st->n_E * st->n_pH != c->M || !st->E_ladder || !st->pH_ladder || !st->E || !st->pH))
            return fail(c, GB_ERR_INVALID_ARG, "exchange grid does not match the batch");
    }
    if (nsteps == 0) return GB_OK;
    DeviceGuard g(c->device);
    if (sites && st->mc_every > 0 && st->mc_mode == 1) {
        rc = ensure_sweep_part(c);
        if (rc) return rc;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // one captured block covers a whole number of MC and exchange periods
    int64_t L = 1;
    auto lcm = [](int64_t a, int64_t b) {
        int64_t x = a, y = b;
        while (y) { int64_t t = x % y; x = y; y = t; }
        return a / x * b;
    };
    if (sites && st->mc_every > 0) L = lcm(L, st->mc_every);
    if (sites && st->grid && st->ex_every > 0) L = lcm(L, st->ex_every);
    const bool graph_ok = (L <= 1000) && ((int64_t)st->step % L == 0) && (nsteps % L == 0);
    GB_CHECK(c, gbk::launch_set_counters(c->ctr, st->step, st->attempt, s));
    if (!graph_ok) {
        rc = enqueue_steps(c, st, sites, nsteps, s);
        if (rc) return rc;
    } else {
        // key: everything baked into the graph
        std::vector<uint8_t> key(sizeof(gb_md_state) + sizeof(gb_sites) + sizeof(int64_t) * 3);
        gb_md_state kst = *st;
        kst.step = 0;
        kst.attempt = 0;
        memcpy(key.data(), &kst, sizeof(kst));
        gb_sites ks{};
        if (sites) ks = *sites;
        memcpy(key.data() + sizeof(kst), &ks, sizeof(ks));
        const int64_t extra[3] = {L, c->wpb * 2 + (c->use_persist ? 1 : 0), (int64_t)c->tpt * 2 + (c->prof ? 1 : 0)};
        memcpy(key.data() + sizeof(kst) + sizeof(ks), extra, sizeof(extra));
        if (c->prof) {
            rc = ensure_prof_events(c, L);
            if (rc) return rc;
        }
        if (!c->md_exec || key != c->md_key) {
            if (c->md_exec) { cudaGraphExecDestroy(c->md_exec); c->md_exec = nullptr; }
            cudaGraph_t graph = nullptr;
            GB_CHECK(c, cudaStreamBeginCapture(c->cs, cudaStreamCaptureModeThreadLocal));
            c->capturing = true;
            rc = enqueue_steps(c, st, sites, L, c->cs);
            c->capturing = false;
            cudaError_t e = cudaStreamEndCapture(c->cs, &graph);
            if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
            if (e != cudaSuccess) return cuda_fail(c, e, "graph capture");
            e = cudaGraphInstantiate(&c->md_exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) { c->md_exec = nullptr; return cuda_fail(c, e, "graph instantiate"); }
            c->md_key = key;
            c->md_len = L;
        }
        GB_CHECK(c, cudaEventRecord(c->ev_in, s));
        GB_CHECK(c, cudaStreamWaitEvent(c->cs, c->ev_in, 0));
        for (int64_t k = 0; k < nsteps / L; ++k) GB_CHECK(c, cudaGraphLaunch(c->md_exec, c->cs));
        GB_CHECK(c, cudaEventRecord(c->ev_out, c->cs));
        GB_CHECK(c, cudaStreamWaitEvent(s, c->ev_out, 0));
    }
    int64_t n_ex = 0;
    if (sites && st->grid && st->ex_every > 0)
        n_ex = ((int64_t)st->step + nsteps) / st->ex_every - (int64_t)st->step / st->ex_every;
    st->step += (uint64_t)nsteps;
    st->attempt += (uint64_t)n_ex;
    return GB_OK;
}

extern "C" int gb_md_segment_host(gb_ctx* c, gb_md_state* st, const gb_sites* sites, int64_t nsteps,
                                  const gb_md_host* h, void* stream) {
    int rc = check_md(c, st);
    if (rc) return rc;
    if (!h) return fail(c, GB_ERR_INVALID_ARG, "host state is NULL");
    if (h->state && (!st->state || h->n_sites < 0)) return fail(c, GB_ERR_INVALID_ARG, "host state array without a device one");
    if (h->grid && !st->grid) return fail(c, GB_ERR_INVALID_ARG, "host grid without a device one");
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t N = (size_t)c->N, M = (size_t)c->M;
    const size_t G = (size_t)st->n_E * (size_t)st->n_pH;
    struct Pair { void* dev; void* host; size_t bytes; };
    const Pair arrays[] = {
        {st->xyzq, h->xyzq, 16 * N},  {st->vel, h->vel, 16 * N},   {st->force, h->force, 16 * N},
        {st->state, h->state, 4 * (size_t)(h->n_sites > 0 ? h->n_sites : 0)},
        {st->pH, h->pH, 8 * M},       {st->E, h->E, 8 * M},        {st->grid, h->grid, 4 * G},
    };
    for (const Pair& a : arrays)
        if (a.host && a.bytes) {
            if (!a.dev) return fail(c, GB_ERR_INVALID_ARG, "host array without a device buffer");
            GB_CHECK(c, cudaMemcpyAsync(a.dev, a.host, a.bytes, cudaMemcpyHostToDevice, s));
        }
    rc = gb_md_segment(c, st, sites, nsteps, stream);
    if (rc) return rc;
    for (const Pair& a : arrays)
        if (a.host && a.bytes) GB_CHECK(c, cudaMemcpyAsync(a.host, a.dev, a.bytes, cudaMemcpyDeviceToHost, s));
    return gb_sync_status(c, stream);
}

// ---------------------------------------------------------------------------------
// Autotuner: time one full force evaluation per candidate tile shape.

extern "C" int gb_autotune(gb_ctx* c, const float* xyzq, const float* rad, void* stream) {
    // Every (warps per block, tiles per task) candidate runs full evaluations
    // with each register cap; the passes are timed one by one, so each pass
    // keeps its own best cap and a candidate scores the sum of its passes' best.
    int rc = check_inputs(c, xyzq, rad);
    if (rc) return rc;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    GB_CHECK(c, cudaStreamSynchronize(s));
    const int wpbs[] = {1, 2, 4, 8};
    // the cutoff kernels come with caps 1 and 3 only
    const bool cut = c->list_ctr != nullptr;
    std::vector<int> caps = cut ? std::vector<int>{1, 3} : std::vector<int>{1, 3, 4};
    std::vector<int> tpts;
    const int base = default_tpt(c);
    for (int f : {1, 2, 4, 8, 16, 32, 64}) {
        int t = std::max(1, base * f / 16);
        if (std::find(tpts.begin(), tpts.end(), t) == tpts.end()) tpts.push_back(t);
    }
    cudaEvent_t ev[6];
    for (auto& e : ev) GB_CHECK(c, cudaEventCreate(&e));
    float best = 1e30f;
    int best_w = c->wpb, best_t = c->tpt, best_cap[3] = {c->tasks.cap[0], c->tasks.cap[1], c->tasks.cap[2]};
    for (int t : tpts) {
        rc = gb_set_tiles(c, c->wpb, t);
        if (rc) break;
        for (int w : wpbs) {
            c->wpb = w;
            float pass_best[3] = {1e30f, 1e30f, 1e30f};
            int pass_cap[3] = {3, 3, 3};
            for (int cap : caps) {
                for (int k = 0; k < 3; ++k) c->tasks.cap[k] = cap;
                float ms_min[3] = {1e30f, 1e30f, 1e30f};
                for (int rep = 0; rep < 5 && !rc; ++rep) {
                    rc = evaluate(c, xyzq, rad, nullptr, 0, nullptr, s, ev);
                    if (rc) break;
                    cudaEventSynchronize(ev[5]);
                    float ms[3] = {0, 0, 0};
                    cudaEventElapsedTime(&ms[0], ev[0], ev[1]);
                    cudaEventElapsedTime(&ms[1], ev[2], ev[3]);
                    cudaEventElapsedTime(&ms[2], ev[4], ev[5]);
                    if (rep > 0)
                        for (int k = 0; k < 3; ++k) ms_min[k] = std::min(ms_min[k], ms[k]);
                }
                if (rc) break;
                for (int k = 0; k < 3; ++k)
                    if (ms_min[k] < pass_best[k]) { pass_best[k] = ms_min[k]; pass_cap[k] = cap; }
            }
            if (rc) break;
            const float total = pass_best[0] + pass_best[1] + pass_best[2];
            if (total < best) {
                best = total;
                best_w = w;
                best_t = t;
                for (int k = 0; k < 3; ++k) best_cap[k] = pass_cap[k];
            }
        }
        if (rc) break;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    // the O(N) kernels left their accumulators cleared; the last evaluation's
    // force and chain accumulators are read out (and cleared) here
    if (!rc) rc = gbk::launch_forces_out(atom_args(c, xyzq, rad), nullptr, nullptr, nullptr, s) == cudaSuccess
                      ? GB_OK : GB_ERR_CUDA;
    if (rc) return rc;
    for (int k = 0; k < 3; ++k) c->tasks.cap[k] = best_cap[k];
    return gb_set_tiles(c, best_w, best_t);
}

extern "C" int gb_set_profiling(gb_ctx* c, int32_t enable) {
    if (!c) return fail(nullptr, GB_ERR_INVALID_ARG, "NULL context");
    c->prof = enable != 0;
    c->prof_steps = 0;
    return GB_OK;
}

extern "C" int gb_pass_times(gb_ctx* c, double* mean_ms) {
    if (!c || !mean_ms) return fail(c, GB_ERR_INVALID_ARG, "NULL argument");
    if (!c->prof || c->prof_steps == 0 || !c->prof_steps_per_launch.empty())
        return fail(c, GB_ERR_INVALID_ARG, "profiling is off or no three-pass segment ran");
    DeviceGuard g(c->device);
    for (int p = 0; p < 3; ++p) {
        double acc = 0.0;
        for (int64_t k = 0; k < c->prof_steps; ++k) {
            float ms = 0.0f;
            GB_CHECK(c, cudaEventSynchronize(c->prof_ev[6 * k + 2 * p + 1]));
            GB_CHECK(c, cudaEventElapsedTime(&ms, c->prof_ev[6 * k + 2 * p], c->prof_ev[6 * k + 2 * p + 1]));
            acc += ms;
        }
        mean_ms[p] = acc / (double)c->prof_steps;
    }
    return GB_OK;
}

extern "C" int gb_set_persistent(gb_ctx* c, int32_t enable) {
    if (!c) return fail(nullptr, GB_ERR_INVALID_ARG, "NULL context");
    c->use_persist = enable != 0;
    if (c->md_exec) { cudaGraphExecDestroy(c->md_exec); c->md_exec = nullptr; c->md_key.clear(); }
    return GB_OK;
}

// Register caps tuned on the MD driver itself: coordinate descent over the
// three passes' caps, each candidate timed on short MD segments (CUDA events
// around the captured graphs, the same launches the driver uses), every trial
// starting from a saved copy of the MD state, which is put back at the end.
extern "C" int gb_autotune_md(gb_ctx* c, gb_md_state* st, const gb_sites* sites, int64_t trial_steps,
                              void* stream) {
    int rc = check_md(c, st);
    if (rc) return rc;
    if (sites && (rc = check_sites(c, sites))) return rc;
    if (trial_steps < 1 || trial_steps > 100000) return fail(c, GB_ERR_INVALID_ARG, "trial_steps must be 1..100000");
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t N = (size_t)c->N, M = (size_t)c->M;
    const size_t n_sites = (sites && st->state) ? (size_t)sites->n_sites : 0;
    struct Buf { void* p; size_t bytes; };
    const Buf bufs[] = {{(void*)st->xyzq, 16 * N}, {(void*)st->vel, 16 * N}, {(void*)st->force, 16 * N},
                        {(void*)st->R, 4 * N},     {(void*)st->state, 4 * n_sites},
                        {(void*)st->pH, st->pH ? 8 * M : 0}, {(void*)st->E, st->E ? 8 * M : 0},
                        {(void*)st->grid, st->grid ? 4 * M : 0},
                        {(void*)st->ex_count, st->ex_count ? 32 * M : 0}};
    size_t total = 0;
    for (const Buf& b : bufs) total += (b.p ? b.bytes : 0);
    unsigned char* save = nullptr;
    GB_CHECK(c, cudaMalloc((void**)&save, std::max<size_t>(total, 16)));
    const gb_md_state st0 = *st;
    auto copy_state = [&](bool out) -> cudaError_t {
        size_t off = 0;
        for (const Buf& b : bufs) {
            if (!b.p || !b.bytes) continue;
            cudaError_t e = out ? cudaMemcpyAsync(save + off, b.p, b.bytes, cudaMemcpyDeviceToDevice, s)
                                : cudaMemcpyAsync(b.p, save + off, b.bytes, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return e;
            off += b.bytes;
        }
        return cudaSuccess;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = copy_state(true);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    const std::vector<int> caps = c->list_ctr ? std::vector<int>{1, 3} : std::vector<int>{1, 3, 4};
    auto trial = [&](const int* cap, float* ms) -> int {
        for (int k = 0; k < 3; ++k) c->tasks.cap[k] = cap[k];
        if (c->md_exec) { cudaGraphExecDestroy(c->md_exec); c->md_exec = nullptr; c->md_key.clear(); }
        float best = 1e30f;
        for (int rep = 0; rep < 5; ++rep) {           // the first run also captures the graph
            *st = st0;
            if (copy_state(false) != cudaSuccess) return fail(c, GB_ERR_CUDA, "state restore failed");
            if (cudaEventRecord(e0, s) != cudaSuccess) return fail(c, GB_ERR_CUDA, "event record failed");
            int r = gb_md_segment(c, st, sites, trial_steps, stream);
            if (r) return r;
            if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
                return fail(c, GB_ERR_CUDA, "event wait failed");
            float t = 0.0f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) best = std::min(best, t);
        }
        *ms = best;
        return GB_OK;
    };
    int best[3] = {c->tasks.cap[0], c->tasks.cap[1], c->tasks.cap[2]};
    for (int& b : best)
        if (std::find(caps.begin(), caps.end(), b) == caps.end()) b = 3;
    float t_best = 0.0f;
    if (ce != cudaSuccess) rc = cuda_fail(c, ce, "gb_autotune_md set-up");
    if (!rc) rc = trial(best, &t_best);
    for (int pass = 0; pass < 3 && !rc; ++pass) {
        for (int cap : caps) {
            if (cap == best[pass]) continue;
            int cand[3] = {best[0], best[1], best[2]};
            cand[pass] = cap;
            float t = 0.0f;
            rc = trial(cand, &t);
            if (rc) break;
            if (t < t_best) {
                t_best = t;
                for (int k = 0; k < 3; ++k) best[k] = cand[k];
            }
        }
    }
    // the chosen caps; the state as it was; no graph captured with other caps
    for (int k = 0; k < 3; ++k) c->tasks.cap[k] = best[k];
    if (c->md_exec) { cudaGraphExecDestroy(c->md_exec); c->md_exec = nullptr; c->md_key.clear(); }
    *st = st0;
    cudaError_t re = copy_state(false);
    if (re == cudaSuccess) re = cudaStreamSynchronize(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(save);
    if (!rc && re != cudaSuccess) rc = cuda_fail(c, re, "state restore");
    return rc;
}

extern "C" int gb_set_wait_limit(gb_ctx* c, int64_t polls) {
    if (!c) return fail(nullptr, GB_ERR_INVALID_ARG, "NULL context");
    if (polls < 0 || polls > 0xffffffffLL) return fail(c, GB_ERR_INVALID_ARG, "polls must be 0 .. 2^32 - 1");
    c->spin_limit = polls == 0 ? (1u << 22) : (unsigned)polls;
    // captured launches carry the limit: rebuild the MD graph on next use
    if (c->md_exec) { cudaGraphExecDestroy(c->md_exec); c->md_exec = nullptr; c->md_key.clear(); }
    return GB_OK;
}

extern "C" int gb_persist_times(gb_ctx* c, double* out) {
    if (!c || !out) return fail(c, GB_ERR_INVALID_ARG, "NULL argument");
    if (!c->prof || c->prof_steps_per_launch.empty())
        return fail(c, GB_ERR_INVALID_ARG, "profiling is off or no persistent launch ran");
    DeviceGuard g(c->device);
    double ms_sum = 0.0, steps = 0.0;
    for (size_t k = 0; k < c->prof_steps_per_launch.size(); ++k) {
        float ms = 0.0f;
        GB_CHECK(c, cudaEventSynchronize(c->prof_ev[2 * k + 1]));
        GB_CHECK(c, cudaEventElapsedTime(&ms, c->prof_ev[2 * k], c->prof_ev[2 * k + 1]));
        ms_sum += ms;
        steps += c->prof_steps_per_launch[k];
    }
    const double nl = (double)c->prof_steps_per_launch.size();
    out[0] = ms_sum / steps;   // ms per MD step inside the persistent kernel
    out[1] = ms_sum / nl;      // ms per launch
    out[2] = steps / nl;       // MD steps per launch
    return GB_OK;
}
