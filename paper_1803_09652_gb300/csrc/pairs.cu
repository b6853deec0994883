// O(N^2) pair passes of the GB hot path on sm_103a.
//
// Every replica's atoms are cut into 32-atom tiles; a warp owns a contiguous
// run of tile pairs (I, J), I <= J, of the upper triangle.  Lane l holds atom
// I*32 + l ("i") in registers for the whole row; the 32 atoms of tile J ("j")
// rotate one lane per step with warp shuffles, carrying their own FP32 force
// partials with them, so each unordered pair is evaluated exactly once
// (Newton's third law) and both of its contributions are summed without
// atomics.  After a tile pair, the j partials are folded into int64 fixed
// point with one global atomic per atom and component; the i partials go to
// int64 registers and are flushed when the row ends.  FP32 partials never
// span more than one 32 x 32 tile pair, and integer sums are associative,
// so the results do not depend on launch order or on the tile-run split.
//
// Pass 1 (Born integrals), pass 2 (GB + Coulomb energy, direct forces, dE/dR,
// optional dE/dq and soft repulsion) and pass 3 (Born-radius chain rule)
// share the walker below; the arithmetic of each pass is in its policy.
#include "common.cuh"
#include "internal.h"
#include "poly_coeffs.h"

namespace gbk {

// --- HCT descreening integral H(r; a, s) --------------------------------------
// H = (1/4pi) * volume integral of |y - x_i|^-4 over the part of the sphere
// (centre x_j, radius s) that lies outside the sphere (x_i, a).  Closed form
// from spherical shells about x_i between L = max(a, |r - s|) and U = r + s;
// when x_i is engulfed (a < s - r) the full shells between a and s - r add
// 1/a - 1/L.  It is used only where the spheres overlap (rare): there its
// terms are O(1) and FP32 keeps them.
__device__ __forceinline__ float hct_closed(float r, float rinv, float a, float s) {
    if (a >= r + s) return 0.0f;
    const float U = r + s;
    const float L = fmaxf(a, fabsf(r - s));
    const float iU = 1.0f / U, iL = 1.0f / L;
    const float iU2 = iU * iU, iL2 = iL * iL;
    float b = (iL - iU) + 0.25f * (r - s * s * rinv) * (iU2 - iL2) + 0.5f * rinv * logf(L * iU);
    if (a < s - r) b += 2.0f * (1.0f / a - iL);
    return 0.5f * b;
}

// -(dH/dr) / r of the closed form.
__device__ __forceinline__ float hct_closed_fr(float r, float rinv, float a, float s) {
    if (a >= r + s) return 0.0f;
    const float U = r + s;
    const float rs = r - s;
    float L, dL;
    if (a > fabsf(rs)) { L = a; dL = 0.0f; }
    else { L = fabsf(rs); dL = rs > 0.0f ? 1.0f : -1.0f; }
    const float iU = 1.0f / U, iL = 1.0f / L;
    const float iU2 = iU * iU, iL2 = iL * iL;
    const float w = r - s * s * rinv;           // r - s^2/r
    const float dw = 1.0f + s * s * rinv * rinv; // d/dr of w
    // b = 1/L - 1/U + (w/4)(1/U^2 - 1/L^2) + (1/(2r)) ln(L/U)
    float db = -dL * iL2 + iU2
             + 0.25f * dw * (iU2 - iL2)
             + 0.5f * w * (dL * iL2 * iL - iU2 * iU)
             - 0.5f * rinv * rinv * logf(L * iU)
             + 0.5f * rinv * (dL * iL - iU);
    if (a < s - r) db += 2.0f * dL * iL2;
    return -0.5f * db * rinv;
}

// Non-overlapping spheres: H = 1/2 x^3/r g(x^2), dH/dr = -1/2 x^3/r^2 h(x^2),
// x = s/r, with g, h the fitted polynomials (no cancellation, no MUFU).
__device__ __forceinline__ float hct(float r, float rinv, float a, float s) {
    const float x = s * rinv, y = x * x;
    if (r >= a + s && y <= GB_POLY_YMAX) return 0.5f * rinv * x * y * gb_poly_g(y);
    return hct_closed(r, rinv, a, s);
}

__device__ __forceinline__ float hct_fr(float r, float rinv, float a, float s) {
    const float x = s * rinv, y = x * x;
    if (r >= a + s && y <= GB_POLY_YMAX) return 0.5f * x * y * rinv * rinv * rinv * gb_poly_h(y);
    return hct_closed_fr(r, rinv, a, s);
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// --- pass 1: Born integrals I_i = sum_j H(r_ij; a_i, s_j) -----------------------
struct Born {
    struct IState { float x, y, z, a, s; long long acc; };
    struct JState { float x, y, z, a, s, acc; };
    struct Part {
        float I;
        __device__ __forceinline__ void zero() { I = 0.0f; }
    };
    static __device__ __forceinline__ void load_i(const PairArgs& A, int64_t base, int n, int i, IState& st) {
        if (i < n) {
            const float4 p = A.xyzq[base + i];
            const float2 rs = A.rad[base + i];
            st.x = p.x; st.y = p.y; st.z = p.z;
            st.a = rs.x - A.offset;
            st.s = rs.y * st.a;
        } else {
            st.x = ghost_x(i - n); st.y = 0.0f; st.z = 0.0f; st.a = 1.0f; st.s = 0.0f;
        }
        st.acc = 0;
    }
    static __device__ __forceinline__ void load_j(const PairArgs& A, int64_t base, int n, int j, JState& st) {
        if (j < n) {
            const float4 p = A.xyzq[base + j];
            const float2 rs = A.rad[base + j];
            st.x = p.x; st.y = p.y; st.z = p.z;
            st.a = rs.x - A.offset;
            st.s = rs.y * st.a;
        } else {
            st.x = ghost_x(j - n); st.y = 0.0f; st.z = 0.0f; st.a = 1.0f; st.s = 0.0f;
        }
        st.acc = 0.0f;
    }
    template <int FLAGS>
    static __device__ __forceinline__ void pair(const PairArgs&, const IState& i, JState& j, Part& p, int, int) {
        const float dx = j.x - i.x, dy = j.y - i.y, dz = j.z - i.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float rinv = rsqrtf(r2);
        const float r = r2 * rinv;
        p.I += hct(r, rinv, i.a, j.s);
        j.acc += hct(r, rinv, j.a, i.s);
    }
    static __device__ __forceinline__ void rotate(JState& j, int src) {
        j.x = shfl(j.x, src); j.y = shfl(j.y, src); j.z = shfl(j.z, src);
        j.a = shfl(j.a, src); j.s = shfl(j.s, src); j.acc = shfl(j.acc, src);
    }
    static __device__ __forceinline__ void home(JState& j, int src) { j.acc = shfl(j.acc, src); }
    static __device__ __forceinline__ void fold_i(IState& i, const Part& p) { i.acc += fix_i(p.I); }
    static __device__ __forceinline__ void flush_j(const PairArgs& A, int64_t base, int n, int j, const JState& st) {
        if (j < n) red_add(&A.I_acc[base + j], fix_i(st.acc));
    }
    static __device__ __forceinline__ void flush_i(const PairArgs& A, int, int64_t base, int n, int i, const IState& st) {
        if (i < n) red_add(&A.I_acc[base + i], st.acc);
    }
};

// --- pass 2: GB + Coulomb pair energy, direct forces, dE/dR, dE/dq --------------
// Pair (i, j), both orderings of the double sum together:
//   e_GB = -tau k_e q_i q_j / f,  f^2 = r^2 + R_i R_j exp(-D),  D = r^2 / (4 R_i R_j)
//   e_C  =  k_c q_i q_j / r
//   -(de/dr)/r = e_GB (1 - exp(-D)/4) / f^2 + e_C / r^2
//   de/dR_i = -e_GB exp(-D)(1 + D) R_j / (2 f^2)       (and i <-> j)
//   de/dq_i = (-tau k_e / f + k_c / r) q_j              (and i <-> j)
struct Energy {
    struct IState {
        float x, y, z, q, R, h;
        long long fx, fy, fz, dR, phi, egb, ec, er;
    };
    struct JState { float x, y, z, q, R, h, fx, fy, fz, dR, phi; };
    struct Part {
        float fx, fy, fz, dR, phi, egb, ec, er;
        __device__ __forceinline__ void zero() { fx = fy = fz = dR = phi = egb = ec = er = 0.0f; }
    };
    static __device__ __forceinline__ void load_common(const PairArgs& A, int64_t base, int n, int i,
                                                       float& x, float& y, float& z, float& q,
                                                       float& R, float& h) {
        if (i < n) {
            const float4 p = A.xyzq[base + i];
            const float2 rh = A.Rh[base + i];
            x = p.x; y = p.y; z = p.z; q = p.w; R = rh.x; h = rh.y;
        } else {
            x = ghost_x(i - n); y = 0.0f; z = 0.0f; q = 0.0f; R = 1.0f; h = 0.5f;
        }
    }
    static __device__ __forceinline__ void load_i(const PairArgs& A, int64_t base, int n, int i, IState& st) {
        load_common(A, base, n, i, st.x, st.y, st.z, st.q, st.R, st.h);
        st.fx = st.fy = st.fz = st.dR = st.phi = st.egb = st.ec = st.er = 0;
    }
    static __device__ __forceinline__ void load_j(const PairArgs& A, int64_t base, int n, int j, JState& st) {
        load_common(A, base, n, j, st.x, st.y, st.z, st.q, st.R, st.h);
        st.fx = st.fy = st.fz = st.dR = st.phi = 0.0f;
    }
    template <int FLAGS>
    static __device__ __forceinline__ void pair(const PairArgs& A, const IState& i, JState& j, Part& p,
                                                int ii, int jj) {
        const float dx = j.x - i.x, dy = j.y - i.y, dz = j.z - i.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float rinv = rsqrtf(r2);
        const float qq = i.q * j.q;
        const float D = r2 * (i.h * j.h);
        const float e = __expf(-D);
        const float f2 = fmaf(i.R * j.R, e, r2);
        const float finv = rsqrtf(f2);
        const float finv2 = finv * finv;
        const float gb = -A.tau_ke * qq * finv;
        const float cl = A.kc * qq * rinv;
        float fr = gb * finv2 * fmaf(-0.25f, e, 1.0f) + cl * rinv * rinv;
        const float G = -0.5f * gb * finv2 * e * (1.0f + D);
        if (FLAGS & EF_REP) {
            const float r = r2 * rinv;
            if (r < A.rep_sigma && (ii - jj > 1 || jj - ii > 1)) {
                const float dd = A.rep_sigma - r;
                fr += 2.0f * A.rep_k * dd * rinv;
                if (FLAGS & EF_ENERGY) p.er += A.rep_k * dd * dd;
            }
        }
        p.fx = fmaf(-fr, dx, p.fx); p.fy = fmaf(-fr, dy, p.fy); p.fz = fmaf(-fr, dz, p.fz);
        j.fx = fmaf(fr, dx, j.fx); j.fy = fmaf(fr, dy, j.fy); j.fz = fmaf(fr, dz, j.fz);
        p.dR = fmaf(G, j.R, p.dR);
        j.dR = fmaf(G, i.R, j.dR);
        if (FLAGS & EF_PHI) {
            const float P = fmaf(-A.tau_ke, finv, A.kc * rinv);
            p.phi = fmaf(P, j.q, p.phi);
            j.phi = fmaf(P, i.q, j.phi);
        }
        if (FLAGS & EF_ENERGY) { p.egb += gb; p.ec += cl; }
    }
    template <int FLAGS>
    static __device__ __forceinline__ void rotate_f(JState& j, int src) {
        j.x = shfl(j.x, src); j.y = shfl(j.y, src); j.z = shfl(j.z, src);
        j.q = shfl(j.q, src); j.R = shfl(j.R, src); j.h = shfl(j.h, src);
        j.fx = shfl(j.fx, src); j.fy = shfl(j.fy, src); j.fz = shfl(j.fz, src);
        j.dR = shfl(j.dR, src);
        if (FLAGS & EF_PHI) j.phi = shfl(j.phi, src);
    }
    template <int FLAGS>
    static __device__ __forceinline__ void home_f(JState& j, int src) {
        j.fx = shfl(j.fx, src); j.fy = shfl(j.fy, src); j.fz = shfl(j.fz, src);
        j.dR = shfl(j.dR, src);
        if (FLAGS & EF_PHI) j.phi = shfl(j.phi, src);
    }
    template <int FLAGS>
    static __device__ __forceinline__ void fold_i_f(IState& i, const Part& p) {
        i.fx += fix(p.fx); i.fy += fix(p.fy); i.fz += fix(p.fz);
        i.dR += fix(p.dR);
        if (FLAGS & EF_PHI) i.phi += fix(p.phi);
        if (FLAGS & EF_ENERGY) {
            i.egb += fix(p.egb); i.ec += fix(p.ec);
            if (FLAGS & EF_REP) i.er += fix(p.er);
        }
    }
    template <int FLAGS>
    static __device__ __forceinline__ void flush_j_f(const PairArgs& A, int64_t base, int n, int j, const JState& st) {
        if (j < n) {
            const int64_t g = base + j;
            red_add(&A.F_acc[g], fix(st.fx));
            red_add(&A.F_acc[A.N + g], fix(st.fy));
            red_add(&A.F_acc[2 * A.N + g], fix(st.fz));
            red_add(&A.dR_acc[g], fix(st.dR));
            if (FLAGS & EF_PHI) red_add(&A.phi_acc[g], fix(st.phi));
        }
    }
    template <int FLAGS>
    static __device__ __forceinline__ void flush_i_f(const PairArgs& A, int r, int64_t base, int n, int i, const IState& st) {
        if (i < n) {
            const int64_t g = base + i;
            red_add(&A.F_acc[g], st.fx);
            red_add(&A.F_acc[A.N + g], st.fy);
            red_add(&A.F_acc[2 * A.N + g], st.fz);
            red_add(&A.dR_acc[g], st.dR);
            if (FLAGS & EF_PHI) red_add(&A.phi_acc[g], st.phi);
        }
        if (FLAGS & EF_ENERGY) {
            const long long egb = warp_sum_ll(st.egb), ec = warp_sum_ll(st.ec);
            const long long er = (FLAGS & EF_REP) ? warp_sum_ll(st.er) : 0;
            if ((threadIdx.x & 31) == 0) {
                red_add(&A.E_acc[4 * r + 0], egb);
                red_add(&A.E_acc[4 * r + 1], ec);
                if (FLAGS & EF_REP) red_add(&A.E_acc[4 * r + 2], er);
            }
        }
    }
};

// --- pass 3: Born-radius chain rule -------------------------------------------
// E depends on R_i(psi_i), psi_i = a_i sum_j H(r_ij; a_i, s_j).  With
// c_i = dE/dR_i * dR_i/dpsi_i * a_i the pair (i, j) carries
//   -(dE/dr)/r = c_i * (-(dH(r; a_i, s_j)/dr)/r) + c_j * (-(dH(r; a_j, s_i)/dr)/r).
struct Chain {
    struct IState { float x, y, z, a, s, c; long long fx, fy, fz; };
    struct JState { float x, y, z, a, s, c, fx, fy, fz; };
    struct Part {
        float fx, fy, fz;
        __device__ __forceinline__ void zero() { fx = fy = fz = 0.0f; }
    };
    static __device__ __forceinline__ void load_common(const PairArgs& A, int64_t base, int n, int i,
                                                       float& x, float& y, float& z, float& a,
                                                       float& s, float& c) {
        if (i < n) {
            const float4 p = A.xyzq[base + i];
            const float2 rs = A.rad[base + i];
            x = p.x; y = p.y; z = p.z;
            a = rs.x - A.offset;
            s = rs.y * a;
            c = A.cc[base + i];
        } else {
            x = ghost_x(i - n); y = 0.0f; z = 0.0f; a = 1.0f; s = 0.0f; c = 0.0f;
        }
    }
    static __device__ __forceinline__ void load_i(const PairArgs& A, int64_t base, int n, int i, IState& st) {
        load_common(A, base, n, i, st.x, st.y, st.z, st.a, st.s, st.c);
        st.fx = st.fy = st.fz = 0;
    }
    static __device__ __forceinline__ void load_j(const PairArgs& A, int64_t base, int n, int j, JState& st) {
        load_common(A, base, n, j, st.x, st.y, st.z, st.a, st.s, st.c);
        st.fx = st.fy = st.fz = 0.0f;
    }
    template <int FLAGS>
    static __device__ __forceinline__ void pair(const PairArgs&, const IState& i, JState& j, Part& p, int, int) {
        const float dx = j.x - i.x, dy = j.y - i.y, dz = j.z - i.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float rinv = rsqrtf(r2);
        const float r = r2 * rinv;
        const float fr = i.c * hct_fr(r, rinv, i.a, j.s) + j.c * hct_fr(r, rinv, j.a, i.s);
        p.fx = fmaf(-fr, dx, p.fx); p.fy = fmaf(-fr, dy, p.fy); p.fz = fmaf(-fr, dz, p.fz);
        j.fx = fmaf(fr, dx, j.fx); j.fy = fmaf(fr, dy, j.fy); j.fz = fmaf(fr, dz, j.fz);
    }
    static __device__ __forceinline__ void rotate(JState& j, int src) {
        j.x = shfl(j.x, src); j.y = shfl(j.y, src); j.z = shfl(j.z, src);
        j.a = shfl(j.a, src); j.s = shfl(j.s, src); j.c = shfl(j.c, src);
        j.fx = shfl(j.fx, src); j.fy = shfl(j.fy, src); j.fz = shfl(j.fz, src);
    }
    static __device__ __forceinline__ void home(JState& j, int src) {
        j.fx = shfl(j.fx, src); j.fy = shfl(j.fy, src); j.fz = shfl(j.fz, src);
    }
    static __device__ __forceinline__ void fold_i(IState& i, const Part& p) {
        i.fx += fix(p.fx); i.fy += fix(p.fy); i.fz += fix(p.fz);
    }
    static __device__ __forceinline__ void flush_j(const PairArgs& A, int64_t base, int n, int j, const JState& st) {
        if (j < n) {
            const int64_t g = base + j;
            red_add(&A.F_acc[g], fix(st.fx));
            red_add(&A.F_acc[A.N + g], fix(st.fy));
            red_add(&A.F_acc[2 * A.N + g], fix(st.fz));
        }
    }
    static __device__ __forceinline__ void flush_i(const PairArgs& A, int, int64_t base, int n, int i, const IState& st) {
        if (i < n) {
            const int64_t g = base + i;
            red_add(&A.F_acc[g], st.fx);
            red_add(&A.F_acc[A.N + g], st.fy);
            red_add(&A.F_acc[2 * A.N + g], st.fz);
        }
    }
};

// Energy's helpers carry the flag set; adapt them to the walker's interface.
template <int FLAGS>
struct EnergyF : Energy {
    static __device__ __forceinline__ void rotate(JState& j, int src) { rotate_f<FLAGS>(j, src); }
    static __device__ __forceinline__ void home(JState& j, int src) { home_f<FLAGS>(j, src); }
    static __device__ __forceinline__ void fold_i(IState& i, const Part& p) { fold_i_f<FLAGS>(i, p); }
    static __device__ __forceinline__ void flush_j(const PairArgs& A, int64_t b, int n, int j, const JState& s) {
        flush_j_f<FLAGS>(A, b, n, j, s);
    }
    static __device__ __forceinline__ void flush_i(const PairArgs& A, int r, int64_t b, int n, int i, const IState& s) {
        flush_i_f<FLAGS>(A, r, b, n, i, s);
    }
};

// --- the warp walker ------------------------------------------------------------
template <class P, int FLAGS>
__global__ void __launch_bounds__(256) k_pairs(PairArgs A, const int4* __restrict__ tasks, int n_tasks) {
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= n_tasks) return;
    const int4 t = tasks[w];
    int r = t.x, I = t.y, J = t.z;
    const int cnt = t.w;
    int64_t base = A.atom_off[r];
    int n = (int)(A.atom_off[r + 1] - base);
    int nb = (n + 31) >> 5;
    typename P::IState is;
    P::load_i(A, base, n, I * 32 + lane, is);
    const int next = (lane + 1) & 31;
    for (int c = 0; c < cnt; ++c) {
        typename P::JState js;
        P::load_j(A, base, n, J * 32 + lane, js);
        typename P::Part ip;
        ip.zero();
        const int ii = I * 32 + lane;
        if (I != J) {
#pragma unroll 4
            for (int k = 0; k < 32; ++k) {
                P::template pair<FLAGS>(A, is, js, ip, ii, J * 32 + ((lane + k) & 31));
                P::rotate(js, next);
            }
        } else {
            // diagonal tile: step k pairs lane l with atom (l + k) mod 32; steps
            // 1..15 and half of step 16 visit every unordered pair once
#pragma unroll 4
            for (int k = 1; k <= 16; ++k) {
                P::rotate(js, next);
                if (k < 16 || lane < 16)
                    P::template pair<FLAGS>(A, is, js, ip, ii, J * 32 + ((lane + k) & 31));
            }
            P::home(js, (lane + 16) & 31);
        }
        P::fold_i(is, ip);
        P::flush_j(A, base, n, J * 32 + lane, js);
        if (c + 1 < cnt) {
            if (++J == nb) {
                P::flush_i(A, r, base, n, I * 32 + lane, is);
                if (++I == nb) {
                    do {
                        ++r;
                        base = A.atom_off[r];
                        n = (int)(A.atom_off[r + 1] - base);
                        nb = (n + 31) >> 5;
                    } while (nb == 0);
                    I = 0;
                }
                J = I;
                P::load_i(A, base, n, I * 32 + lane, is);
            }
        }
    }
    P::flush_i(A, r, base, n, I * 32 + lane, is);
}

template <class P, int FLAGS>
static cudaError_t go(const PairArgs& a, const TaskList& t, int wpb, cudaStream_t s) {
    if (t.n_tasks == 0) return cudaSuccess;
    const int blocks = (t.n_tasks + wpb - 1) / wpb;
    k_pairs<P, FLAGS><<<blocks, 32 * wpb, 0, s>>>(a, t.d_tasks, t.n_tasks);
    return cudaGetLastError();
}

cudaError_t launch_pairs(int pass, int flags, const PairArgs& a, const TaskList& t, int wpb,
                         cudaStream_t s) {
    if (pass == PASS_BORN) return go<Born, 0>(a, t, wpb, s);
    if (pass == PASS_CHAIN) return go<Chain, 0>(a, t, wpb, s);
    switch (flags & 7) {
        case 0: return go<EnergyF<0>, 0>(a, t, wpb, s);
        case 1: return go<EnergyF<1>, 1>(a, t, wpb, s);
        case 2: return go<EnergyF<2>, 2>(a, t, wpb, s);
        case 3: return go<EnergyF<3>, 3>(a, t, wpb, s);
        case 4: return go<EnergyF<4>, 4>(a, t, wpb, s);
        case 5: return go<EnergyF<5>, 5>(a, t, wpb, s);
        case 6: return go<EnergyF<6>, 6>(a, t, wpb, s);
        default: return go<EnergyF<7>, 7>(a, t, wpb, s);
    }
}

}  // namespace gbk
