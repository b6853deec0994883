// Per-atom bodies shared by the one-pass-per-launch kernels (atoms.cu) and
// the persistent MD kernel (persist.cu).
#pragma once

#include "common.cuh"
#include "internal.h"

namespace gbk {

__device__ __forceinline__ void set_err(int* err, int code) { atomicCAS(err, 0, code); }

// --- Born radii: I -> psi -> R (OBC) -------------------------------------------
// R = 1 / (1/a - tanh(Phi)/rho), Phi = alpha psi - beta psi^2 + gamma psi^3.
// Written without cancellation: with t = exp(-2|Phi|),
//   1/a - tanh(Phi)/rho = (offset (1 + t) + 2 a t) / (a rho (1 + t))   (Phi >= 0)
// and 1 - tanh^2 = 4 t / (1 + t)^2.  The small difference rho - a enters as
// the offset itself: taken as rho - fl(rho - offset) it would carry the
// rounding of a (up to 6e-8 A, 7e-7 of the 0.09 A offset), and since R ->
// a rho / offset for buried atoms every radius came out low by ~2.4e-7, a
// bias the self energies of a molecule summed (a 2470-atom replica whose GB
// and Coulomb energies cancel 14-fold missed the 1e-6 energy bar).  FP32
// throughout with the accurate expf: the same transform in FP64 met the bar
// by little more and cost 10 % of an 8 x 2048 MD step on this GPU's FP64
// units.  The integral is read in FP64.
// Writes (R, 1/(2R)), the chain prefactor a dR/dpsi, and clears the integral.
__device__ __forceinline__ void born_finalize_atom(const AtomArgs& A, int64_t g, float* R_out) {
    const float I = (float)((double)(long long)__ldcg(&A.I_acc[g]) * FIX_I_INV);
    A.I_acc[g] = 0;
    const float2 rs = A.rad[g];
    const float rho = rs.x;
    const float a = rho - A.offset;
    const float psi = a * I;
    const float Phi = psi * fmaf(psi, fmaf(A.gamma, psi, -A.beta), A.alpha);
    const float t = expf(-2.0f * fabsf(Phi));
    const float onet = 1.0f + t;
    float R;
    if (Phi >= 0.0f) {
        R = (a * rho * onet) / fmaf(A.offset, onet, 2.0f * a * t);
    } else {  // tanh < 0: 1/a + |tanh|/rho, no cancellation either
        R = 1.0f / (1.0f / a + (1.0f - t) / (onet * rho));
    }
    const float sech2 = 4.0f * t / (onet * onet);
    const float dRdpsi = R * R * sech2 * fmaf(psi, fmaf(3.0f * A.gamma, psi, -2.0f * A.beta), A.alpha) / rho;
    if (!(R > 0.0f) || !isfinite(R) || !isfinite(dRdpsi)) set_err(A.err, GB_ERR_NONFINITE);
    A.Rh[g] = make_float2(R, 0.5f / R);
    A.cfac[g] = dRdpsi * a;
    if (R_out) R_out[g] = R;
}

// Screened solvent factors at distance f (FP64): with ek = exp(-kappa f),
//   tE = k_e (1/eps_in - ek/eps_out)              (GB term -1/2 q q tE / f)
//   tF = k_e (1/eps_in - ek (1 + kappa f)/eps_out)  (d/df (tE/f) = -tF / f^2);
// both equal (1/eps_in - 1/eps_out) k_e without salt.
__device__ __forceinline__ double2 gb_screen(double kc, double ke_out, double kappa, double f) {
    if (kappa == 0.0) return make_double2(kc - ke_out, kc - ke_out);
    const double ek = exp(-kappa * f);
    return make_double2(kc - ke_out * ek, kc - ke_out * ek * (1.0 + kappa * f));
}

// Chain factor c = dE/dR * a dR/dpsi of atom g from the pair part of R dE/dR
// (the pair pass sums R_i dE/dR_i; cleared here) plus the self term
// 1/2 tF(R) q^2 / R^2.  Returns q.
__device__ __forceinline__ double chain_factor_atom(const AtomArgs& A, int64_t g, double* R_used) {
    const double q = __ldcg(&A.xyzq[g]).w;
    const double R = __ldcg(&A.Rh[g]).x;
    const double2 t = gb_screen(A.kc, A.ke_out, A.kappa, R);
    const double iR = 1.0 / R;
    const double dEdR = (unfix(__ldcg(&A.dR_acc[g])) + 0.5 * t.y * q * q * iR) * iR;
    A.dR_acc[g] = 0;
    A.cc[g] = (float)(dEdR * (double)__ldcg(&A.cfac[g]));
    *R_used = R;
    return q;
}

// Standard normals from Philox4x64-10 (key (seed, 0), counter (replica, step,
// 4, atom)) by Box-Muller on (u1, u2) and (u3, u4), u1, u3 in (0, 1].
__device__ __forceinline__ float3 md_normals(u64 seed, u64 r, u64 step, u64 atom) {
    const Philox4 w = philox4x64(r, step, 4, atom, seed, 0);
    const float u1 = (float)(((double)(w.w[0] >> 11) + 1.0) * (1.0 / 9007199254740992.0));
    const float u2 = (float)unif53(w.w[1]);
    const float u3 = (float)(((double)(w.w[2] >> 11) + 1.0) * (1.0 / 9007199254740992.0));
    const float u4 = (float)unif53(w.w[3]);
    const float m1 = sqrtf(-2.0f * logf(u1)), m2 = sqrtf(-2.0f * logf(u3));
    float s2, c2, s4, c4;
    sincospif(2.0f * u2, &s2, &c2);
    sincospif(2.0f * u4, &s4, &c4);
    return make_float3(m1 * c2, m1 * s2, m2 * c4);
}

// B (half kick), A (half drift), O (exact Ornstein-Uhlenbeck), A (half drift)
// of one atom with force f; z holds three standard normals.
__device__ __forceinline__ void baoab_first(const MDArgs& m, float4& x, float4& v, float4 f, float3 z) {
    v.x = fmaf(m.h * m.inv_m, f.x, v.x);
    v.y = fmaf(m.h * m.inv_m, f.y, v.y);
    v.z = fmaf(m.h * m.inv_m, f.z, v.z);
    x.x = fmaf(m.h, v.x, x.x); x.y = fmaf(m.h, v.y, x.y); x.z = fmaf(m.h, v.z, x.z);
    v.x = fmaf(m.c1, v.x, m.c2 * z.x);
    v.y = fmaf(m.c1, v.y, m.c2 * z.y);
    v.z = fmaf(m.c1, v.z, m.c2 * z.z);
    x.x = fmaf(m.h, v.x, x.x); x.y = fmaf(m.h, v.y, x.y); x.z = fmaf(m.h, v.z, x.z);
}

// Harmonic chain bonds k (r - r0)^2 with atoms i-1 and i+1 of the replica:
// force on atom i.
__device__ __forceinline__ float3 bond_force_kr(float k, float r0, const float4* xyzq, int64_t base, int i, int n) {
    float3 f = make_float3(0.0f, 0.0f, 0.0f);
    if (k == 0.0f) return f;
    const float4 xi = __ldcg(&xyzq[base + i]);
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const int j = side ? i + 1 : i - 1;
        if (j < 0 || j >= n) continue;
        const float4 xj = __ldcg(&xyzq[base + j]);
        const float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
        const float rr = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        // dE/dr = 2 k (r - r0); the force on i points along +d when stretched
        const float sc = 2.0f * k * (rr - r0) / rr;
        f.x = fmaf(sc, dx, f.x); f.y = fmaf(sc, dy, f.y); f.z = fmaf(sc, dz, f.z);
    }
    return f;
}
__device__ __forceinline__ float3 bond_force(const MDArgs& m, const float4* xyzq, int64_t base, int i, int n) {
    return bond_force_kr(m.bond_k, m.bond_r0, xyzq, base, i, n);
}

}  // namespace gbk
