// O(N^2) pair passes of the GB hot path on sm_103a.
//
// Every replica's atoms are cut into 32-atom tiles.  A warp owns a contiguous
// run of the upper triangle's work, walked as 64-atom super-rows: lane l holds
// the two atoms 64K + l and 64K + 32 + l ("i", one FP32x2 register pair per
// quantity) for the whole row, while the 32 atoms of tile J ("j") rotate one
// lane per step with warp shuffles, carrying their FP32 partial sums.  Each
// step therefore evaluates two pairs per lane with packed FP32x2 arithmetic
// (FFMA2 / FMUL2 / FADD2: one issue slot for two lanes' worth of FP32 work)
// and one set of shuffles, and every unordered pair is evaluated exactly once
// (Newton's third law).  The first two tiles of a super-row touch the
// diagonal and are masked.  After each tile the j partials are folded into
// int64 fixed point with one global atomic per atom and component; the i
// partials go to int64 registers, flushed when the row ends.  FP32 partials
// never span more than one 64 x 32 block and integer sums are associative,
// so results are the same for every run, task split and launch order.
//
// Pass 1 (Born integrals), pass 2 (GB + Coulomb energy, direct forces, dE/dR,
// optional dE/dq and soft repulsion) and pass 3 (Born-radius chain rule)
// share the walker below; the arithmetic of each pass is in its policy.
#pragma once

#include "common.cuh"
#include "internal.h"
#include "poly_coeffs.h"

namespace gbk {

// Disjoint spheres (r >= a + s) with x = s/r <= 0.6: H = 1/2 s^3 r^-4 g(x^2) and
// -(dH/dr)/r = 1/2 s^3 r^-6 h(x^2), with g, h the fitted polynomials: no
// cancellation and no MUFU.  Every lane evaluates the polynomial; the closed
// form runs only when some lane of the warp holds an overlapping pair (a warp
// vote), so the common path carries no divergent branch.
__device__ __forceinline__ bool far_ok(float r, float lim, float y) { return (r >= lim) && (y <= GB_POLY_YMAX); }

// True (warp-uniform) when every pair of this warp step has y <= GB_POLY_YFAR,
// where the lower-degree far-field polynomials reach the same FP32 accuracy.
// The chain's tiles are spatially compact, so most steps qualify.
__device__ __forceinline__ bool all_far(float2 a, float2 b) {
    const float m = fmaxf(fmaxf(a.x, a.y), fmaxf(b.x, b.y));
    return __all_sync(0xffffffffu, m <= GB_POLY_YFAR);
}

// --- packed FP32x2 helpers ----------------------------------------------------------
typedef float2 f2;
__device__ __forceinline__ f2 F2(float v) { return make_float2(v, v); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }

// MUFU reciprocal square root and base-2 exponential; inputs here are never
// denormal, so the flush-to-zero forms need no fix-up instructions.
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_ftz(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ f2 rsqrt2(f2 x) { return make_float2(rsqrt_ftz(x.x), rsqrt_ftz(x.y)); }
__device__ __forceinline__ f2 ex22(f2 x) { return make_float2(ex2_ftz(x.x), ex2_ftz(x.y)); }
// 1/sqrt(x) refined by one Newton step y (3 - x y^2) / 2
__device__ __forceinline__ f2 rsqrt2_nr(f2 x) {
    const f2 y = rsqrt2(x);
    return mul2(y, fma2(F2(-0.5f), mul2(x, mul2(y, y)), F2(1.5f)));
}

constexpr float SQRT_LOG2E = 1.2011224087864498f;  // sqrt(log2(e))
constexpr float LN2 = 0.69314718055994531f;
constexpr float LOG2E = 1.4426950408889634f;
constexpr float FAR_R2 = 1.0e30f;                  // r^2 given to masked-off lanes

__device__ __forceinline__ f2 neg2(f2 v) { return make_float2(-v.x, -v.y); }
// Compensated summation (Kahan): sum + c carries the running total, with c
// the negated rounding error of the additions so far.
__device__ __forceinline__ void kahan_add(f2& sum, f2& c, f2 term) {
    const f2 y = add2(term, neg2(c));
    const f2 t = add2(sum, y);
    c = add2(add2(t, neg2(sum)), neg2(y));
    sum = t;
}
// Reciprocal: MUFU estimate (flush-to-zero; arguments here are O(1) lengths)
// and one Newton step y + y (1 - x y), which brings it to about half an ulp.
__device__ __forceinline__ float rcp_ftz(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ f2 rcp2(f2 x) {
    const f2 y = make_float2(rcp_ftz(x.x), rcp_ftz(x.y));
    return fma2(y, fma2(neg2(x), y, F2(1.0f)), y);
}
__device__ __forceinline__ f2 logv(f2 x) { return make_float2(logf(x.x), logf(x.y)); }

// --- HCT descreening integral H(r; a, s), closed form -----------------------------
// H = (1/4pi) * volume integral of |y - x_i|^-4 over the part of the sphere
// (centre x_j, radius s) that lies outside the sphere (x_i, a).  Closed form
// from spherical shells about x_i between L = max(a, |r - s|) and U = r + s:
//   H = 1/2 [1/L - 1/U + (r - s^2/r)/4 (1/U^2 - 1/L^2) + ln(L/U) / (2r)],
// plus 1/a - 1/L inside the bracket when x_i is engulfed (a < s - r), and 0
// when sphere j lies inside sphere i (a >= r + s).  It serves only pairs whose
// spheres overlap or nearly touch (chain neighbours and contacts), where its
// O(1) terms cancel to about a tenth of their size: the reciprocals and the
// logarithm are kept to FP32 rounding.  Both pairs of a lane (x and y halves)
// are evaluated at once, branch-free.
__device__ __forceinline__ f2 hct_closed2(f2 r, f2 rinv, f2 a, f2 s) {
    const f2 U = add2(r, s);
    const f2 rs = add2(r, neg2(s));
    const f2 L = make_float2(fmaxf(a.x, fabsf(rs.x)), fmaxf(a.y, fabsf(rs.y)));
    const f2 iU = rcp2(U), iL = rcp2(L);
    const f2 dU2 = add2(mul2(iU, iU), neg2(mul2(iL, iL)));        // 1/U^2 - 1/L^2
    const f2 w = fma2(neg2(mul2(s, s)), rinv, r);                 // r - s^2/r
    f2 b = fma2(mul2(F2(0.25f), w), dU2, add2(iL, neg2(iU)));
    b = fma2(mul2(F2(0.5f), rinv), logv(mul2(L, iU)), b);        // ln(L/U) / (2r)
    const f2 eng = mul2(F2(2.0f), add2(rcp2(a), neg2(iL)));       // engulfed: 2 (1/a - 1/L)
    b.x += (a.x < -rs.x) ? eng.x : 0.0f;
    b.y += (a.y < -rs.y) ? eng.y : 0.0f;
    return make_float2(a.x >= U.x ? 0.0f : 0.5f * b.x, a.y >= U.y ? 0.0f : 0.5f * b.y);
}

// -(dH/dr) / r of the closed form, for both pairs of a lane.  With dL = dL/dr
// (0 while L = a, sign(r - s) while L = |r - s|) and w = r - s^2/r:
//   dB/dr = -dL/L^2 + 1/U^2 + (1 + s^2/r^2)/4 (1/U^2 - 1/L^2)
//           + w/2 (dL/L^3 - 1/U^3) - ln(L/U) / (2 r^2) + (dL/L - 1/U) / (2r)
// plus 2 dL/L^2 when engulfed; -(dH/dr)/r = -dB/dr / (2r).
__device__ __forceinline__ f2 hct_closed_fr2(f2 r, f2 rinv, f2 a, f2 s) {
    const f2 U = add2(r, s);
    const f2 rs = add2(r, neg2(s));
    const bool on_x = a.x > fabsf(rs.x), on_y = a.y > fabsf(rs.y);   // L = a
    const f2 L = make_float2(on_x ? a.x : fabsf(rs.x), on_y ? a.y : fabsf(rs.y));
    const f2 dL = make_float2(on_x ? 0.0f : (rs.x > 0.0f ? 1.0f : -1.0f),
                              on_y ? 0.0f : (rs.y > 0.0f ? 1.0f : -1.0f));
    const f2 iU = rcp2(U), iL = rcp2(L);
    const f2 iU2 = mul2(iU, iU), iL2 = mul2(iL, iL);
    const f2 s2r2 = mul2(mul2(s, s), mul2(rinv, rinv));           // s^2 / r^2
    const f2 w = fma2(neg2(s2r2), r, r);                          // r - s^2/r
    const f2 dLiL = mul2(dL, iL);
    f2 db = fma2(neg2(dLiL), iL, iU2);                            // -dL/L^2 + 1/U^2
    db = fma2(mul2(F2(0.25f), add2(F2(1.0f), s2r2)), add2(iU2, neg2(iL2)), db);
    db = fma2(mul2(F2(0.5f), w), add2(mul2(dLiL, iL2), neg2(mul2(iU2, iU))), db);
    const f2 hr = mul2(F2(0.5f), rinv);
    db = fma2(neg2(mul2(hr, rinv)), logv(mul2(L, iU)), db);
    db = fma2(hr, add2(dLiL, neg2(iU)), db);
    db.x += (a.x < -rs.x) ? 2.0f * dLiL.x * iL.x : 0.0f;
    db.y += (a.y < -rs.y) ? 2.0f * dLiL.y * iL.y : 0.0f;
    const f2 fr = mul2(mul2(F2(-0.5f), db), rinv);
    return make_float2(a.x >= U.x ? 0.0f : fr.x, a.y >= U.y ? 0.0f : fr.y);
}

// --- the same integral restricted to the ball |y - x_i| < rc (Born-radius cutoff) ---
// Shells about x_i now run from L to U' = min(U, rc): the bracket of
// hct_closed2 with U' in place of U when L < U' (else no shell term), and the
// engulfed part 2 (1/a - 1/min(L, rc)) when a < s - r and a < rc.  irc = 1/rc.
// Serves the pairs of blocks that straddle the cutoff, where sphere j reaches
// past rc (r + s > rc); it is exact (to rounding) for every geometry, so the
// lanes of such a step that do not reach past rc may take it too.
__device__ __forceinline__ f2 hct_cut2(f2 r, f2 rinv, f2 a, f2 s, float rc, float irc) {
    const f2 U = add2(r, s);
    const f2 Up = make_float2(fminf(U.x, rc), fminf(U.y, rc));
    const f2 rs = add2(r, neg2(s));
    const f2 L = make_float2(fmaxf(a.x, fabsf(rs.x)), fmaxf(a.y, fabsf(rs.y)));
    const f2 iU = rcp2(Up), iL = rcp2(L);
    const f2 dU2 = add2(mul2(iU, iU), neg2(mul2(iL, iL)));
    const f2 w = fma2(neg2(mul2(s, s)), rinv, r);
    f2 b = fma2(mul2(F2(0.25f), w), dU2, add2(iL, neg2(iU)));
    b = fma2(mul2(F2(0.5f), rinv), logv(mul2(L, iU)), b);
    b.x = (L.x < Up.x) ? b.x : 0.0f;
    b.y = (L.y < Up.y) ? b.y : 0.0f;
    const f2 iLc = make_float2(L.x < rc ? iL.x : irc, L.y < rc ? iL.y : irc);
    const f2 eng = mul2(F2(2.0f), add2(rcp2(a), neg2(iLc)));
    b.x += (a.x < -rs.x && a.x < rc) ? eng.x : 0.0f;
    b.y += (a.y < -rs.y && a.y < rc) ? eng.y : 0.0f;
    return mul2(F2(0.5f), b);
}

// -(dH/dr)/r of hct_cut2.  As hct_closed_fr2 with dU = dU'/dr (1 while
// U < rc, 0 once U' = rc) in the terms that came from the upper limit:
//   dB/dr = -dL/L^2 + dU/U'^2 + (1 + s^2/r^2)/4 (1/U'^2 - 1/L^2)
//           + w/2 (dL/L^3 - dU/U'^3) - ln(L/U') / (2 r^2) + (dL/L - dU/U') / (2r)
// (0 when L >= U'), plus 2 dL/L^2 when engulfed with L < rc.
// (out of line: the chain pass's straddle code would not fit the instruction
// cache with it inlined into every block mode)
static __device__ __noinline__ f2 hct_cut_fr2(f2 r, f2 rinv, f2 a, f2 s, float rc) {
    const f2 U = add2(r, s);
    const bool cx = U.x > rc, cy = U.y > rc;
    const f2 Up = make_float2(cx ? rc : U.x, cy ? rc : U.y);
    const f2 rs = add2(r, neg2(s));
    const bool on_x = a.x > fabsf(rs.x), on_y = a.y > fabsf(rs.y);
    const f2 L = make_float2(on_x ? a.x : fabsf(rs.x), on_y ? a.y : fabsf(rs.y));
    const f2 dL = make_float2(on_x ? 0.0f : (rs.x > 0.0f ? 1.0f : -1.0f),
                              on_y ? 0.0f : (rs.y > 0.0f ? 1.0f : -1.0f));
    const f2 iU = rcp2(Up), iL = rcp2(L);
    const f2 iUd = make_float2(cx ? 0.0f : iU.x, cy ? 0.0f : iU.y);   // dU / U'
    const f2 iU2 = mul2(iU, iU), iL2 = mul2(iL, iL);
    const f2 s2r2 = mul2(mul2(s, s), mul2(rinv, rinv));
    const f2 w = fma2(neg2(s2r2), r, r);
    const f2 dLiL = mul2(dL, iL);
    f2 db = fma2(neg2(dLiL), iL, mul2(iUd, iU));
    db = fma2(mul2(F2(0.25f), add2(F2(1.0f), s2r2)), add2(iU2, neg2(iL2)), db);
    db = fma2(mul2(F2(0.5f), w), add2(mul2(dLiL, iL2), neg2(mul2(iUd, iU2))), db);
    const f2 hr = mul2(F2(0.5f), rinv);
    db = fma2(neg2(mul2(hr, rinv)), logv(mul2(L, iU)), db);
    db = fma2(hr, add2(dLiL, neg2(iUd)), db);
    db.x = (L.x < Up.x) ? db.x : 0.0f;
    db.y = (L.y < Up.y) ? db.y : 0.0f;
    db.x += (a.x < -rs.x && a.x < rc && L.x < rc) ? 2.0f * dLiL.x * iL.x : 0.0f;
    db.y += (a.y < -rs.y && a.y < rc && L.y < rc) ? 2.0f * dLiL.y * iL.y : 0.0f;
    return mul2(mul2(F2(-0.5f), db), rinv);
}

// Disjoint spheres (r >= a + s) reaching past rc: the shells run from
// L = r - s to U' = min(r + s, rc), and with w = U' - L, z = w / U' the
// integral takes a form without cancelling O(1/L) terms,
//   H = 1/(4r) [ (s/L) z^2 - J(z) ],   J(z) = -ln(1 - z) - z - z^2/2 = z^3 q(z)
// (J = int_0^z t^2/(1-t) dt; q the fitted series of positive terms of
// poly_coeffs.h: gb_poly_q for z <= 1/2, gb_poly_q_hi for z <= 3/4, which
// covers every pair of disjoint spheres of the usual radius sets, and beyond
// that J from the logarithm, where its terms cancel by less than a factor 10;
// each range behind a warp vote over the lanes that use this form).  w is formed as
// min((rc - r) + s, 2s): rc - r is exact for the pairs near the cutoff, so w
// carries one rounding.  Lanes with w <= 0 (sphere j wholly past rc, masked
// lanes) give 0.
struct CutFar {
    f2 z, w, iL, iU, B;
    bool cx, cy;                      // U' = rc (the cutoff limits the shells)
};
__device__ __forceinline__ CutFar hct_cut_far_terms(f2 r, f2 s, float rc, bool use0 = true, bool use1 = true) {
    CutFar c;
    const f2 L = add2(r, neg2(s));
    c.iL = rcp2(L);
    const f2 wc = add2(add2(F2(rc), neg2(r)), s);
    const f2 s2 = add2(s, s);
    c.cx = wc.x < s2.x;
    c.cy = wc.y < s2.y;
    c.w = make_float2(fmaxf(0.0f, c.cx ? wc.x : s2.x), fmaxf(0.0f, c.cy ? wc.y : s2.y));
    const f2 U = add2(L, c.w);
    c.iU = rcp2(U);
    c.z = mul2(c.w, c.iU);
    const f2 z2 = mul2(c.z, c.z), z3 = mul2(z2, c.z);
    f2 J = mul2(z3, gb_poly_q2(c.z));
    if (__any_sync(0xffffffffu, (use0 && c.z.x > GB_POLY_ZJ) || (use1 && c.z.y > GB_POLY_ZJ))) {
        const f2 Jh = mul2(z3, gb_poly_q_hi2(add2(c.z, F2(-GB_POLY_ZMID))));
        J = make_float2(c.z.x > GB_POLY_ZJ ? Jh.x : J.x, c.z.y > GB_POLY_ZJ ? Jh.y : J.y);
        if (__any_sync(0xffffffffu, (use0 && c.z.x > GB_POLY_ZJ2) || (use1 && c.z.y > GB_POLY_ZJ2))) {
            const f2 Jl = add2(logv(mul2(U, c.iL)), neg2(fma2(F2(0.5f), z2, c.z)));   // ln(U'/L) - z - z^2/2
            J = make_float2(c.z.x > GB_POLY_ZJ2 ? Jl.x : J.x, c.z.y > GB_POLY_ZJ2 ? Jl.y : J.y);
        }
    }
    c.B = fma2(mul2(s, c.iL), z2, neg2(J));
    return c;
}
__device__ __forceinline__ f2 hct_cut_far2(f2 r, f2 rinv, f2 s, float rc, bool use0, bool use1) {
    return mul2(mul2(F2(0.25f), rinv), hct_cut_far_terms(r, s, rc, use0, use1).B);
}
// -(dH/dr)/r of hct_cut_far2: with z' = -1/U' while the cutoff limits the
// shells and -z/U' otherwise (dJ/dz = z^2/(1-z), z/(1-z) = w/L),
//   dB/dr = -(s/L^2) z^2 + z' z (2s - w) / L,   dH/dr = (dB/dr - B/r) / (4r),
// where no two terms cancel.
__device__ __forceinline__ f2 hct_cut_far_fr2(f2 r, f2 rinv, f2 s, float rc, bool use0, bool use1) {
    const CutFar c = hct_cut_far_terms(r, s, rc, use0, use1);
    const f2 zp = neg2(make_float2(c.cx ? c.iU.x : c.z.x * c.iU.x, c.cy ? c.iU.y : c.z.y * c.iU.y));
    const f2 t = mul2(mul2(zp, c.z), mul2(fma2(F2(2.0f), s, neg2(c.w)), c.iL));
    const f2 dB = fma2(neg2(mul2(s, mul2(c.iL, c.iL))), mul2(c.z, c.z), t);
    const f2 dH = mul2(mul2(F2(0.25f), rinv), fma2(neg2(c.B), rinv, dB));
    return mul2(neg2(dH), rinv);
}
// One direction (descreened atom radius a, descreening sphere s) of every
// lane of a step in which some sphere crosses rc: disjoint spheres take the
// restricted form above (the whole sphere while it lies inside the ball, 0
// once it lies wholly past rc), overlapping ones the general restricted
// closed form behind a vote.
__device__ __forceinline__ f2 hct_cut_dir2(f2 r, f2 rinv, f2 a, f2 s, float rc) {
    const bool d0 = r.x >= a.x + s.x, d1 = r.y >= a.y + s.y;
    f2 h = hct_cut_far2(r, rinv, s, rc, d0, d1);
    if (__any_sync(0xffffffffu, !(d0 && d1))) {
        const f2 g = hct_cut2(r, rinv, a, s, rc, 1.0f / rc);
        h = make_float2(d0 ? h.x : g.x, d1 ? h.y : g.y);
    }
    return h;
}
__device__ __forceinline__ f2 hct_cut_dir_fr2(f2 r, f2 rinv, f2 a, f2 s, float rc) {
    const bool d0 = r.x >= a.x + s.x, d1 = r.y >= a.y + s.y;
    f2 h = hct_cut_far_fr2(r, rinv, s, rc, d0, d1);
    if (__any_sync(0xffffffffu, !(d0 && d1))) {
        const f2 g = hct_cut_fr2(r, rinv, a, s, rc);
        h = make_float2(d0 ? h.x : g.x, d1 ? h.y : g.y);
    }
    return h;
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// --- diagonal masks -------------------------------------------------------------------
// Step k pairs lane l's i atoms with tile atom (l + k) mod 32.  A tile that
// holds the same atoms as an i half ("diagonal") keeps steps 1..15 and the
// lower half of step 16, which visit each unordered pair once.  Mode DX: the
// tile is the x half's own tile and the y half is below the diagonal (off);
// mode DY: the tile is the y half's own tile (x half fully on).
enum { M_FULL = 0, M_DX = 1, M_DY = 2 };
// Per-block bounds (see block_info): far block; r^2 >= t_near proves the
// far-field form valid for both directions of a pair.
struct BlockInfo {
    bool far;
    bool straddle;    // EF_CUT kernels: some pairs of the block on each side of the cutoff
    float t_near;
    float skip2;      // EF_STRADDLE blocks: a step whose pairs all have r^2 > skip2 adds nothing
};
struct Mask {
    bool x, y;
};
template <int MODE>
__device__ __forceinline__ Mask step_mask(int k, int lane) {
    const bool diag = (k >= 1 && k <= 15) || (k == 16 && lane < 16);
    Mask m;
    m.x = (MODE == M_DX) ? diag : true;
    m.y = (MODE == M_FULL) ? true : (MODE == M_DY ? diag : false);
    return m;
}
template <int MODE>
__device__ __forceinline__ f2 keep(f2 v, Mask m) {
    if (MODE == M_FULL) return v;
    return make_float2(m.x ? v.x : 0.0f, m.y ? v.y : 0.0f);
}
template <int MODE>
__device__ __forceinline__ f2 safe_r2(f2 r2, Mask m) {
    if (MODE == M_FULL) return r2;
    return make_float2(m.x ? r2.x : FAR_R2, m.y ? r2.y : FAR_R2);
}

__device__ __forceinline__ f2 sel2(f2 v, Mask m) { return make_float2(m.x ? v.x : 0.0f, m.y ? v.y : 0.0f); }

// Lanes past a replica's end hold ghost atoms (see ghost_x): zero charge,
// zero descreening radius, zero chain factor, parked far away.
__device__ __forceinline__ void load_xas(const PairArgs& A, int64_t base, int n, int i, float& x,
                                         float& y, float& z, float& a, float& s) {
    if (i < n) {
        const float4 p = __ldcg(&A.xyzq[base + i]);
        const float2 rs = A.rad[base + i];
        x = p.x; y = p.y; z = p.z;
        a = rs.x - A.offset;
        s = rs.y * a;
    } else {
        x = ghost_x(i - n); y = 0.0f; z = 0.0f; a = 1.0f; s = 0.0f;
    }
}

// --- pass 1: Born integrals I_i = sum_j H(r_ij; a_i, s_j) -----------------------
struct Born {
    static constexpr int NQ = 1;      // int64 i-side accumulators per atom (shared memory)
    static constexpr int UNROLL = 2;  // rotation steps unrolled (measured best per pass) ...
    static constexpr int UNROLL_FAR = 4;   // ... and in far blocks
    static constexpr bool RADIUS_CUT = true;   // EF_CUT: the cutoff is rgbmax
    struct IState {
        f2 nx, ny, nz, a, s, s2, hs3;   // nx = -x
    };
    // s2 = s^2 and hs3 = s^3 / 2 travel with the j atom through far blocks
    // (one shuffle more, three multiplies fewer per step)
    struct JState { float x, y, z, a, s, acc, s2, hs3; };
    struct Part {
        f2 I;
        __device__ __forceinline__ void zero() { I = F2(0.0f); }
    };
    static __device__ __forceinline__ void load_i(const PairArgs& A, int64_t base, int n, int i0, int lane, IState& st) {
        float x0, y0, z0, a0, s0, x1, y1, z1, a1, s1;
        load_xas(A, base, n, i0 + lane, x0, y0, z0, a0, s0);
        load_xas(A, base, n, i0 + 32 + lane, x1, y1, z1, a1, s1);
        st.nx = make_float2(-x0, -x1); st.ny = make_float2(-y0, -y1); st.nz = make_float2(-z0, -z1);
        st.a = make_float2(a0, a1); st.s = make_float2(s0, s1);
        st.s2 = mul2(st.s, st.s);
        st.hs3 = mul2(mul2(F2(0.5f), st.s2), st.s);
    }
    static __device__ __forceinline__ void load_j(const PairArgs& A, int64_t base, int n, int j, JState& st) {
        load_xas(A, base, n, j, st.x, st.y, st.z, st.a, st.s);
        st.acc = 0.0f;
        st.s2 = st.s * st.s;
        st.hs3 = 0.5f * st.s2 * st.s;
    }
    template <int FLAGS, int MODE, bool FAR>
    static __device__ __forceinline__ void pair(const PairArgs& A, const IState& i, JState& j, Part& p, Mask m,
                                                const BlockInfo& bi, int, int, int) {
        const f2 dx = add2(F2(j.x), i.nx), dy = add2(F2(j.y), i.ny), dz = add2(F2(j.z), i.nz);
        const f2 r2 = safe_r2<MODE>(fma2(dx, dx, fma2(dy, dy, mul2(dz, dz))), m);
        // near blocks hold the few large terms that dominate an atom's
        // integral (and the closed form, which cancels its terms about
        // tenfold): there 1/r gets a Newton step, since the MUFU estimate's
        // error enters r^-4 four times; far blocks sum many small terms
        const f2 rinv = FAR ? rsqrt2(r2) : rsqrt2_nr(r2);
        const f2 rinv2 = mul2(rinv, rinv), rinv4 = mul2(rinv2, rinv2);
        const float sj2 = FAR ? j.s2 : j.s * j.s;
        const float hs3j = FAR ? j.hs3 : 0.5f * sj2 * j.s;
        const f2 y_ij = mul2(F2(sj2), rinv2), y_ji = mul2(i.s2, rinv2);
        // EF_STRADDLE: lanes whose sphere lies wholly past rgbmax give 0; a step
        // with some sphere across it takes the restricted form for every lane
        bool out_ij0 = false, out_ij1 = false, out_ji0 = false, out_ji1 = false;
        if (FLAGS & EF_STRADDLE) {
            const f2 r = mul2(r2, rinv);
            const float rc = A.rgbmax;
            out_ij0 = r.x - j.s >= rc; out_ij1 = r.y - j.s >= rc;
            out_ji0 = r.x - i.s.x >= rc; out_ji1 = r.y - i.s.y >= rc;
            const bool sh = (!out_ij0 && r.x + j.s > rc) || (!out_ij1 && r.y + j.s > rc) ||
                            (!out_ji0 && r.x + i.s.x > rc) || (!out_ji1 && r.y + i.s.y > rc);
            if (__any_sync(0xffffffffu, sh)) {
                const f2 h_ij = keep<MODE>(hct_cut_dir2(r, rinv, i.a, F2(j.s), rc), m);
                const f2 h_ji = keep<MODE>(hct_cut_dir2(r, rinv, F2(j.a), i.s, rc), m);
                p.I = add2(p.I, h_ij);
                j.acc += h_ji.x + h_ji.y;
                return;
            }
        }
        if (FAR) {  // whole block proven disjoint and far: no votes, short polynomial
            p.I = fma2(F2(hs3j), mul2(rinv4, gb_poly_gf2(y_ij)), p.I);
            const f2 h = mul2(i.hs3, mul2(rinv4, gb_poly_gf2(y_ji)));
            j.acc += h.x + h.y;
            return;
        }
        // the block bound t_near decides most steps with one compare per lane;
        // the exact per-direction tests run only on steps where some pair is
        // closer
        const float r2min = fminf(r2.x, r2.y);
        f2 g_ij, g_ji;
        if (all_far(y_ij, y_ji)) {
            g_ij = gb_poly_gf2(y_ij);
            g_ji = gb_poly_gf2(y_ji);
        } else {
            g_ij = gb_poly_g2(y_ij);
            g_ji = gb_poly_g2(y_ji);
        }
        f2 h_ij = mul2(F2(hs3j), mul2(rinv4, g_ij));
        f2 h_ji = mul2(i.hs3, mul2(rinv4, g_ji));
        if (__any_sync(0xffffffffu, r2min < bi.t_near)) {
            const f2 r = mul2(r2, rinv);
            const f2 lim_ij = add2(i.a, F2(j.s)), lim_ji = add2(F2(j.a), i.s);
            const bool b0 = !far_ok(r.x, lim_ij.x, y_ij.x), b1 = !far_ok(r.y, lim_ij.y, y_ij.y);
            const bool c0 = !far_ok(r.x, lim_ji.x, y_ji.x), c1 = !far_ok(r.y, lim_ji.y, y_ji.y);
            if (__any_sync(0xffffffffu, b0 || b1)) {
                const f2 hc = hct_closed2(r, rinv, i.a, F2(j.s));
                h_ij = make_float2(b0 ? hc.x : h_ij.x, b1 ? hc.y : h_ij.y);
            }
            if (__any_sync(0xffffffffu, c0 || c1)) {
                const f2 hc = hct_closed2(r, rinv, F2(j.a), i.s);
                h_ji = make_float2(c0 ? hc.x : h_ji.x, c1 ? hc.y : h_ji.y);
            }
        }
        if (FLAGS & EF_STRADDLE) {   // no sphere across rgbmax: wholly inside or past it
            h_ij = make_float2(out_ij0 ? 0.0f : h_ij.x, out_ij1 ? 0.0f : h_ij.y);
            h_ji = make_float2(out_ji0 ? 0.0f : h_ji.x, out_ji1 ? 0.0f : h_ji.y);
        }
        h_ij = keep<MODE>(h_ij, m);
        h_ji = keep<MODE>(h_ji, m);
        p.I = add2(p.I, h_ij);
        j.acc += h_ji.x + h_ji.y;
    }
    static __device__ __forceinline__ void rotate_data(JState& j, int src) {
        j.x = shfl(j.x, src); j.y = shfl(j.y, src); j.z = shfl(j.z, src);
        j.a = shfl(j.a, src); j.s = shfl(j.s, src);
    }
    // far blocks never read a: it is left behind (the block reloads it)
    static __device__ __forceinline__ void rotate_far(JState& j, int src) {
        j.x = shfl(j.x, src); j.y = shfl(j.y, src); j.z = shfl(j.z, src);
        j.s2 = shfl(j.s2, src); j.hs3 = shfl(j.hs3, src);
    }
    static __device__ __forceinline__ void rotate_acc(JState& j, int src) { j.acc = shfl(j.acc, src); }
    static __device__ __forceinline__ void take_data(JState& j, const JState& d) {
        j.x = d.x; j.y = d.y; j.z = d.z; j.a = d.a; j.s = d.s; j.s2 = d.s2; j.hs3 = d.hs3;
    }
    static __device__ __forceinline__ void fold_i(IState&, long long* sa, int lane, const Part& p) {
        sa[lane] += fix_i(p.I.x);
        sa[32 + lane] += fix_i(p.I.y);
    }
    // Two atoms at the same position (r = 0; masked pairs read as far first):
    // r = r^2 / r is NaN, the closed form carries it through U = r + s and
    // the restricted form of the cutoff through w = r - s^2/r, so both atoms'
    // sums turn NaN.  One test per block and lane, on the j side, records it
    // before the fixed-point conversion would hide it.
    static __device__ __forceinline__ void flush_j(const PairArgs& A, int64_t base, int n, int j, const JState& st) {
        if (!isfinite(st.acc) && A.err) atomicCAS(A.err, 0, GB_ERR_NONFINITE);
        if (j < n) red_add(&A.I_acc[base + j], fix_i(st.acc));
    }
    static __device__ __forceinline__ void flush_i(const PairArgs& A, int, int64_t base, int n, int i0, int lane,
                                                   const IState&, long long* sa) {
        if (i0 + lane < n) red_add(&A.I_acc[base + i0 + lane], sa[lane]);
        if (i0 + 32 + lane < n) red_add(&A.I_acc[base + i0 + 32 + lane], sa[32 + lane]);
    }
};

// --- pass 2: GB + Coulomb pair energy, direct forces, dE/dR, dE/dq --------------
// Pair (i, j), both orderings of the double sum together:
//   e_GB = -tau k_e q_i q_j / f,  f^2 = r^2 + R_i R_j exp(-D),  D = r^2 / (4 R_i R_j)
//   e_C  =  k_c q_i q_j / r
//   -(de/dr)/r = k_c q_i q_j / r^3 - tau k_e q_i q_j (1 - exp(-D)/4) / f^3
//   R_i de/dR_i = tau k_e q_i q_j exp(-D)(R_i R_j + r^2/4) / (2 f^3)   (and i <-> j:
//                 (1 + D) R_i R_j = R_i R_j + r^2/4, the same value on both sides)
//   de/dq_i = (-tau k_e / f + k_c / r) q_j                  (and i <-> j)
// Each atom carries h = sqrt(log2 e) / (2R) (negated for i), so that
// exp(-D) = 2^(r^2 (-h_i) h_j) is two multiplies and one ex2.
struct Energy {
    static constexpr int NQ = 5;      // fx, fy, fz, R dE/dR, dE/dq (shared memory)
    static constexpr int UNROLL = 2;
    static constexpr int UNROLL_FAR = 2;
    static constexpr bool RADIUS_CUT = false;  // EF_CUT: the cutoff is `cut`
    struct IState {
        f2 nx, ny, nz, q, R, nh;
        f2 qa, qk;                    // q tau k_e / 2 and q k_c (unscreened pair factors)
        long long egb, ec, er;
    };
    struct JState { float x, y, z, q, R, h, fx, fy, fz, dR, phi; };
    struct Part {
        f2 sx, sy, sz, dR, phi, egb, ec, er;   // s* = sum of fr d (the i force is -s)
        f2 kgb, kc, kr;                        // compensation terms of the energy sums
        __device__ __forceinline__ void zero() {
            sx = sy = sz = dR = phi = egb = ec = er = kgb = kc = kr = F2(0.0f);
        }
    };
    static __device__ __forceinline__ void load_one(const PairArgs& A, int64_t base, int n, int i, float& x,
                                                    float& y, float& z, float& q, float& R, float& h) {
        if (i < n) {
            const float4 p = __ldcg(&A.xyzq[base + i]);
            const float2 rh = __ldcg(&A.Rh[base + i]);
            x = p.x; y = p.y; z = p.z; q = p.w; R = rh.x; h = rh.y * SQRT_LOG2E;
        } else {
            x = ghost_x(i - n); y = 0.0f; z = 0.0f; q = 0.0f; R = 1.0f; h = 0.5f * SQRT_LOG2E;
        }
    }
    static __device__ __forceinline__ void load_i(const PairArgs& A, int64_t base, int n, int i0, int lane, IState& st) {
        float x0, y0, z0, q0, R0, h0, x1, y1, z1, q1, R1, h1;
        load_one(A, base, n, i0 + lane, x0, y0, z0, q0, R0, h0);
        load_one(A, base, n, i0 + 32 + lane, x1, y1, z1, q1, R1, h1);
        st.nx = make_float2(-x0, -x1); st.ny = make_float2(-y0, -y1); st.nz = make_float2(-z0, -z1);
        st.q = make_float2(q0, q1); st.R = make_float2(R0, R1); st.nh = make_float2(-h0, -h1);
        st.qa = mul2(st.q, F2(0.5f * A.tau_ke));
        st.qk = mul2(st.q, F2(A.kc));
        st.egb = st.ec = st.er = 0;
    }
    static __device__ __forceinline__ void load_j(const PairArgs& A, int64_t base, int n, int j, JState& st) {
        load_one(A, base, n, j, st.x, st.y, st.z, st.q, st.R, st.h);
        st.fx = st.fy = st.fz = st.dR = st.phi = 0.0f;
    }
    template <int FLAGS, int MODE, bool FAR>
    static __device__ __forceinline__ void pair(const PairArgs& A, const IState& i, JState& j, Part& p, Mask m,
                                                const BlockInfo&, int i0, int jbase, int k) {
        const f2 dx = add2(F2(j.x), i.nx), dy = add2(F2(j.y), i.ny), dz = add2(F2(j.z), i.nz);
        const f2 r2 = safe_r2<MODE>(fma2(dx, dx, fma2(dy, dy, mul2(dz, dz))), m);
        // energies are sums of large terms that cancel: when they are wanted,
        // one Newton step takes the MUFU reciprocal square roots to FP32 rounding
        const f2 rinv = (FLAGS & EF_ENERGY) ? rsqrt2_nr(r2) : rsqrt2(r2);
        const f2 rinv2 = mul2(rinv, rinv);
        const f2 qq = mul2(i.q, F2(j.q));
        const f2 nDl = mul2(r2, mul2(i.nh, F2(j.h)));                 // -D log2(e)
        const f2 e = ex22(nDl);                                       // exp(-D)
        const f2 RR = mul2(i.R, F2(j.R));
        const f2 fsq = fma2(RR, e, r2);
        const f2 finv = (FLAGS & EF_ENERGY) ? rsqrt2_nr(fsq) : rsqrt2(fsq);
        const f2 finv3 = mul2(mul2(finv, finv), finv);
        // solvent factors: tE in the energy (-tE q q / f), tF in its f-derivative;
        // both (1/eps_in - 1/eps_out) k_e without salt, screened by
        // exp(-kappa f) with it (Debye-Hueckel)
        f2 tE = F2(A.tau_ke), w;
        if (FLAGS & EF_SALT) {
            const f2 f = mul2(fsq, finv);
            const f2 ekv = mul2(F2(A.ke_out), ex22(mul2(F2(-A.kappa * LOG2E), f)));   // k_e e^{-kappa f} / eps_out
            tE = add2(F2(A.kc), neg2(ekv));
            const f2 tF = fma2(neg2(ekv), mul2(F2(A.kappa), f), tE);
            w = mul2(mul2(qq, F2(0.5f)), mul2(tF, finv3));           // tF q q / (2 f^3)
        } else {
            w = mul2(mul2(i.qa, F2(j.q)), finv3);
        }
        const f2 nu = fma2(F2(0.5f), e, F2(-2.0f));                   // -2 (1 - e/4)
        const f2 qc = mul2(i.qk, F2(j.q));
        f2 fr = fma2(qc, mul2(rinv2, rinv), mul2(w, nu));
        f2 G = mul2(mul2(w, e), fma2(r2, F2(0.25f), RR));              // w e (1 + D) R_i R_j
        Mask cm{true, true};          // pair within the cutoff (EF_STRADDLE blocks test it)
        if (FLAGS & EF_STRADDLE) {
            cm.x = r2.x <= A.cut2;
            cm.y = r2.y <= A.cut2;
            fr = sel2(fr, cm);
            G = sel2(G, cm);
        }
        f2 er = F2(0.0f);
        if ((FLAGS & EF_REP) && !FAR) {
            const float sig2 = A.rep_sigma * A.rep_sigma;
            const bool n0 = r2.x < sig2, n1 = r2.y < sig2;
            if (__any_sync(0xffffffffu, n0 || n1)) {
                const int jj = jbase + ((threadIdx.x + k) & 31);
                const int ia = i0 + (threadIdx.x & 31), ib = ia + 32;
                if (n0 && (ia - jj > 1 || jj - ia > 1)) {
                    const float dd = A.rep_sigma - r2.x * rinv.x;
                    fr.x = fmaf(2.0f * A.rep_k * dd, rinv.x, fr.x);
                    er.x = A.rep_k * dd * dd;
                }
                if (n1 && (ib - jj > 1 || jj - ib > 1)) {
                    const float dd = A.rep_sigma - r2.y * rinv.y;
                    fr.y = fmaf(2.0f * A.rep_k * dd, rinv.y, fr.y);
                    er.y = A.rep_k * dd * dd;
                }
            }
        }
        fr = keep<MODE>(fr, m);
        G = keep<MODE>(G, m);
        p.sx = fma2(fr, dx, p.sx); p.sy = fma2(fr, dy, p.sy); p.sz = fma2(fr, dz, p.sz);
        j.fx = fmaf(fr.y, dx.y, fmaf(fr.x, dx.x, j.fx));
        j.fy = fmaf(fr.y, dy.y, fmaf(fr.x, dy.x, j.fy));
        j.fz = fmaf(fr.y, dz.y, fmaf(fr.x, dz.x, j.fz));
        p.dR = add2(p.dR, G);
        j.dR += G.x + G.y;
        if (FLAGS & EF_PHI) {
            f2 P = keep<MODE>(fma2(neg2(tE), finv, mul2(F2(A.kc), rinv)), m);
            if (FLAGS & EF_STRADDLE) P = sel2(P, cm);
            p.phi = fma2(P, F2(j.q), p.phi);
            j.phi = fmaf(P.y, i.q.y, fmaf(P.x, i.q.x, j.phi));
        }
        if (FLAGS & EF_ENERGY) {
            // the pair energies are large terms that cancel: compensated
            // (Kahan) FP32 sums within the block
            f2 eg = keep<MODE>(mul2(neg2(tE), mul2(qq, finv)), m), ecl = keep<MODE>(mul2(qc, rinv), m);
            if (FLAGS & EF_STRADDLE) {
                eg = sel2(eg, cm);
                ecl = sel2(ecl, cm);
            }
            kahan_add(p.egb, p.kgb, eg);
            kahan_add(p.ec, p.kc, ecl);
            if (FLAGS & EF_REP) kahan_add(p.er, p.kr, keep<MODE>(er, m));
        }
    }
    static __device__ __forceinline__ void rotate_data(JState& j, int src) {
        j.x = shfl(j.x, src); j.y = shfl(j.y, src); j.z = shfl(j.z, src);
        j.q = shfl(j.q, src); j.R = shfl(j.R, src); j.h = shfl(j.h, src);
    }
    static __device__ __forceinline__ void rotate_far(JState& j, int src) { rotate_data(j, src); }
    template <int FLAGS>
    static __device__ __forceinline__ void rotate_acc_f(JState& j, int src) {
        j.fx = shfl(j.fx, src); j.fy = shfl(j.fy, src); j.fz = shfl(j.fz, src);
        j.dR = shfl(j.dR, src);
        if (FLAGS & EF_PHI) j.phi = shfl(j.phi, src);
    }
    static __device__ __forceinline__ void take_data(JState& j, const JState& d) {
        j.x = d.x; j.y = d.y; j.z = d.z; j.q = d.q; j.R = d.R; j.h = d.h;
    }
    template <int FLAGS>
    static __device__ __forceinline__ void fold_i_f(IState& i, long long* sa, int lane, const Part& p) {
        sa[lane] -= fix(p.sx.x); sa[32 + lane] -= fix(p.sx.y);
        sa[64 + lane] -= fix(p.sy.x); sa[96 + lane] -= fix(p.sy.y);
        sa[128 + lane] -= fix(p.sz.x); sa[160 + lane] -= fix(p.sz.y);
        sa[192 + lane] += fix(p.dR.x); sa[224 + lane] += fix(p.dR.y);
        if (FLAGS & EF_PHI) {
            sa[256 + lane] += fix(p.phi.x);
            sa[288 + lane] += fix(p.phi.y);
        }
        if (FLAGS & EF_ENERGY) {
            i.egb += (fix(p.egb.x) + fix(p.egb.y)) - (fix(p.kgb.x) + fix(p.kgb.y));
            i.ec += (fix(p.ec.x) + fix(p.ec.y)) - (fix(p.kc.x) + fix(p.kc.y));
            if (FLAGS & EF_REP) i.er += (fix(p.er.x) + fix(p.er.y)) - (fix(p.kr.x) + fix(p.kr.y));
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
    static __device__ __forceinline__ void flush_i_f(const PairArgs& A, int r, int64_t base, int n, int i0, int lane,
                                                     const IState& st, long long* sa) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = i0 + 32 * h + lane;
            if (i < n) {
                const int64_t g = base + i;
                const int o = 32 * h + lane;
                red_add(&A.F_acc[g], sa[o]);
                red_add(&A.F_acc[A.N + g], sa[64 + o]);
                red_add(&A.F_acc[2 * A.N + g], sa[128 + o]);
                red_add(&A.dR_acc[g], sa[192 + o]);
                if (FLAGS & EF_PHI) red_add(&A.phi_acc[g], sa[256 + o]);
            }
        }
        if (FLAGS & EF_ENERGY) {
            const long long egb = warp_sum_ll(st.egb), ec = warp_sum_ll(st.ec);
            const long long er = (FLAGS & EF_REP) ? warp_sum_ll(st.er) : 0;
            if (lane == 0) {
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
    static constexpr int NQ = 3;      // fx, fy, fz (shared memory)
    static constexpr int UNROLL = 2;
    static constexpr int UNROLL_FAR = 4;
    static constexpr bool RADIUS_CUT = true;   // EF_CUT: the cutoff is rgbmax
    struct IState {
        f2 nx, ny, nz, a, s, s2, hs3, c;
    };
    // s2 = s^2 and hs3 = s^3 / 2 travel with the j atom through far blocks
    struct JState { float x, y, z, a, s, c, fx, fy, fz, s2, hs3; };
    struct Part {
        f2 sx, sy, sz;
        __device__ __forceinline__ void zero() { sx = sy = sz = F2(0.0f); }
    };
    static __device__ __forceinline__ void load_one(const PairArgs& A, int64_t base, int n, int i, float& x,
                                                    float& y, float& z, float& a, float& s, float& c) {
        load_xas(A, base, n, i, x, y, z, a, s);
        c = (i < n) ? __ldcg(&A.cc[base + i]) : 0.0f;
    }
    static __device__ __forceinline__ void load_i(const PairArgs& A, int64_t base, int n, int i0, int lane, IState& st) {
        float x0, y0, z0, a0, s0, c0, x1, y1, z1, a1, s1, c1;
        load_one(A, base, n, i0 + lane, x0, y0, z0, a0, s0, c0);
        load_one(A, base, n, i0 + 32 + lane, x1, y1, z1, a1, s1, c1);
        st.nx = make_float2(-x0, -x1); st.ny = make_float2(-y0, -y1); st.nz = make_float2(-z0, -z1);
        st.a = make_float2(a0, a1); st.s = make_float2(s0, s1); st.c = make_float2(c0, c1);
        st.s2 = mul2(st.s, st.s);
        st.hs3 = mul2(mul2(F2(0.5f), st.s2), st.s);
    }
    static __device__ __forceinline__ void load_j(const PairArgs& A, int64_t base, int n, int j, JState& st) {
        load_one(A, base, n, j, st.x, st.y, st.z, st.a, st.s, st.c);
        st.fx = st.fy = st.fz = 0.0f;
        st.s2 = st.s * st.s;
        st.hs3 = 0.5f * st.s2 * st.s;
    }
    template <int FLAGS, int MODE, bool FAR>
    static __device__ __forceinline__ void pair(const PairArgs& A, const IState& i, JState& j, Part& p, Mask m,
                                                const BlockInfo& bi, int, int, int) {
        const f2 dx = add2(F2(j.x), i.nx), dy = add2(F2(j.y), i.ny), dz = add2(F2(j.z), i.nz);
        const f2 r2 = safe_r2<MODE>(fma2(dx, dx, fma2(dy, dy, mul2(dz, dz))), m);
        const f2 rinv = rsqrt2(r2);
        const f2 rinv2 = mul2(rinv, rinv);
        const float sj2 = FAR ? j.s2 : j.s * j.s;
        const float hs3j = FAR ? j.hs3 : 0.5f * sj2 * j.s;
        const f2 y_ij = mul2(F2(sj2), rinv2), y_ji = mul2(i.s2, rinv2);
        // EF_STRADDLE: as in Born; a lane with one direction wholly past rgbmax
        // has the other across it or past it too
        bool out0 = false, out1 = false;
        if (FLAGS & EF_STRADDLE) {
            const f2 r = mul2(r2, rinv);
            const float rc = A.rgbmax;
            out0 = r.x - j.s >= rc && r.x - i.s.x >= rc;
            out1 = r.y - j.s >= rc && r.y - i.s.y >= rc;
            const bool sh = (!out0 && (r.x + j.s > rc || r.x + i.s.x > rc)) ||
                            (!out1 && (r.y + j.s > rc || r.y + i.s.y > rc));
            if (__any_sync(0xffffffffu, sh)) {
                const f2 fr = keep<MODE>(fma2(i.c, hct_cut_dir_fr2(r, rinv, i.a, F2(j.s), rc),
                                              mul2(F2(j.c), hct_cut_dir_fr2(r, rinv, F2(j.a), i.s, rc))), m);
                p.sx = fma2(fr, dx, p.sx); p.sy = fma2(fr, dy, p.sy); p.sz = fma2(fr, dz, p.sz);
                j.fx = fmaf(fr.y, dx.y, fmaf(fr.x, dx.x, j.fx));
                j.fy = fmaf(fr.y, dy.y, fmaf(fr.x, dy.x, j.fy));
                j.fz = fmaf(fr.y, dz.y, fmaf(fr.x, dz.x, j.fz));
                return;
            }
        }
        if (FAR) {  // whole block proven disjoint and far: no votes, short polynomial
            const f2 t = fma2(mul2(i.c, F2(hs3j)), gb_poly_hf2(y_ij),
                              mul2(mul2(F2(j.c), i.hs3), gb_poly_hf2(y_ji)));
            const f2 fr = mul2(t, mul2(rinv2, mul2(rinv2, rinv2)));
            p.sx = fma2(fr, dx, p.sx); p.sy = fma2(fr, dy, p.sy); p.sz = fma2(fr, dz, p.sz);
            j.fx = fmaf(fr.y, dx.y, fmaf(fr.x, dx.x, j.fx));
            j.fy = fmaf(fr.y, dy.y, fmaf(fr.x, dy.x, j.fy));
            j.fz = fmaf(fr.y, dz.y, fmaf(fr.x, dz.x, j.fz));
            return;
        }
        // c_i s_j^3/2 h(y_ij) + c_j s_i^3/2 h(y_ji), times r^-6
        const float r2min = fminf(r2.x, r2.y);
        f2 p_ij, p_ji;
        if (all_far(y_ij, y_ji)) {
            p_ij = gb_poly_hf2(y_ij);
            p_ji = gb_poly_hf2(y_ji);
        } else {
            p_ij = gb_poly_h2(y_ij);
            p_ji = gb_poly_h2(y_ji);
        }
        const f2 t_ij = mul2(mul2(i.c, F2(hs3j)), p_ij);
        const f2 t_ji = mul2(mul2(F2(j.c), i.hs3), p_ji);
        const f2 rinv6 = mul2(rinv2, mul2(rinv2, rinv2));
        f2 fr = mul2(add2(t_ij, t_ji), rinv6);
        if (__any_sync(0xffffffffu, r2min < bi.t_near)) {
            const f2 r = mul2(r2, rinv);
            const f2 lim_ij = add2(i.a, F2(j.s)), lim_ji = add2(F2(j.a), i.s);
            const bool b0 = !far_ok(r.x, lim_ij.x, y_ij.x), b1 = !far_ok(r.y, lim_ij.y, y_ij.y);
            const bool c0 = !far_ok(r.x, lim_ji.x, y_ji.x), c1 = !far_ok(r.y, lim_ji.y, y_ji.y);
            f2 fb = mul2(t_ij, rinv6), fc = mul2(t_ji, rinv6);
            if (__any_sync(0xffffffffu, b0 || b1)) {
                const f2 hc = mul2(i.c, hct_closed_fr2(r, rinv, i.a, F2(j.s)));
                fb = make_float2(b0 ? hc.x : fb.x, b1 ? hc.y : fb.y);
            }
            if (__any_sync(0xffffffffu, c0 || c1)) {
                const f2 hc = mul2(F2(j.c), hct_closed_fr2(r, rinv, F2(j.a), i.s));
                fc = make_float2(c0 ? hc.x : fc.x, c1 ? hc.y : fc.y);
            }
            const f2 fbc = add2(fb, fc);
            fr = make_float2(b0 || c0 ? fbc.x : fr.x, b1 || c1 ? fbc.y : fr.y);
        }
        if (FLAGS & EF_STRADDLE) fr = make_float2(out0 ? 0.0f : fr.x, out1 ? 0.0f : fr.y);
        fr = keep<MODE>(fr, m);
        p.sx = fma2(fr, dx, p.sx); p.sy = fma2(fr, dy, p.sy); p.sz = fma2(fr, dz, p.sz);
        j.fx = fmaf(fr.y, dx.y, fmaf(fr.x, dx.x, j.fx));
        j.fy = fmaf(fr.y, dy.y, fmaf(fr.x, dy.x, j.fy));
        j.fz = fmaf(fr.y, dz.y, fmaf(fr.x, dz.x, j.fz));
    }
    static __device__ __forceinline__ void rotate_data(JState& j, int src) {
        j.x = shfl(j.x, src); j.y = shfl(j.y, src); j.z = shfl(j.z, src);
        j.a = shfl(j.a, src); j.s = shfl(j.s, src); j.c = shfl(j.c, src);
    }
    static __device__ __forceinline__ void rotate_far(JState& j, int src) {
        j.x = shfl(j.x, src); j.y = shfl(j.y, src); j.z = shfl(j.z, src);
        j.s2 = shfl(j.s2, src); j.hs3 = shfl(j.hs3, src); j.c = shfl(j.c, src);
    }
    static __device__ __forceinline__ void rotate_acc(JState& j, int src) {
        j.fx = shfl(j.fx, src); j.fy = shfl(j.fy, src); j.fz = shfl(j.fz, src);
    }
    static __device__ __forceinline__ void take_data(JState& j, const JState& d) {
        j.x = d.x; j.y = d.y; j.z = d.z; j.a = d.a; j.s = d.s; j.c = d.c; j.s2 = d.s2; j.hs3 = d.hs3;
    }
    static __device__ __forceinline__ void fold_i(IState&, long long* sa, int lane, const Part& p) {
        sa[lane] -= fix(p.sx.x); sa[32 + lane] -= fix(p.sx.y);
        sa[64 + lane] -= fix(p.sy.x); sa[96 + lane] -= fix(p.sy.y);
        sa[128 + lane] -= fix(p.sz.x); sa[160 + lane] -= fix(p.sz.y);
    }
    static __device__ __forceinline__ void flush_j(const PairArgs& A, int64_t base, int n, int j, const JState& st) {
        if (j < n) {
            const int64_t g = base + j;
            red_add(&A.F_acc[g], fix(st.fx));
            red_add(&A.F_acc[A.N + g], fix(st.fy));
            red_add(&A.F_acc[2 * A.N + g], fix(st.fz));
        }
    }
    static __device__ __forceinline__ void flush_i(const PairArgs& A, int, int64_t base, int n, int i0, int lane,
                                                   const IState&, long long* sa) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = i0 + 32 * h + lane;
            if (i < n) {
                const int64_t g = base + i;
                const int o = 32 * h + lane;
                red_add(&A.F_acc[g], sa[o]);
                red_add(&A.F_acc[A.N + g], sa[64 + o]);
                red_add(&A.F_acc[2 * A.N + g], sa[128 + o]);
            }
        }
    }
};

// Energy's helpers carry the flag set; adapt them to the walker's interface.
template <int FLAGS>
struct EnergyF : Energy {
    static __device__ __forceinline__ void rotate_acc(JState& j, int src) { rotate_acc_f<FLAGS>(j, src); }
    static __device__ __forceinline__ void fold_i(IState& i, long long* sa, int lane, const Part& p) {
        fold_i_f<FLAGS>(i, sa, lane, p);
    }
    static __device__ __forceinline__ void flush_j(const PairArgs& A, int64_t b, int n, int j, const JState& s) {
        flush_j_f<FLAGS>(A, b, n, j, s);
    }
    static __device__ __forceinline__ void flush_i(const PairArgs& A, int r, int64_t b, int n, int i0, int lane,
                                                   const IState& s, long long* sa) {
        flush_i_f<FLAGS>(A, r, b, n, i0, lane, s, sa);
    }
};

// --- the warp walker ------------------------------------------------------------
// The steps of one (super-row, tile) block: after 32 rotations every j value is
// back in its home lane.
template <class P, int FLAGS, int MODE, bool FAR>
__device__ __forceinline__ void run_tile(const PairArgs& A, const typename P::IState& is, typename P::JState& js,
                                         typename P::Part& ip, const BlockInfo& bi, int i0, int jbase, int lane,
                                         int next) {
    // a DX block pairs the x half with its own tile: only steps 1 .. 16 carry
    // pairs (js enters rotated by one and leaves rotated by 17)
    constexpr int K0 = (MODE == M_DX) ? 1 : 0, K1 = (MODE == M_DX) ? 17 : 32;
    // straddling blocks carry the long restricted-integral code: not unrolled,
    // so that it fits the instruction cache
    constexpr int U = (FLAGS & EF_STRADDLE) ? 1 : (FAR ? P::UNROLL_FAR : P::UNROLL);
#pragma unroll U
    for (int k = K0; k < K1; ++k) {
        // the next step's j data are fetched before this step's arithmetic, so
        // that only the short accumulator chain is serial between steps
        typename P::JState nx = js;
        if (FAR) P::rotate_far(nx, next);
        else P::rotate_data(nx, next);
        const Mask m = step_mask<MODE>(k, lane);
        bool busy = true;
        if (FLAGS & EF_STRADDLE) {   // every pair of this step wholly past the cutoff's reach
            const float dx0 = js.x + is.nx.x, dy0 = js.y + is.ny.x, dz0 = js.z + is.nz.x;
            const float dx1 = js.x + is.nx.y, dy1 = js.y + is.ny.y, dz1 = js.z + is.nz.y;
            const float q0 = fmaf(dx0, dx0, fmaf(dy0, dy0, dz0 * dz0));
            const float q1 = fmaf(dx1, dx1, fmaf(dy1, dy1, dz1 * dz1));
            busy = __any_sync(0xffffffffu, fminf(q0, q1) <= bi.skip2);
        }
        if (busy) P::template pair<FLAGS, MODE, FAR>(A, is, js, ip, m, bi, i0, jbase, k);
        P::rotate_acc(js, next);
        P::take_data(js, nx);
    }
}

// Classification of a block (super-row K, tile J) from the bounding boxes of
// its tiles (lo.xyz with max a, hi.xyz with max s, from k_tile_boxes).  The
// block is "far" when the boxes prove, for every pair, r >= a_i + s_j
// (disjoint spheres), (s/r)^2 <= YFAR (short polynomial exact to FP32) and
// r >= the soft-repulsion range.  Otherwise r^2 >= t_near proves both
// directions of a pair disjoint with (s/r)^2 <= YMAX (far-field form valid),
// so only steps with a closer pair need the exact tests.  Without boxes
// nothing is proven.
// Bounds between the box of super-row K (tiles 2K, 2K+1) and the box of tile
// J: least and greatest distance squared, largest a and largest s of both.
struct BoxPair {
    float rmin2, rmax2, amax, smax;
};
__device__ __forceinline__ float4 row_box_lo(const PairArgs& A, int t0, int K, int nb, float4* hi) {
    float4 il = __ldcg(&A.boxes[2 * (t0 + 2 * K)]), ih = __ldcg(&A.boxes[2 * (t0 + 2 * K) + 1]);
    if (2 * K + 1 < nb) {
        const float4 l1 = __ldcg(&A.boxes[2 * (t0 + 2 * K + 1)]), h1 = __ldcg(&A.boxes[2 * (t0 + 2 * K + 1) + 1]);
        il = make_float4(fminf(il.x, l1.x), fminf(il.y, l1.y), fminf(il.z, l1.z), fmaxf(il.w, l1.w));
        ih = make_float4(fmaxf(ih.x, h1.x), fmaxf(ih.y, h1.y), fmaxf(ih.z, h1.z), fmaxf(ih.w, h1.w));
    }
    *hi = ih;
    return il;
}
__device__ __forceinline__ BoxPair box_pair(float4 il, float4 ih, float4 jl, float4 jh) {
    BoxPair b;
    const float gx = fmaxf(0.0f, fmaxf(il.x - jh.x, jl.x - ih.x));
    const float gy = fmaxf(0.0f, fmaxf(il.y - jh.y, jl.y - ih.y));
    const float gz = fmaxf(0.0f, fmaxf(il.z - jh.z, jl.z - ih.z));
    const float mx = fmaxf(ih.x - jl.x, jh.x - il.x);
    const float my = fmaxf(ih.y - jl.y, jh.y - il.y);
    const float mz = fmaxf(ih.z - jl.z, jh.z - il.z);
    b.rmin2 = gx * gx + gy * gy + gz * gz;
    b.rmax2 = mx * mx + my * my + mz * mz;
    b.amax = fmaxf(il.w, jl.w);
    b.smax = fmaxf(ih.w, jh.w);
    return b;
}

// Cutoff classes of a block from its box bounds (rmin / rmax the least /
// greatest distance between the boxes, smax the largest screened radius):
//   Born-radius cutoff (Born and chain passes): in range when
//     rmin < rgbmax + smax (some sphere j reaches into the ball about some
//     i), straddling when rmax + smax > rgbmax (some sphere reaches past it);
//   pair cutoff (energy pass): in range when rmin <= max(cut, rep_sigma),
//     straddling when rmax > cut.
// The bounds carry a 0.1 % margin, so that FP32 rounding of a pair's r^2 can
// never move it across a decision taken for its block.  A block that is not
// straddling needs no per-pair test; one out of range adds nothing.
__device__ __forceinline__ void cut_class(const PairArgs& A, bool radius_cut, const BoxPair& b, bool& in,
                                          bool& st) {
    if (radius_cut) {
        const float reach = A.rgbmax + b.smax, inner = A.rgbmax - b.smax;
        in = b.rmin2 <= 1.001f * reach * reach;
        st = inner <= 0.0f || b.rmax2 >= 0.999f * inner * inner;
    } else {
        in = b.rmin2 <= 1.001f * A.e_range2;
        st = b.rmax2 >= 0.999f * A.cut2;
    }
}

template <class P>
__device__ __forceinline__ BlockInfo block_info(const PairArgs& A, int r, int K, int J, int nb) {
    BlockInfo bi;
    bi.skip2 = INFINITY;
    if (!A.boxes) {   // nothing proven: near, and straddling when a cutoff is applied
        bi.far = false;
        bi.straddle = true;
        bi.t_near = INFINITY;
        return bi;
    }
    const int t0 = A.tile_off[r];
    const float4 jl = __ldcg(&A.boxes[2 * (t0 + J)]), jh = __ldcg(&A.boxes[2 * (t0 + J) + 1]);
    float4 ih;
    const float4 il = row_box_lo(A, t0, K, nb, &ih);
    const BoxPair b = box_pair(il, ih, jl, jh);
    const float as = b.amax + b.smax;
    bi.far = b.rmin2 >= as * as && b.smax * b.smax <= GB_POLY_YFAR * b.rmin2;
    if (A.rep_k != 0.0f) bi.far = bi.far && b.rmin2 >= A.rep_sigma * A.rep_sigma;
    // thresholds rounded up a little, so that rounding in r^2 cannot admit a
    // pair the exact test would reject
    bi.t_near = 1.0001f * fmaxf(as * as, b.smax * b.smax * (1.0f / GB_POLY_YMAX));
    // EF_CUT kernels: the block's cutoff class, and the reach past which a
    // pair adds exact zeros (Born and chain passes r >= rgbmax + s for both
    // spheres, energy pass r > max(cut, rep_sigma))
    bool in;
    cut_class(A, P::RADIUS_CUT, b, in, bi.straddle);
    if (P::RADIUS_CUT) {
        const float reach = A.rgbmax + b.smax;
        bi.skip2 = 1.001f * reach * reach;
    } else {
        bi.skip2 = 1.001f * A.e_range2;
    }
    return bi;
}

// Work of replica r is walked as super-rows K = 0 .. ceil(nb/2) - 1 (nb tiles
// of 32 atoms), each over tiles J = 2K .. nb-1; a task is (replica, K, J,
// number of tiles) and may continue into the next super-rows and replicas.
// One warp task walks (replica, K, J, count); sa is the warp's shared-memory
// slot of P::NQ x 64 int64 i-side accumulators (each lane owns its two atoms'
// entries).  Loads of data that kernels rewrite (coordinates, radii, chain
// factors, boxes) go through L2 (ld.global.cg): a persistent launch reads
// them again after other SMs changed them, and L1 is not coherent.
template <class P, int FLAGS>
__device__ __forceinline__ void walk_task(const PairArgs& A, const int4 t, long long* sa, int lane) {
#pragma unroll
    for (int q = 0; q < 2 * P::NQ; ++q) sa[32 * q + lane] = 0;
    int r = t.x, K = t.y, J = t.z;
    const int cnt = t.w;
    int64_t base = A.atom_off[r];
    int n = (int)(A.atom_off[r + 1] - base);
    int nb = (n + 31) >> 5;
    int nk = (nb + 1) >> 1;
    typename P::IState is;
    P::load_i(A, base, n, 64 * K, lane, is);
    const int next = (lane + 1) & 31;
    // EF_CUT: straddling blocks run the pair code with EF_STRADDLE.  The task
    // list is the block neighbour list (k_block_list: in-range blocks only),
    // or, without tile boxes, every block, each counted as straddling.
    constexpr int FS = (FLAGS & EF_CUT) ? (FLAGS | EF_STRADDLE) : FLAGS;
    for (int c = 0; c < cnt; ++c) {
        const bool dx = (J == 2 * K);          // see run_tile: entry / exit rotation of a DX block
        typename P::JState js;
        P::load_j(A, base, n, 32 * J + ((lane + (dx ? 1 : 0)) & 31), js);
        typename P::Part ip;
        ip.zero();
        const BlockInfo bi = block_info<P>(A, r, K, J, nb);
        const bool straddle = (FLAGS & EF_CUT) && bi.straddle;
        if (J >= 2 * K + 2) {
            if (bi.far && !straddle) run_tile<P, FLAGS, M_FULL, true>(A, is, js, ip, bi, 64 * K, 32 * J, lane, next);
            else if (straddle) run_tile<P, FS, M_FULL, false>(A, is, js, ip, bi, 64 * K, 32 * J, lane, next);
            else run_tile<P, FLAGS, M_FULL, false>(A, is, js, ip, bi, 64 * K, 32 * J, lane, next);
        } else if (J == 2 * K) {
            if (straddle) run_tile<P, FS, M_DX, false>(A, is, js, ip, bi, 64 * K, 32 * J, lane, next);
            else run_tile<P, FLAGS, M_DX, false>(A, is, js, ip, bi, 64 * K, 32 * J, lane, next);
        } else {
            if (straddle) run_tile<P, FS, M_DY, false>(A, is, js, ip, bi, 64 * K, 32 * J, lane, next);
            else run_tile<P, FLAGS, M_DY, false>(A, is, js, ip, bi, 64 * K, 32 * J, lane, next);
        }
        P::fold_i(is, sa, lane, ip);
        P::flush_j(A, base, n, 32 * J + ((lane + (dx ? 17 : 0)) & 31), js);
        if (c + 1 < cnt && ++J == nb) {
            P::flush_i(A, r, base, n, 64 * K, lane, is, sa);
#pragma unroll
            for (int q = 0; q < 2 * P::NQ; ++q) sa[32 * q + lane] = 0;
            if (++K == nk) {
                do {
                    ++r;
                    base = A.atom_off[r];
                    n = (int)(A.atom_off[r + 1] - base);
                    nb = (n + 31) >> 5;
                } while (nb == 0);
                nk = (nb + 1) >> 1;
                K = 0;
            }
            J = 2 * K;
            P::load_i(A, base, n, 64 * K, lane, is);
        }
    }
    P::flush_i(A, r, base, n, 64 * K, lane, is, sa);
}


// --- the pair-pass kernel --------------------------------------------------------
// One warp per task.  MINB = 1 leaves the register count to the compiler;
// MINB = 3 or 4 caps it so that three or four 256-thread blocks fit on an SM
// (more warps, some spills).
template <class P, int FLAGS, int MINB>
__global__ void __launch_bounds__(256, MINB) k_pairs(PairArgs A, const int4* __restrict__ tasks, int n_tasks) {
    pdl_enter();
    extern __shared__ long long s_acc[];
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= n_tasks) return;
    walk_task<P, FLAGS>(A, tasks[w], s_acc + (threadIdx.x >> 5) * P::NQ * 64, lane);
}

// The same pass over a task list built on the device (cutoff passes: the
// in-range blocks of k_block_list): the number of tasks is ctr[count_idx],
// and warps take tasks one at a time from the queue head ctr[head_idx] until
// it runs dry, so the grid only needs to fill the GPU.
template <class P, int FLAGS, int MINB>
__global__ void __launch_bounds__(256, MINB) k_pairs_dyn(PairArgs A, const int4* __restrict__ tasks, int* ctr,
                                                         int count_idx, int head_idx) {
    pdl_enter();
    extern __shared__ long long s_acc[];
    const int lane = threadIdx.x & 31;
    long long* sa = s_acc + (threadIdx.x >> 5) * P::NQ * 64;
    const int n_tasks = __ldcg(&ctr[count_idx]);
    for (;;) {
        int w = 0;
        if (lane == 0) w = atomicAdd(&ctr[head_idx], 1);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= n_tasks) break;
        walk_task<P, FLAGS>(A, __ldcg(&tasks[w]), sa, lane);
    }
}

// Launch of pass policy P over a task list; MAXCAP limits the register caps
// instantiated (a larger cap request takes the largest one available).
template <class P, int FLAGS, int MAXCAP = 4>
cudaError_t launch_pass(const PairArgs& a, const TaskList& t, int cap, int wpb, cudaStream_t s) {
    if (t.n_tasks == 0) return cudaSuccess;
    const int blocks = (t.n_tasks + wpb - 1) / wpb;
    const size_t smem = (size_t)wpb * P::NQ * 64 * sizeof(long long);
    const dim3 g(blocks), b(32 * wpb);
    if constexpr (MAXCAP >= 4) {
        if (cap >= 4) return launch_pdl(k_pairs<P, FLAGS, 4>, g, b, smem, s, a, t.d_tasks, t.n_tasks);
    }
    if (cap >= 3) return launch_pdl(k_pairs<P, FLAGS, 3>, g, b, smem, s, a, t.d_tasks, t.n_tasks);
    return launch_pdl(k_pairs<P, FLAGS, 1>, g, b, smem, s, a, t.d_tasks, t.n_tasks);
}

// Bounding boxes of every 32-atom tile (one warp per tile): lo.xyz with the
// largest a = rho - offset, hi.xyz with the largest screened radius s.
__device__ __forceinline__ void tile_box_warp(const PairArgs& A, int M, int t, int lane) {
    int lo = 0, hi = M;               // replica r with tile_off[r] <= t < tile_off[r+1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (A.tile_off[mid] <= t) lo = mid;
        else hi = mid;
    }
    const int r = lo;
    const int64_t base = A.atom_off[r];
    const int n = (int)(A.atom_off[r + 1] - base);
    const int i = 32 * (t - A.tile_off[r]) + lane;
    float x = 0.0f, y = 0.0f, z = 0.0f, q = 0.0f, am = 0.0f, sm = 0.0f;
    if (i < n) {
        const float4 p = __ldcg(&A.xyzq[base + i]);
        const float2 rs = A.rad[base + i];
        x = p.x; y = p.y; z = p.z; q = p.w;
        am = rs.x - A.offset;
        sm = rs.y * am;
    }
    tile_box_store(A.boxes, t, i < n, x, y, z, am, sm, q, A.err);
}


}  // namespace gbk
