// Device helpers shared by the GB300 kernels: constants, fixed-point
// accumulation, ghost atoms for ragged tails, Philox4x64-10.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gbremd.h"

namespace gbk {

// Coulomb constant (kcal A / (mol e^2)), Faraday constant (kcal / (mol V)).
constexpr double KE = 332.0522173;
constexpr double FARADAY = 23.0605478;
constexpr double LN10 = 2.302585092994045684;
// (kcal/mol/A) / amu -> A / ps^2
constexpr double ACCEL = 418.4;

// Fixed-point scales: forces, dE/dR, dE/dq and energies carry 32 fractional
// bits; Born integrals (values below ~10 / A) carry 40.
constexpr float FIX = 4294967296.0f;
constexpr double FIX_INV = 1.0 / 4294967296.0;
constexpr float FIX_I = 1099511627776.0f;
constexpr double FIX_I_INV = 1.0 / 1099511627776.0;

typedef unsigned long long u64;

__device__ __forceinline__ long long fix(float v) { return __float2ll_rn(v * FIX); }
__device__ __forceinline__ long long fix_i(float v) { return __float2ll_rn(v * FIX_I); }
__device__ __forceinline__ long long fix_d(double v) { return __double2ll_rn(v * 4294967296.0); }
__device__ __forceinline__ void red_add(u64* p, long long v) {
    atomicAdd(p, (u64)v);
}
__device__ __forceinline__ double unfix(u64 v) { return (double)(long long)v * FIX_INV; }

// Lanes past the end of a replica hold "ghost" atoms: zero charge, zero
// descreening radius, zero chain factor, parked far away at distinct spots.
// Every term a ghost contributes to a real atom is then exactly +-0.
__device__ __forceinline__ float ghost_x(int local) { return 1.0e7f + 16.0f * (float)local; }

__device__ __forceinline__ float shfl(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// Bounding box of one 32-atom tile, reduced over the warp (every lane calls
// it; lanes without an atom pass valid = false): lo.xyz with the largest
// a = rho - offset, hi.xyz with the largest screened radius s, stored by
// lane 0 at boxes[2t], boxes[2t + 1].
// Also the finiteness check of the evaluation's input: a lane whose atom has a
// non-finite coordinate or charge records GB_ERR_NONFINITE (err nullable; the
// int64 fixed-point sums would otherwise turn NaN into a silent zero).
__device__ __forceinline__ void tile_box_store(float4* boxes, int64_t t, bool valid, float x, float y, float z,
                                               float a, float s, float q, int* err) {
    if (valid && err && !(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(q)))
        atomicCAS(err, 0, GB_ERR_NONFINITE);
    float x0 = valid ? x : INFINITY, y0 = valid ? y : INFINITY, z0 = valid ? z : INFINITY;
    float x1 = valid ? x : -INFINITY, y1 = valid ? y : -INFINITY, z1 = valid ? z : -INFINITY;
    float am = valid ? a : 0.0f, sm = valid ? s : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x0 = fminf(x0, __shfl_xor_sync(0xffffffffu, x0, o));
        y0 = fminf(y0, __shfl_xor_sync(0xffffffffu, y0, o));
        z0 = fminf(z0, __shfl_xor_sync(0xffffffffu, z0, o));
        x1 = fmaxf(x1, __shfl_xor_sync(0xffffffffu, x1, o));
        y1 = fmaxf(y1, __shfl_xor_sync(0xffffffffu, y1, o));
        z1 = fmaxf(z1, __shfl_xor_sync(0xffffffffu, z1, o));
        am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
        sm = fmaxf(sm, __shfl_xor_sync(0xffffffffu, sm, o));
    }
    if ((threadIdx.x & 31) == 0) {
        boxes[2 * t] = make_float4(x0, y0, z0, am);
        boxes[2 * t + 1] = make_float4(x1, y1, z1, sm);
    }
}

// Programmatic dependent launch.  Kernels are launched with launch_pdl, so the
// next kernel in the stream may be scheduled onto SMs while this one drains.
// Every kernel therefore starts with pdl_wait() (returns once the previous
// kernel in the stream has completed and its writes are visible; immediately
// when there is none) before it touches memory, and then calls pdl_trigger()
// to let its own successor be scheduled.  Results are those of plain stream
// order; only launch latency and the block ramp are overlapped.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_enter() {
    pdl_wait();
    pdl_trigger();
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Philox4x64-10 (Salmon et al., SC'11): 10 rounds of two 64x64->128 multiplies
// with the published multipliers, key bumped by the published Weyl constants.
struct Philox4 {
    u64 w[4];
};

__device__ __forceinline__ Philox4 philox4x64(u64 c0, u64 c1, u64 c2, u64 c3, u64 k0, u64 k1) {
    const u64 M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        u64 hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        u64 hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        u64 n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B97F4A7C15ULL;
        k1 += 0xBB67AE8584CAA73BULL;
    }
    Philox4 r;
    r.w[0] = c0; r.w[1] = c1; r.w[2] = c2; r.w[3] = c3;
    return r;
}

// u in [0, 1) from the top 53 bits; integer in [0, n) from the top 32 bits.
__device__ __forceinline__ double unif53(u64 w) { return (double)(w >> 11) * (1.0 / 9007199254740992.0); }
__device__ __forceinline__ int pick_int(u64 w, int n) { return (int)(((w >> 32) * (u64)n) >> 32); }

}  // namespace gbk
