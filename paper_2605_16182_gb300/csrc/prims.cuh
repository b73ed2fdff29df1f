// prims.cuh -- device building blocks of the engine: the counter-based RNG,
// the closed-form samplers and warp / block scans.  The scans, compactions
// and the radix sort built on them are in sortscan.cuh.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tw {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11).  Each walk owns the counter space
// (hop, 0, walk_lo, walk_hi) under key = seed, so a draw depends only on
// (seed, walk, hop) and never on how walks are scheduled.
// ---------------------------------------------------------------------------
struct Rand4 {
    uint32_t r0, r1, r2, r3;
};

__device__ __forceinline__ Rand4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int i = 0; i < 10; i++) {
        const uint32_t a0 = c0, a2 = c2;
        const uint32_t hi0 = __umulhi(0xD2511F53u, a0), lo0 = 0xD2511F53u * a0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, a2), lo1 = 0xCD9E8D57u * a2;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return Rand4{c0, c1, c2, c3};
}

__device__ __forceinline__ Rand4 walk_rand(uint64_t seed, uint64_t walk, uint32_t hop)
{
    return philox4x32_10(hop, 0u, (uint32_t)walk, (uint32_t)(walk >> 32), (uint32_t)seed,
                         (uint32_t)(seed >> 32));
}

// The block of draw `word1` of a hop (the Node2Vec rejection loop: proposal k
// uses word1 = k, its acceptance uniform word1 = 2^31 + k; word1 = 0 is
// walk_rand's block).
__device__ __forceinline__ Rand4 walk_rand2(uint64_t seed, uint64_t walk, uint32_t hop, uint32_t word1)
{
    return philox4x32_10(hop, word1, (uint32_t)walk, (uint32_t)(walk >> 32), (uint32_t)seed,
                         (uint32_t)(seed >> 32));
}

// 53-bit uniform in [0, 1): exact in double.
__device__ __forceinline__ double u53(uint32_t hi, uint32_t lo)
{
    const uint64_t b = ((((uint64_t)hi) << 32) | lo) >> 11;
    return __dmul_rn(__ull2double_rn(b), 1.1102230246251565404236316680908203125e-16);
}

// ---------------------------------------------------------------------------
// Closed-form inverse-CDF samplers over an index i in [0, n) (Sec. 2.5).
// Every step is an explicitly rounded IEEE operation so that no multiply-add
// is contracted: the result is the same as a left-to-right double evaluation
// on any IEEE machine, except for the last-place behaviour of exp / log.
// ---------------------------------------------------------------------------
enum : int { BIAS_UNIFORM = 0, BIAS_LINEAR = 1, BIAS_EXP = 2 };

__device__ __forceinline__ double sampler_x(double u, int64_t n, int bias, double lambda)
{
    const double nd = __ll2double_rn(n);
    if (bias == BIAS_UNIFORM) return __dmul_rn(u, nd);  // Eq. 1
    if (bias == BIAS_LINEAR) {                          // Eq. 2, weight i+1
        double t = __dmul_rn(4.0, u);
        t = __dmul_rn(t, nd);
        t = __dmul_rn(t, __dadd_rn(nd, 1.0));
        t = __dadd_rn(1.0, t);
        return __dmul_rn(__dadd_rn(__dsqrt_rn(t), -1.0), 0.5);
    }
    // weight exp(lambda*i): x = n + log(u + (1-u) exp(-lambda n)) / lambda
    const double e = exp(__dmul_rn(-lambda, nd));
    const double s = __dadd_rn(u, __dmul_rn(__dadd_rn(1.0, -u), e));
    return __dadd_rn(nd, __ddiv_rn(log(s), lambda));
}

__device__ __forceinline__ int64_t sampler_index(double u, int64_t n, int bias, double lambda)
{
    const double x = sampler_x(u, n, bias, lambda);
    if (!(x >= 0.0)) return 0;  // NaN, -inf, negative
    const double f = floor(x);
    if (f >= __ll2double_rn(n - 1)) return n - 1;
    return (int64_t)f;
}

__device__ __forceinline__ int64_t uniform_index(double u, int64_t n)
{
    return sampler_index(u, n, BIAS_UNIFORM, 1.0);
}

// ---------------------------------------------------------------------------
// The same samplers without FP64 on the common path.  GB300 issues FP64 at a
// small fraction of its FP32 / integer rate, so a walk that spends ~75 FP64
// instructions per hop is bound by the FP64 pipe.  Each function below
// returns exactly what the double-precision formula above returns.
// A uniform is carried as its 53-bit integer k (u = k * 2^-53).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t u53_bits(uint32_t hi, uint32_t lo)
{
    return ((((uint64_t)hi) << 32) | lo) >> 11;
}

// floor(fl64(u * n)) clamped to n-1, for 1 <= n < 2^31, computed with
// integers: P = k * n is exact in 128 bits; an IEEE double product keeps the
// top 53 bits of P rounded to nearest-even, and the floor of that value is
// a shift of the rounded significand.
__device__ __forceinline__ int64_t uniform_index_k(uint64_t k, int64_t n)
{
    const uint64_t nn = (uint64_t)n;
    const uint64_t lo = k * nn;
    const uint64_t hi = __umul64hi(k, nn);
    const int b = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);
    if (b <= 53) return 0;  // P < 2^53: u * n < 1, no rounding
    const int s = b - 53;   // 1 <= s <= 31 for n < 2^31
    uint64_t q = (lo >> s) | (hi << (64 - s));
    const uint64_t rem = lo & ((1ull << s) - 1ull);
    const uint64_t half = 1ull << (s - 1);
    if (rem > half || (rem == half && (q & 1ull))) q++;
    const int64_t f = (int64_t)(q >> (53 - s));
    return f < n - 1 ? f : n - 1;
}

// Exponential bias (weight exp(lambda*i), i in [0, n)).  The double formula
// x = n + log(u + (1-u) exp(-lambda n)) / lambda is first evaluated in FP32
// with a bound e on |y32 - y| (y = x - n), derived by first-order rounding
// analysis with rho = 2^-24: u, n, lambda and lambda*n rounded (3 rho
// relative on t = lambda n), expf <= 2 ulp, logf <= 1 ulp, the product with a
// rounded 1/lambda:
//   |s32 - s| / s <= rho (4 + m (5 + 3 t)),  m = min(1, E/u), E = e^-t
//   e32 <= rho (4 + m (5 + 3 t)) / lambda + 4 rho |y|
// (u is formed from two 32-bit conversions and one add: 2 rho; only 32-bit
// integer <-> float conversions are used, 64-bit ones run on the FP64 pipe)
// plus the error of the double evaluation itself (e64, about 1e-16 n) and a
// 1.5x margin.  When [y32 - e, y32 + e] holds no integer, floor(x) is n +
// floor(y32) for both the exact value and the double evaluation; otherwise
// the double formula decides.
struct ExpRate {
    double lambda;
    float lam32;   // (float)lambda
    float inv32;   // (float)(1 / lambda)
};

__device__ __forceinline__ int64_t exp_index_k(uint64_t k, int64_t n, const ExpRate &R)
{
    if (k == 0) return 0;  // u = 0 draws the oldest group for every n
    const float rho = 5.9604644775390625e-8f;  // 2^-24
    // u = k * 2^-53 from the high 32 and low 21 bits of k
    const float u = __uint2float_rn((uint32_t)(k >> 21)) * 2.3283064365386963e-10f +   // 2^-32
                    __uint2float_rn((uint32_t)(k & 0x1FFFFFu)) * 1.1102230246251565e-16f;  // 2^-53
    const float nf = __int2float_rn((int32_t)n);
    const float t = R.lam32 * nf;
    const float E = expf(-t);
    const float s = u + (1.0f - u) * E;
    const float L = logf(s);
    const float y = L * R.inv32;
    if (s > 0.0f && isfinite(y) && y > -2.0e9f) {
        const float m = fminf(1.0f, __fdividef(2.0f * E, u));
        const float ay = fabsf(y);
        float e = rho * (4.0f + m * (5.0f + 3.0f * t)) * R.inv32 + 4.0f * rho * ay;
        e = 1.5f * e + 5e-16f * (nf + ay) + 1e-15f * R.inv32 + 2.0f * rho * ay + 1e-37f;
        const float flo = floorf(y - e), fhi = floorf(y + e);
        if (flo == fhi) {
            const int64_t i = n + (int64_t)__float2int_rn(flo);
            return i < 0 ? 0 : (i > n - 1 ? n - 1 : i);
        }
    }
    const double ud = __dmul_rn(__ull2double_rn(k), 1.1102230246251565404236316680908203125e-16);
    return sampler_index(ud, n, BIAS_EXP, R.lambda);
}

// Linear bias (weight i+1).  The exact inverse is the largest i with
// i(i+1) <= Q, Q = u n (n+1), i.e. (2i+1)^2 <= A = 4Q + 1.  With
// u = k 2^-53, A 2^51 = k n(n+1) + 2^51 is an integer, so i follows from
// 128-bit integer comparisons inside a bracket found by an FP32 estimate.
// The double formula of Eq. 2 is within (X+1) 4.4e-16 of the exact X; when
// A is more than 64 (i+2)^2 units of 2^-51 away from both bucket edges
// (well beyond that error) the double formula floors to the same i,
// otherwise the double formula decides.
__device__ __forceinline__ int64_t linear_index_k(uint64_t k, int64_t n)
{
    typedef unsigned __int128 u128;
    const uint64_t nn = (uint64_t)n * (uint64_t)(n + 1);
    const u128 A = (u128)k * nn + ((u128)1 << 51);
    const float uf = __uint2float_rn((uint32_t)(k >> 21)) * 2.3283064365386963e-10f +
                     __uint2float_rn((uint32_t)(k & 0x1FFFFFu)) * 1.1102230246251565e-16f;
    const float nf = __int2float_rn((int32_t)n);
    const float Af = 4.0f * uf * nf * (nf + 1.0f) + 1.0f;
    const float Xf = fminf((sqrtf(Af) - 1.0f) * 0.5f, 4.0e9f);
    const uint32_t e_lo = __float2uint_rz(Xf * (1.0f - 9.5367431640625e-07f));  // 1 - 2^-20
    const uint32_t e_hi = __float2uint_rz(Xf * (1.0f + 9.5367431640625e-07f));
    uint64_t lo = e_lo > 2u ? (uint64_t)e_lo - 2u : 0u;
    uint64_t hi = (uint64_t)e_hi + 3u;
    bool ok = (((u128)(2 * lo + 1) * (2 * lo + 1)) << 51) <= A;
    if (ok) {
        while (lo < hi) {  // largest m in [lo, hi] with (2m+1)^2 2^51 <= A
            const uint64_t mid = (lo + hi + 1) >> 1;
            if ((((u128)(2 * mid + 1) * (2 * mid + 1)) << 51) <= A) lo = mid;
            else hi = mid - 1;
        }
        const uint64_t i = lo;
        const u128 b0 = ((u128)(2 * i + 1) * (2 * i + 1)) << 51;
        const u128 b1 = ((u128)(2 * i + 3) * (2 * i + 3)) << 51;
        if (b1 > A) {
            const u128 thr = (u128)64 * (u128)((i + 2) * (i + 2));
            if (A - b0 > thr && b1 - A > thr) return (int64_t)i < n - 1 ? (int64_t)i : n - 1;
        }
    }
    const double ud = __dmul_rn(__ull2double_rn(k), 1.1102230246251565404236316680908203125e-16);
    return sampler_index(ud, n, BIAS_LINEAR, 1.0);
}

// Index of the group / edge a draw selects, for any bias.
__device__ __forceinline__ int64_t sampler_index_k(uint64_t k, int64_t n, int bias, const ExpRate &R)
{
    if (bias == BIAS_UNIFORM) return uniform_index_k(k, n);
    if (bias == BIAS_EXP) return exp_index_k(k, n, R);
    return linear_index_k(k, n);
}

// ---------------------------------------------------------------------------
// warp / block helpers
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T o = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += o;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

// Exclusive block scan; blockDim.x must be a multiple of 32 and <= 1024.
// `sh` is caller-provided shared scratch of 33 elements.  Returns the
// exclusive prefix of v; `total` receives the block total.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T *sh, T &total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const T inc = warp_incl_scan(v);
    if (lane == 31) sh[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const T t = lane < nw ? sh[lane] : T(0);
        const T ti = warp_incl_scan(t);
        if (lane < nw) sh[lane] = ti - t;
        if (lane == 31) sh[32] = ti;
    }
    __syncthreads();
    const T res = sh[wid] + inc - v;
    total = sh[32];
    __syncthreads();
    return res;
}

}  // namespace tw
