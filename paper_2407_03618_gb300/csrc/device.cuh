// Device-side helpers: block scans, the ordered (score, doc) key, status word.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "bm25.h"

namespace bm25 {

__device__ __forceinline__ void set_status(int* status, int code)
{
    atomicCAS(status, 0, code);
}

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Inclusive warp scan (sum).
template <typename T>
__device__ __forceinline__ T warp_inclusive_sum(T v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o)
            v += n;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Exclusive scan across the block (blockDim.x a multiple of 32, <= 1024).
// `warp_buf` holds 33 elements of shared memory.  Returns the exclusive
// prefix of v; *total receives the block sum.  Contains __syncthreads().
template <typename T>
__device__ __forceinline__ T block_exclusive_sum(T v, T* warp_buf, T* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    T inc = warp_inclusive_sum(v);
    if (lane == 31)
        warp_buf[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = (lane < nwarps) ? warp_buf[lane] : T(0);
        T wi = warp_inclusive_sum(w);
        if (lane < nwarps)
            warp_buf[lane] = wi - w;  // exclusive
        if (lane == nwarps - 1)
            warp_buf[32] = wi;
    }
    __syncthreads();
    T r = warp_buf[warp] + inc - v;
    *total = warp_buf[32];
    __syncthreads();
    return r;
}

// ---- ranking keys -------------------------------------------------------
// A candidate is a 64-bit key whose unsigned order is the ranking order:
// high word = FP32 score mapped to an order-preserving uint32 (-0.0 folded
// onto +0.0), low word = ~doc so that the lower doc id wins a tie.  Every
// non-NaN score maps to a high word >= 0x007fffff, so key 0 never names a
// real candidate and serves as the empty slot.
__device__ __forceinline__ uint32_t order_f32(float s)
{
    uint32_t u = __float_as_uint(s == 0.0f ? 0.0f : s);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float unorder_f32(uint32_t o)
{
    uint32_t u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
    return __uint_as_float(u);
}

__device__ __forceinline__ unsigned long long make_key(float s, uint32_t doc)
{
    return ((unsigned long long)order_f32(s) << 32) | (unsigned long long)(~doc);
}

__device__ __forceinline__ uint32_t key_doc(unsigned long long k)
{
    return ~(uint32_t)(k & 0xffffffffull);
}

__device__ __forceinline__ float key_score(unsigned long long k)
{
    return unorder_f32((uint32_t)(k >> 32));
}

// ---- per-entry score (Sec. 2, Sec. 2.1) ------------------------------------
// FP32 per entry, in forms free of cancellation (S - S0 written out):
//   Lucene, Robertson:  c TF / (TF + k1 K_D)                  c = IDF
//   ATIRE, BM25+:       c TF / (TF + k1 K_D)                  c = IDF (k1+1)
//   BM25L:              c p / (k1 + delta + p), p = TF / K_D  c = IDF (k1+1) k1/(k1+delta)
//   TF_ldp:             c log1p(log1p(p / delta) / (1 + ln delta)), p = TF / K_D,
//                       c = IDF  (= IDF [ln(1 + ln(p + delta)) - ln(1 + ln delta)])
// with the length factor a = k1 K_D (1 / K_D for BM25L and TF_ldp) and the
// term coefficient c.  The build, the rescoring of a shard and query-time
// scoring all use this one function.
struct ScoreConsts {
    float k1_plus_delta;  // BM25L
    float inv_delta;      // TF_ldp: 1 / delta
    float inv_l0;         // TF_ldp: 1 / (1 + ln delta)
};

inline ScoreConsts score_consts(double k1, double delta)
{
    ScoreConsts k;
    k.k1_plus_delta = (float)(k1 + delta);
    k.inv_delta = delta > 0.0 ? (float)(1.0 / delta) : 0.0f;
    k.inv_l0 = (1.0 + std::log(delta) > 0.0) ? (float)(1.0 / (1.0 + std::log(delta))) : 0.0f;
    return k;
}

// Never -0.0: retrieval uses -0.0 as "untouched".
__device__ __forceinline__ float entry_score(int variant, float f, float a, float c,
                                             const ScoreConsts& k)
{
    float sc;
    if (variant == BM25_L) {
        const float cc = f * a;
        sc = c * cc / (k.k1_plus_delta + cc);
    } else if (variant == BM25_TFLDP) {
        const float cc = f * a;
        sc = c * log1pf(log1pf(cc * k.inv_delta) * k.inv_l0);
    } else {
        sc = c * f / (f + a);
    }
    return (sc == 0.0f) ? 0.0f : sc;
}

// Per-term coefficient c and non-occurrence score S0 from IDF (FP64).
__host__ __device__ inline void term_coef(int variant, double w, double k1, double delta,
                                          double* c, double* s0)
{
    *s0 = 0.0;
    *c = w;
    if (variant == BM25_ATIRE || variant == BM25_PLUS)
        *c = w * (k1 + 1.0);
    if (variant == BM25_L) {
        *s0 = w * (k1 + 1.0) * delta / (k1 + delta);
        *c = w * (k1 + 1.0) * k1 / (k1 + delta);
    } else if (variant == BM25_PLUS) {
        *s0 = w * delta;
    } else if (variant == BM25_TFLDP) {
        *s0 = w * (1.0 + log(1.0 + log(delta)));
    }
}

// The length factor of a document of |D| = len: k1 K_D, or 1 / K_D for
// BM25L and TF_ldp, with K_D = 1 - b + b |D| / Lavg in FP64.
__host__ __device__ inline float length_factor(int variant, double k1, double b, double len,
                                               double lavg)
{
    const double kd = 1.0 - b + b * len / lavg;
    return (variant == BM25_L || variant == BM25_TFLDP) ? (float)(1.0 / kd) : (float)(k1 * kd);
}

}  // namespace bm25
