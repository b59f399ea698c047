// Eager index build (arXiv 2407.03618 Sec. 2 "Eager index-time scoring" and
// "Efficient Matrix Sparsity"; Sec. 2.1 for the non-occurrence shift).
//
// Pipeline, all on the caller's stream:
//   K1 k_doc_prep        |D| per document, the doc id of every token, and the
//                        per-document length factor of the score
//   K2 k_radix_*         stable LSD radix sort of the tokens by term id with
//                        the doc id as payload.  The input is in document order,
//                        so the result is term-major with doc ids ascending
//                        inside each term, and equal (term, doc) pairs adjacent
//   K3 k_rle_*           run-length reduce of the sorted pairs: one run per
//                        distinct (term, doc) = one CSC entry, TF = run length
//   K4/K5 k_indptr       column starts (the exclusive prefix sum of DF) by a
//                        lower bound over the term of each run; DF = difference
//   K6 k_idf             IDF and S0 per term in FP64, FP32 score coefficient
//   K7 k_pad_posts       padding slots of the packed (doc, score) copy
//   K8 k_score           S(t,D) - S0(t) per CSC entry in FP32, written to the
//                        CSC and to the packed copy that staged retrieval
//                        reads (each column 16-byte aligned)
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "device.cuh"
#include "internal.h"

namespace bm25 {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortIpt = 16;
constexpr int kSortTile = kSortThreads * kSortIpt;  // 4096 items per tile
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kMaxDigitBits = 9;  // 18-bit vocabularies (<= 262,144 terms) sort in two passes
constexpr int kMaxBuckets = 1 << kMaxDigitBits;
constexpr int kSortedTileBytes = 2 * kSortTile * (int)sizeof(uint32_t);  // downsweep dynamic smem

// ---- K1 -------------------------------------------------------------------
// One warp per group of 32 documents (lane l: document g*32 + l): |D|, the
// FP32 length factor used by the score kernel (k1 * K_D, or 1 / K_D for
// BM25L, with K_D = 1 - b + b |D| / Lavg evaluated in FP64), and the doc id
// of every token of the group, written coalesced: each position finds its
// document by a 5-step search over the lanes' start offsets.  Offsets are
// checked; a malformed range records BM25_E_TOKEN_RANGE and nothing is
// written outside [0, n_tokens).
__global__ void k_doc_prep(const int64_t* __restrict__ off, int64_t n_docs, int64_t n_tokens,
                           int32_t* __restrict__ tok_doc, int32_t* __restrict__ doc_len,
                           float* __restrict__ len_factor, int variant, double k1, double b,
                           double lavg, int* status)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    if (warp0 == 0 && lane == 0 && (off[0] != 0 || off[n_docs] != n_tokens))
        set_status(status, BM25_E_TOKEN_RANGE);
    const int64_t n_groups = (n_docs + 31) >> 5;
    for (int64_t g = warp0; g < n_groups; g += nwarps) {
        const int64_t d = (g << 5) + lane;
        const bool has = d < n_docs;
        int64_t lo = has ? off[d] : 0, hi = has ? off[d + 1] : 0;
        const bool bad = has && (lo < 0 || hi < lo || hi > n_tokens);
        if (bad)
            set_status(status, BM25_E_TOKEN_RANGE);
        if (has) {
            const int64_t len = bad ? 0 : hi - lo;
            doc_len[d] = (int32_t)len;
            len_factor[d] = length_factor(variant, k1, b, (double)len, lavg);
        }
        if (__any_sync(0xffffffffu, bad))
            continue;  // the build fails; only in-range writes happen above
        if (!has)
            lo = hi = n_tokens;  // lanes past the last document start nothing
        // the group's tokens are [first lo, last hi); lane l's document owns
        // [lo_l, hi_l), and documents are contiguous
        const int64_t start = __shfl_sync(0xffffffffu, lo, 0);
        int last = 31;
        {
            const unsigned has_mask = __ballot_sync(0xffffffffu, has);
            last = 31 - __clz(has_mask);
        }
        const int64_t end = __shfl_sync(0xffffffffu, hi, last);
        // warp-uniform loop over windows of 32 positions.  Position p belongs
        // to the last lane whose document starts at or before p: the lanes
        // started by the window's first position are counted by one ballot,
        // and the few documents starting inside the window (a window holds
        // ~32 / mean length of them) are added one by one.  Lanes past the
        // last document start at n_tokens and never count.
        const uint32_t live = (last == 31) ? 0xffffffffu : ((2u << last) - 1u);
        for (int64_t pb = start; pb < end; pb += 32) {
            const int64_t p = pb + lane;
            const uint32_t before = __ballot_sync(0xffffffffu, lo <= pb) & live;
            uint32_t inside = __ballot_sync(0xffffffffu, lo > pb && lo <= pb + 31) & live;
            int idx = __popc(before) - 1;  // >= 0: lane 0 starts at `start` <= pb
            while (inside) {               // warp-uniform
                const int l = __ffs(inside) - 1;
                inside &= inside - 1u;
                idx += (__shfl_sync(0xffffffffu, lo, l) <= p) ? 1 : 0;
            }
            if (p < end)
                tok_doc[p] = (int32_t)((g << 5) + idx);
        }
    }
}

// ---- K2: stable LSD radix sort -------------------------------------------
// Reduce-then-scan per pass (Satish et al. 2009; Merrill and Grimshaw 2011),
// partitioned the way those papers do it for a resident grid: block b of the
// G-block downsweep grid owns the consecutive tiles [b*nt/G, (b+1)*nt/G) of
// the input and walks them in order, ranking each tile's items stably and
// advancing its per-digit output bases by the tile's counts.  The upsweep
// splits each of those ranges over S blocks (a full wave of small blocks)
// and counts their digits; one exclusive scan over the [digit][b][s] table
// gives every (digit, b) its first output position at s = 0.  No kernel
// waits on another block.  The table has 2^bits * G * S words instead of
// one column per tile, and the writes of one digit by consecutive tiles of
// a block continue each other.

// First and last+1 tile of downsweep block b.
__device__ __forceinline__ void sort_block_tiles(int64_t b, int64_t G, int64_t n_tiles,
                                                 int64_t& t0, int64_t& t1)
{
    t0 = b * n_tiles / G;
    t1 = (b + 1) * n_tiles / G;
}

// Digit histogram of upsweep block (b, s) = (blockIdx.x / S, blockIdx.x % S):
// counts[(d * G + b) * S + s].  One private histogram per warp, plain shared
// atomics (grouping a warp's equal digits with __match_any_sync first was
// slower).  With vocab > 0 it also checks every key against [0, vocab).
__global__ void __launch_bounds__(kSortThreads)
    k_radix_upsweep(const uint32_t* __restrict__ keys, int64_t n, int shift, int bits,
                    uint32_t* __restrict__ counts, int64_t n_tiles, int S, uint32_t vocab,
                    int* status)
{
    __shared__ uint32_t whist[kSortWarps][kMaxBuckets];
    const int nb = 1 << bits;
    const uint32_t mask = (uint32_t)nb - 1u;
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kSortWarps * kMaxBuckets; i += kSortThreads)
        (&whist[0][0])[i] = 0;
    __syncthreads();
    const int64_t G = gridDim.x / S, b = blockIdx.x / S, sub = blockIdx.x % S;
    int64_t t0, t1;
    sort_block_tiles(b, G, n_tiles, t0, t1);
    const int64_t lo = (t0 + sub * (t1 - t0) / S) * kSortTile;
    const int64_t hi = min((t0 + (sub + 1) * (t1 - t0) / S) * kSortTile, n);
    bool bad = false;
    // rounds of 4 x 256 items, the loads of a round issued together
    for (int64_t p0 = lo; p0 < hi; p0 += 4 * kSortThreads) {
        uint32_t k[4];
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int64_t p = p0 + i * kSortThreads + threadIdx.x;
            k[i] = p < hi ? keys[p] : 0u;
        }
#pragma unroll
        for (int i = 0; i < 4; i++) {
            if (p0 + i * kSortThreads + threadIdx.x < hi) {
                bad |= (vocab != 0u && k[i] >= vocab);
                atomicAdd(&whist[warp][(k[i] >> shift) & mask], 1u);
            }
        }
    }
    if (bad)
        set_status(status, BM25_E_TOKEN_RANGE);
    __syncthreads();
    for (int d = threadIdx.x; d < nb; d += kSortThreads) {
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; w++)
            c += whist[w][d];
        counts[((int64_t)d * G + b) * S + sub] = c;
    }
}

// Stable scatter of the block's tiles, in order.  Per tile: warp w owns
// items [w*512, w*512+512) and walks them in 16 rounds of 32 consecutive
// items; __match_any_sync groups a round's lanes by digit, so each item's
// rank among equal digits follows its position.  Per-warp counters become
// per-warp bases by an exclusive scan over warps (warp order = item order),
// the items are reordered in shared memory into the tile's digit order, and
// consecutive threads write consecutive global positions of one digit.
// Thread t keeps the block's running global base of digits 2t and 2t+1 in
// registers.  The next tile's keys and doc ids are loaded while the current
// tile is written out.
__global__ void __launch_bounds__(kSortThreads, 2)
    k_radix_downsweep(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                      uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, int64_t n,
                      int shift, int bits, const uint32_t* __restrict__ offsets, int64_t n_tiles,
                      int S)
{
    __shared__ uint32_t wcnt[kSortWarps][kMaxBuckets];  // per-warp counts, then tile positions
    __shared__ uint32_t gofs[kMaxBuckets];  // global position - position in the sorted tile
    __shared__ uint32_t scan_buf[33];
    // kSortTile sorted keys, then kSortTile sorted doc ids
    extern __shared__ uint32_t sorted_tile[];
    uint32_t* sk = sorted_tile;
    uint32_t* sv = sorted_tile + kSortTile;
    const int nb = 1 << bits;
    const uint32_t mask = (uint32_t)nb - 1u;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();
    static_assert(kMaxBuckets <= 2 * kSortThreads, "two digits per thread");
    uint32_t run[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int d = 2 * (int)threadIdx.x + h;
        run[h] = d < nb ? offsets[((int64_t)d * gridDim.x + blockIdx.x) * S] : 0u;
    }
    int64_t t0, t1;
    sort_block_tiles(blockIdx.x, gridDim.x, n_tiles, t0, t1);
    uint32_t k[kSortIpt], v[kSortIpt];
    const int wbase = warp * (kSortIpt * 32) + lane;  // item index in the tile, round 0
    auto load_tile = [&](int64_t tile) {
        const int64_t first = tile * kSortTile + wbase;
        const uint32_t* kp = keys_in + first;
        const uint32_t* vp = vals_in + first;
        const int rem = (int)min((int64_t)kSortTile, n - first);  // may be <= 0
#pragma unroll
        for (int r = 0; r < kSortIpt; r++) {
            const bool ok = r * 32 < rem;
            k[r] = ok ? kp[r * 32] : 0u;
            v[r] = ok ? vp[r * 32] : 0u;
        }
    };
    if (t0 < t1)
        load_tile(t0);
    for (int64_t tile = t0; tile < t1; tile++) {
        const int64_t tile0 = tile * kSortTile;
        const int tile_n = (int)min((int64_t)kSortTile, n - tile0);
        for (int i = threadIdx.x; i < kSortWarps * kMaxBuckets; i += kSortThreads)
            (&wcnt[0][0])[i] = 0;
        __syncthreads();
        uint32_t rank[kSortIpt];
#pragma unroll
        for (int r = 0; r < kSortIpt; r++) {
            const bool ok = wbase + r * 32 < tile_n;
            const uint32_t dg = ok ? ((k[r] >> shift) & mask) : 0xffffffffu;
            const uint32_t peers = __match_any_sync(0xffffffffu, dg);
            const uint32_t before = ok ? wcnt[warp][dg] : 0u;
            __syncwarp();
            if (ok && (peers & lt) == 0)
                wcnt[warp][dg] = before + (uint32_t)__popc(peers);
            __syncwarp();
            rank[r] = before + (uint32_t)__popc(peers & lt);
        }
        __syncthreads();
        // per digit: the tile total and the exclusive scan over warps; then
        // the digit's start in the tile, folded into the warp bases
        uint32_t tot2[2] = {0u, 0u};
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int d = 2 * (int)threadIdx.x + h;
            if (d < nb) {
#pragma unroll
                for (int w = 0; w < kSortWarps; w++)
                    tot2[h] += wcnt[w][d];
            }
        }
        uint32_t all;
        const uint32_t ds = block_exclusive_sum(tot2[0] + tot2[1], scan_buf, &all);
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int d = 2 * (int)threadIdx.x + h;
            if (d < nb) {
                uint32_t c = ds + (h ? tot2[0] : 0u);  // the digit's start in the tile
                gofs[d] = run[h] - c;
                run[h] += tot2[h];
#pragma unroll
                for (int w = 0; w < kSortWarps; w++) {
                    const uint32_t t = wcnt[w][d];
                    wcnt[w][d] = c;
                    c += t;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kSortIpt; r++) {
            if (wbase + r * 32 < tile_n) {
                const uint32_t local = wcnt[warp][(k[r] >> shift) & mask] + rank[r];
                sk[local] = k[r];
                sv[local] = v[r];
            }
        }
        __syncthreads();
        if (tile + 1 < t1)
            load_tile(tile + 1);
        for (int i = threadIdx.x; i < tile_n; i += kSortThreads) {
            const uint32_t kk = sk[i];
            const uint32_t pos = gofs[(kk >> shift) & mask] + (uint32_t)i;
            keys_out[pos] = kk;
            vals_out[pos] = sv[i];
        }
        // (the next tile's first barrier orders these reads of sk, sv and
        // gofs before their next writes)
    }
}

// ---- K3: run-length reduce -------------------------------------------------
// Tile of 4096 sorted positions, striped: in round i, warp w covers the 32
// consecutive positions tile + i*256 + w*32 + lane.  A position starts a run
// (a distinct (term, doc) pair) when its pair differs from the previous
// position's.  Runs are numbered in position order, i.e. by (round, warp,
// lane), so the writes of one warp-round are consecutive.
// All four loads are unconditional (clamped at the ends), so that a thread's
// loads for several positions are in flight together.
__device__ __forceinline__ bool is_head(const uint32_t* __restrict__ keys,
                                        const uint32_t* __restrict__ vals, int64_t p, int64_t n,
                                        uint32_t& kk, uint32_t& vv)
{
    const int64_t pc = p < n ? p : n - 1;
    const int64_t pp = pc > 0 ? pc - 1 : 0;
    kk = keys[pc];
    vv = vals[pc];
    const uint32_t kp = keys[pp], vp = vals[pp];
    return p < n && (p == 0 || kk != kp || vv != vp);
}

__global__ void __launch_bounds__(kSortThreads)
    k_rle_count(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals, int64_t n,
                uint32_t* __restrict__ tile_heads)
{
    __shared__ uint32_t buf[33];
    const int lane = threadIdx.x & 31;
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    uint32_t c = 0;
#pragma unroll 4
    for (int i = 0; i < kSortIpt; i++) {
        const int64_t p = base + i * kSortThreads + threadIdx.x;
        uint32_t kk, vv;
        const bool h = is_head(keys, vals, p, n, kk, vv);
        const uint32_t bal = __ballot_sync(0xffffffffu, h);
        if (lane == 0)
            c += __popc(bal);
    }
    uint32_t tot;
    block_exclusive_sum(c, buf, &tot);
    if (threadIdx.x == 0)
        tile_heads[blockIdx.x] = tot;
}

// Writes one CSC entry per run: its start position (TF = distance to the next
// start), its term (for the score kernel) and its doc id (the CSC row index).
__global__ void __launch_bounds__(kSortThreads)
    k_rle_emit(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals, int64_t n,
               const uint32_t* __restrict__ tile_off, const uint32_t* __restrict__ d_nnz,
               int32_t* __restrict__ run_pos, int32_t* __restrict__ run_term,
               int32_t* __restrict__ indices)
{
    __shared__ uint32_t seg_cnt[kSortIpt * kSortWarps];
    __shared__ uint32_t buf[33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    uint32_t kk[kSortIpt], vv[kSortIpt], bals[kSortIpt];
#pragma unroll
    for (int i = 0; i < kSortIpt; i++) {
        const int64_t p = base + i * kSortThreads + threadIdx.x;
        const bool h = is_head(keys, vals, p, n, kk[i], vv[i]);
        bals[i] = __ballot_sync(0xffffffffu, h);
        if (lane == 0)
            seg_cnt[i * kSortWarps + warp] = __popc(bals[i]);
    }
    __syncthreads();
    // exclusive scan of the 128 (round, warp) counts in (round, warp) order
    const uint32_t c = (threadIdx.x < kSortIpt * kSortWarps) ? seg_cnt[threadIdx.x] : 0u;
    uint32_t tot;
    const uint32_t ex = block_exclusive_sum(c, buf, &tot);
    if (threadIdx.x < kSortIpt * kSortWarps)
        seg_cnt[threadIdx.x] = ex;
    __syncthreads();
    const uint32_t t0 = tile_off[blockIdx.x];
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < kSortIpt; i++) {
        if (bals[i] & (1u << lane)) {
            const int64_t p = base + i * kSortThreads + threadIdx.x;
            const uint32_t j = t0 + seg_cnt[i * kSortWarps + warp] + __popc(bals[i] & lt);
            run_pos[j] = (int32_t)p;
            run_term[j] = (int32_t)kk[i];
            indices[j] = (int32_t)vv[i];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        run_pos[*d_nnz] = (int32_t)n;
}

// ---- K4/K5: column starts -------------------------------------------------
// indptr[t] = number of runs whose term is < t (runs are term-major), i.e.
// the exclusive prefix sum of DF; found by a lower bound per term.
__global__ void k_indptr(const int32_t* __restrict__ run_term, const uint32_t* __restrict__ d_nnz,
                         int32_t vocab, int64_t* __restrict__ indptr)
{
    const int64_t nnz = *d_nnz;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= vocab;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = nnz;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (run_term[mid] < t)
                lo = mid + 1;
            else
                hi = mid;
        }
        indptr[t] = lo;
    }
}

// ---- K6: per-term IDF, S0 and FP32 coefficient ------------------------------
// Written in simplified but equal forms: Lucene's argument
// (N - DF + 0.5)/(DF + 0.5) + 1 equals (N + 1)/(DF + 0.5).
__device__ double idf_of(int variant, double n, double df)
{
    if (df <= 0.0)
        return 0.0;  // a term that occurs nowhere contributes nothing
    switch (variant) {
    case BM25_LUCENE:
    case BM25_L:
        return log((n + 1.0) / (df + 0.5));
    case BM25_ROBERTSON:
        return log((n - df + 0.5) / (df + 0.5));
    case BM25_ATIRE:
        return log(n / df);
    default:  // BM25_PLUS, BM25_TFLDP
        return log((n + 1.0) / df);
    }
}

// df_out gets the index's own DF (its column lengths); IDF is taken from
// df_global[t] and n_docs when df_global is given (a doc-range shard scored
// with the whole collection's statistics), else from the own DF.
__global__ void k_idf(const int64_t* __restrict__ indptr, int32_t vocab, int64_t n_docs,
                      int variant, double k1, double delta, const int32_t* __restrict__ df_global,
                      int32_t* __restrict__ df_out, double* __restrict__ idf_out,
                      double* __restrict__ s0_out, float* __restrict__ coef)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < vocab;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t df_own = indptr[t + 1] - indptr[t];
        const int64_t df = df_global ? (int64_t)df_global[t] : df_own;
        double w = idf_of(variant, (double)n_docs, (double)df);
        double s0, c;
        term_coef(variant, w, k1, delta, &c, &s0);
        df_out[t] = (int32_t)df_own;
        idf_out[t] = w;
        s0_out[t] = s0;
        coef[t] = (float)c;
    }
}

// ---- K7: scores ----------------------------------------------------------
// FP32 S(t,D) - S0(t) per entry (entry_score in device.cuh), written to the
// CSC and to the packed copy staged retrieval reads.
__global__ void k_score(const int32_t* __restrict__ run_pos, const int32_t* __restrict__ run_term,
                        const int32_t* __restrict__ indices, const uint32_t* __restrict__ d_nnz,
                        const float* __restrict__ coef, const float* __restrict__ len_factor,
                        int variant, ScoreConsts kc, const int64_t* __restrict__ indptr,
                        int32_t* __restrict__ tf_out, float* __restrict__ data,
                        uint2* __restrict__ posts)
{
    const int64_t nnz = *d_nnz;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    constexpr int U = 4;  // entries per thread and iteration, their loads issued together
    for (int64_t j0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j0 < nnz; j0 += U * stride) {
        int32_t tf[U], doc[U], term[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int64_t j = j0 + u * stride;
            const bool ok = j < nnz;
            tf[u] = ok ? run_pos[j + 1] - run_pos[j] : 0;
            doc[u] = ok ? indices[j] : 0;
            term[u] = ok ? run_term[j] : 0;
        }
        float a[U], c[U];
        int64_t c0[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const bool ok = j0 + u * stride < nnz;
            a[u] = ok ? len_factor[doc[u]] : 1.0f;
            c[u] = ok ? coef[term[u]] : 0.0f;
            c0[u] = ok ? indptr[term[u]] : 0;
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int64_t j = j0 + u * stride;
            if (j >= nnz)
                break;
            const float sc = entry_score(variant, (float)tf[u], a[u], c[u], kc);
            tf_out[j] = tf[u];
            data[j] = sc;
            posts[post_start(c0[u], term[u]) + (j - c0[u])] =
                make_uint2((uint32_t)doc[u], __float_as_uint(sc));
        }
    }
}

// The length factor of every document from |D| and a given Lavg (as
// k_doc_prep computes it).
__global__ void k_len_factor(const int32_t* __restrict__ doc_len, int64_t n_docs, int variant,
                             double k1, double b, double lavg, float* __restrict__ len_factor)
{
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < n_docs;
         d += (int64_t)gridDim.x * blockDim.x) {
        len_factor[d] = length_factor(variant, k1, b, (double)doc_len[d], lavg);
    }
}

// Scores of the stored entries from their TF, |D| and the term coefficients
// (a doc-range shard after the collection's statistics are known): the same
// arithmetic as k_score.  Each block takes a contiguous range of entries and
// finds the terms that range spans once; each entry then finds its term
// inside that span.
constexpr int kRescoreItems = 2048;  // entries per block
__global__ void k_rescore(const int64_t* __restrict__ indptr, int32_t vocab, int64_t nnz,
                          const int32_t* __restrict__ indices, const int32_t* __restrict__ tf,
                          const float* __restrict__ coef, const float* __restrict__ len_factor,
                          int variant, ScoreConsts kc, float* __restrict__ data,
                          uint2* __restrict__ posts)
{
    __shared__ int32_t span[2];
    auto term_of = [&](int64_t j, int32_t lo, int32_t hi) {  // last t in [lo, hi) with indptr[t] <= j
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if (indptr[mid] <= j)
                lo = mid;
            else
                hi = mid;
        }
        return lo;
    };
    for (int64_t j0 = (int64_t)blockIdx.x * kRescoreItems; j0 < nnz;
         j0 += (int64_t)gridDim.x * kRescoreItems) {
        const int64_t j1 = min(nnz, j0 + kRescoreItems);
        __syncthreads();  // the previous range's readers of span are done
        if (threadIdx.x == 0)
            span[0] = term_of(j0, 0, vocab);
        if (threadIdx.x == 32)
            span[1] = term_of(j1 - 1, 0, vocab) + 1;
        __syncthreads();
        const int32_t t_lo = span[0], t_hi = span[1];
        for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
            const int32_t t = term_of(j, t_lo, t_hi);
            const int32_t d = indices[j];
            const float sc = entry_score(variant, (float)tf[j], len_factor[d], coef[t], kc);
            data[j] = sc;
            const int64_t c0 = indptr[t];
            posts[post_start(c0, t) + (j - c0)] = make_uint2((uint32_t)d, __float_as_uint(sc));
        }
    }
}

// The padding slots of the packed layout: after column t up to the start of
// column t+1, and past the last column up to n_posts.
__global__ void k_pad_posts(const int64_t* __restrict__ indptr, int32_t vocab, int64_t n_posts,
                            uint2* __restrict__ posts)
{
    const uint2 pad = make_uint2(kPostPad, 0u);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= vocab;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t from, to;
        if (t < vocab) {
            from = post_start(indptr[t], t) + (indptr[t + 1] - indptr[t]);
            to = post_start(indptr[t + 1], t + 1);
        } else {
            from = post_start(indptr[vocab], vocab);
            to = n_posts;
        }
        for (int64_t p = from; p < to; p++)
            posts[p] = pad;
    }
}

// Packed entries from the CSC arrays (after an import): one thread per
// entry finds its column by a binary search over indptr.
__global__ void k_pack_posts(const int64_t* __restrict__ indptr, int32_t vocab, int64_t nnz,
                             const int32_t* __restrict__ indices, const float* __restrict__ data,
                             uint2* __restrict__ posts)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nnz;
         j += (int64_t)gridDim.x * blockDim.x) {
        int32_t lo = 0, hi = vocab;  // last t with indptr[t] <= j
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if (indptr[mid] <= j)
                lo = mid;
            else
                hi = mid;
        }
        const int64_t c0 = indptr[lo];
        posts[post_start(c0, lo) + (j - c0)] =
            make_uint2((uint32_t)indices[j], __float_as_uint(data[j]));
    }
}

// ---- memory --------------------------------------------------------------
cudaMemPool_t g_pools[64];
std::mutex g_pool_mu;

int pool_for_device(int dev, cudaMemPool_t* out)
{
    std::lock_guard<std::mutex> g(g_pool_mu);
    if (dev < 0 || dev >= 64)
        return set_error(BM25_E_CUDA, "device ordinal %d out of range", dev);
    if (!g_pools[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        BM25_CUDA_TRY(cudaMemPoolCreate(&g_pools[dev], &props));
        uint64_t keep = ~0ull;  // keep freed blocks for the next build
        BM25_CUDA_TRY(cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &keep));
    }
    *out = g_pools[dev];
    return BM25_OK;
}

template <typename T>
int pool_alloc(T** p, int64_t count, cudaMemPool_t pool, cudaStream_t s)
{
    size_t bytes = (size_t)(count > 0 ? count : 1) * sizeof(T);
    if (forced_alloc_failure()) {
        *p = nullptr;
        return set_error(BM25_E_OOM, "device allocation of %zu bytes failed (forced by "
                         "bm25_debug_fail_allocs)", bytes);
    }
    cudaError_t e = cudaMallocFromPoolAsync((void**)p, bytes, pool, s);
    if (e != cudaSuccess) {
        *p = nullptr;
        return set_error(e == cudaErrorMemoryAllocation ? BM25_E_OOM : BM25_E_CUDA,
                         "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    return BM25_OK;
}

struct TempSet {
    std::vector<void*> ptrs;
    cudaStream_t s;
    explicit TempSet(cudaStream_t st) : s(st) {}
    template <typename T>
    int alloc(T** p, int64_t count, cudaMemPool_t pool)
    {
        int r = pool_alloc(p, count, pool, s);
        if (r == BM25_OK)
            ptrs.push_back((void*)*p);
        return r;
    }
    ~TempSet()
    {
        for (void* p : ptrs)
            cudaFreeAsync(p, s);
    }
};

int grid_for(int64_t n, int threads, int max_blocks)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1)
        b = 1;
    if (b > max_blocks)
        b = max_blocks;
    return (int)b;
}

}  // namespace

int pool_for_current_device(cudaMemPool_t* out)
{
    int dev = 0;
    BM25_CUDA_TRY(cudaGetDevice(&dev));
    return pool_for_device(dev, out);
}

// Index arrays live in the library's stream-ordered pool (freed blocks are
// kept for the next build).  Sizes come from the index's scalars.
int alloc_index_arrays(bm25_index* ix, cudaStream_t s, bool fixed, bool per_entry)
{
    cudaMemPool_t pool;
    BM25_TRY(pool_for_current_device(&pool));
    if (fixed) {
        BM25_TRY(pool_alloc(&ix->indptr, (int64_t)ix->vocab + 1, pool, s));
        BM25_TRY(pool_alloc(&ix->df, ix->vocab, pool, s));
        BM25_TRY(pool_alloc(&ix->doc_len, ix->n_docs, pool, s));
        BM25_TRY(pool_alloc(&ix->idf, ix->vocab, pool, s));
        BM25_TRY(pool_alloc(&ix->s0, ix->vocab, pool, s));
        BM25_TRY(pool_alloc(&ix->status, 1, pool, s));
        BM25_CUDA_TRY(cudaMemsetAsync(ix->status, 0, sizeof(int), s));
    }
    if (per_entry) {
        BM25_TRY(pool_alloc(&ix->indices, ix->nnz, pool, s));
        BM25_TRY(pool_alloc(&ix->data, ix->nnz, pool, s));
        BM25_TRY(pool_alloc(&ix->tf, ix->nnz, pool, s));
        ix->n_posts = ix->nnz + ix->vocab + 3;
        BM25_TRY(pool_alloc(&ix->posts, ix->n_posts, pool, s));
    }
    return BM25_OK;
}

int pack_posts(bm25_index* ix, cudaStream_t s)
{
    DeviceInfo di;
    BM25_TRY(device_info(&di));
    const int max_blocks = di.sm_count * 16;
    {
        ProfileScope ps_("k_pad_posts", s);
        k_pad_posts<<<grid_for((int64_t)ix->vocab + 1, 256, max_blocks), 256, 0, s>>>(
            ix->indptr, ix->vocab, ix->n_posts, ix->posts);
    }
    count_launch();
    BM25_LAUNCH_CHECK();
    if (ix->nnz > 0) {
        ProfileScope ps_("k_pack_posts", s);
        k_pack_posts<<<grid_for(ix->nnz, 256, max_blocks), 256, 0, s>>>(
            ix->indptr, ix->vocab, ix->nnz, ix->indices, ix->data, ix->posts);
        count_launch();
        BM25_LAUNCH_CHECK();
    }
    return BM25_OK;
}

// Rescores a built index with statistics of a larger collection (a doc-range
// shard): IDF and S0 from df_global (device, [vocab]; NULL = the index's own
// DF) and n_docs_global, Lavg = n_tokens_global / n_docs_global, then every
// stored S(t,D) - S0(t) and its packed copy with the arithmetic of the build.
int rescore_index(bm25_index* ix, const int32_t* df_global, int64_t n_docs_global,
                  int64_t n_tokens_global, cudaStream_t s)
{
    DeviceInfo di;
    BM25_TRY(device_info(&di));
    cudaMemPool_t pool;
    BM25_TRY(pool_for_device(di.device, &pool));
    const int max_blocks = di.sm_count * 16;
    const double lavg = (double)n_tokens_global / (double)n_docs_global;
    TempSet tmp(s);
    float* len_factor = nullptr;
    float* coef = nullptr;
    BM25_TRY(tmp.alloc(&len_factor, ix->n_docs, pool));
    BM25_TRY(tmp.alloc(&coef, ix->vocab, pool));
    {
        ProfileScope ps_("k_len_factor", s);
        k_len_factor<<<grid_for(ix->n_docs, 256, max_blocks), 256, 0, s>>>(
            ix->doc_len, ix->n_docs, ix->variant, ix->k1, ix->b, lavg, len_factor);
    }
    count_launch();
    BM25_LAUNCH_CHECK();
    {
        ProfileScope ps_("k_idf", s);
        k_idf<<<grid_for(ix->vocab, 256, max_blocks), 256, 0, s>>>(
            ix->indptr, ix->vocab, n_docs_global, ix->variant, ix->k1, ix->delta, df_global,
            ix->df, ix->idf, ix->s0, coef);
    }
    count_launch();
    BM25_LAUNCH_CHECK();
    if (ix->nnz > 0) {
        const int64_t blocks = (ix->nnz + kRescoreItems - 1) / kRescoreItems;
        ProfileScope ps_("k_rescore", s);
        k_rescore<<<(unsigned)std::min<int64_t>(blocks, max_blocks), 256, 0, s>>>(
            ix->indptr, ix->vocab, ix->nnz, ix->indices, ix->tf, coef, len_factor, ix->variant,
            score_consts(ix->k1, ix->delta), ix->data, ix->posts);
        count_launch();
        BM25_LAUNCH_CHECK();
    }
    ix->lavg = lavg;
    ix->stat_docs = n_docs_global;
    ix->stat_tokens = n_tokens_global;
    return BM25_OK;
}

namespace {

// The largest TF and |D| of an index (atomicMax into mx[0], mx[1]).
__global__ void k_max_tf_len(const int32_t* __restrict__ tf, int64_t nnz,
                             const int32_t* __restrict__ doc_len, int64_t n_docs, int32_t* mx)
{
    int32_t a = 0, b = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nnz; j += stride)
        a = max(a, tf[j]);
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < n_docs; d += stride)
        b = max(b, doc_len[d]);
    a = __reduce_max_sync(0xffffffffu, a);
    b = __reduce_max_sync(0xffffffffu, b);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&mx[0], a);
        atomicMax(&mx[1], b);
    }
}

// Lazy postings: each packed entry's second word becomes TF | |D| << 16
// (packed) or TF; padding slots are copied as they are.
__global__ void k_lazy_posts(const int64_t* __restrict__ indptr, int32_t vocab, int64_t nnz,
                             const int32_t* __restrict__ indices, const int32_t* __restrict__ tf,
                             const int32_t* __restrict__ doc_len, int packed,
                             uint2* __restrict__ posts_lazy)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nnz;
         j += (int64_t)gridDim.x * blockDim.x) {
        int32_t lo = 0, hi = vocab;  // last t with indptr[t] <= j
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if (indptr[mid] <= j)
                lo = mid;
            else
                hi = mid;
        }
        const int64_t c0 = indptr[lo];
        const int32_t d = indices[j];
        const uint32_t w =
            packed ? ((uint32_t)tf[j] | ((uint32_t)doc_len[d] << 16)) : (uint32_t)tf[j];
        posts_lazy[post_start(c0, lo) + (j - c0)] = make_uint2((uint32_t)d, w);
    }
}

}  // namespace

int enable_lazy(bm25_index* ix, cudaStream_t s)
{
    if (ix->posts_lazy)
        return BM25_OK;
    DeviceInfo di;
    BM25_TRY(device_info(&di));
    cudaMemPool_t pool;
    BM25_TRY(pool_for_device(di.device, &pool));
    const int max_blocks = di.sm_count * 16;
    int32_t h_mx[2] = {0, 0};
    {
        TempSet tmp(s);
        int32_t* mx = nullptr;
        BM25_TRY(tmp.alloc(&mx, 2, pool));
        BM25_CUDA_TRY(cudaMemsetAsync(mx, 0, 2 * sizeof(int32_t), s));
        {
            ProfileScope ps_("k_max_tf_len", s);
            k_max_tf_len<<<grid_for(std::max(ix->nnz, ix->n_docs), 256, max_blocks), 256, 0, s>>>(
                ix->tf, ix->nnz, ix->doc_len, ix->n_docs, mx);
        }
        count_launch();
        BM25_LAUNCH_CHECK();
        BM25_CUDA_TRY(cudaMemcpyAsync(h_mx, mx, sizeof(h_mx), cudaMemcpyDeviceToHost, s));
        BM25_CUDA_TRY(cudaStreamSynchronize(s));
    }
    const bool packed = h_mx[0] <= 0xffff && h_mx[1] <= 0xffff;
    uint2* pl = nullptr;
    BM25_TRY(pool_alloc(&pl, ix->n_posts, pool, s));
    cudaError_t e = cudaMemcpyAsync(pl, ix->posts, sizeof(uint2) * (size_t)ix->n_posts,
                                    cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && ix->nnz > 0) {
        {
            ProfileScope ps_("k_lazy_posts", s);
            k_lazy_posts<<<grid_for(ix->nnz, 256, max_blocks), 256, 0, s>>>(
                ix->indptr, ix->vocab, ix->nnz, ix->indices, ix->tf, ix->doc_len, packed ? 1 : 0,
                pl);
        }
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFreeAsync(pl, s);
        return set_error(BM25_E_CUDA, "building the lazy postings failed: %s",
                         cudaGetErrorString(e));
    }
    ix->posts_lazy = pl;
    ix->lazy_packed = packed;
    return BM25_OK;
}

void free_index_arrays(bm25_index* ix, cudaStream_t s)
{
    if (ix->posts_lazy)
        cudaFreeAsync(ix->posts_lazy, s);
    ix->posts_lazy = nullptr;
    void* ps[] = {ix->indptr, ix->indices, ix->data, ix->tf, ix->df,
                  ix->doc_len, ix->idf, ix->s0, ix->status, ix->posts};
    for (void* p : ps)
        if (p)
            cudaFreeAsync(p, s);
    ix->indptr = nullptr;
    ix->indices = nullptr;
    ix->data = nullptr;
    ix->tf = nullptr;
    ix->df = nullptr;
    ix->doc_len = nullptr;
    ix->idf = nullptr;
    ix->s0 = nullptr;
    ix->status = nullptr;
    ix->posts = nullptr;
    ix->n_posts = 0;
}

int build_index_device(const int32_t* d_tokens, int64_t n_tokens, const int64_t* d_offsets,
                       int64_t n_docs, int32_t vocab, int variant, double k1, double b,
                       double delta, cudaStream_t s, bm25_index** out)
{
    DeviceInfo di;
    BM25_TRY(device_info(&di));
    cudaMemPool_t pool;
    BM25_TRY(pool_for_device(di.device, &pool));
    const int max_blocks = di.sm_count * 16;
    const double lavg = (double)n_tokens / (double)n_docs;
    const int64_t T = n_tokens;

    bm25_index* ix = new bm25_index();
    ix->device = di.device;
    ix->n_docs = n_docs;
    ix->n_tokens = n_tokens;
    ix->vocab = vocab;
    ix->variant = variant;
    ix->k1 = k1;
    ix->b = b;
    ix->delta = delta;
    ix->lavg = lavg;
    ix->stat_docs = n_docs;
    ix->stat_tokens = n_tokens;
    auto fail = [&](int code) {
        free_index_arrays(ix, s);
        delete ix;
        return code;
    };
    {
        int r = alloc_index_arrays(ix, s, true, false);  // arrays sized by V and N
        if (r != BM25_OK)
            return fail(r);
    }
    int rc = BM25_OK;
    uint32_t h_nnz = 0;
    int h_status = 0;
    {
        TempSet tmp(s);
        int32_t* tok_doc = nullptr;
        float* len_factor = nullptr;
        uint32_t *ka = nullptr, *va = nullptr, *kb = nullptr, *vb = nullptr;
        uint32_t *counts = nullptr, *scan_tmp = nullptr, *tile_heads = nullptr, *d_total = nullptr;
        int32_t *run_pos = nullptr, *run_term = nullptr;
        float* coef = nullptr;
        const int64_t n_tiles = (T + kSortTile - 1) / kSortTile;
        int nbits = 1;
        while (nbits < 31 && ((int64_t)1 << nbits) < (int64_t)vocab)
            nbits++;
        const int passes = (nbits + kMaxDigitBits - 1) / kMaxDigitBits;
        const int dbits = (nbits + passes - 1) / passes;
        // the sort's grid: one wave of resident downsweep blocks (both sort
        // kernels of a pass use it: it fixes which tiles each block owns)
        if (cudaFuncSetAttribute(k_radix_downsweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSortedTileBytes) != cudaSuccess)
            return fail(set_error(BM25_E_CUDA, "cannot give the sort kernel %d bytes of shared "
                                               "memory", kSortedTileBytes));
        int sort_bps = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sort_bps, k_radix_downsweep, kSortThreads,
                                                          kSortedTileBytes) != cudaSuccess)
            sort_bps = 1;
        const int64_t sort_grid = std::max<int64_t>(
            1, std::min<int64_t>(n_tiles, (int64_t)std::max(sort_bps, 1) * di.sm_count));
        // upsweep blocks per downsweep block: about 8 resident 256-thread
        // blocks per SM in all
        const int sort_split = (int)std::max<int64_t>(
            1, std::min<int64_t>((8LL * di.sm_count + sort_grid - 1) / sort_grid,
                                 n_tiles / sort_grid));
        const int64_t ncounts = ((int64_t)1 << dbits) * sort_grid * sort_split;
        int r = BM25_OK;
        if (r == BM25_OK) r = tmp.alloc(&tok_doc, T, pool);
        if (r == BM25_OK) r = tmp.alloc(&len_factor, n_docs, pool);
        if (r == BM25_OK) r = tmp.alloc(&ka, T, pool);
        if (r == BM25_OK) r = tmp.alloc(&va, T, pool);
        if (r == BM25_OK) r = tmp.alloc(&kb, T, pool);
        if (r == BM25_OK) r = tmp.alloc(&counts, ncounts, pool);
        if (r == BM25_OK) r = tmp.alloc(&scan_tmp, scan_tmp_elems(ncounts > n_tiles ? ncounts : n_tiles), pool);
        if (r == BM25_OK) r = tmp.alloc(&tile_heads, n_tiles, pool);
        if (r == BM25_OK) r = tmp.alloc(&d_total, 2, pool);
        if (r == BM25_OK) r = tmp.alloc(&coef, vocab, pool);
        if (r != BM25_OK)
            return fail(r);
        vb = (uint32_t*)tok_doc;  // reused once pass 0 has consumed the doc ids

        {

            ProfileScope ps_("k_doc_prep", s);

            k_doc_prep<<<grid_for(n_docs, 256, max_blocks), 256, 0, s>>>(
                d_offsets, n_docs, T, tok_doc, ix->doc_len, len_factor, variant, k1, b, lavg,
                ix->status);

        }
        count_launch();
        BM25_LAUNCH_CHECK();

        const uint32_t* kin = (const uint32_t*)d_tokens;
        const uint32_t* vin = (const uint32_t*)tok_doc;
        if (T > 0) {
            for (int pass = 0; pass < passes; pass++) {
                uint32_t* kout = (pass % 2 == 0) ? ka : kb;
                uint32_t* vout = (pass % 2 == 0) ? va : vb;
                const int shift = pass * dbits;
                const int bits = (nbits - shift < dbits) ? nbits - shift : dbits;
                {
                    ProfileScope ps_("k_radix_upsweep", s);
                    k_radix_upsweep<<<(unsigned)(sort_grid * sort_split), kSortThreads, 0, s>>>(
                        kin, T, shift, bits, counts, n_tiles, sort_split,
                        pass == 0 ? (uint32_t)vocab : 0u, ix->status);
                }
                count_launch();
                BM25_LAUNCH_CHECK();
                BM25_TRY(exclusive_scan_u32(counts, counts,
                                            ((int64_t)1 << bits) * sort_grid * sort_split,
                                            d_total, scan_tmp, s));
                {
                    ProfileScope ps_("k_radix_downsweep", s);
                    k_radix_downsweep<<<(unsigned)sort_grid, kSortThreads, kSortedTileBytes, s>>>(
                        kin, vin, kout, vout, T, shift, bits, counts, n_tiles, sort_split);
                }
                count_launch();
                BM25_LAUNCH_CHECK();
                kin = kout;
                vin = vout;
            }
            {
                ProfileScope ps_("k_rle_count", s);
                k_rle_count<<<(unsigned)n_tiles, kSortThreads, 0, s>>>(kin, vin, T, tile_heads);
            }
            count_launch();
            BM25_LAUNCH_CHECK();
            BM25_TRY(exclusive_scan_u32(tile_heads, tile_heads, n_tiles, d_total, scan_tmp, s));
        } else {
            BM25_CUDA_TRY(cudaMemsetAsync(d_total, 0, sizeof(uint32_t), s));
        }
        BM25_CUDA_TRY(cudaMemcpyAsync(&h_nnz, d_total, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        BM25_CUDA_TRY(cudaMemcpyAsync(&h_status, ix->status, sizeof(int), cudaMemcpyDeviceToHost, s));
        BM25_CUDA_TRY(cudaStreamSynchronize(s));
        if (h_status != 0) {
            rc = set_error(h_status, "index build: a token id is outside [0, %d) or the doc "
                                     "offsets are malformed", vocab);
        } else {
            const int64_t nnz = h_nnz;
            ix->nnz = nnz;
            int r2 = alloc_index_arrays(ix, s, false, true);  // arrays sized by nnz
            if (r2 == BM25_OK) r2 = tmp.alloc(&run_pos, nnz + 1, pool);
            if (r2 == BM25_OK) r2 = tmp.alloc(&run_term, nnz, pool);
            if (r2 != BM25_OK)
                return fail(r2);
            if (T > 0) {
                {
                    ProfileScope ps_("k_rle_emit", s);
                    k_rle_emit<<<(unsigned)n_tiles, kSortThreads, 0, s>>>(
                        kin, vin, T, tile_heads, d_total, run_pos, run_term, ix->indices);
                }
                count_launch();
                BM25_LAUNCH_CHECK();
            }
            {
                ProfileScope ps_("k_indptr", s);
                k_indptr<<<grid_for((int64_t)vocab + 1, 256, max_blocks), 256, 0, s>>>(
                    run_term, d_total, vocab, ix->indptr);
            }
            {
                ProfileScope ps_("k_idf", s);
                k_idf<<<grid_for(vocab, 256, max_blocks), 256, 0, s>>>(
                    ix->indptr, vocab, n_docs, variant, k1, delta, nullptr, ix->df, ix->idf,
                    ix->s0, coef);
            }
            {
                ProfileScope ps_("k_pad_posts", s);
                k_pad_posts<<<grid_for((int64_t)vocab + 1, 256, max_blocks), 256, 0, s>>>(
                    ix->indptr, vocab, ix->n_posts, ix->posts);
            }
            count_launch(3);
            BM25_LAUNCH_CHECK();
            if (nnz > 0) {
                {
                    ProfileScope ps_("k_score", s);
                    k_score<<<grid_for(nnz, 256, max_blocks), 256, 0, s>>>(
                        run_pos, run_term, ix->indices, d_total, coef, len_factor, variant,
                        score_consts(k1, delta), ix->indptr, ix->tf, ix->data, ix->posts);
                }
                count_launch();
                BM25_LAUNCH_CHECK();
            }
        }
    }  // temporaries are released (stream-ordered) here
    if (rc != BM25_OK)
        return fail(rc);
    *out = ix;
    return BM25_OK;
}

}  // namespace bm25
