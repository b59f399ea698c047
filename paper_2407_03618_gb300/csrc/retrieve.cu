// Batched top-k retrieval over the eager term-major index (arXiv 2407.03618
// Sec. 2 "Assigning Query Scores" and "Top-k selection"; Sec. 2.1 for the
// shift added back to every returned score).
//
// Doc-tiled shared-memory path, four launches per call:
//   R0 k_query_prep   sum_i S0(q_i) per query in FP64; token / offset checks
//   R1 k_seg_bounds   for every query token and every doc-tile boundary, the
//                     first posting of the token's column at or past the
//                     boundary (binary search: doc ids ascend in a column)
//   R2 k_tile_topk    persistent CTAs over (query, doc tile) items: each item
//                     scatter-adds its postings into FP32 accumulators in
//                     shared memory, marks touched documents in a bitmask,
//                     and radix-selects the tile's best k' candidates,
//                     including the lowest-id untouched documents (score 0)
//   R3 k_merge        per query: radix-select k' of the tiles' candidates,
//                     sort them and write (id, score + shift)
#include <algorithm>
#include <cstdio>

#include "device.cuh"
#include "internal.h"

namespace bm25 {
namespace {

typedef unsigned long long u64;

constexpr int kTileThreads = 512;
constexpr int kTokChunk = 64;     // query tokens staged in shared memory at a time
constexpr int kMergeThreads = 512;

// ---- R0 ---------------------------------------------------------------------
__global__ void k_query_prep(const int32_t* __restrict__ q_tokens, int64_t n_tok,
                             const int64_t* __restrict__ q_off, int32_t nq,
                             const double* __restrict__ s0, int32_t vocab,
                             double* __restrict__ shift, uint32_t* __restrict__ thresh,
                             uint32_t* __restrict__ ccount, int* status)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq;
         q += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = q_off[q], hi = q_off[q + 1];
        if (lo < 0 || hi < lo || hi > n_tok || (q == 0 && lo != 0) ||
            (q == nq - 1 && hi != n_tok))
            set_status(status, BM25_E_TOKEN_RANGE);
        lo = lo < 0 ? 0 : (lo > n_tok ? n_tok : lo);
        hi = hi < lo ? lo : (hi > n_tok ? n_tok : hi);
        double sum = 0.0;
        for (int64_t m = lo; m < hi; m++) {
            int32_t t = q_tokens[m];
            if (t < 0 || t >= vocab) {
                set_status(status, BM25_E_TOKEN_RANGE);
                continue;
            }
            sum += s0[t];
        }
        shift[q] = sum;
        thresh[q] = 0u;  // below every real score key
        ccount[q] = 0u;
    }
}

// ---- R1 ---------------------------------------------------------------------
// seg[m * (n_tiles + 1) + j] = first position p in column q_tokens[m] with
// indices[p] >= j * W (j = n_tiles gives the column end).  A token outside
// the vocabulary gets an empty column.
__global__ void k_seg_bounds(const int32_t* __restrict__ q_tokens, int64_t n_tok,
                             const int64_t* __restrict__ indptr,
                             const int32_t* __restrict__ indices, int32_t vocab, int32_t W,
                             int32_t n_tiles, int32_t* __restrict__ seg)
{
    const int64_t per = (int64_t)n_tiles + 1;
    const int64_t total = n_tok * per;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t m = i / per;
        int32_t j = (int32_t)(i - m * per);
        int32_t t = q_tokens[m];
        int64_t lo = 0, hi = 0;
        if (t >= 0 && t < vocab) {
            lo = indptr[t];
            hi = indptr[t + 1];
        }
        if (j == 0) {
            seg[i] = (int32_t)lo;
        } else if (j == n_tiles) {
            seg[i] = (int32_t)hi;
        } else {
            const int32_t target = j * W;
            while (lo < hi) {
                int64_t mid = (lo + hi) >> 1;
                if (indices[mid] < target)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            seg[i] = (int32_t)lo;
        }
    }
}

// ---- block-level radix select of the k largest 64-bit keys ------------------
// MSD, 8-bit digits.  Each pass histograms the digit of the candidates that
// still match the selected prefix, picks the bucket holding the k-th largest
// key, and stops as soon as that bucket is taken whole.  Keys are distinct
// (the low word is the doc id), so exactly k keys end up at or above the
// final prefix.
struct SelectState {
    uint32_t hist[256];
    u64 prefix, pmask, minkey;
    uint32_t need, bucket, ctr, cnt, tau, base;
    uint32_t red[33];
};

// Finds the bucket (warp 0).  Bins are visited from digit 255 down.
__device__ __forceinline__ void select_bucket(SelectState& st, int shift)
{
    const int lane = threadIdx.x & 31;
    // lane l owns digits 255-8l .. 248-8l
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < 8; i++)
        s += st.hist[255 - 8 * lane - i];
    uint32_t inc = warp_inclusive_sum(s);
    uint32_t before = inc - s;
    uint32_t need = st.need;
    bool mine = before < need && need <= inc;
    if (mine) {
        uint32_t cum = before;
        int d = 255 - 8 * lane;
        for (int i = 0; i < 8; i++, d--) {
            uint32_t h = st.hist[d];
            if (cum + h >= need)
                break;
            cum += h;
        }
        st.prefix |= (u64)d << shift;
        st.pmask |= (u64)0xff << shift;
        st.need = need - cum;
        st.bucket = st.hist[d];
    }
}

// for_each(f) must call f(key) for every candidate owned by this thread.
// emit(key) is called for each of the min(k, n) selected keys (any order).
// n = number of candidates.  All threads of the block must call this.
template <class ForEach, class Emit>
__device__ void block_select(SelectState& st, uint32_t n, uint32_t k, ForEach for_each,
                             Emit emit)
{
    if (n <= k) {
        for_each([&](u64 key) { emit(key); });
        __syncthreads();
        return;
    }
    if (threadIdx.x == 0) {
        st.prefix = 0;
        st.pmask = 0;
        st.need = k;
    }
    for (int pass = 0; pass < 8; pass++) {
        const int shift = 56 - 8 * pass;
        for (int i = threadIdx.x; i < 256; i += blockDim.x)
            st.hist[i] = 0;
        __syncthreads();
        const u64 pm = st.pmask, pf = st.prefix;
        for_each([&](u64 key) {
            if ((key & pm) == pf)
                atomicAdd(&st.hist[(key >> shift) & 0xff], 1u);
        });
        __syncthreads();
        if (threadIdx.x < 32)
            select_bucket(st, shift);
        __syncthreads();
        if (st.bucket == st.need)
            break;
    }
    const u64 pm = st.pmask, pf = st.prefix;
    for_each([&](u64 key) {
        if ((key & pm) >= pf)
            emit(key);
    });
    __syncthreads();
}

// Same selection over an indexable candidate set: get(i) returns the key of
// candidate i < n.  The loops are warp-uniform, so histogram updates are
// aggregated per warp with __match_any_sync (candidates that share a score
// prefix would otherwise serialise on one counter).
template <class Get, class Emit>
__device__ void block_select_idx(SelectState& st, uint32_t n, uint32_t k, Get get, Emit emit)
{
    const int lane = threadIdx.x & 31;
    const uint32_t stride = blockDim.x;
    const uint32_t base0 = threadIdx.x & ~31u;
    if (n <= k) {
        for (uint32_t i = threadIdx.x; i < n; i += stride)
            emit(get(i));
        __syncthreads();
        return;
    }
    if (threadIdx.x == 0) {
        st.prefix = 0;
        st.pmask = 0;
        st.need = k;
    }
    for (int pass = 0; pass < 8; pass++) {
        const int shift = 56 - 8 * pass;
        for (int i = threadIdx.x; i < 256; i += blockDim.x)
            st.hist[i] = 0;
        __syncthreads();
        const u64 pm = st.pmask, pf = st.prefix;
        for (uint32_t b = base0; b < n; b += stride) {
            const uint32_t i = b + lane;
            uint32_t dg = 0xffffffffu;
            if (i < n) {
                u64 key = get(i);
                if ((key & pm) == pf)
                    dg = (uint32_t)(key >> shift) & 0xffu;
            }
            uint32_t peers = __match_any_sync(0xffffffffu, dg);
            if (dg != 0xffffffffu && (peers & lanemask_lt()) == 0)
                atomicAdd(&st.hist[dg], (uint32_t)__popc(peers));
        }
        __syncthreads();
        if (threadIdx.x < 32)
            select_bucket(st, shift);
        __syncthreads();
        if (st.bucket == st.need)
            break;
    }
    const u64 pm = st.pmask, pf = st.prefix;
    for (uint32_t i = threadIdx.x; i < n; i += stride) {
        u64 key = get(i);
        if ((key & pm) >= pf)
            emit(key);
    }
    __syncthreads();
}

// ---- R2 -----------------------------------------------------------------------
// Dynamic shared memory: acc[W] FP32 | mask[W/32] | SelectState | token stage.
constexpr uint32_t kSurvCap = 2048;  // survivors kept in shared memory per item

struct TileStage {
    int32_t lo[kTokChunk];
    int32_t pre[kTokChunk + 1];
    uint32_t scan[33];
    uint32_t n_surv, n_pos;
    uint16_t surv[kSurvCap];  // local doc ids of the item's candidates
};

__global__ void __launch_bounds__(kTileThreads, 3)
    k_tile_topk(const int32_t* __restrict__ q_tokens, int64_t n_tok,
                const int64_t* __restrict__ q_off, int32_t nq, int64_t n_docs,
                const int32_t* __restrict__ indices, const float* __restrict__ data,
                const int32_t* __restrict__ seg, int32_t W, int32_t n_tiles, int32_t kprime,
                uint32_t* __restrict__ thresh, uint32_t* __restrict__ ccount,
                u64* __restrict__ cand, int64_t cand_cap)
{
    extern __shared__ __align__(16) unsigned char smem[];
    float* acc = reinterpret_cast<float*>(smem);
    uint32_t* mask = reinterpret_cast<uint32_t*>(acc + W);
    SelectState& st = *reinterpret_cast<SelectState*>(mask + W / 32);
    TileStage& ts = *reinterpret_cast<TileStage*>(&st + 1);

    const int tid = threadIdx.x;
    for (int i = tid; i < W; i += kTileThreads)
        acc[i] = 0.0f;
    for (int i = tid; i < W / 32; i += kTileThreads)
        mask[i] = 0u;
    __syncthreads();

    const int64_t n_items = (int64_t)nq * n_tiles;
    const int64_t per = (int64_t)n_tiles + 1;
    // tile-major order: tile 0 of every query first, so that the running
    // per-query threshold is usually known when a query's later tiles run,
    // and the segments in flight at once all belong to one doc tile
    auto item_qt = [&](int64_t item, int64_t& q, int32_t& tile) {
        tile = (int32_t)(item / nq);
        q = item - (int64_t)tile * nq;
    };
    // warp 0 prefetches the first token chunk's segment bounds of its next
    // item (lane l: tokens 2l, 2l+1) and thread 0 the query's threshold
    int32_t pf_lo0 = 0, pf_lo1 = 0, pf_hi0 = 0, pf_hi1 = 0;
    uint32_t pf_tau = 0;
#define BM25_PREFETCH(ITEM)                                                          \
    do {                                                                             \
        const int64_t it_ = (ITEM);                                                  \
        if (tid < 32 && it_ < n_items) {                                             \
            int64_t q_;                                                              \
            int32_t t_;                                                              \
            item_qt(it_, q_, t_);                                                    \
            int64_t a_ = q_off[q_], b_ = q_off[q_ + 1];                              \
            a_ = a_ < 0 ? 0 : (a_ > n_tok ? n_tok : a_);                             \
            b_ = b_ < a_ ? a_ : (b_ > n_tok ? n_tok : b_);                           \
            const int64_t m_ = a_ + 2 * tid;                                         \
            pf_lo0 = pf_hi0 = pf_lo1 = pf_hi1 = 0;                                   \
            if (m_ < b_) {                                                           \
                pf_lo0 = seg[m_ * per + t_];                                         \
                pf_hi0 = seg[m_ * per + t_ + 1];                                     \
            }                                                                        \
            if (m_ + 1 < b_) {                                                       \
                pf_lo1 = seg[(m_ + 1) * per + t_];                                   \
                pf_hi1 = seg[(m_ + 1) * per + t_ + 1];                               \
            }                                                                        \
            if (tid == 0)                                                            \
                pf_tau = *(volatile uint32_t*)&thresh[q_];                           \
        }                                                                            \
    } while (0)
    BM25_PREFETCH(blockIdx.x);

    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        int64_t q;
        int32_t tile;
        item_qt(item, q, tile);
        const int64_t d0 = (int64_t)tile * W;
        const int32_t wd = (int32_t)min((int64_t)W, n_docs - d0);
        const int32_t nwords = (wd + 31) >> 5;
        int64_t m0 = q_off[q], m1 = q_off[q + 1];
        m0 = m0 < 0 ? 0 : (m0 > n_tok ? n_tok : m0);
        m1 = m1 < m0 ? m0 : (m1 > n_tok ? n_tok : m1);
        const uint32_t my_tau = pf_tau;  // thread 0's copy is the one used

        // scatter-add the item's postings, a chunk of query tokens at a time
        for (int64_t mb = m0; mb < m1; mb += kTokChunk) {
            const int cnt = (int)min((int64_t)kTokChunk, m1 - mb);
            if (tid < 32) {
                int32_t len[2];
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int i = 2 * tid + h;
                    int32_t l = 0, hh = 0;
                    if (mb == m0) {  // prefetched
                        l = h ? pf_lo1 : pf_lo0;
                        hh = h ? pf_hi1 : pf_hi0;
                    } else if (i < cnt) {
                        const int32_t* sg = seg + (mb + i) * per + tile;
                        l = sg[0];
                        hh = sg[1];
                    }
                    if (i >= cnt)
                        l = hh = 0;
                    len[h] = hh - l;
                    ts.lo[i] = l;
                }
                int32_t s2 = len[0] + len[1];
                int32_t inc = warp_inclusive_sum(s2);
                ts.pre[2 * tid] = inc - s2;
                ts.pre[2 * tid + 1] = inc - s2 + len[0];
                if (tid == 31)
                    ts.pre[kTokChunk] = inc;
            }
            if (mb == m0)
                BM25_PREFETCH(item + gridDim.x);  // overlaps with this item's work
            __syncthreads();
            const int32_t total = ts.pre[kTokChunk];
            constexpr int U = 4;  // postings in flight per thread
            for (int32_t e0 = tid; e0 < total; e0 += U * kTileThreads) {
                int32_t dd[U];
                float vv[U];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int32_t e = e0 + u * kTileThreads;
                    dd[u] = -1;
                    if (e < total) {
                        int a = 0, b = cnt;  // pre[a] <= e < pre[b]
                        while (b - a > 1) {
                            int mid = (a + b) >> 1;
                            if (ts.pre[mid] <= e)
                                a = mid;
                            else
                                b = mid;
                        }
                        const int32_t j = ts.lo[a] + (e - ts.pre[a]);
                        dd[u] = __ldg(indices + j) - (int32_t)d0;
                        vv[u] = __ldg(data + j);
                    }
                }
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int32_t d = dd[u];
                    if ((uint32_t)d < (uint32_t)wd) {  // holds for any well-formed index
                        atomicAdd(&acc[d], vv[u]);
                        atomicOr(&mask[d >> 5], 1u << (d & 31));
                    }
                }
            }
            __syncthreads();
        }
        if (m0 == m1)
            BM25_PREFETCH(item + gridDim.x);

        // ---- selection ------------------------------------------------------
        // tau = the query's running threshold: some tile already holds k'
        // documents scoring at least tau, so a document below tau cannot be
        // in the top k' (documents AT tau can, through the doc-id tie rule).
        if (tid == 0) {
            st.tau = my_tau;
            st.ctr = 0;
            st.minkey = ~0ull;
            ts.n_surv = 0;
            ts.n_pos = 0;
        }
        __syncthreads();
        const uint32_t tau = st.tau;
        const uint32_t kp = (uint32_t)min(kprime, wd);
        {
            uint32_t pos = 0;
            for (int w = tid; w < nwords; w += kTileThreads) {
                uint32_t bits = mask[w];
                while (bits) {
                    const int bpos = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const int d = (w << 5) + bpos;
                    const float a = acc[d];
                    pos += (a > 0.0f);
                    if (order_f32(a) >= tau) {
                        uint32_t slot = atomicAdd(&ts.n_surv, 1u);
                        if (slot < kSurvCap)
                            ts.surv[slot] = (uint16_t)d;
                    }
                }
            }
            pos = warp_sum(pos);
            if ((tid & 31) == 0 && pos)
                atomicAdd(&ts.n_pos, pos);
        }
        __syncthreads();
        // Untouched documents score exactly 0.  They can enter the tile's top
        // k' only if 0 clears tau and fewer than k' touched documents score
        // above 0; then the k' lowest-id untouched ones join the candidates.
        if (tau <= 0x80000000u && ts.n_pos < kp) {
            uint32_t carry = 0;
            for (int w0 = 0; w0 < nwords && carry < kp; w0 += kTileThreads) {
                const int w = w0 + tid;
                uint32_t zeros = 0;
                if (w < nwords) {
                    uint32_t valid = (w == nwords - 1 && (wd & 31)) ? ((1u << (wd & 31)) - 1u)
                                                                    : 0xffffffffu;
                    zeros = ~mask[w] & valid;
                }
                uint32_t z = __popc(zeros);
                uint32_t tot;
                uint32_t ex = block_exclusive_sum(z, ts.scan, &tot) + carry;
                if (w < nwords && ex < kp) {
                    uint32_t take = kp - ex;
                    uint32_t fill = zeros;
                    if (take < z) {  // keep only the lowest `take` zero bits
                        uint32_t f = 0;
                        for (uint32_t c = 0; c < take; c++) {
                            uint32_t low = fill & (0u - fill);
                            f |= low;
                            fill ^= low;
                        }
                        fill = f;
                    }
                    mask[w] |= fill;
                    while (fill) {
                        const int bpos = __ffs(fill) - 1;
                        fill &= fill - 1;
                        uint32_t slot = atomicAdd(&ts.n_surv, 1u);
                        if (slot < kSurvCap)
                            ts.surv[slot] = (uint16_t)((w << 5) + bpos);
                    }
                }
                carry += tot;
            }
            __syncthreads();
        }
        const uint32_t n_cand = ts.n_surv;
        const uint32_t n_emit = n_cand < kp ? n_cand : kp;
        if (tid == 0)
            st.base = n_emit ? atomicAdd(&ccount[q], n_emit) : 0u;
        __syncthreads();
        if (n_emit > 0) {
            u64* out = cand + q * cand_cap + st.base;
            auto emit = [&](u64 key) {
                uint32_t slot = atomicAdd(&st.ctr, 1u);
                if (slot < n_emit) {
                    out[slot] = key;
                    atomicMin(&st.minkey, key);
                }
            };
            if (n_cand <= kSurvCap) {
                block_select_idx(st, n_cand, kp,
                                 [&](uint32_t i) {
                                     const int d = ts.surv[i];
                                     return make_key(acc[d], (uint32_t)(d0 + d));
                                 },
                                 emit);
            } else {  // more survivors than the buffer holds: walk the bitmask
                auto for_each = [&](auto f) {
                    for (int w = tid; w < nwords; w += kTileThreads) {
                        uint32_t bits = mask[w];
                        while (bits) {
                            const int bpos = __ffs(bits) - 1;
                            bits &= bits - 1;
                            const int d = (w << 5) + bpos;
                            const float a = acc[d];
                            if (order_f32(a) >= tau)
                                f(make_key(a, (uint32_t)(d0 + d)));
                        }
                    }
                };
                block_select(st, n_cand, kp, for_each, emit);
            }
            // a full set of k' candidates raises the query's threshold to the
            // score of the weakest of them
            if (tid == 0 && n_emit == kp)
                atomicMax(&thresh[q], (uint32_t)(st.minkey >> 32));
        }

        // reset the touched accumulators and the bitmask for the next item
        for (int w = tid; w < nwords; w += kTileThreads) {
            uint32_t bits = mask[w];
            while (bits) {
                int bpos = __ffs(bits) - 1;
                bits &= bits - 1;
                acc[(w << 5) + bpos] = 0.0f;
            }
            mask[w] = 0u;
        }
        __syncthreads();
    }
}

#undef BM25_PREFETCH

// ---- R3 -----------------------------------------------------------------------
// Per query: the k' best of the tiles' candidates, re-keyed on the final FP32
// score (shift added) so that equal returned scores list the lower doc id
// first, then sorted.
__global__ void __launch_bounds__(kMergeThreads)
    k_merge(const u64* __restrict__ cand, int64_t cand_cap, const uint32_t* __restrict__ ccount,
            int32_t kprime, int32_t k, const double* __restrict__ shift,
            int32_t* __restrict__ out_ids, float* __restrict__ out_scores)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SelectState st;
    u64* sel = reinterpret_cast<u64*>(smem);
    const int q = blockIdx.x;
    const int tid = threadIdx.x;
    const int64_t n = min((int64_t)ccount[q], cand_cap);
    const u64* c = cand + (int64_t)q * cand_cap;

    int sz = 1;
    while (sz < kprime)
        sz <<= 1;
    for (int i = tid; i < sz; i += kMergeThreads)
        sel[i] = 0ull;
    if (tid == 0)
        st.ctr = 0;
    __syncthreads();
    auto for_each = [&](auto f) {
        for (int64_t i = tid; i < n; i += kMergeThreads)
            f(c[i]);
    };
    block_select(st, (uint32_t)n, (uint32_t)kprime, for_each, [&](u64 key) {
        uint32_t slot = atomicAdd(&st.ctr, 1u);
        if (slot < (uint32_t)kprime)
            sel[slot] = key;
    });
    const double sh = shift[q];
    for (int i = tid; i < kprime; i += kMergeThreads) {
        u64 key = sel[i];
        if (key != 0ull)
            sel[i] = make_key((float)((double)key_score(key) + sh), key_doc(key));
    }
    __syncthreads();
    // bitonic sort, descending
    for (int size = 2; size <= sz; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < sz / 2; i += kMergeThreads) {
                int lo = 2 * i - (i & (stride - 1));
                int hi = lo + stride;
                bool desc = ((lo & size) == 0);
                u64 a = sel[lo], b = sel[hi];
                if ((a < b) == desc) {
                    sel[lo] = b;
                    sel[hi] = a;
                }
            }
            __syncthreads();
        }
    }
    for (int r = tid; r < k; r += kMergeThreads) {
        int64_t o = (int64_t)q * k + r;
        if (r < kprime) {
            u64 key = sel[r];
            out_ids[o] = (int32_t)key_doc(key);
            out_scores[o] = key_score(key);
        } else {
            out_ids[o] = -1;
            out_scores[o] = -__int_as_float(0x7f800000);
        }
    }
}

size_t tile_smem_bytes(int32_t W)
{
    return (size_t)W * 4 + (size_t)(W / 32) * 4 + sizeof(SelectState) + sizeof(TileStage);
}

template <typename T>
int grow(T** p, size_t* cap, size_t need)
{
    if (need <= *cap && *p)
        return BM25_OK;
    if (*p)
        cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    size_t n = need > 0 ? need : 1;
    BM25_CUDA_TRY(cudaMalloc((void**)p, n * sizeof(T)));
    *cap = n;
    return BM25_OK;
}

}  // namespace

int workspace_reserve(const bm25_index* ix, bm25_workspace* ws, int32_t nq, int64_t n_tok,
                      int32_t kprime, int64_t n_tiles)
{
    (void)ix;
    size_t shift_cap = (size_t)ws->max_queries;
    if ((size_t)nq > shift_cap || !ws->shift) {
        for (void* p : {(void*)ws->shift, (void*)ws->thresh, (void*)ws->ccount})
            if (p)
                cudaFree(p);
        ws->shift = nullptr;
        ws->thresh = nullptr;
        ws->ccount = nullptr;
        const size_t m = (size_t)std::max(nq, 1);
        BM25_CUDA_TRY(cudaMalloc((void**)&ws->shift, sizeof(double) * m));
        BM25_CUDA_TRY(cudaMalloc((void**)&ws->thresh, sizeof(uint32_t) * m));
        BM25_CUDA_TRY(cudaMalloc((void**)&ws->ccount, sizeof(uint32_t) * m));
        ws->max_queries = (int32_t)m;
    }
    BM25_TRY(grow(&ws->seg, &ws->seg_cap, (size_t)n_tok * (size_t)(n_tiles + 1)));
    BM25_TRY(grow(&ws->cand, &ws->cand_cap, (size_t)nq * (size_t)n_tiles * (size_t)kprime));
    return BM25_OK;
}

void workspace_release(bm25_workspace* ws)
{
    void* ps[] = {ws->shift, ws->thresh, ws->ccount, ws->seg, ws->cand};
    for (void* p : ps)
        if (p)
            cudaFree(p);
    if (ws->owns_staging) {
        void* st[] = {ws->q_tokens, ws->q_offsets, ws->out_ids, ws->out_scores};
        for (void* p : st)
            if (p)
                cudaFree(p);
    }
    ws->shift = nullptr;
    ws->thresh = nullptr;
    ws->ccount = nullptr;
    ws->seg = nullptr;
    ws->cand = nullptr;
}

int retrieve_device(const bm25_index* ix, bm25_workspace* ws, const int32_t* q_tokens,
                    const int64_t* q_off, int32_t nq, int64_t n_tok, int32_t k, int32_t* out_ids,
                    float* out_scores, int accumulator, int32_t tile_docs, cudaStream_t s)
{
    (void)accumulator;
    if (nq == 0)
        return BM25_OK;
    DeviceInfo di;
    BM25_TRY(device_info(&di));
    const int64_t N = ix->n_docs;
    const int32_t kprime = (int32_t)std::min<int64_t>(k, N);
    int32_t W = tile_docs > 0 ? tile_docs : ix->plan.tile_docs;
    // multiples of 128 keep the shared-memory carve-up 16-byte aligned
    int64_t w_need = (N + 127) / 128 * 128;
    if (W > w_need)
        W = (int32_t)w_need;
    const int32_t n_tiles = (int32_t)((N + W - 1) / W);
    BM25_TRY(workspace_reserve(ix, ws, nq, n_tok, kprime, n_tiles));

    const int max_blocks = di.sm_count * 16;
    int g0 = (int)std::min<int64_t>((nq + 255) / 256, max_blocks);
    {
        ProfileScope ps_("k_query_prep", s);
        k_query_prep<<<std::max(g0, 1), 256, 0, s>>>(q_tokens, n_tok, q_off, nq, ix->s0, ix->vocab,
                                                      ws->shift, ws->thresh, ws->ccount,
                                                      ix->status);
    }
    count_launch();
    BM25_LAUNCH_CHECK();
    const int64_t n_seg = n_tok * ((int64_t)n_tiles + 1);
    if (n_seg > 0) {
        int g1 = (int)std::min<int64_t>((n_seg + 255) / 256, max_blocks);
        {
            ProfileScope ps_("k_seg_bounds", s);
            k_seg_bounds<<<g1, 256, 0, s>>>(q_tokens, n_tok, ix->indptr, ix->indices, ix->vocab, W,
                                            n_tiles, ws->seg);
        }
        count_launch();
        BM25_LAUNCH_CHECK();
    }
    const size_t smem = tile_smem_bytes(W);
    BM25_CUDA_TRY(cudaFuncSetAttribute(k_tile_topk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    int per_sm = 0;
    BM25_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_topk,
                                                                kTileThreads, smem));
    if (per_sm < 1)
        return set_error(BM25_E_INVALID, "doc tile of %d documents does not fit on an SM", W);
    const int64_t n_items = (int64_t)nq * n_tiles;
    int g2 = (int)std::min<int64_t>(n_items, (int64_t)di.sm_count * per_sm);
    {
        ProfileScope ps_("k_tile_topk", s);
        k_tile_topk<<<g2, kTileThreads, smem, s>>>(q_tokens, n_tok, q_off, nq, N, ix->indices,
                                                   ix->data, ws->seg, W, n_tiles, kprime,
                                                   ws->thresh, ws->ccount, ws->cand,
                                                   (int64_t)n_tiles * kprime);
    }
    count_launch();
    BM25_LAUNCH_CHECK();
    int sz = 1;
    while (sz < kprime)
        sz <<= 1;
    const size_t msmem = (size_t)sz * sizeof(u64);
    BM25_CUDA_TRY(cudaFuncSetAttribute(k_merge, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)msmem));
    {
        ProfileScope ps_("k_merge", s);
        k_merge<<<nq, kMergeThreads, msmem, s>>>(ws->cand, (int64_t)n_tiles * kprime, ws->ccount,
                                                 kprime, k, ws->shift, out_ids, out_scores);
    }
    count_launch();
    BM25_LAUNCH_CHECK();
    return BM25_OK;
}

}  // namespace bm25
