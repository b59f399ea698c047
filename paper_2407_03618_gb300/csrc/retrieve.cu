// Batched top-k retrieval over the eager term-major index (arXiv 2407.03618
// Sec. 2 "Assigning Query Scores" and "Top-k selection"; Sec. 2.1 for the
// shift added back to every returned score).
//
// Doc-tiled shared-memory path, four launches per call:
//   R0 k_query_prep   sum_i S0(q_i) per query in FP64; token / offset checks;
//                     resets the per-query running threshold; counts the
//                     query's postings (a bound on the documents it touches)
//   R1 k_seg_bounds   for every query token and every doc-tile boundary, the
//                     first posting of the token's column at or past the
//                     boundary (binary search: doc ids ascend in a column)
//   R2 k_tile_topk    persistent CTAs over (doc tile, query) items: each item
//                     scatter-adds its postings into FP32 accumulators in
//                     shared memory, marks touched documents in a bitmask,
//                     keeps the documents that clear the query's running
//                     threshold, and radix-selects the tile's best k' of them
//                     (including the lowest-id untouched documents, score 0,
//                     when they can matter)
//   R3 k_merge        per query: the k' best of the tiles' candidates,
//                     re-keyed on the final score, sorted, written out
#include <algorithm>
#include <cstdio>
#include <cstdlib>

#include "device.cuh"
#include "internal.h"

namespace bm25 {
namespace {

typedef unsigned long long u64;

constexpr int kTokChunk = 64;          // query tokens staged in shared memory at a time
constexpr int kMergeThreads = 256;
constexpr int kMergeBufCap = 4096;     // candidates a merge gathers into shared memory
constexpr uint32_t kZeroKey = 0x80000000u;  // order_f32(0.0f)

// ---- R0 ---------------------------------------------------------------------
__global__ void k_query_prep(const int32_t* __restrict__ q_tokens, int64_t n_tok,
                             const int64_t* __restrict__ q_off, int32_t nq,
                             const double* __restrict__ s0, const int64_t* __restrict__ indptr,
                             int32_t vocab, double* __restrict__ shift,
                             uint32_t* __restrict__ thresh, uint32_t* __restrict__ qpost,
                             int* status)
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
        int64_t post = 0;
        for (int64_t m = lo; m < hi; m++) {
            int32_t t = q_tokens[m];
            if (t < 0 || t >= vocab) {
                set_status(status, BM25_E_TOKEN_RANGE);
                continue;
            }
            sum += s0[t];
            post += indptr[t + 1] - indptr[t];
        }
        shift[q] = sum;
        thresh[q] = 0u;  // below every real score key
        qpost[q] = post > 0xffffffffll ? 0xffffffffu : (uint32_t)post;
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
    uint32_t need, bucket, ctr, tau;
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

// Selection over an indexable candidate set: get(i) for i < n_index is the
// key of candidate i, or 0 where index i holds no candidate; n_real is the
// number of non-zero keys.  Every key starts with the `skip` bytes of
// `common` (bytes all candidates share, so their passes are skipped).
// emit(key, slot) runs once per selected key with distinct slots
// 0 .. min(k, n_real) - 1.  The loops are warp-uniform, so histogram updates
// and output slots are aggregated per warp (__match_any_sync /
// __ballot_sync): keys sharing a prefix would otherwise serialise on one
// shared-memory counter.  st.ctr must be 0 on entry.  With TRAIL_SYNC false
// the block is not synchronised after the emit loop.
template <bool TRAIL_SYNC, class Get, class Emit>
__device__ void block_select_idx(SelectState& st, uint32_t n_index, uint32_t n_real, uint32_t k,
                                 int skip, u64 common, Get get, Emit emit)
{
    const int lane = threadIdx.x & 31;
    const uint32_t stride = blockDim.x;
    const uint32_t base0 = threadIdx.x & ~31u;
    u64 pm = 0, pf = 0;
    if (n_real > k) {
        if (threadIdx.x == 0) {
            const u64 m0 = skip >= 8 ? ~0ull : (skip <= 0 ? 0ull : ~0ull << (64 - 8 * skip));
            st.prefix = common & m0;
            st.pmask = m0;
            st.need = k;
        }
        for (int pass = skip; pass < 8; pass++) {
            const int shift = 56 - 8 * pass;
            for (int i = threadIdx.x; i < 256; i += blockDim.x)
                st.hist[i] = 0;
            __syncthreads();
            const u64 cpm = st.pmask, cpf = st.prefix;
            for (uint32_t b = base0; b < n_index; b += stride) {
                const uint32_t i = b + lane;
                uint32_t dg = 0xffffffffu;
                if (i < n_index) {
                    const u64 key = get(i);
                    if (key != 0ull && (key & cpm) == cpf)
                        dg = (uint32_t)(key >> shift) & 0xffu;
                }
                const uint32_t peers = __match_any_sync(0xffffffffu, dg);
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
        pm = st.pmask;
        pf = st.prefix;
    }
    for (uint32_t b = base0; b < n_index; b += stride) {
        const uint32_t i = b + lane;
        u64 key = 0;
        bool take = false;
        if (i < n_index) {
            key = get(i);
            take = key != 0ull && (key & pm) >= pf;
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, take);
        if (bal) {
            uint32_t base = 0;
            if (lane == __ffs(bal) - 1)
                base = atomicAdd(&st.ctr, (uint32_t)__popc(bal));
            base = __shfl_sync(0xffffffffu, base, __ffs(bal) - 1);
            if (take)
                emit(key, base + __popc(bal & lanemask_lt()));
        }
    }
    if (TRAIL_SYNC)
        __syncthreads();
}

// Number of leading bytes shared by every key whose high word lies in
// [kmin, kmax] (the low word, a doc id, is assumed to vary).
__device__ __forceinline__ int common_bytes(uint32_t kmin, uint32_t kmax)
{
    uint32_t x = kmin ^ kmax;
    return x ? (__clz(x) >> 3) : 4;
}

// ---- R2 -----------------------------------------------------------------------
// Dynamic shared memory: acc[W] FP32 | SelectState | TileStage |
// surv_val[WARPS * SPW] FP32 | surv_doc[WARPS * SPW] (doc id within the tile).
//
// An accumulator holds -0.0 until a posting lands on it (stored scores are
// never -0.0 and -0.0 + x == x, so a touched accumulator is never -0.0).
// Postings are added with fire-and-forget shared-memory reductions.  In the
// common case an item's postings fit in one round of U per thread, and each
// thread keeps the doc ids of its postings in registers; after the barrier
// it claims each of those documents with an atomic exchange that returns the
// document's sum and leaves a mark behind: the first claimer of a document
// gets its score, later claimers (the document appeared in several columns)
// see the mark.  With the query's threshold above 0 the mark is -0.0, so the
// claim also resets the accumulator for the next item; otherwise (untouched
// documents may compete) the mark is a NaN pattern, which keeps touched and
// untouched documents apart until the tile is done.  Documents that clear
// the threshold go, with their score, to a list of the claiming warp, sized
// to the postings the warp owns (no overflow, no shared counters).  Items
// with more postings than one round, or more tokens than one chunk, take a
// path that walks the whole tile.
#ifdef BM25_PHASE_TIMING
// Diagnostic build only: per-phase cycle totals of k_tile_topk, summed over
// CTAs (thread 0's view), and item statistics.
__device__ unsigned long long g_phase[16];
#define BM25_PHASE(I)                                                                \
    do {                                                                             \
        if (tid == 0) {                                                              \
            const long long now_ = clock64();                                        \
            ph_acc[I] += (unsigned long long)(now_ - ph_t);                          \
            ph_t = now_;                                                             \
        }                                                                            \
    } while (0)
#else
#define BM25_PHASE(I) \
    do {              \
    } while (0)
#endif
constexpr uint32_t kUntouched = 0x80000000u;  // bits of -0.0f
constexpr uint32_t kMarked = 0x7fffffffu;     // a NaN: claimed while untouched ones still count
constexpr int kMaxWarps = 16;
constexpr int kPostU = 8;                     // postings per thread in one round
constexpr uint32_t kOutCap = 128;             // candidates an item stages for a deferred write

struct TileStage {
    int32_t lo[kTokChunk];
    int32_t pre[kTokChunk + 1];
    uint32_t scan[33];
    int32_t qoff[2][2];                   // token range of the current / next item
    uint32_t w_surv[kMaxWarps];           // per warp: its candidates
    uint32_t w_pos[kMaxWarps];            // per warp: claimed documents scoring > 0
    uint32_t w_kmin[kMaxWarps], w_kmax[kMaxWarps];  // per warp: candidate score keys
    uint32_t list_pre[kMaxWarps + 1];     // exclusive prefix of the candidate lists
    // The previous item's result, written to global memory by the next item
    // once its first barrier has passed, so that no barrier waits on those
    // writes: its candidates (when at most kOutCap), count and threshold.
    u64 obuf[kOutCap];
    int32_t o_item, o_q;
    uint32_t o_count, o_tau, o_staged;  // o_staged = 0: written directly already
    uint32_t q_post;                    // the current query's postings (all columns)
    uint32_t cutoff;                    // fill: docs [0, cutoff) hold the k' lowest untouched
};

// Bitonic sort of one 64-bit key per lane, descending across the warp.
__device__ __forceinline__ u64 warp_sort_desc(u64 key)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const u64 other = __shfl_xor_sync(0xffffffffu, key, stride);
            const bool lower = (lane & stride) == 0;  // the lower index of the pair
            const bool desc = (lane & size) == 0;     // this block sorts descending
            // the lower index keeps the larger key in a descending block
            const bool keep_max = (lower == desc);
            key = keep_max ? (key > other ? key : other) : (key < other ? key : other);
        }
    }
    return key;
}

// Counts the untouched documents (accumulator -0.0) among the tile's first
// wd, up to k of them, and stores in *cutoff the smallest c such that docs
// [0, c) hold min(k, untouched) of them.  All threads call it (block scans
// over words of 32 documents); ends with __syncthreads().
__device__ uint32_t first_untouched(const float* acc, int32_t wd, uint32_t k, uint32_t* scan_buf,
                                    uint32_t* cutoff)
{
    const int32_t nwords = (wd + 31) >> 5;
    uint32_t carry = 0;
    if (threadIdx.x == 0)
        *cutoff = (uint32_t)wd;
    for (int w0 = 0; w0 < nwords && carry < k; w0 += blockDim.x) {
        const int w = w0 + threadIdx.x;
        uint32_t zeros = 0;
        if (w < nwords) {
            const int dmax = min(32, wd - (w << 5));
            for (int b = 0; b < dmax; b++)
                if (__float_as_uint(acc[(w << 5) + b]) == 0x80000000u)
                    zeros |= 1u << b;
        }
        const uint32_t z = __popc(zeros);
        uint32_t tot;
        const uint32_t ex = block_exclusive_sum(z, scan_buf, &tot) + carry;
        if (w < nwords && ex < k && ex + z >= k) {  // the k-th untouched one is here
            uint32_t f = zeros;
            for (uint32_t c = ex + 1; c < k; c++)
                f &= f - 1;
            *cutoff = (uint32_t)((w << 5) + __ffs(f));  // one past it
        }
        carry += tot;
    }
    __syncthreads();
    return carry < k ? carry : k;
}

template <int THREADS>
constexpr size_t tile_lists_bytes()
{
    return (size_t)(THREADS / 32) * (kPostU * 32) * (sizeof(float) + sizeof(uint16_t));
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS, 3)  // three 12K-document tiles per SM
    k_tile_topk(const int32_t* __restrict__ q_tokens, int64_t n_tok,
                const int64_t* __restrict__ q_off, int32_t nq, int64_t n_docs,
                const int32_t* __restrict__ indices, const float* __restrict__ data,
                const int32_t* __restrict__ seg, int32_t W, int32_t n_tiles, int32_t kprime,
                uint32_t* __restrict__ thresh, const uint32_t* __restrict__ qpost,
                uint32_t* __restrict__ tcount, u64* __restrict__ cand)
{
    constexpr int WARPS = THREADS / 32;
    constexpr int U = kPostU;
    constexpr uint32_t SPW = U * 32;  // candidates a warp can claim in one round
    static_assert(WARPS <= kMaxWarps, "too many warps");
    extern __shared__ __align__(16) unsigned char smem[];
    float* acc = reinterpret_cast<float*>(smem);
    SelectState& st = *reinterpret_cast<SelectState*>(acc + W);
    TileStage& ts = *reinterpret_cast<TileStage*>(&st + 1);
    float* surv_val = reinterpret_cast<float*>(&ts + 1);
    uint16_t* surv_doc = reinterpret_cast<uint16_t*>(surv_val + WARPS * SPW);

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const uint32_t ltmask = lanemask_lt();
    const float neg0 = __uint_as_float(kUntouched);
    float* my_sval = surv_val + warp * SPW;
    uint16_t* my_sdoc = surv_doc + warp * SPW;
    for (int i = tid; i < W; i += THREADS)
        acc[i] = neg0;

    const int32_t n_items = nq * n_tiles;  // < 2^31 (checked by the host)
    const int64_t per = (int64_t)n_tiles + 1;
    // Tile-major order: item = tile * nq + q, tile 0 of every query first, so
    // the running threshold of a query is usually known when its later tiles
    // run, and the segments in flight at once all belong to one doc tile.
    // (tile, q) advance by the grid stride without dividing.
    const int32_t step_t = (int32_t)(gridDim.x / nq), step_q = (int32_t)(gridDim.x % nq);
    auto advance = [&](int32_t& t, int32_t& qq) {
        t += step_t;
        qq += step_q;
        if (qq >= nq) {
            qq -= nq;
            t++;
        }
    };
    const int32_t ntok32 = (int32_t)n_tok;  // < 2^31 (checked by the host)
    auto clamp_off = [&](int64_t v) -> int32_t {
        return v < 0 ? 0 : (v > n_tok ? ntok32 : (int32_t)v);
    };
    // Warp 0 runs a two-stage pipeline over the CTA's items: while item i is
    // processed it loads the segment bounds of item i+1 (lane l: tokens 2l
    // and 2l+1 of the first chunk) from the token range it loaded during item
    // i-1, and the (raw, unclamped) token range of item i+2.  Thread 0 also
    // loads item i+1's threshold.  No load of the pipeline is consumed in the
    // item it is issued in.
    int32_t tile = (int32_t)(blockIdx.x / nq), q = (int32_t)(blockIdx.x % nq);
    int32_t t1 = tile, q1 = q;
    advance(t1, q1);
    int32_t t2 = t1, q2 = q1;
    advance(t2, q2);
    int32_t a1 = 0, b1 = 0;                 // clamped token range of item i+1
    int64_t ra2 = 0, rb2 = 0;               // raw token range of item i+2
    int32_t pf_lo0 = 0, pf_lo1 = 0, pf_hi0 = 0, pf_hi1 = 0;
    uint32_t pf_tau = 0, pf_post = 0;
    auto load_seg = [&](int32_t t_, int32_t a_, int32_t b_) {
        const int32_t m_ = a_ + 2 * tid;
        pf_lo0 = pf_hi0 = pf_lo1 = pf_hi1 = 0;
        if (m_ < b_) {
            pf_lo0 = seg[(int64_t)m_ * per + t_];
            pf_hi0 = seg[(int64_t)m_ * per + t_ + 1];
        }
        if (m_ + 1 < b_) {
            pf_lo1 = seg[(int64_t)(m_ + 1) * per + t_];
            pf_hi1 = seg[(int64_t)(m_ + 1) * per + t_ + 1];
        }
    };
    if (tid == 0)
        ts.o_item = -1;
    if (tid < 32) {
        const int32_t a0 = clamp_off(q_off[q]);
        const int32_t b0 = max(a0, clamp_off(q_off[q + 1]));
        load_seg(tile, a0, b0);
        if (tid == 0) {
            ts.qoff[0][0] = a0;
            ts.qoff[0][1] = b0;
            pf_tau = *(volatile uint32_t*)&thresh[q];
            pf_post = qpost[q];
        }
        if ((int64_t)blockIdx.x + gridDim.x < n_items) {
            a1 = clamp_off(q_off[q1]);
            b1 = max(a1, clamp_off(q_off[q1 + 1]));
        }
        if ((int64_t)blockIdx.x + 2 * (int64_t)gridDim.x < n_items) {
            ra2 = q_off[q2];
            rb2 = q_off[q2 + 1];
        }
    }
    __syncthreads();
#ifdef BM25_PHASE_TIMING
    unsigned long long ph_acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long ph_t = clock64();
#endif

    // writes the previous item's staged result (all threads; call between
    // two barriers)
    auto flush = [&]() {
        const int32_t pi = ts.o_item;
        if (pi < 0)
            return;
        const uint32_t pc = ts.o_count;
        if (ts.o_staged) {
            for (uint32_t t = tid; t < pc; t += THREADS)
                cand[(int64_t)pi * kprime + t] = ts.obuf[t];
            if (tid == 0)
                tcount[pi] = pc;
        }
        if (tid == 0 && ts.o_tau != 0u)
            atomicMax(&thresh[ts.o_q], ts.o_tau);
    };
    int parity = 0;
    for (int32_t item = blockIdx.x; item < n_items; item += gridDim.x, parity ^= 1) {
        const int64_t d0 = (int64_t)tile * W;
        const int32_t wd = (int32_t)min((int64_t)W, n_docs - d0);
        const int32_t m0 = ts.qoff[parity][0], m1 = ts.qoff[parity][1];
        // warp 0: advance the pipeline once this item's prefetched values are used
        auto pipeline = [&]() {
            if (tid < 32) {
                const int32_t nitem = item + (int32_t)gridDim.x;
                if (nitem < n_items) {
                    load_seg(t1, a1, b1);
                    if (tid == 0) {
                        ts.qoff[parity ^ 1][0] = a1;
                        ts.qoff[parity ^ 1][1] = b1;
                        pf_tau = *(volatile uint32_t*)&thresh[q1];
                        pf_post = qpost[q1];
                    }
                }
                a1 = clamp_off(ra2);
                b1 = max(a1, clamp_off(rb2));
                int32_t t3 = t2, q3 = q2;
                advance(t3, q3);
                if ((int64_t)nitem + 2 * (int64_t)gridDim.x < n_items) {
                    ra2 = q_off[q3];
                    rb2 = q_off[q3 + 1];
                }
                t1 = t2;
                q1 = q2;
                t2 = t3;
                q2 = q3;
            }
        };
        if (tid == 0) {
            st.tau = pf_tau;  // thread 0 holds the threshold; the others read st.tau
            ts.q_post = pf_post;
        }
        int32_t dd[U];        // doc ids (within the tile) of this thread's postings
#pragma unroll
        for (int u = 0; u < U; u++)
            dd[u] = -1;
        bool one_round = true;  // one chunk of tokens, one round of postings (uniform)

        // ---- scatter-add the item's postings, a chunk of tokens at a time ----
        for (int32_t mb = m0; mb < m1; mb += kTokChunk) {
            const int cnt = min(kTokChunk, m1 - mb);
            if (tid < 32) {
                int32_t len[2];
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int i = 2 * tid + h;
                    int32_t l = 0, hh = 0;
                    if (mb == m0) {  // prefetched during the previous item
                        l = h ? pf_lo1 : pf_lo0;
                        hh = h ? pf_hi1 : pf_hi0;
                    } else if (i < cnt) {
                        const int32_t* sg = seg + (int64_t)(mb + i) * per + tile;
                        l = sg[0];
                        hh = sg[1];
                    }
                    if (i >= cnt)
                        l = hh = 0;
                    len[h] = hh - l;
                    ts.lo[i] = l;
                }
                const int32_t s2 = len[0] + len[1];
                const int32_t inc = warp_inclusive_sum(s2);
                ts.pre[2 * tid] = inc - s2;
                ts.pre[2 * tid + 1] = inc - s2 + len[0];
                if (tid == 31)
                    ts.pre[kTokChunk] = inc;
                if (mb == m0)
                    pipeline();
            }
            __syncthreads();
            BM25_PHASE(0);
            if (mb == m0)
                flush();
            const int32_t total = ts.pre[kTokChunk];
            if (mb != m0 || total > U * THREADS)
                one_round = false;
            // Warp w takes runs of 32 consecutive postings, r = w, w + WARPS, ...
            // The token of its first run comes from one warp-uniform binary
            // search; runs only move forward, so each later one (and each
            // lane) steps on from there over finished or empty segments.
            for (int32_t r0 = warp; r0 * 32 < total; r0 += U * WARPS) {
                float vv[U];
                int a = 0;
                {
                    const int32_t eb = r0 * 32;
                    int b = cnt;  // pre[a] <= eb < pre[b]
                    while (b - a > 1) {
                        const int mid = (a + b) >> 1;
                        if (ts.pre[mid] <= eb)
                            a = mid;
                        else
                            b = mid;
                    }
                }
                // runs this warp owns in this round (warp-uniform)
                const int32_t n_runs = (total + 31) >> 5;
                const int32_t u_max = (n_runs - r0 + WARPS - 1) / WARPS;
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int32_t r = r0 + u * WARPS;
                    const int32_t e = r * 32 + lane;
                    dd[u] = -1;
                    if (u < u_max && e < total) {
                        while (ts.pre[a + 1] <= e)
                            a++;
                        const int32_t j = ts.lo[a] + (e - ts.pre[a]);
                        dd[u] = __ldg(indices + j) - (int32_t)d0;
                        vv[u] = __ldg(data + j);
                    }
                }
#pragma unroll
                for (int u = 0; u < U; u++) {
                    if (u < u_max) {
                        if ((uint32_t)dd[u] < (uint32_t)wd)  // holds for any well-formed index
                            atomicAdd(&acc[dd[u]], vv[u]);   // result unused: a reduction
                        else
                            dd[u] = -1;
                    }
                }
            }
            __syncthreads();
            BM25_PHASE(1);
        }
        if (m0 == m1) {
            pipeline();
            __syncthreads();
            flush();
            __syncthreads();  // the flush reads the staged result before it is replaced
        }

        // tau = the query's running threshold: some tile already holds k'
        // documents scoring at least tau, so a document below tau cannot be
        // in the top k' (documents AT tau can, through the doc-id tie rule).
        const uint32_t tau = st.tau;
        const uint32_t kp = (uint32_t)min(kprime, wd);
        // Untouched documents score exactly 0: they can matter only if 0
        // clears tau (and then only if fewer than k' touched ones score > 0),
        // and only the k' lowest-id untouched documents of the whole corpus
        // can: a tile whose predecessors hold at least k' untouched documents
        // (true once t * W - postings of the query >= k') adds none.
        const bool zero_counts = tau <= kZeroKey;
        const bool may_fill = zero_counts && (int64_t)tile * W < (int64_t)kp + ts.q_post;
        // candidates go to the staging buffer when they fit (kp <= kOutCap),
        // else straight to the item's slots
        u64* out = kp <= kOutCap ? ts.obuf : cand + (int64_t)item * kprime;
        uint32_t n_emit = 0;
        uint32_t new_tau = 0;  // score key of (a lower bound on) the weakest emitted
        bool tau_ok = false;   // new_tau is a valid bound to publish

        if (one_round) {
            // ---- claim each posting's document once; keep the candidates ---------
            const uint32_t mark = zero_counts ? kMarked : kUntouched;
            uint32_t pos = 0, kmin = 0xffffffffu, kmax = 0u, n_keep = 0;
            // slots this warp filled in the single round (warp-uniform)
            const int32_t u_max = (((ts.pre[kTokChunk] + 31) >> 5) - warp + WARPS - 1) / WARPS;
            float cv[U];  // all exchanges first, so their latencies overlap
#pragma unroll
            for (int u = 0; u < U; u++)
                cv[u] = (u < u_max && dd[u] >= 0)
                            ? atomicExch(&acc[dd[u]], __uint_as_float(mark))
                            : __uint_as_float(kUntouched);
#pragma unroll
            for (int u = 0; u < U; u++) {
                if (u >= u_max)
                    break;
                bool keep = false;
                const float v = cv[u];
                const uint32_t vb = __float_as_uint(v);
                uint32_t o = 0;
                if (vb != kUntouched && vb != kMarked) {  // the first claim of the document
                    o = order_f32(v);
                    if (zero_counts)
                        pos += (v > 0.0f);
                    keep = o >= tau;
                }
                const uint32_t bal = __ballot_sync(0xffffffffu, keep);
                if (keep) {
                    const uint32_t slot = n_keep + __popc(bal & ltmask);  // < SPW
                    my_sval[slot] = v;
                    my_sdoc[slot] = (uint16_t)dd[u];
                    kmin = min(kmin, o);
                    kmax = max(kmax, o);
                }
                n_keep += __popc(bal);
            }
            pos = __reduce_add_sync(0xffffffffu, pos);
            kmin = __reduce_min_sync(0xffffffffu, kmin);
            kmax = __reduce_max_sync(0xffffffffu, kmax);
            if (lane == 0) {
                ts.w_surv[warp] = n_keep;
                ts.w_pos[warp] = pos;
                ts.w_kmin[warp] = kmin;
                ts.w_kmax[warp] = kmax;
            }
            __syncthreads();
            BM25_PHASE(2);
            uint32_t n_cand, n_pos, my_base;
            {
                const bool has = lane < WARPS;
                const uint32_t sv = has ? ts.w_surv[lane] : 0u;
                const uint32_t inc = warp_inclusive_sum(sv);
                n_cand = __shfl_sync(0xffffffffu, inc, 31);
                my_base = __shfl_sync(0xffffffffu, inc - sv, warp);
                n_pos = __reduce_add_sync(0xffffffffu, has ? ts.w_pos[lane] : 0u);
                kmin = __reduce_min_sync(0xffffffffu, has ? ts.w_kmin[lane] : 0xffffffffu);
                kmax = __reduce_max_sync(0xffffffffu, has ? ts.w_kmax[lane] : 0u);
                if (warp == 0 && lane <= WARPS)
                    ts.list_pre[lane] = inc - sv;
            }
            const bool fill_on = may_fill && n_pos < kp;
            if (!fill_on) {
                if (zero_counts) {  // lift the marks: the accumulators start the next item clean
#pragma unroll
                    for (int u = 0; u < U; u++)
                        if (dd[u] >= 0)
                            acc[dd[u]] = neg0;
                }
                n_emit = n_cand < kp ? n_cand : kp;
                if (n_cand <= kp) {
                    // every candidate is kept: warp w writes its own at its offset
                    const uint32_t nw = ts.w_surv[warp];
                    for (uint32_t i = lane; i < nw; i += 32)
                        out[my_base + i] = make_key(my_sval[i], (uint32_t)(d0 + my_sdoc[i]));
                    new_tau = kmin;
                    tau_ok = true;
                } else if (n_cand <= 32) {
                    // a few candidates too many (kp < n_cand <= 32): warp 0 sorts
                    // them in registers, no block barrier
                    if (warp == 0) {
                        u64 key = 0ull;
                        if ((uint32_t)lane < n_cand) {
                            int a = 0, b = WARPS;  // list_pre[a] <= lane < list_pre[b]
                            while (b - a > 1) {
                                const int mid = (a + b) >> 1;
                                if (ts.list_pre[mid] <= (uint32_t)lane)
                                    a = mid;
                                else
                                    b = mid;
                            }
                            const uint32_t sl = a * SPW + (lane - ts.list_pre[a]);
                            key = make_key(surv_val[sl], (uint32_t)(d0 + surv_doc[sl]));
                        }
                        key = warp_sort_desc(key);
                        if ((uint32_t)lane < kp)
                            out[lane] = key;
                        new_tau = (uint32_t)(__shfl_sync(0xffffffffu, key, kp - 1) >> 32);
                    }
                    tau_ok = true;
                } else {
#ifdef BM25_PHASE_TIMING
                    if (tid == 0)
                        ph_acc[6] += 1;
#endif
                    if (tid == 0)
                        st.ctr = 0;
                    __syncthreads();
                    auto get = [&](uint32_t i) -> u64 {
                        int a = 0, b = WARPS;  // list_pre[a] <= i < list_pre[b]
                        while (b - a > 1) {
                            const int mid = (a + b) >> 1;
                            if (ts.list_pre[mid] <= i)
                                a = mid;
                            else
                                b = mid;
                        }
                        const uint32_t s = a * SPW + (i - ts.list_pre[a]);
                        return make_key(surv_val[s], (uint32_t)(d0 + surv_doc[s]));
                    };
                    block_select_idx<true>(st, n_cand, n_cand, kp, common_bytes(kmin, kmax),
                                           (u64)kmax << 32, get,
                                           [&](u64 key, uint32_t slot) { out[slot] = key; });
                    // the selected keys are those at or above the final prefix,
                    // so its score word bounds the weakest of them from below
                    new_tau = (uint32_t)(st.prefix >> 32);
                    tau_ok = true;
                }
            } else {
#ifdef BM25_PHASE_TIMING
                if (tid == 0)
                    ph_acc[7] += 1;
#endif
                // Untouched documents compete (rare): put the candidates' sums
                // back (so -0.0 again means untouched and the mark means
                // touched below tau), find the k' lowest untouched documents,
                // and select among the candidate lists and those.
                const uint32_t nw = ts.w_surv[warp];
                for (uint32_t i = lane; i < nw; i += 32)
                    acc[my_sdoc[i]] = my_sval[i];
                __syncthreads();
                const uint32_t n_unt = first_untouched(acc, wd, kp, ts.scan, &ts.cutoff);
                const uint32_t cut = ts.cutoff;
                const uint32_t n_all = n_cand + n_unt;
                n_emit = n_all < kp ? n_all : kp;
                if (tid == 0)
                    st.ctr = 0;
                __syncthreads();
                auto get = [&](uint32_t i) -> u64 {
                    if (i < n_cand) {
                        int a = 0, b = WARPS;  // list_pre[a] <= i < list_pre[b]
                        while (b - a > 1) {
                            const int mid = (a + b) >> 1;
                            if (ts.list_pre[mid] <= i)
                                a = mid;
                            else
                                b = mid;
                        }
                        const uint32_t s = a * SPW + (i - ts.list_pre[a]);
                        return make_key(surv_val[s], (uint32_t)(d0 + surv_doc[s]));
                    }
                    const uint32_t d = i - n_cand;
                    return __float_as_uint(acc[d]) == kUntouched
                               ? make_key(0.0f, (uint32_t)(d0 + d))
                               : 0ull;
                };
                block_select_idx<true>(st, n_cand + cut, n_all, kp, 0, 0ull, get,
                                       [&](u64 key, uint32_t slot) { out[slot] = key; });
                if (n_all > kp) {
                    new_tau = (uint32_t)(st.prefix >> 32);
                    tau_ok = true;
                }
#pragma unroll
                for (int u = 0; u < U; u++)
                    if (dd[u] >= 0)
                        acc[dd[u]] = neg0;
            }
        } else {
            // ---- many postings or tokens: walk the whole tile --------------------
            uint32_t c = 0, p = 0;
            for (int d = tid; d < wd; d += THREADS) {
                const float a = acc[d];
                if (__float_as_uint(a) != kUntouched) {
                    c += order_f32(a) >= tau;
                    p += a > 0.0f;
                }
            }
            uint32_t n_cand, n_pos, n_untouched = 0, cut = 0;
            block_exclusive_sum(c, ts.scan, &n_cand);
            block_exclusive_sum(p, ts.scan, &n_pos);
            const bool fill_on = may_fill && n_pos < kp;
            if (fill_on) {
                n_untouched = first_untouched(acc, wd, kp, ts.scan, &ts.cutoff);
                cut = ts.cutoff;
            }            const uint32_t n_all = n_cand + n_untouched;
            n_emit = n_all < kp ? n_all : kp;
            if (tid == 0)
                st.ctr = 0;
            __syncthreads();
            auto get = [&](uint32_t d) -> u64 {
                const float a = acc[d];
                const bool touched = __float_as_uint(a) != kUntouched;
                return (touched ? order_f32(a) >= tau : d < cut)
                           ? make_key(a, (uint32_t)(d0 + d))
                           : 0ull;
            };
            block_select_idx<true>(st, (uint32_t)wd, n_all, kp, 0, 0ull, get,
                                   [&](u64 key, uint32_t slot) { out[slot] = key; });
            if (n_all > kp) {
                new_tau = (uint32_t)(st.prefix >> 32);
                tau_ok = true;
            }
            for (int i = tid; i < wd; i += THREADS)
                acc[i] = neg0;
        }
        BM25_PHASE(3);
        if (tid == 0) {
            // staged for the next item's flush; a full set of k' candidates
            // raises the query's threshold to (a lower bound on) the score of
            // the weakest of them
            ts.o_item = item;
            ts.o_q = q;
            ts.o_count = n_emit;
            ts.o_staged = kp <= kOutCap;
            ts.o_tau = (tau_ok && n_emit == kp && kp > 0) ? new_tau : 0u;
            if (kp > kOutCap)
                tcount[item] = n_emit;  // its candidates were written directly
        }
        __syncthreads();
        BM25_PHASE(4);
#ifdef BM25_PHASE_TIMING
        if (tid == 0)
            ph_acc[5] += one_round ? 1 : 0;
#endif
        advance(tile, q);
    }
    flush();  // the CTA's last item
#ifdef BM25_PHASE_TIMING
    if (tid == 0)
        for (int i = 0; i < 8; i++)
            atomicAdd(&g_phase[i], ph_acc[i]);
#endif
}

// ---- R3 -----------------------------------------------------------------------
// Per query: gather the tiles' candidates (tcount[tile * nq + q] of them in
// item tile * nq + q's slots), select the k' best, re-key them on the final
// FP32 score (shift added) so that equal returned scores list the lower doc
// id first, sort, and write (id, score).  Dynamic shared memory:
// sel[pow2 >= k'] | buf[buf_cap] keys | pre[n_tiles + 1].
__global__ void __launch_bounds__(kMergeThreads)
    k_merge(const u64* __restrict__ cand, const uint32_t* __restrict__ tcount, int32_t nq,
            int32_t n_tiles, int32_t kprime, int32_t k, const double* __restrict__ shift,
            int32_t* __restrict__ out_ids, float* __restrict__ out_scores, int32_t buf_cap)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SelectState st;
    int sz = 1;
    while (sz < kprime)
        sz <<= 1;
    u64* sel = reinterpret_cast<u64*>(smem);
    u64* buf = sel + sz;
    uint32_t* pre = reinterpret_cast<uint32_t*>(buf + buf_cap);
    const int q = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // exclusive scan of the per-tile counts
    uint32_t carry = 0;
    for (int t0 = 0; t0 < n_tiles; t0 += kMergeThreads) {
        const int t = t0 + tid;
        const uint32_t c = t < n_tiles ? tcount[(int64_t)t * nq + q] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_sum(c, st.red, &tot);
        if (t < n_tiles)
            pre[t] = carry + ex;
        carry += tot;
    }
    if (tid == 0)
        pre[n_tiles] = carry;
    for (int i = tid; i < sz; i += kMergeThreads)
        sel[i] = 0ull;
    if (tid == 0)
        st.ctr = 0;
    __syncthreads();
    const uint32_t total = pre[n_tiles];  // > 0: the tiles hold at least k' candidates
    const bool gathered = total <= (uint32_t)buf_cap;
    if (gathered) {  // one warp per tile copies its candidates
        for (int t = warp; t < n_tiles; t += kMergeThreads / 32) {
            const uint32_t c = pre[t + 1] - pre[t];
            const u64* src = cand + ((int64_t)t * nq + q) * kprime;
            for (uint32_t s = lane; s < c; s += 32)
                buf[pre[t] + s] = src[s];
        }
        __syncthreads();
    }
    auto get = [&](uint32_t i) -> u64 {
        if (gathered)
            return buf[i];
        int a = 0, b = n_tiles;  // pre[a] <= i < pre[b]
        while (b - a > 1) {
            int mid = (a + b) >> 1;
            if (pre[mid] <= i)
                a = mid;
            else
                b = mid;
        }
        return cand[((int64_t)a * nq + q) * kprime + (i - pre[a])];
    };
    block_select_idx<true>(st, total, total, (uint32_t)kprime, 0, 0ull, get,
                           [&](u64 key, uint32_t slot) {
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
        const u64 key = r < kprime ? sel[r] : 0ull;
        if (key != 0ull) {
            out_ids[o] = (int32_t)key_doc(key);
            out_scores[o] = key_score(key);
        } else {
            out_ids[o] = -1;
            out_scores[o] = -__int_as_float(0x7f800000);
        }
    }
}

size_t tile_smem_bytes(int32_t W, int threads)
{
    const size_t lists = threads == 128   ? tile_lists_bytes<128>()
                         : threads == 256 ? tile_lists_bytes<256>()
                                          : tile_lists_bytes<512>();
    return (size_t)W * 4 + sizeof(SelectState) + sizeof(TileStage) + lists;
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

#ifdef BM25_PHASE_TIMING
extern "C" int bm25_debug_phase_read(unsigned long long* out, int reset)
{
    if (cudaMemcpyFromSymbol(out, g_phase, sizeof(unsigned long long) * 8) != cudaSuccess)
        return -4;
    if (reset) {
        unsigned long long z[16] = {0};
        cudaMemcpyToSymbol(g_phase, z, sizeof(z));
    }
    return 0;
}
#endif

int workspace_reserve(const bm25_index* ix, bm25_workspace* ws, int32_t nq, int64_t n_tok,
                      int32_t kprime, int64_t n_tiles)
{
    (void)ix;
    if (nq > ws->max_queries || !ws->shift) {
        for (void* p : {(void*)ws->shift, (void*)ws->thresh, (void*)ws->qpost})
            if (p)
                cudaFree(p);
        ws->shift = nullptr;
        ws->thresh = nullptr;
        ws->qpost = nullptr;
        const size_t m = (size_t)std::max(nq, 1);
        BM25_CUDA_TRY(cudaMalloc((void**)&ws->shift, sizeof(double) * m));
        BM25_CUDA_TRY(cudaMalloc((void**)&ws->thresh, sizeof(uint32_t) * m));
        BM25_CUDA_TRY(cudaMalloc((void**)&ws->qpost, sizeof(uint32_t) * m));
        ws->max_queries = (int32_t)m;
    }
    BM25_TRY(grow(&ws->seg, &ws->seg_cap, (size_t)n_tok * (size_t)(n_tiles + 1)));
    BM25_TRY(grow(&ws->tcount, &ws->tcount_cap, (size_t)nq * (size_t)n_tiles));
    BM25_TRY(grow(&ws->cand, &ws->cand_cap, (size_t)nq * (size_t)n_tiles * (size_t)kprime));
    return BM25_OK;
}

void workspace_release(bm25_workspace* ws)
{
    void* ps[] = {ws->shift, ws->thresh, ws->qpost, ws->tcount, ws->seg, ws->cand};
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
    ws->qpost = nullptr;
    ws->tcount = nullptr;
    ws->seg = nullptr;
    ws->cand = nullptr;
}

int retrieve_device(const bm25_index* ix, bm25_workspace* ws, const int32_t* q_tokens,
                    const int64_t* q_off, int32_t nq, int64_t n_tok, int32_t k, int32_t* out_ids,
                    float* out_scores, const Plan& plan, cudaStream_t s)
{
    const int32_t tile_docs = plan.tile_docs;
    if (nq == 0)
        return BM25_OK;
    DeviceInfo di;
    BM25_TRY(device_info(&di));
    const int64_t N = ix->n_docs;
    const int32_t kprime = (int32_t)std::min<int64_t>(k, N);
    int32_t W = tile_docs > 0 ? tile_docs : 12288;
    // multiples of 128 keep the shared-memory carve-up 16-byte aligned
    int64_t w_need = (N + 127) / 128 * 128;
    if (W > w_need)
        W = (int32_t)w_need;
    const int64_t n_tiles64 = (N + W - 1) / W;
    if (n_tiles64 > 65536)
        return set_error(BM25_E_INVALID, "%lld doc tiles of %d documents: use wider tiles",
                         (long long)n_tiles64, W);
    const int32_t n_tiles = (int32_t)n_tiles64;
    if ((int64_t)nq * n_tiles >= INT32_MAX)
        return set_error(BM25_E_INVALID, "%d queries x %d doc tiles is too many work items for "
                         "one call", nq, n_tiles);
    BM25_TRY(workspace_reserve(ix, ws, nq, n_tok, kprime, n_tiles));

    const int max_blocks = di.sm_count * 16;
    int g0 = (int)std::min<int64_t>((nq + 255) / 256, max_blocks);
    {
        ProfileScope ps_("k_query_prep", s);
        k_query_prep<<<std::max(g0, 1), 256, 0, s>>>(q_tokens, n_tok, q_off, nq, ix->s0,
                                                      ix->indptr, ix->vocab, ws->shift,
                                                      ws->thresh, ws->qpost, ix->status);
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
    const size_t smem = tile_smem_bytes(W, plan.threads);
    const int64_t n_items = (int64_t)nq * n_tiles;
    auto launch_tile = [&](auto kernel, int threads) -> int {
        BM25_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
        int per_sm = 0;
        BM25_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads,
                                                                    smem));
        if (per_sm < 1)
            return set_error(BM25_E_INVALID, "doc tile of %d documents does not fit on an SM", W);
#ifdef BM25_PHASE_TIMING
        if (const char* e = getenv("BM25_CTAS_PER_SM"))
            per_sm = std::min(per_sm, atoi(e));
#endif
        const int g2 = (int)std::min<int64_t>(n_items, (int64_t)di.sm_count * per_sm);
        {
            ProfileScope ps_("k_tile_topk", s);
            kernel<<<g2, threads, smem, s>>>(q_tokens, n_tok, q_off, nq, N, ix->indices, ix->data,
                                             ws->seg, W, n_tiles, kprime, ws->thresh, ws->qpost,
                                             ws->tcount, ws->cand);
        }
        count_launch();
        BM25_LAUNCH_CHECK();
        return BM25_OK;
    };
    if (plan.threads == 128)
        BM25_TRY(launch_tile(k_tile_topk<128>, 128));
    else if (plan.threads == 256)
        BM25_TRY(launch_tile(k_tile_topk<256>, 256));
    else
        BM25_TRY(launch_tile(k_tile_topk<512>, 512));
    int sz = 1;
    while (sz < kprime)
        sz <<= 1;
    const int32_t buf_cap =
        (int32_t)std::min<int64_t>(kMergeBufCap, (int64_t)n_tiles * kprime);
    const size_t msmem = (size_t)sz * sizeof(u64) + (size_t)buf_cap * sizeof(u64) +
                         (size_t)(n_tiles + 1) * sizeof(uint32_t);
    BM25_CUDA_TRY(cudaFuncSetAttribute(k_merge, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)msmem));
    {
        ProfileScope ps_("k_merge", s);
        k_merge<<<nq, kMergeThreads, msmem, s>>>(ws->cand, ws->tcount, nq, n_tiles, kprime, k,
                                                 ws->shift, out_ids, out_scores, buf_cap);
    }
    count_launch();
    BM25_LAUNCH_CHECK();
    return BM25_OK;
}

}  // namespace bm25
