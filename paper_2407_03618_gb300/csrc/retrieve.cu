// Batched top-k retrieval over the eager term-major index (arXiv 2407.03618
// Sec. 2 "Assigning Query Scores" and "Top-k selection"; Sec. 2.1 for the
// shift added back to every returned score).
//
// Launches per call (per sub-batch for R0, R2, R3, R4):
//   R0 k_query_prep   sum_i S0(q_i) per query in FP64; token / offset checks;
//                     the query's postings (sum of DF); routes each query to
//                     the dense path (few postings) or the doc-tiled path and
//                     resets the running threshold of the tiled ones
//   R1 k_seg_bounds   for every query token and every doc-tile boundary, the
//                     first posting of the token's column at or past the
//                     boundary (binary search: doc ids ascend in a column),
//                     as a slot of the packed (doc, score) layout
//   R2 k_tile_staged  persistent CTAs over (doc tile, query) items taken from
//                     a device work queue: a producer warp stages each
//                     item's posting segments into shared memory with
//                     bulk asynchronous copies; consumer
//                     warps scatter-add them into the tile's FP32
//                     accumulators, claim each touched document once, keep
//                     the ones that clear the query's running threshold and
//                     select the tile's best k' (including the lowest-id
//                     untouched documents, score 0, when they can matter)
//   R3 k_merge_level  (large k' over many tiles) merge tree: groups of tiles
//                     of one query cut to their k' best, in place, until
//                     the candidates left fit one block's shared memory
//      k_merge        per tiled query: the k' best of the tiles' candidates,
//                     re-keyed on the final score, sorted, written out
//   R4 k_dense_topk   per dense-path query: scatter into a dense FP32 vector
//                     in global memory (L2-resident), claim, select, write out
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
constexpr int kTreeKeys = 8192;        // candidates a merge-tree block gathers at most
constexpr uint32_t kZeroKey = 0x80000000u;  // order_f32(0.0f)
// A tiled-path record's k field: k' in the low 16 bits, and kNegScores when
// one of the query's columns holds negative scores (Robertson terms with
// DF > N/2), so that its documents' sums need not grow monotonically.
constexpr int32_t kNegScores = 1 << 30;
constexpr int32_t kKpMask = 0xffff;

// ---- R0 ---------------------------------------------------------------------
// Per query: checks its token range (clamped where malformed), sum_i S0(q_i)
// in FP64, k' = min(k_q, N), and the postings of its columns (an upper bound
// on the documents it touches).  Queries with at most dense_max postings go
// to the list of the dense path (sq, count in ctr[1]); the others get a
// record {q, first token, end token, k' (+ kNegScores)} on the list of the tiled path
// (lrec / lpost / thresh, count in ctr[0]), with their running threshold
// reset.  List order follows the atomic appends; results do not depend on it.
__global__ void k_query_prep(const int32_t* __restrict__ q_tokens, int64_t n_tok,
                             const int64_t* __restrict__ q_off, int32_t nq, int check_first,
                             int check_last, const int32_t* __restrict__ qk, int32_t kmax,
                             int64_t n_docs, const double* __restrict__ s0,
                             const double* __restrict__ idf,
                             const int64_t* __restrict__ indptr, int32_t vocab, int64_t dense_max,
                             double* __restrict__ shift, int32_t* __restrict__ qkp,
                             int4* __restrict__ lrec, uint32_t* __restrict__ lpost,
                             uint32_t* __restrict__ thresh, int32_t* __restrict__ sq,
                             uint32_t* __restrict__ ctr, int* status, int lazy_variant,
                             double lazy_k1, double lazy_delta)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // warp-uniform loop: the list appends are aggregated per warp
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < nq;
         base += stride) {
        const int64_t q = base + lane;
        const bool act = q < nq;
        int64_t lo = 0, hi = 0, post = 0;
        int32_t kp = 0;
        bool neg = false;
        if (act) {
            lo = q_off[q];
            hi = q_off[q + 1];
            if (lo < 0 || hi < lo || hi > n_tok || (check_first && q == 0 && lo != 0) ||
                (check_last && q == nq - 1 && hi != n_tok))
                set_status(status, BM25_E_TOKEN_RANGE);
            lo = lo < 0 ? 0 : (lo > n_tok ? n_tok : lo);
            hi = hi < lo ? lo : (hi > n_tok ? n_tok : hi);
            int32_t kq = qk ? qk[q] : kmax;
            if (kq < 1 || kq > kmax) {
                set_status(status, BM25_E_INVALID);
                kq = kq < 1 ? 1 : kmax;
            }
            kp = (int64_t)kq < n_docs ? kq : (int32_t)n_docs;
            double sum = 0.0;
            for (int64_t m = lo; m < hi; m++) {
                const int32_t t = q_tokens[m];
                if (t < 0 || t >= vocab) {
                    set_status(status, BM25_E_TOKEN_RANGE);
                    continue;
                }
                if (lazy_variant >= 0) {  // S0 at the call's k1, delta
                    double c, z;
                    term_coef(lazy_variant, idf[t], lazy_k1, lazy_delta, &c, &z);
                    sum += z;
                } else {
                    sum += s0[t];
                }
                post += indptr[t + 1] - indptr[t];
                neg |= idf[t] < 0.0;
            }
            shift[q] = sum;
            qkp[q] = kp;
        }
        const bool dense = act && post <= dense_max;
        const bool tiled = act && !dense;
        const uint32_t bd = __ballot_sync(0xffffffffu, dense);
        const uint32_t bt = __ballot_sync(0xffffffffu, tiled);
        uint32_t base_d = 0, base_t = 0;
        if (lane == 0) {
            if (bd)
                base_d = atomicAdd(&ctr[1], (uint32_t)__popc(bd));
            if (bt)
                base_t = atomicAdd(&ctr[0], (uint32_t)__popc(bt));
        }
        base_d = __shfl_sync(0xffffffffu, base_d, 0);
        base_t = __shfl_sync(0xffffffffu, base_t, 0);
        const uint32_t lt = lanemask_lt();
        if (dense)
            sq[base_d + __popc(bd & lt)] = (int32_t)q;
        if (tiled) {
            const uint32_t li = base_t + __popc(bt & lt);
            lrec[li] = make_int4((int32_t)q, (int32_t)lo, (int32_t)hi, kp | (neg ? kNegScores : 0));
            lpost[li] = post > 0xffffffffll ? 0xffffffffu : (uint32_t)post;
            thresh[li] = 0u;  // below every real score key
        }
    }
}

// ---- R1 ---------------------------------------------------------------------
// seg[m * (n_tiles + 1) + j] = first position p in column q_tokens[m] with
// indices[p] >= j * W (j = n_tiles gives the column end).  A token outside
// the vocabulary gets an empty column.
// PACKED: the positions are slots of the packed layout (bm25_index::posts,
// column t shifted by post_start(indptr[t], t) - indptr[t]), as uint32.
template <bool PACKED>
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
        int64_t lo = 0, hi = 0, shift = 0;
        if (t >= 0 && t < vocab) {
            lo = indptr[t];
            hi = indptr[t + 1];
            if (PACKED)
                shift = post_start(lo, t) - lo;
        }
        int64_t pos;
        if (j == 0) {
            pos = lo;
        } else if (j == n_tiles) {
            pos = hi;
        } else {
            const int32_t target = j * W;
            while (lo < hi) {
                int64_t mid = (lo + hi) >> 1;
                if (indices[mid] < target)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            pos = lo;
        }
        if (PACKED)
            reinterpret_cast<uint32_t*>(seg)[i] = (uint32_t)(pos + shift);
        else
            seg[i] = (int32_t)pos;
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
// The selection runs on threads 0 .. nthreads-1 (whole warps), which meet at
// sync() (__syncthreads() for a whole block, a named barrier for a subset).
template <bool TRAIL_SYNC, class Sync, class Get, class Emit>
__device__ void select_top(SelectState& st, uint32_t nthreads, Sync sync, uint32_t n_index,
                           uint32_t n_real, uint32_t k, int skip, u64 common, Get get, Emit emit)
{
    const int lane = threadIdx.x & 31;
    const uint32_t stride = nthreads;
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
            for (uint32_t i = threadIdx.x; i < 256; i += nthreads)
                st.hist[i] = 0;
            sync();
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
            sync();
            if (threadIdx.x < 32)
                select_bucket(st, shift);
            sync();
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
        sync();
}

template <bool TRAIL_SYNC, class Get, class Emit>
__device__ void block_select_idx(SelectState& st, uint32_t n_index, uint32_t n_real, uint32_t k,
                                 int skip, u64 common, Get get, Emit emit)
{
    select_top<TRAIL_SYNC>(st, blockDim.x, [] { __syncthreads(); }, n_index, n_real, k, skip,
                           common, get, emit);
}

// Number of leading bytes shared by every key whose high word lies in
// [kmin, kmax] (the low word, a doc id, is assumed to vary).
__device__ __forceinline__ int common_bytes(uint32_t kmin, uint32_t kmax)
{
    uint32_t x = kmin ^ kmax;
    return x ? (__clz(x) >> 3) : 4;
}

constexpr uint32_t kUntouched = 0x80000000u;  // bits of -0.0f

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

// ---- R2 -----------------------------------------------------------------------
// The tiled path as a producer/consumer pipeline.  One producer warp walks
// the CTA's (doc tile, query) items ahead of the consumers: for each query
// token it copies the token's posting segment inside the tile from the
// packed (doc, score) layout into a shared-memory staging buffer with a
// bulk asynchronous copy (cp.async.bulk, completion counted in bytes on an
// mbarrier).  Segments start on 16-byte boundaries, so each copy is
// widened to whole pairs: the extra slots hold postings of the same column
// outside the tile, or padding, and are dropped by the doc-range test.
// Staging buffers form a ring of plan.stages; an item larger than one buffer
// spans several.  The consumer warps (named barrier 1):
//   scatter  every staged posting in the tile is added to the tile's FP32
//            accumulator in shared memory (Sec. 2 "Assigning Query Scores":
//            the column slices summed per document); the atomic add returns
//            the old value, and -0.0 there (untouched; stored scores are
//            never -0.0) marks the document's first touch, which appends it
//            to the tile's touched list;
//   claim    the touched list is walked once: each document's sum is read,
//            its accumulator reset to -0.0, and a sum that clears the
//            query's running threshold becomes a candidate key (score, ~doc);
//   select   the k' best candidates of the tile go to the item's slots, and
//            a full set of k' raises the query's threshold (Sec. 2 "Top-k
//            selection", restated as a radix select with exact pruning).
// While a document scoring 0 can still rank (threshold at or below the key
// of 0), an item counts over its touched list first, adds the lowest-id
// untouched documents when fewer than k' touched ones score above 0,
// selects over both, and resets through the list.  Candidates beyond
// kCandCap in a claim are put back and selected by a scan of the tile.
constexpr int kMaxStages = 8;        // staging buffers in the ring at most
constexpr int kCandCap = 256;        // candidate keys an item collects in the common case
constexpr uint32_t kTouchCap = 2048; // touched-list entries kept (an item touching more
                                     // documents walks its whole tile instead)
constexpr int kWaitPolls = kHandshakePolls;  // mbarrier polls before a copy wait gives up


// Query-time scoring (an index with lazy postings: doc id and TF | |D| <<
// 16, or TF alone with |D| read from doc_len when either exceeds 16 bits).
// The scores are computed while scattering, with the call's k1, b, delta:
// length factor from |D| and the index's Lavg, coefficient per query token
// from its IDF (entry_score, term_coef).
struct LazyArgs {
    const int32_t* q_tokens;   // the batch's tokens (to look up each token's IDF)
    const double* idf;         // [vocab]
    const int32_t* doc_len;    // [n_docs] (unpacked layout)
    int variant;
    int packed;                // 1: second word = TF | |D| << 16
    double k1, delta;
    float one_minus_b, b_over_lavg;  // K_D = 1 - b + b |D| / Lavg
    float k1f;
    ScoreConsts kc;
};

// Per staging buffer of the lazy kernel: where each of the chunk's (up to)
// 64 query tokens starts in the buffer (start[64] = entries in the buffer;
// tokens with no entries start where the next one does) and its coefficient.
struct __align__(16) SegTable {
    uint16_t start[68];
    float coef[64];
};

constexpr int32_t kModeList = 0;   // first touches listed, claimed after the scatter
constexpr int32_t kModeCross = 1;  // threshold crossings listed, the tile reset in bulk
constexpr int32_t kModeEnd = 3;    // no item: the CTA's work is done

struct __align__(16) StageHdr {
    int32_t n;       // entries in the buffer
    int32_t last;    // 1: the item's last buffer
    int32_t mode;    // kModeList or kModeCross (the same for all buffers of an item), or kModeEnd
    int32_t item, qi;        // the item (doc tile * n_long + query record) and its query record
    uint32_t kp, post, tau;  // the query's k', postings, threshold when staged
};

struct StagedFront {
    unsigned long long full[kMaxStages];   // producer -> consumers (bytes landed)
    unsigned long long empty[kMaxStages];  // consumers -> producer (buffer free)
    StageHdr hdr[kMaxStages];
    uint32_t lc[2], ovf[2];                // candidate count / overflow, per item parity
    uint32_t tl_count[2];                  // touched-list length, per item parity
    uint32_t abort_flag;
    uint32_t scan[33];
    uint32_t cutoff;
    SelectState st;
};
constexpr size_t kStagedFront = (sizeof(StagedFront) + 15) / 16 * 16;

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// Global -> shared bulk copy; bytes a multiple of 16, both addresses 16-byte
// aligned; completion is counted on `bar`.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              unsigned long long* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"((unsigned long long)__cvta_generic_to_global(src)), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Warp-uniform bounded wait for the phase of `bar` with the given parity (a
// producer/consumer handshake).  Gives up (false) after `polls` polls or once
// another warp has given up.
__device__ __forceinline__ bool warp_wait(unsigned long long* bar, uint32_t parity,
                                          const volatile uint32_t* abort_flag, int polls)
{
    for (int i = 0; i < polls; i++) {
        if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity)))
            return true;
        if (__any_sync(0xffffffffu, *abort_flag != 0u))
            return false;
    }
    return false;
}

// Warp-uniform wait for the bulk copies of one fill to land, bounded by
// kWaitPolls whatever the other warps do: a copy completes in bounded time,
// and a CTA must not exit while one still writes its shared memory.
__device__ __forceinline__ bool warp_drain(unsigned long long* bar, uint32_t parity)
{
    for (int i = 0; i < kWaitPolls; i++)
        if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity)))
            return true;
    return false;
}

// acc[dl] += v in shared memory when dl < wd, returning the old value;
// -0.0 (the untouched mark) when nothing is added.  A predicated atomic, so
// that lanes outside the tile do not split the warp.
__device__ __forceinline__ float atom_add_if(float* acc, uint32_t dl, uint32_t wd, float v)
{
    float old = __uint_as_float(0x80000000u);
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.lt.u32 p, %1, %2;\n\t"
        "@p atom.shared.add.f32 %0, [%3], %4;\n\t}"
        : "+f"(old)
        : "r"(dl), "r"(wd), "r"(smem_addr(acc) + dl * 4u), "f"(v)
        : "memory");
    return old;
}

template <int NT>
__device__ __forceinline__ void consumer_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}

// consumer_sync that also returns, to every consumer thread, whether any of
// them passed v = true (barrier reduction).
template <int NT>
__device__ __forceinline__ bool consumer_sync_any(bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, 1, %2, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(NT)
        : "memory");
    return r != 0u;
}

// Exclusive scan across the NT consumer threads (see block_exclusive_sum).
template <int NT, typename T>
__device__ __forceinline__ T consumer_exclusive_sum(T v, T* warp_buf, T* total)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = warp_inclusive_sum(v);
    if (lane == 31)
        warp_buf[warp] = inc;
    consumer_sync<NT>();
    if (warp == 0) {
        T w = (lane < NW) ? warp_buf[lane] : T(0);
        T wi = warp_inclusive_sum(w);
        if (lane < NW)
            warp_buf[lane] = wi - w;
        if (lane == NW - 1)
            warp_buf[32] = wi;
    }
    consumer_sync<NT>();
    T r = warp_buf[warp] + inc - v;
    *total = warp_buf[32];
    consumer_sync<NT>();
    return r;
}

// first_untouched over the consumer threads.
template <int NT>
__device__ uint32_t consumer_first_untouched(const float* acc, int32_t wd, uint32_t k,
                                             uint32_t* scan_buf, uint32_t* cutoff)
{
    const int32_t nwords = (wd + 31) >> 5;
    uint32_t carry = 0;
    if (threadIdx.x == 0)
        *cutoff = (uint32_t)wd;
    for (int w0 = 0; w0 < nwords && carry < k; w0 += NT) {
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
        const uint32_t ex = consumer_exclusive_sum<NT>(z, scan_buf, &tot) + carry;
        if (w < nwords && ex < k && ex + z >= k) {
            uint32_t f = zeros;
            for (uint32_t c = ex + 1; c < k; c++)
                f &= f - 1;
            *cutoff = (uint32_t)((w << 5) + __ffs(f));
        }
        carry += tot;
    }
    consumer_sync<NT>();
    return carry < k ? carry : k;
}

// Shared memory of k_tile_staged: the front, W accumulators, the candidate
// list, `stages` staging buffers of `entries` packed postings, the touched
// list (tl_cap 16-bit entries, rounded to 16 bytes).
size_t staged_smem_bytes(int32_t W, int stages, int entries, uint32_t tl_cap, bool lazy)
{
    return kStagedFront + (size_t)W * sizeof(float) + (size_t)kCandCap * sizeof(u64) +
           (size_t)stages * entries * sizeof(uint2) + ((size_t)tl_cap * sizeof(uint16_t) + 15) / 16 * 16 +
           (lazy ? (size_t)stages * sizeof(SegTable) : 0);
}

// seg (packed): for query token m and tile boundary j, the first slot of the
// token's packed column at or past document j * W (j = n_tiles: the column
// end), from k_seg_bounds<true>.
// Up to four CTAs per SM: the register bound allows four (67 registers per
// thread at 6 consumer warps, the default, 56 at 8); shared memory allows
// four up to W = 7168 and three at the default W = 10240 (73 KB).
template <int CW, bool LAZY>
__global__ void __launch_bounds__((CW + 1) * 32, CW >= 16 ? 2 : (LAZY ? 3 : 4))
    k_tile_staged(int64_t n_docs, const uint2* __restrict__ posts, const uint32_t* __restrict__ seg,
                  int32_t W, int32_t n_tiles, int32_t kstride, const int4* __restrict__ lrec,
                  const uint32_t* __restrict__ lpost, const uint32_t* __restrict__ ctr,
                  uint32_t* queue, uint32_t* __restrict__ thresh, uint32_t* __restrict__ tcount,
                  u64* __restrict__ cand, int* __restrict__ status, int wait_polls,
                  int n_stages, int stage_entries, uint32_t tl_cap, LazyArgs lz)
{
    constexpr int NT = CW * 32;  // consumer threads
    constexpr int OW = CW - 1;   // the output warp (the fewest postings per item)
    extern __shared__ __align__(16) unsigned char smem[];
    StagedFront& sh = *reinterpret_cast<StagedFront*>(smem);
    float* acc = reinterpret_cast<float*>(smem + kStagedFront);
    u64* clist = reinterpret_cast<u64*>(acc + W);
    uint2* stage = reinterpret_cast<uint2*>(clist + kCandCap);
    uint16_t* tl = reinterpret_cast<uint16_t*>(stage + (size_t)n_stages * stage_entries);
    SegTable* segt = reinterpret_cast<SegTable*>(
        reinterpret_cast<unsigned char*>(tl) + ((size_t)tl_cap * sizeof(uint16_t) + 15) / 16 * 16);
    SelectState& st = sh.st;

    const int32_t nq = (int32_t)ctr[0];
    const int32_t n_items = nq * n_tiles;  // < 2^31 (checked by the host)
    if ((int32_t)blockIdx.x >= n_items)
        return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float neg0 = __uint_as_float(kUntouched);
    for (int i = tid; i < W; i += blockDim.x)
        acc[i] = neg0;
    if (tid == 0) {
        for (int s = 0; s < n_stages; s++) {
            mbar_init(&sh.full[s], 1);
            mbar_init(&sh.empty[s], CW);
        }
        sh.lc[0] = sh.lc[1] = 0;
        sh.ovf[0] = sh.ovf[1] = 0;
        sh.tl_count[0] = sh.tl_count[1] = 0;
        sh.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const volatile uint32_t* abort_flag = &sh.abort_flag;
    // Tile-major items (item = tile * nq + q) from a work queue: CTA b starts
    // with item b, then takes the next unclaimed one, G + (*queue)++, so that
    // CTAs that drew cheap items take more of them and all finish together.
    const int64_t per = (int64_t)n_tiles + 1;

    if (warp == CW) {
        // ================================ producer ================================
        // Items are claimed two ahead of the one being staged; loads run one
        // item (segments, threshold) and two items (records) ahead of it.
        // Once the queue is empty the warp stages one fill of kModeEnd.
        const int32_t G = (int32_t)gridDim.x;
        auto claim = [&]() -> int32_t {  // n_items when none is left
            uint32_t v = 0u;
            if (lane == 0)
                v = atomicAdd(queue, 1u);
            v = __shfl_sync(0xffffffffu, v, 0);
            return (int64_t)G + v < (int64_t)n_items ? G + (int32_t)v : n_items;
        };
        int32_t it0 = (int32_t)blockIdx.x;
        int32_t it1 = claim();
        int32_t it2 = claim();
        int32_t t0 = it0 / nq, q0 = it0 - t0 * nq;
        int32_t t1 = it1 / nq, q1 = it1 - t1 * nq;
        int32_t t2 = it2 / nq, q2 = it2 - t2 * nq;
        auto load_pair = [&](int32_t t_, int4 r_, uint32_t* lo, uint32_t* hi) {
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int32_t m = r_.y + 2 * lane + h;
                lo[h] = hi[h] = 0u;
                if (m < r_.z) {
                    lo[h] = seg[(int64_t)m * per + t_];
                    hi[h] = seg[(int64_t)m * per + t_ + 1];
                }
            }
        };
        int4 rec0 = lrec[q0];
        int4 rec1 = make_int4(0, 0, 0, 0), rec2 = make_int4(0, 0, 0, 0);
        if (it1 < n_items)
            rec1 = lrec[q1];
        uint32_t lo0[2], hi0[2];
        load_pair(t0, rec0, lo0, hi0);
        uint32_t tau0 = *(const volatile uint32_t*)&thresh[q0];
        uint32_t post0 = lpost[q0];
        int s = 0;
        uint32_t round = 0;
        bool aborted = false;
        while (it0 < n_items) {
            // next items' loads (consumed in the next iteration)
            const bool has1 = it1 < n_items;
            const bool has2 = it2 < n_items;
            if (has2)
                rec2 = lrec[q2];
            uint32_t lo1[2] = {0u, 0u}, hi1[2] = {0u, 0u}, tau1 = 0u, post1 = 0u;
            if (has1) {
                load_pair(t1, rec1, lo1, hi1);
                tau1 = *(const volatile uint32_t*)&thresh[q1];
                post1 = lpost[q1];
            }
            // stage item (t0, q0)
            const int32_t m0 = rec0.y, m1 = rec0.z;
            for (int32_t mb = m0;; mb += 64) {
                const int cnt = (int)min((int64_t)64, (int64_t)m1 - mb);  // may be <= 0
                uint32_t a[2], n[2];
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    uint32_t lo = lo0[h], hi = hi0[h];
                    if (mb != m0) {  // tokens past the first 64: loaded here
                        lo = hi = 0u;
                        const int32_t m = mb + 2 * lane + h;
                        if (m < m1) {
                            lo = seg[(int64_t)m * per + t0];
                            hi = seg[(int64_t)m * per + t0 + 1];
                        }
                    }
                    const bool live = (2 * lane + h) < cnt && lo < hi;
                    a[h] = lo & ~1u;
                    n[h] = live ? ((hi + 1u) & ~1u) - a[h] : 0u;
                }
                const uint32_t s2 = n[0] + n[1];
                const uint32_t inc = warp_inclusive_sum(s2);
                const uint32_t off[2] = {inc - s2, inc - s2 + n[0]};
                float cf[2] = {0.0f, 0.0f};
                if (LAZY) {  // the chunk's per-token coefficients at the call's k1, delta
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        const int32_t m = mb + 2 * lane + h;
                        if (n[h] > 0u && m < m1) {
                            double c, s0;
                            term_coef(lz.variant, lz.idf[lz.q_tokens[m]], lz.k1, lz.delta, &c, &s0);
                            cf[h] = (float)c;
                        }
                    }
                }
                const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
                const bool last_chunk = (int64_t)mb + 64 >= (int64_t)m1;
                if (total == 0u && !last_chunk)
                    continue;
                const uint32_t se = (uint32_t)stage_entries;
                const uint32_t nst = total == 0u ? 1u : (total + se - 1) / se;
                for (uint32_t k = 0; k < nst; k++) {
                    const uint32_t e0 = k * se;
                    const uint32_t e1 = min(total, e0 + se);
                    // After giving up, nothing more is staged: a buffer whose
                    // consumers gave up may still be receiving its copies.
                    if (!warp_wait(&sh.empty[s], (round & 1u) ^ 1u, abort_flag, wait_polls)) {
                        aborted = true;
                        if (lane == 0) {
                            set_status(status, BM25_E_TIMEOUT);
                            *(volatile uint32_t*)&sh.abort_flag = 1u;
                        }
                        break;
                    }
                    if (LAZY) {  // where each token's entries start in this buffer
                        SegTable& tb = segt[s];
#pragma unroll
                        for (int h = 0; h < 2; h++) {
                            const uint32_t st0 = min(max(off[h], e0), e1) - e0;
                            tb.start[2 * lane + h] = (uint16_t)st0;
                            tb.coef[2 * lane + h] = cf[h];
                        }
                        if (lane == 0)
                            tb.start[64] = (uint16_t)(e1 - e0);
                        __syncwarp();
                    }
                    if (lane == 0) {
                        StageHdr& hd = sh.hdr[s];
                        hd.n = (int32_t)(e1 - e0);
                        hd.last = (last_chunk && k + 1 == nst) ? 1 : 0;
                        // a sum can cross the threshold only once when it only grows
                        hd.mode = (tau0 > kZeroKey && !(rec0.w & kNegScores)) ? kModeCross
                                                                              : kModeList;
                        hd.item = it0;
                        hd.qi = q0;
                        hd.kp = (uint32_t)(rec0.w & kKpMask);
                        hd.post = post0;
                        hd.tau = tau0;
                        mbar_arrive_expect_tx(&sh.full[s], (e1 - e0) * (uint32_t)sizeof(uint2));
                    }
                    __syncwarp();
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        const uint32_t lo_e = max(off[h], e0);
                        const uint32_t hi_e = min(off[h] + n[h], e1);
                        if (lo_e < hi_e)
                            bulk_copy_g2s(stage + (size_t)s * stage_entries + (lo_e - e0),
                                          posts + a[h] + (lo_e - off[h]),
                                          (hi_e - lo_e) * (uint32_t)sizeof(uint2), &sh.full[s]);
                    }
                    if (++s == n_stages) {
                        s = 0;
                        round++;
                    }
                }
                if (last_chunk || aborted)
                    break;
            }
            if (aborted)
                break;
            // shift the pipeline
            rec0 = rec1;
            rec1 = rec2;
            lo0[0] = lo1[0];
            lo0[1] = lo1[1];
            hi0[0] = hi1[0];
            hi0[1] = hi1[1];
            tau0 = tau1;
            post0 = post1;
            it0 = it1;
            t0 = t1;
            q0 = q1;
            it1 = it2;
            t1 = t2;
            q1 = q2;
            it2 = claim();
            t2 = it2 / nq;
            q2 = it2 - t2 * nq;
        }
        if (!aborted) {  // the end: a fill without postings that names no item
            if (!warp_wait(&sh.empty[s], (round & 1u) ^ 1u, abort_flag, wait_polls)) {
                if (lane == 0) {
                    set_status(status, BM25_E_TIMEOUT);
                    *(volatile uint32_t*)&sh.abort_flag = 1u;
                }
            } else {
                if (lane == 0) {
                    StageHdr& hd = sh.hdr[s];
                    hd.n = 0;
                    hd.last = 1;
                    hd.mode = kModeEnd;
                    mbar_arrive_expect_tx(&sh.full[s], 0u);
                }
                __syncwarp();
                if (++s == n_stages) {
                    s = 0;
                    round++;
                }
            }
        }
        // The copies of the last fill of every stage have landed before the
        // warp leaves, also after giving up (an earlier fill of a stage
        // completed before its buffer was released for the next one).
        for (int k = 0; k < n_stages; k++) {
            if (s == 0) {
                s = n_stages;
                if (round == 0)
                    break;
                round--;
            }
            s--;
            warp_drain(&sh.full[s], round & 1u);
        }
        return;
    }

    // ================================ consumers ================================
    int s = 0;
    uint32_t round = 0, par = 0;
    bool aborted = false;
    auto csync = [] { consumer_sync<NT>(); };
    const uint32_t ltmask = lanemask_lt();
    for (;; par ^= 1u) {
        int32_t item = 0, tile = 0, qi = 0, mode = kModeList;
        bool done = false;
        uint32_t qkp = 1, post = 0, tau = 0;
        uint32_t d0u = 0, wdu = 0;
        float tau_f = 0.0f;
        bool cross = false, first_fill = true;
        // ---- scatter the item's staged postings ----------------------------------
        for (;;) {
            if (!warp_wait(&sh.full[s], round & 1u, abort_flag, wait_polls)) {
                // give up without releasing the buffer (its copies may still
                // be landing; the producer waits for them before it leaves)
                aborted = true;
                if (lane == 0) {
                    set_status(status, BM25_E_TIMEOUT);
                    *(volatile uint32_t*)&sh.abort_flag = 1u;
                }
                break;
            }
            const StageHdr& hd = sh.hdr[s];
            const int2 nl = *reinterpret_cast<const int2*>(&hd.n);  // entries, last fill
            if (first_fill) {  // the item's fields, the same in all its fills
                first_fill = false;
                if (hd.mode == kModeEnd) {  // (the same fill for every consumer warp)
                    done = true;
                    break;
                }
                item = hd.item;
                qi = hd.qi;
                tile = (item - qi) / nq;
                qkp = hd.kp;
                post = hd.post;
                tau = hd.tau;
                mode = hd.mode;
                cross = mode == kModeCross;  // warp-uniform
                tau_f = unorder_f32(tau);    // (used when tau is above the key of 0)
                d0u = (uint32_t)tile * (uint32_t)W;
                wdu = (uint32_t)min((int64_t)W, n_docs - (int64_t)d0u);
            }
            // Lane l of a warp takes entries 64 j + l and 64 j + 32 + l of the
            // buffer (chunk j of 64 entries to warp j % CW), so the 32 adds of one
            // instruction go to consecutive postings: a dense column's documents
            // then fall in distinct shared-memory banks.
            const int32_t n_e = min(max(nl.x, 0), stage_entries);
            const uint2* sb = stage + (size_t)s * stage_entries;
            for (int32_t e0 = warp * 64; e0 < n_e; e0 += 2 * NT) {
                const int32_t ea = e0 + lane, eb = ea + 32;
                const uint2 pa = ea < n_e ? sb[ea] : make_uint2(kPostPad, 0u);
                const uint2 pb = eb < n_e ? sb[eb] : make_uint2(kPostPad, 0u);
                const uint32_t dl0 = pa.x - d0u, dl1 = pb.x - d0u;
                float v0 = __uint_as_float(pa.y), v1 = __uint_as_float(pb.y);
                if (LAZY) {
                    // an entry's token: the last one starting at or before it
                    const SegTable& tb = segt[s];
                    auto coef_of = [&](int32_t e) {
                        int lo = 0, hi = 65;
                        while (hi - lo > 1) {
                            const int mid = (lo + hi) >> 1;
                            if ((int32_t)tb.start[mid] <= e)
                                lo = mid;
                            else
                                hi = mid;
                        }
                        return tb.coef[min(lo, 63)];
                    };
                    auto lazy_v = [&](uint32_t w, uint32_t dl, float c) {
                        uint32_t tfv, len;
                        if (lz.packed) {
                            tfv = w & 0xffffu;
                            len = w >> 16;
                        } else {
                            tfv = w;
                            len = dl < wdu ? (uint32_t)lz.doc_len[d0u + dl] : 0u;
                        }
                        const float kd = fmaf(lz.b_over_lavg, (float)len, lz.one_minus_b);
                        const float a = (lz.variant == BM25_L || lz.variant == BM25_TFLDP)
                                            ? 1.0f / kd
                                            : lz.k1f * kd;
                        return entry_score(lz.variant, (float)tfv, a, c, lz.kc);
                    };
                    v0 = lazy_v(pa.y, dl0, coef_of(ea));
                    v1 = lazy_v(pb.y, dl1, coef_of(eb));
                }
                // the sums before the adds (-0.0 where nothing was added)
                const float o0 = atom_add_if(acc, dl0, wdu, v0);
                const float o1 = atom_add_if(acc, dl1, wdu, v1);
                // listed: a first touch (the old value is -0.0), or in the crossing
                // mode the posting that lifts the sum to the threshold
                bool f0, f1;
                if (cross) {
                    f0 = dl0 < wdu && o0 + v0 >= tau_f && !(o0 >= tau_f);
                    f1 = dl1 < wdu && o1 + v1 >= tau_f && !(o1 >= tau_f);
                } else {
                    f0 = dl0 < wdu && __float_as_uint(o0) == kUntouched;
                    f1 = dl1 < wdu && __float_as_uint(o1) == kUntouched;
                }
                const uint32_t b0 = __ballot_sync(0xffffffffu, f0);
                const uint32_t b1 = __ballot_sync(0xffffffffu, f1);
                if (b0 | b1) {
                    const uint32_t n0 = __popc(b0);
                    uint32_t base = 0;
                    if (lane == 0)
                        base = atomicAdd(&sh.tl_count[par], n0 + (uint32_t)__popc(b1));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    const uint32_t p0 = base + __popc(b0 & ltmask);
                    const uint32_t p1 = base + n0 + __popc(b1 & ltmask);
                    if (f0 && p0 < tl_cap)  // beyond the cap only counted
                        tl[p0] = (uint16_t)dl0;
                    if (f1 && p1 < tl_cap)
                        tl[p1] = (uint16_t)dl1;
                }
            }
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&sh.empty[s]);
            if (++s == n_stages) {
                s = 0;
                round++;
            }
            if (nl.y != 0)
                break;
        }
        if (done)
            return;
        // every posting added, every first touch (crossing) listed; if any
        // consumer warp gave up, all of them leave here together, so that no
        // warp waits at a later barrier for one that left
        if (consumer_sync_any<NT>(aborted))
            return;

        const int64_t d0 = (int64_t)tile * W;
        const int32_t wd = (int32_t)min((int64_t)W, n_docs - d0);
        const uint32_t n_t = sh.tl_count[par];
        if (tid == 0) {  // counters of the next item (used after its scatter barrier)
            sh.lc[par ^ 1u] = 0;
            sh.ovf[par ^ 1u] = 0;
            sh.tl_count[par ^ 1u] = 0;
        }
        const uint32_t kp = min(qkp, (uint32_t)wd);
        u64* out = cand + (int64_t)item * kstride;
        uint32_t n_emit = 0, new_tau = 0;
        bool tau_ok = false;
        auto emit = [&](u64 key, uint32_t slot) { out[slot] = key; };
        const bool zero_counts = tau <= kZeroKey;
        // the k' best of the candidate keys clist[0 .. n_c) (n_c <= kCandCap) to the
        // item's slots; a full set raises the threshold
        auto select_clist = [&](uint32_t n_c) {
            if (n_c <= kp) {
                if (warp == OW) {
                    uint32_t m = 0xffffffffu;
                    for (uint32_t i = lane; i < n_c; i += 32) {
                        const u64 key = clist[i];
                        out[i] = key;
                        m = min(m, (uint32_t)(key >> 32));
                    }
                    new_tau = __reduce_min_sync(0xffffffffu, m);
                    tau_ok = n_c > 0;
                }
                n_emit = n_c;
            } else if (n_c <= 32) {
                if (warp == OW) {  // a few too many: sorted in registers
                    u64 key = (uint32_t)lane < n_c ? clist[lane] : 0ull;
                    key = warp_sort_desc(key);
                    if ((uint32_t)lane < kp)
                        out[lane] = key;
                    new_tau = (uint32_t)(__shfl_sync(0xffffffffu, key, kp - 1) >> 32);
                    tau_ok = true;
                }
                n_emit = kp;
            } else {
                if (tid == 0)
                    st.ctr = 0;
                select_top<false>(st, NT, csync, n_c, n_c, kp, 0, 0ull,
                                  [&](uint32_t i) -> u64 { return clist[i]; }, emit);
                new_tau = (uint32_t)(st.prefix >> 32);
                tau_ok = true;
                n_emit = kp;
            }
        };
        auto reset_tile = [&]() {  // every accumulator of the tile back to -0.0
            float4* a4 = reinterpret_cast<float4*>(acc);
            const float4 z = make_float4(neg0, neg0, neg0, neg0);
#pragma unroll 8
            for (int32_t i = tid; i < (wd + 3) / 4; i += NT)
                a4[i] = z;
        };

        if (mode == kModeCross) {
            // ---- the listed documents are exactly those at or above the threshold -----
            if (n_t <= (uint32_t)kCandCap) {
                for (uint32_t i = tid; i < n_t; i += NT) {
                    const uint32_t dl = tl[i];
                    clist[i] = make_key(acc[dl], (uint32_t)(d0 + dl));
                }
                if (n_t > 0)
                    consumer_sync<NT>();  // every candidate's sum read before the reset
                reset_tile();
                select_clist(n_t);
            } else {
                if (tid == 0)
                    st.ctr = 0;
                consumer_sync<NT>();  // (with n_t <= k' the select emits at once)
                select_top<true>(st, NT, csync, (uint32_t)wd, n_t, kp, 0, 0ull,
                                 [&](uint32_t d) -> u64 {
                                     const float v = acc[d];
                                     return __float_as_uint(v) != kUntouched &&
                                                    order_f32(v) >= tau
                                                ? make_key(v, (uint32_t)(d0 + d))
                                                : 0ull;
                                 },
                                 emit);
                n_emit = min(n_t, kp);
                if (n_t > kp) {
                    new_tau = (uint32_t)(st.prefix >> 32);
                    tau_ok = true;
                }
                reset_tile();
            }
            consumer_sync<NT>();  // the tile is clean before the next scatter
        } else if (!zero_counts) {
            // ---- claim: read and reset each touched document once ------------------
            // (through the touched list, or over the whole tile when the list
            // overflowed; a touched sum is never -0.0)
            const bool walk = n_t > tl_cap;
            const uint32_t n_w = walk ? (uint32_t)wd : n_t;
            for (uint32_t b0 = warp * 32; b0 < n_w; b0 += NT) {  // warp-uniform
                const uint32_t t = b0 + lane;
                bool keep = false;
                uint32_t dl = 0;
                float v = 0.0f;
                if (t < n_w) {
                    dl = walk ? t : tl[t];
                    v = acc[dl];
                    if (__float_as_uint(v) != kUntouched) {
                        acc[dl] = neg0;
                        keep = order_f32(v) >= tau;
                    }
                }
                const uint32_t bal = __ballot_sync(0xffffffffu, keep);
                if (bal) {
                    const int leader = __ffs(bal) - 1;
                    uint32_t base = 0;
                    if (lane == leader)
                        base = atomicAdd(&sh.lc[par], (uint32_t)__popc(bal));
                    base = __shfl_sync(0xffffffffu, base, leader);
                    if (keep) {
                        const uint32_t pos = base + __popc(bal & ltmask);
                        if (pos < (uint32_t)kCandCap) {
                            clist[pos] = make_key(v, (uint32_t)(d0 + dl));
                        } else {  // no room: the sum goes back for the general select
                            acc[dl] = v;
                            sh.ovf[par] = 1;
                        }
                    }
                }
            }
            consumer_sync<NT>();
            const uint32_t n_c = sh.lc[par];
            if (!sh.ovf[par]) {
                select_clist(n_c);
            } else {
                // more candidates than the list holds: select over the list and
                // the sums put back in the tile
                if (tid == 0)
                    st.ctr = 0;
                consumer_sync<NT>();  // (with n_c <= k' the select emits at once)
                select_top<true>(st, NT, csync, (uint32_t)kCandCap + (uint32_t)wd, n_c, kp, 0, 0ull,
                                 [&](uint32_t i) -> u64 {
                                     if (i < (uint32_t)kCandCap)
                                         return clist[i];
                                     const uint32_t d = i - kCandCap;
                                     const float v = acc[d];
                                     return __float_as_uint(v) != kUntouched
                                                ? make_key(v, (uint32_t)(d0 + d))
                                                : 0ull;
                                 },
                                 emit);
                n_emit = min(n_c, kp);
                if (n_c > kp) {
                    new_tau = (uint32_t)(st.prefix >> 32);
                    tau_ok = true;
                }
                for (int32_t d = tid; d < wd; d += NT)
                    acc[d] = neg0;
                consumer_sync<NT>();
            }
        } else {
            // ---- a score of 0 can still rank: count, fill, select over the lists -------
            // (through the touched list, or over the whole tile when it overflowed)
            const bool walk = n_t > tl_cap;
            uint32_t c = 0, p = 0;
            for (uint32_t t = tid; t < (walk ? (uint32_t)wd : n_t); t += NT) {
                const float v = acc[walk ? t : tl[t]];
                c += __float_as_uint(v) != kUntouched && order_f32(v) >= tau;
                p += v > 0.0f;
            }
            uint32_t n_cand, n_pos, n_unt = 0, cut = 0;
            consumer_exclusive_sum<NT>(c, sh.scan, &n_cand);
            consumer_exclusive_sum<NT>(p, sh.scan, &n_pos);
            const bool may_fill = (int64_t)tile * W < (int64_t)qkp + (int64_t)post;
            if (may_fill && n_pos < kp) {
                n_unt = consumer_first_untouched<NT>(acc, wd, kp, sh.scan, &sh.cutoff);
                cut = sh.cutoff;
            }
            // indexes: the listed documents, then the tile's first `cut`
            // documents (untouched ones score 0); walking, the tile itself
            const uint32_t n_l = walk ? 0u : n_t;
            const uint32_t n_all = n_cand + n_unt;
            n_emit = min(n_all, kp);
            if (tid == 0)
                st.ctr = 0;
            consumer_sync<NT>();
            select_top<true>(st, NT, csync, walk ? (uint32_t)wd : n_l + cut, n_all, kp, 0, 0ull,
                             [&](uint32_t i) -> u64 {
                                 if (walk) {
                                     const float v = acc[i];
                                     if (__float_as_uint(v) != kUntouched)
                                         return order_f32(v) >= tau
                                                    ? make_key(v, (uint32_t)(d0 + i))
                                                    : 0ull;
                                     return i < cut ? make_key(0.0f, (uint32_t)(d0 + i)) : 0ull;
                                 }
                                 if (i < n_l) {
                                     const uint32_t dl = tl[i];
                                     const float v = acc[dl];
                                     return order_f32(v) >= tau ? make_key(v, (uint32_t)(d0 + dl))
                                                                : 0ull;
                                 }
                                 const uint32_t d = i - n_l;
                                 return __float_as_uint(acc[d]) == kUntouched
                                            ? make_key(0.0f, (uint32_t)(d0 + d))
                                            : 0ull;
                             },
                             emit);
            if (n_all > kp) {
                new_tau = (uint32_t)(st.prefix >> 32);
                tau_ok = true;
            }
            if (walk) {
                reset_tile();
            } else {
                for (uint32_t t = tid; t < n_t; t += NT)
                    acc[tl[t]] = neg0;
            }
            consumer_sync<NT>();
        }
        // the output warp's first lane records the item (select paths: every
        // thread holds the result; the others computed it in warp OW)
        if (tid == OW * 32) {
            tcount[item] = n_emit;
            // a full set of the query's k' candidates raises its threshold to (a
            // lower bound on) the weakest of them (a tile narrower than k' never does)
            if (tau_ok && n_emit == qkp && qkp > 0)
                atomicMax(&thresh[qi], new_tau);
        }
    }
}

// ---- finishing a query's row (R3 and R4) ------------------------------------
// sel[0 .. sz) holds the k' selected keys (slots past them 0; sz a power of
// two >= k').  Re-keys them on the final FP32 score B = S + sum_i S0(q_i)
// (Sec. 2.1), so that equal returned scores list the lower doc id first,
// sorts them descending (bitonic) and writes row slots 0 .. kout-1: ids and
// scores, -1 / -inf past the k' documents.  All threads of the block call it.
__device__ void finish_row(u64* sel, int sz, uint32_t kp, int32_t kout, double sh,
                           int32_t* __restrict__ ids, float* __restrict__ scores,
                           int32_t id_base)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < sz; i += nt) {
        const u64 key = sel[i];
        if ((uint32_t)i < kp && key != 0ull)
            sel[i] = make_key((float)((double)key_score(key) + sh), key_doc(key));
    }
    __syncthreads();
    for (int size = 2; size <= sz; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < sz / 2; i += nt) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool desc = ((lo & size) == 0);
                const u64 a = sel[lo], b = sel[hi];
                if ((a < b) == desc) {
                    sel[lo] = b;
                    sel[hi] = a;
                }
            }
            __syncthreads();
        }
    }
    for (int r = tid; r < kout; r += nt) {
        const u64 key = (uint32_t)r < kp ? sel[r] : 0ull;
        if (key != 0ull) {
            ids[r] = (int32_t)key_doc(key) + id_base;
            scores[r] = key_score(key);
        } else {
            ids[r] = -1;
            scores[r] = -__int_as_float(0x7f800000);
        }
    }
}

// ---- R3 -----------------------------------------------------------------------
// Merge tree.  A query's tiles all start with no threshold when they run in
// the same wave (a small batch), so each hands over its k' best: up to
// n_tiles x k' candidates, too many for one block to select from quickly
// when k' is large.  One level merges groups of `fan` consecutive virtual
// tiles (tile j * tstride, j = 0, 1, ...) of each query in place: block
// (g, b) = (blockIdx.x / nb, blockIdx.x % nb) gathers the candidates of
// group g of query record b into shared memory (fan * kstride keys at
// most), keeps their k' best (all of them when there are no more than k')
// and writes them, with their count, to the slots of the group's first
// tile.  The next level, or k_merge, then reads the tiles at stride
// tstride * fan.  A group of one tile is left as it is.  A key left out of
// its group's k' best has k' keys above it and so is not among the query's
// k' best either: the result is the one selection over all the candidates
// would give.
__global__ void __launch_bounds__(kMergeThreads)
    k_merge_level(u64* __restrict__ cand, uint32_t* __restrict__ tcount,
                  const int4* __restrict__ lrec, const uint32_t* __restrict__ ctr,
                  int32_t n_tiles, int32_t tstride, int32_t fan, int32_t kstride, int32_t nb)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SelectState st;
    __shared__ uint32_t pre[kMergeThreads + 1];
    const int32_t nl = (int32_t)ctr[0];
    const int32_t b = (int32_t)(blockIdx.x % (uint32_t)nb);
    const int32_t g = (int32_t)(blockIdx.x / (uint32_t)nb);
    if (b >= nl)
        return;
    const int64_t n_v = ((int64_t)n_tiles + tstride - 1) / tstride;
    const int64_t v0 = (int64_t)g * fan;
    const int32_t nv = (int32_t)min((int64_t)fan, n_v - v0);  // fan <= kMergeThreads
    if (nv <= 1)
        return;
    const uint32_t kp = (uint32_t)(lrec[b].w & kKpMask);
    u64* buf = reinterpret_cast<u64*>(smem);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    auto slot0 = [&](int64_t v) { return (v * tstride * nl + b); };  // item of virtual tile v
    const uint32_t c = tid < nv ? min(tcount[slot0(v0 + tid)], (uint32_t)kstride) : 0u;
    uint32_t tot;
    const uint32_t ex = block_exclusive_sum(c, st.red, &tot);
    if (tid < nv)
        pre[tid] = ex;
    if (tid == 0) {
        pre[nv] = tot;
        st.ctr = 0;
    }
    __syncthreads();
    for (int j = warp; j < nv; j += kMergeThreads / 32) {  // one warp per tile
        const u64* src = cand + slot0(v0 + j) * kstride;
        const uint32_t a = pre[j], cj = pre[j + 1] - a;
        for (uint32_t s = lane; s < cj; s += 32)
            buf[a + s] = src[s];
    }
    __syncthreads();  // every key read before the group's first slots are rewritten
    u64* out = cand + slot0(v0) * kstride;
    if (tot <= kp) {
        for (uint32_t i = tid; i < tot; i += kMergeThreads)
            out[i] = buf[i];
    } else {
        block_select_idx<false>(st, tot, tot, kp, 0, 0ull, [&](uint32_t i) { return buf[i]; },
                                [&](u64 key, uint32_t slot) { out[slot] = key; });
    }
    if (tid == 0)
        tcount[slot0(v0)] = min(tot, kp);
}

// Per query of the tiled path (block b: record b): gather the candidates of
// the virtual tiles j * tstride (tcount[tile * n_long + b] of them in that
// item's kstride slots), select the k' best and finish the query's row.
// Dynamic shared memory: sel[pow2 >= kstride] | buf[buf_cap] keys |
// pre[n_v + 1], n_v = ceil(n_tiles / tstride).
__global__ void __launch_bounds__(kMergeThreads)
    k_merge(const u64* __restrict__ cand, const uint32_t* __restrict__ tcount,
            const int4* __restrict__ lrec, const uint32_t* __restrict__ ctr, int32_t n_tiles,
            int32_t tstride, int32_t kstride, int32_t kout, const double* __restrict__ shift,
            int32_t* __restrict__ out_ids, float* __restrict__ out_scores, int32_t buf_cap,
            int32_t id_base)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SelectState st;
    const int32_t nl = (int32_t)ctr[0];
    const int b = blockIdx.x;
    if (b >= nl)
        return;
    const int4 rec = lrec[b];
    const int32_t q = rec.x;
    const uint32_t kp = (uint32_t)(rec.w & kKpMask);
    int sz_all = 1;
    while (sz_all < kstride)
        sz_all <<= 1;
    int sz = 1;
    while ((uint32_t)sz < kp)
        sz <<= 1;
    u64* sel = reinterpret_cast<u64*>(smem);
    u64* buf = sel + sz_all;
    uint32_t* pre = reinterpret_cast<uint32_t*>(buf + buf_cap);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t n_v = (int32_t)(((int64_t)n_tiles + tstride - 1) / tstride);
    auto item_of = [&](int32_t v) { return (int64_t)v * tstride * nl + b; };

    // exclusive scan of the per-tile counts
    uint32_t carry = 0;
    for (int t0 = 0; t0 < n_v; t0 += kMergeThreads) {
        const int t = t0 + tid;
        // (at most kstride: a count left unwritten by a tile kernel that gave
        // up must not send the gather past the item's slots)
        const uint32_t c = t < n_v ? min(tcount[item_of(t)], (uint32_t)kstride) : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_sum(c, st.red, &tot);
        if (t < n_v)
            pre[t] = carry + ex;
        carry += tot;
    }
    if (tid == 0)
        pre[n_v] = carry;
    for (int i = tid; i < sz; i += kMergeThreads)
        sel[i] = 0ull;
    if (tid == 0)
        st.ctr = 0;
    __syncthreads();
    const uint32_t total = pre[n_v];  // >= k': the tiles hold enough candidates
    const bool gathered = total <= (uint32_t)buf_cap;
    if (gathered) {  // one warp per tile copies its candidates
        for (int t = warp; t < n_v; t += kMergeThreads / 32) {
            const uint32_t c = pre[t + 1] - pre[t];
            const u64* src = cand + item_of(t) * kstride;
            for (uint32_t s = lane; s < c; s += 32)
                buf[pre[t] + s] = src[s];
        }
        __syncthreads();
    }
    auto get = [&](uint32_t i) -> u64 {
        if (gathered)
            return buf[i];
        int a = 0, e = n_v;  // pre[a] <= i < pre[e]
        while (e - a > 1) {
            const int mid = (a + e) >> 1;
            if (pre[mid] <= i)
                a = mid;
            else
                e = mid;
        }
        return cand[item_of(a) * kstride + (i - pre[a])];
    };
    block_select_idx<true>(st, total, total, kp, 0, 0ull, get, [&](u64 key, uint32_t slot) {
        if (slot < kp)
            sel[slot] = key;
    });
    finish_row(sel, sz, kp, kout, shift[q], out_ids + (int64_t)q * kout,
               out_scores + (int64_t)q * kout, id_base);
}

// ---- R4 -----------------------------------------------------------------------
// The dense path for queries with few postings: one CTA per query, taken from
// the short list by an atomic counter (ctr[2]).  The CTA owns a dense FP32
// vector of N accumulators in global memory, all -0.0 between queries; only
// the sectors the query touches are brought in, and they stay in L2 while the
// query runs.
//   1. scatter: every posting (d, S) of the query's columns is added to
//      acc[d] with a fire-and-forget reduction (Sec. 2 "Assigning Query
//      Scores": the summed column slices);
//   2. claim: each posting's document is exchanged for -0.0, so the first
//      claimer of a document gets its sum and the vector is clean again; the
//      first claims go, as keys, to the CTA's candidate list (global memory);
//   3. fill: if fewer than k' touched documents score > 0, the untouched
//      documents (score 0) can rank: the k' lowest-id ones lie below
//      R = k' + touched, found through a shared-memory bitmap of the touched
//      documents below R, and are appended to the list;
//   4. select the k' best of the list (radix select) and finish the row.
constexpr int kDenseThreads = 256;

struct DenseStage {
    int32_t lo[kTokChunk];
    int32_t pre[kTokChunk + 1];
    uint32_t scan[33];
    uint32_t n_first, n_pos, kmin, kmax;
    uint32_t item;
};

// Loads the columns of query tokens [mb, mb + cnt) into ds.lo / ds.pre
// (warp 0; cnt <= kTokChunk).  A token outside the vocabulary has an empty
// column.
__device__ __forceinline__ void dense_columns(DenseStage& ds, const int32_t* __restrict__ q_tokens,
                                              const int64_t* __restrict__ indptr, int32_t vocab,
                                              int64_t mb, int cnt)
{
    const int lane = threadIdx.x & 31;
    int32_t len[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int i = 2 * lane + h;
        int32_t l = 0, n = 0;
        if (i < cnt) {
            const int32_t t = q_tokens[mb + i];
            if (t >= 0 && t < vocab) {
                const int64_t a = indptr[t];
                l = (int32_t)a;  // positions < nnz <= 2^31 - 2
                n = (int32_t)(indptr[t + 1] - a);
            }
        }
        len[h] = n;
        ds.lo[i] = l;
    }
    const int32_t s2 = len[0] + len[1];
    const int32_t inc = warp_inclusive_sum(s2);
    ds.pre[2 * lane] = inc - s2;
    ds.pre[2 * lane + 1] = inc - s2 + len[0];
    if (lane == 31)
        ds.pre[kTokChunk] = inc;
}

// Token of the first posting of run r0 (ds.pre[a] <= 32 r0 < ds.pre[a+1]).
__device__ __forceinline__ int dense_first_token(const DenseStage& ds, int cnt, int32_t eb)
{
    int a = 0, b = cnt;
    while (b - a > 1) {
        const int mid = (a + b) >> 1;
        if (ds.pre[mid] <= eb)
            a = mid;
        else
            b = mid;
    }
    return a;
}

__global__ void __launch_bounds__(kDenseThreads)
    k_dense_topk(const int32_t* __restrict__ q_tokens, int64_t n_tok,
                 const int64_t* __restrict__ q_off, const int32_t* __restrict__ qkp,
                 const double* __restrict__ shift, const int64_t* __restrict__ indptr,
                 const int32_t* __restrict__ indices, const float* __restrict__ data,
                 int32_t vocab, int64_t n_docs, const int32_t* __restrict__ sq,
                 uint32_t* __restrict__ ctr, float* __restrict__ slots, u64* __restrict__ lists,
                 int64_t list_cap, int32_t kstride, int32_t kout, int32_t* __restrict__ out_ids,
                 float* __restrict__ out_scores, int32_t id_base)
{
    constexpr int WARPS = kDenseThreads / 32;
    constexpr int U = 8;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SelectState st;
    __shared__ DenseStage ds;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int sz_all = 1;
    while (sz_all < kstride)
        sz_all <<= 1;
    u64* sel = reinterpret_cast<u64*>(smem);
    uint32_t* bits = reinterpret_cast<uint32_t*>(sel + sz_all);
    float* acc = slots + (size_t)blockIdx.x * (size_t)n_docs;
    u64* list = lists + (size_t)blockIdx.x * (size_t)list_cap;
    const uint32_t n_short = ctr[1];
    const uint32_t ltmask = lanemask_lt();
    const uint32_t N32 = (uint32_t)n_docs;  // n_docs < 2^31

    for (;;) {
        if (tid == 0) {
            ds.item = atomicAdd(&ctr[2], 1u);
            ds.n_first = 0;
            ds.n_pos = 0;
            ds.kmin = 0xffffffffu;
            ds.kmax = 0u;
            st.ctr = 0;
        }
        __syncthreads();
        const uint32_t item = ds.item;
        if (item >= n_short)
            break;
        const int32_t q = sq[item];
        int64_t lo = q_off[q], hi = q_off[q + 1];  // checked by k_query_prep; clamped here
        lo = lo < 0 ? 0 : (lo > n_tok ? n_tok : lo);
        hi = hi < lo ? lo : (hi > n_tok ? n_tok : hi);
        const uint32_t kp = (uint32_t)qkp[q];
        const bool one_chunk = hi - lo <= kTokChunk;

        // ---- 1 and 2: scatter, then claim ----------------------------------------
        uint32_t pos = 0, kmin = 0xffffffffu, kmax = 0u;
        for (int pass = 0; pass < 2; pass++) {
            for (int64_t mb = lo; mb < hi; mb += kTokChunk) {
                const int cnt = (int)min((int64_t)kTokChunk, hi - mb);
                if (pass == 0 || !one_chunk) {
                    __syncthreads();  // earlier readers of ds.lo / ds.pre are done
                    if (warp == 0)
                        dense_columns(ds, q_tokens, indptr, vocab, mb, cnt);
                    __syncthreads();
                }
                const int32_t total = ds.pre[kTokChunk];
                for (int32_t r0 = warp; r0 * 32 < total; r0 += U * WARPS) {
                    int a = dense_first_token(ds, cnt, r0 * 32);
                    int32_t dd[U];
                    float vv[U];
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        const int32_t e = (r0 + u * WARPS) * 32 + lane;
                        dd[u] = -1;
                        vv[u] = 0.0f;
                        if (e < total) {
                            while (ds.pre[a + 1] <= e)
                                a++;
                            const int32_t j = ds.lo[a] + (e - ds.pre[a]);
                            const int32_t d = __ldg(indices + j);
                            if ((uint32_t)d < N32) {  // holds for any well-formed index
                                dd[u] = d;
                                if (pass == 0)
                                    vv[u] = __ldg(data + j);
                            }
                        }
                    }
                    if (pass == 0) {
#pragma unroll
                        for (int u = 0; u < U; u++)
                            if (dd[u] >= 0)
                                atomicAdd(acc + dd[u], vv[u]);  // result unused: a reduction
                    } else {
                        float cv[U];  // all exchanges first, so their latencies overlap
#pragma unroll
                        for (int u = 0; u < U; u++)
                            cv[u] = dd[u] >= 0 ? atomicExch(acc + dd[u], __uint_as_float(kUntouched))
                                               : __uint_as_float(kUntouched);
#pragma unroll
                        for (int u = 0; u < U; u++) {
                            const bool first = __float_as_uint(cv[u]) != kUntouched;
                            const uint32_t bal = __ballot_sync(0xffffffffu, first);
                            if (bal) {
                                uint32_t base = 0;
                                if (lane == __ffs(bal) - 1)
                                    base = atomicAdd(&ds.n_first, (uint32_t)__popc(bal));
                                base = __shfl_sync(0xffffffffu, base, __ffs(bal) - 1);
                                if (first) {
                                    const uint32_t o = order_f32(cv[u]);
                                    list[base + __popc(bal & ltmask)] = make_key(cv[u], (uint32_t)dd[u]);
                                    pos += cv[u] > 0.0f;
                                    kmin = min(kmin, o);
                                    kmax = max(kmax, o);
                                }
                            }
                        }
                    }
                }
            }
            __syncthreads();  // pass 0: every reduction precedes every exchange
        }
        pos = __reduce_add_sync(0xffffffffu, pos);
        kmin = __reduce_min_sync(0xffffffffu, kmin);
        kmax = __reduce_max_sync(0xffffffffu, kmax);
        if (lane == 0) {
            if (pos)
                atomicAdd(&ds.n_pos, pos);
            atomicMin(&ds.kmin, kmin);
            atomicMax(&ds.kmax, kmax);
        }
        __syncthreads();
        const uint32_t n_first = ds.n_first;
        const bool fill = ds.n_pos < kp;
        uint32_t n_all = n_first;

        // ---- 3: the lowest-id untouched documents, when they can rank -------------
        if (fill) {
            const int64_t R = min(n_docs, (int64_t)kp + (int64_t)n_first);
            const int32_t nw = (int32_t)((R + 31) >> 5);
            for (int w = tid; w < nw; w += kDenseThreads)
                bits[w] = 0u;
            __syncthreads();
            for (uint32_t i = tid; i < n_first; i += kDenseThreads) {
                const uint32_t d = key_doc(list[i]);
                if ((int64_t)d < R)
                    atomicOr(&bits[d >> 5], 1u << (d & 31));
            }
            __syncthreads();
            uint32_t carry = 0;  // block-uniform
            for (int w0 = 0; w0 < nw && carry < kp; w0 += kDenseThreads) {
                const int w = w0 + tid;
                uint32_t z = 0;
                if (w < nw) {
                    const int rem = (int)(R - ((int64_t)w << 5));
                    const uint32_t valid = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
                    z = ~bits[w] & valid;
                }
                uint32_t tot;
                uint32_t r = block_exclusive_sum((uint32_t)__popc(z), ds.scan, &tot) + carry;
                while (z && r < kp) {
                    const int bpos = __ffs(z) - 1;
                    z &= z - 1;
                    list[n_first + r] = make_key(0.0f, (uint32_t)((w << 5) + bpos));
                    r++;
                }
                carry += tot;
            }
            n_all = n_first + min(carry, kp);
            __syncthreads();
        }

        // ---- 4: select and finish -------------------------------------------------
        int sz = 1;
        while ((uint32_t)sz < kp)
            sz <<= 1;
        for (int i = tid; i < sz; i += kDenseThreads)
            sel[i] = 0ull;
        __syncthreads();
        const int skip = fill ? 0 : common_bytes(ds.kmin, ds.kmax);
        const u64 common = fill ? 0ull : (u64)ds.kmax << 32;
        block_select_idx<true>(st, n_all, n_all, kp, skip, common,
                               [&](uint32_t i) -> u64 { return list[i]; },
                               [&](u64 key, uint32_t slot) {
            if (slot < kp)
                sel[slot] = key;
        });
        finish_row(sel, sz, kp, kout, shift[q], out_ids + (int64_t)q * kout,
                   out_scores + (int64_t)q * kout, id_base);
        // finish_row ends with global writes only; the next query's first
        // barrier orders the reuse of sel and the stage
    }
}

// Sets n 32-bit words to v (the dense vectors start at -0.0).
__global__ void k_fill_u32(uint32_t* __restrict__ p, int64_t n, uint32_t v)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// ---- merge of doc-range shards --------------------------------------------
// Per query (block q): the shards' rows, n_shards * k slots of (global id,
// final score), empty slots id -1; selects the k' = min(k, valid slots) best
// by (score desc, id asc) and writes the sorted row (then -1 / -inf).  The
// scores are final (shift included), so no shift is added.
__global__ void __launch_bounds__(kMergeThreads)
    k_merge_shards(const int32_t* __restrict__ cand_ids, const float* __restrict__ cand_scores,
                   int32_t n_shards, int32_t nq, int32_t k, int32_t* __restrict__ out_ids,
                   float* __restrict__ out_scores)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SelectState st;
    const int q = blockIdx.x;
    const uint32_t n_index = (uint32_t)n_shards * (uint32_t)k;
    auto slot = [&](uint32_t i) -> int64_t {  // shard i / k, rank i % k of query q
        return ((int64_t)(i / (uint32_t)k) * nq + q) * k + (i % (uint32_t)k);
    };
    auto get = [&](uint32_t i) -> u64 {
        const int64_t p = slot(i);
        const int32_t id = cand_ids[p];
        return id >= 0 ? make_key(cand_scores[p], (uint32_t)id) : 0ull;
    };
    uint32_t valid = 0;
    for (uint32_t i = threadIdx.x; i < n_index; i += blockDim.x)
        valid += cand_ids[slot(i)] >= 0;
    uint32_t n_valid;
    block_exclusive_sum(valid, st.red, &n_valid);
    const uint32_t kp = min(n_valid, (uint32_t)k);
    int sz = 1;
    while ((uint32_t)sz < kp)
        sz <<= 1;
    u64* sel = reinterpret_cast<u64*>(smem);
    for (int i = threadIdx.x; i < sz; i += blockDim.x)
        sel[i] = 0ull;
    if (threadIdx.x == 0)
        st.ctr = 0;
    __syncthreads();
    block_select_idx<true>(st, n_index, n_valid, kp, 0, 0ull, get, [&](u64 key, uint32_t s) {
        if (s < kp)
            sel[s] = key;
    });
    finish_row(sel, sz, kp, k, 0.0, out_ids + (int64_t)q * k, out_scores + (int64_t)q * k, 0);
}

constexpr int64_t kCandBudget = int64_t(2) << 30;   // bytes of tile candidates per sub-batch
constexpr int64_t kDenseBudget = int64_t(2) << 30;  // bytes of dense vectors per workspace
constexpr int kDenseCtasPerSm = 2;
constexpr int32_t kDenseMaxL2 = 1 << 19;  // postings bound of the dense path in L2_DENSE mode

// Everything a call's launches depend on, derived from the index, plan and
// batch shape alone (so that reserving and retrieving agree).
struct Geometry {
    int32_t W = 0, n_tiles = 0, kstride = 0, nq_sub = 0;
    int64_t dense_max = -1;  // -1: no dense path
    int32_t dense_ctas = 0;
    int64_t list_cap = 0;
    size_t dense_smem = 0;
};

size_t dense_smem_bytes(int32_t kstride, int64_t dense_max)
{
    int sz = 1;
    while (sz < kstride)
        sz <<= 1;
    const int64_t bit_words = ((int64_t)kstride + dense_max + 31) / 32 + 1;
    return (size_t)sz * sizeof(u64) + (size_t)bit_words * sizeof(uint32_t);
}

int geometry(const bm25_index* ix, const bm25_workspace* ws, int32_t nq, int32_t kmax,
             const Plan& plan, Geometry* g)
{
    DeviceInfo di;
    BM25_TRY(device_info(&di));
    const int64_t N = ix->n_docs;
    g->kstride = (int32_t)std::min<int64_t>(kmax, N);
    g->W = tile_width(plan, N);
    const int64_t n_tiles64 = (N + g->W - 1) / g->W;
    if (n_tiles64 > 65536)
        return set_error(BM25_E_INVALID, "%lld doc tiles of %d documents: use wider tiles",
                         (long long)n_tiles64, g->W);
    g->n_tiles = (int32_t)n_tiles64;
    // queries per sub-batch: tile candidates within kCandBudget, work items < 2^31
    const int64_t per_q = (int64_t)g->n_tiles * g->kstride * (int64_t)sizeof(u64);
    int64_t sub = std::max<int64_t>(1, kCandBudget / per_q);
    sub = std::min<int64_t>(sub, (INT32_MAX - 1) / g->n_tiles);
    if (ws->fixed)  // a lent workspace holds the whole batch or the caller splits it
        sub = nq;
    g->nq_sub = (int32_t)std::min<int64_t>(std::max(nq, 1), sub);
    if ((int64_t)g->nq_sub * g->n_tiles >= INT32_MAX)
        return set_error(BM25_E_INVALID, "%d queries x %d doc tiles is too many work items for "
                         "one call", g->nq_sub, g->n_tiles);
    g->dense_max = -1;
    g->dense_ctas = 0;
    if (plan.accumulator != BM25_ACC_SMEM_TILED && !ws->fixed) {
        const int64_t dmax = plan.accumulator == BM25_ACC_L2_DENSE
                                 ? std::max<int64_t>(plan.dense_max, kDenseMaxL2)
                                 : plan.dense_max;
        // CTAs in flight: the dense vectors within kDenseBudget, and the
        // sectors their queries touch (32 bytes per posting at most) within
        // half of L2, so that scatter and claim meet in L2
        const int64_t by_mem = kDenseBudget / ((int64_t)sizeof(float) * N);
        const int64_t by_l2 = std::max<int64_t>(1, (int64_t)di.l2_bytes / 2 / (32 * dmax));
        const int64_t ctas = std::min<int64_t>(
            std::min<int64_t>((int64_t)di.sm_count * kDenseCtasPerSm, by_mem), by_l2);
        const size_t smem = dense_smem_bytes(g->kstride, dmax);
        if (dmax > 0 && ctas >= 1 && smem + sizeof(SelectState) + sizeof(DenseStage) <=
                                         (size_t)di.max_smem_optin) {
            g->dense_max = dmax;
            g->dense_ctas = (int32_t)ctas;
            g->list_cap = dmax + g->kstride;
            g->dense_smem = smem;
        }
    }
    return BM25_OK;
}

template <typename T>
int grow(T** p, size_t* cap, size_t need, bool capturing)
{
    if (need <= *cap && *p)
        return BM25_OK;
    if (capturing)
        return set_error(BM25_E_INVALID, "the workspace must grow, which cannot happen during "
                         "stream capture: reserve it for this call first");
    if (*p)
        cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    size_t n = need > 0 ? need : 1;
    if (forced_alloc_failure())
        return set_error(BM25_E_OOM, "device allocation of %zu bytes failed (forced by "
                         "bm25_debug_fail_allocs)", n * sizeof(T));
    BM25_CUDA_TRY(cudaMalloc((void**)p, n * sizeof(T)));
    *cap = n;
    return BM25_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int reserve(const bm25_index* ix, bm25_workspace* ws, const Geometry& g, int64_t n_tok,
            cudaStream_t s)
{
    const size_t m = (size_t)g.nq_sub;
    const size_t n_seg = (size_t)n_tok * (size_t)(g.n_tiles + 1);
    const size_t n_tc = m * (size_t)g.n_tiles;
    const size_t n_cand = n_tc * (size_t)g.kstride;
    const size_t n_slots = (size_t)g.dense_ctas * (size_t)ix->n_docs;
    const size_t n_lists = (size_t)g.dense_ctas * (size_t)g.list_cap;
    if (ws->fixed) {
        if ((int32_t)m > ws->max_queries || n_seg > ws->seg_cap || n_tc > ws->tcount_cap ||
            n_cand > ws->cand_cap)
            return set_error(BM25_E_INVALID, "the lent scratch is too small for this batch");
        return BM25_OK;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    BM25_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
    const bool capturing = cs != cudaStreamCaptureStatusNone;
    if ((int32_t)m > ws->max_queries || !ws->qbuf) {
        const size_t bytes = query_arrays_bytes((int64_t)m);
        BM25_TRY(grow(&ws->qbuf, &ws->qbuf_cap, bytes, capturing));
        carve_queries(ws, ws->qbuf, (int32_t)m);
    }
    BM25_TRY(grow(&ws->seg, &ws->seg_cap, n_seg, capturing));
    BM25_TRY(grow(&ws->tcount, &ws->tcount_cap, n_tc, capturing));
    BM25_TRY(grow(&ws->cand, &ws->cand_cap, n_cand, capturing));
    if (n_slots > 0 && (n_slots > ws->dslots_cap || !ws->dslots)) {
        BM25_TRY(grow(&ws->dslots, &ws->dslots_cap, n_slots, capturing));
        // every dense accumulator starts untouched (-0.0); queries leave them so
        k_fill_u32<<<1024, 256, 0, s>>>(reinterpret_cast<uint32_t*>(ws->dslots),
                                        (int64_t)ws->dslots_cap, kUntouched);
        count_launch();
        BM25_LAUNCH_CHECK();
    }
    if (n_lists > 0)
        BM25_TRY(grow(&ws->dlists, &ws->dlists_cap, n_lists, capturing));
    return BM25_OK;
}

}  // namespace

int merge_topk_device(const int32_t* cand_ids, const float* cand_scores, int32_t n_shards,
                      int32_t nq, int32_t k, int32_t* out_ids, float* out_scores, cudaStream_t s)
{
    if (nq == 0)
        return BM25_OK;
    int sz = 1;
    while (sz < k)
        sz <<= 1;
    const size_t smem = (size_t)sz * sizeof(u64);
    BM25_CUDA_TRY(cudaFuncSetAttribute(k_merge_shards, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    {
        ProfileScope ps_("k_merge_shards", s);
        k_merge_shards<<<nq, kMergeThreads, smem, s>>>(cand_ids, cand_scores, n_shards, nq, k,
                                                       out_ids, out_scores);
    }
    count_launch();
    BM25_LAUNCH_CHECK();
    return BM25_OK;
}

int32_t tile_width(const Plan& plan, int64_t n_docs)
{
    int32_t W = plan.tile_docs > 0 ? plan.tile_docs : Plan().tile_docs;
    // multiples of 128 keep the shared-memory carve-up 16-byte aligned
    const int64_t w_need = (n_docs + 127) / 128 * 128;
    if (W > w_need)
        W = (int32_t)w_need;
    return W;
}

size_t query_arrays_bytes(int64_t m)
{
    const size_t q = (size_t)std::max<int64_t>(m, 1);
    return align256(4 * sizeof(uint32_t)) + align256(q * sizeof(double)) +
           align256(q * sizeof(int4)) + 4 * align256(q * sizeof(uint32_t));
}

void carve_queries(bm25_workspace* ws, unsigned char* base, int32_t m)
{
    const size_t q = (size_t)std::max(m, 1);
    unsigned char* p = base;
    ws->ctr = reinterpret_cast<uint32_t*>(p);
    p += align256(4 * sizeof(uint32_t));
    ws->shift = reinterpret_cast<double*>(p);
    p += align256(q * sizeof(double));
    ws->lrec = reinterpret_cast<int4*>(p);
    p += align256(q * sizeof(int4));
    ws->qkp = reinterpret_cast<int32_t*>(p);
    p += align256(q * sizeof(uint32_t));
    ws->lpost = reinterpret_cast<uint32_t*>(p);
    p += align256(q * sizeof(uint32_t));
    ws->thresh = reinterpret_cast<uint32_t*>(p);
    p += align256(q * sizeof(uint32_t));
    ws->sq = reinterpret_cast<int32_t*>(p);
    ws->max_queries = (int32_t)q;
}

int workspace_bytes_for(const bm25_index* ix, int32_t nq, int64_t n_tok, int32_t kmax,
                        const Plan& plan, size_t* bytes)
{
    bm25_workspace probe;
    Geometry g;
    BM25_TRY(geometry(ix, &probe, nq, kmax, plan, &g));
    const size_t m = (size_t)g.nq_sub;
    *bytes = query_arrays_bytes((int64_t)m) +
             sizeof(int32_t) * (size_t)n_tok * (size_t)(g.n_tiles + 1) +
             m * (size_t)g.n_tiles * (sizeof(uint32_t) + sizeof(u64) * (size_t)g.kstride) +
             (size_t)g.dense_ctas * ((size_t)ix->n_docs * sizeof(float) +
                                     (size_t)g.list_cap * sizeof(u64));
    return BM25_OK;
}

size_t workspace_bytes_held(const bm25_workspace* ws)
{
    if (ws->fixed)
        return 0;
    return ws->qbuf_cap + ws->seg_cap * sizeof(int32_t) + ws->tcount_cap * sizeof(uint32_t) +
           ws->cand_cap * sizeof(u64) + ws->dslots_cap * sizeof(float) +
           ws->dlists_cap * sizeof(u64);
}

int workspace_reserve_for(const bm25_index* ix, bm25_workspace* ws, int32_t nq, int64_t n_tok,
                          int32_t kmax, const Plan& plan, cudaStream_t s)
{
    Geometry g;
    BM25_TRY(geometry(ix, ws, nq, kmax, plan, &g));
    return reserve(ix, ws, g, n_tok, s);
}

void workspace_release(bm25_workspace* ws)
{
    if (!ws->fixed) {
        void* ps[] = {ws->qbuf, ws->tcount, ws->seg, ws->cand, ws->dslots, ws->dlists};
        for (void* p : ps)
            if (p)
                cudaFree(p);
    }
    if (ws->owns_staging) {
        void* st[] = {ws->q_tokens, ws->q_offsets, ws->q_k, ws->out_ids, ws->out_scores};
        for (void* p : st)
            if (p)
                cudaFree(p);
    }
    bm25_workspace clean;
    clean.device = ws->device;
    *ws = clean;
}

int retrieve_device(const bm25_index* ix, bm25_workspace* ws, const int32_t* q_tokens,
                    const int64_t* q_off, int32_t nq, int64_t n_tok, const int32_t* q_k,
                    int32_t kmax, int32_t* out_ids, float* out_scores, const Plan& plan,
                    cudaStream_t s, const QueryParams* qp)
{
    if (nq == 0)
        return BM25_OK;
    const bool lazy = qp != nullptr;
    DeviceInfo di;
    BM25_TRY(device_info(&di));
    const int64_t N = ix->n_docs;
    Geometry g;
    BM25_TRY(geometry(ix, ws, nq, kmax, plan, &g));
    BM25_TRY(reserve(ix, ws, g, n_tok, s));
    const int32_t W = g.W, n_tiles = g.n_tiles, kstride = g.kstride;
    const int max_blocks = di.sm_count * 16;

    // R1 once for every token of the batch
    const int64_t n_seg = n_tok * ((int64_t)n_tiles + 1);
    if (n_seg > 0) {
        const int g1 = (int)std::min<int64_t>((n_seg + 255) / 256, max_blocks);
        {
            ProfileScope ps_("k_seg_bounds", s);
            k_seg_bounds<true><<<g1, 256, 0, s>>>(q_tokens, n_tok, ix->indptr, ix->indices,
                                                  ix->vocab, W, n_tiles, ws->seg);
        }
        count_launch();
        BM25_LAUNCH_CHECK();
    }

    // launch shapes that do not depend on the sub-batch
    const uint32_t tl_cap = std::min<uint32_t>((uint32_t)W, kTouchCap);
    const size_t smem = staged_smem_bytes(W, plan.stages, plan.stage_entries, tl_cap, lazy);
    // plan.threads consumer threads (4, 8 or 16 warps) and one producer warp
    auto tile_kernel = lazy ? (plan.threads == 128   ? k_tile_staged<4, true>
                               : plan.threads == 192 ? k_tile_staged<6, true>
                               : plan.threads == 256 ? k_tile_staged<8, true>
                                                     : k_tile_staged<16, true>)
                            : (plan.threads == 128   ? k_tile_staged<4, false>
                               : plan.threads == 192 ? k_tile_staged<6, false>
                               : plan.threads == 256 ? k_tile_staged<8, false>
                                                     : k_tile_staged<16, false>);
    LazyArgs lz = {};
    if (lazy) {
        lz.q_tokens = q_tokens;
        lz.idf = ix->idf;
        lz.doc_len = ix->doc_len;
        lz.variant = ix->variant;
        lz.packed = ix->lazy_packed ? 1 : 0;
        lz.k1 = qp->k1;
        lz.delta = qp->delta;
        lz.one_minus_b = (float)(1.0 - qp->b);
        lz.b_over_lavg = (float)(qp->b / ix->lavg);
        lz.k1f = (float)qp->k1;
        lz.kc = score_consts(qp->k1, qp->delta);
    }
    const int tile_threads = plan.threads + 32;
    BM25_CUDA_TRY(cudaFuncSetAttribute(tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    int per_sm = 0;
    BM25_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tile_kernel,
                                                                tile_threads, smem));
    if (per_sm < 1)
        return set_error(BM25_E_INVALID, "doc tile of %d documents does not fit on an SM", W);
    // the merge tree's levels: groups of `fan` tiles while the candidates a
    // query can have left exceed what k_merge gathers
    const int32_t fan = (int32_t)std::min<int64_t>(kMergeThreads,
                                                   std::max<int64_t>(2, kTreeKeys / kstride));
    const size_t tsmem = (size_t)fan * kstride * sizeof(u64);
    int32_t tstride = 1, levels = 0;
    if (tsmem <= (size_t)di.max_smem_optin) {
        for (int64_t n_v = n_tiles; n_v > 1 && n_v * kstride > kMergeBufCap;
             n_v = (n_v + fan - 1) / fan)
            levels++;
        if (levels > 0)
            BM25_CUDA_TRY(cudaFuncSetAttribute(
                k_merge_level, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem));
    }
    int32_t n_final = n_tiles;
    for (int l = 0; l < levels; l++)
        n_final = (n_final + fan - 1) / fan;
    int sz_all = 1;
    while (sz_all < kstride)
        sz_all <<= 1;
    const int32_t buf_cap = (int32_t)std::min<int64_t>(kMergeBufCap, (int64_t)n_final * kstride);
    const size_t msmem = (size_t)sz_all * sizeof(u64) + (size_t)buf_cap * sizeof(u64) +
                         (size_t)(n_final + 1) * sizeof(uint32_t);
    BM25_CUDA_TRY(cudaFuncSetAttribute(k_merge, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)msmem));
    if (g.dense_ctas > 0)
        BM25_CUDA_TRY(cudaFuncSetAttribute(k_dense_topk,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)g.dense_smem));

    for (int32_t q0 = 0; q0 < nq; q0 += g.nq_sub) {
        const int32_t nb = std::min(g.nq_sub, nq - q0);
        int32_t* ids = out_ids + (int64_t)q0 * kmax;
        float* scores = out_scores + (int64_t)q0 * kmax;
        const int64_t* qo = q_off + q0;
        BM25_CUDA_TRY(cudaMemsetAsync(ws->ctr, 0, 4 * sizeof(uint32_t), s));
        {
            const int g0 = (int)std::min<int64_t>((nb + 255) / 256, max_blocks);
            ProfileScope ps_("k_query_prep", s);
            k_query_prep<<<std::max(g0, 1), 256, 0, s>>>(
                q_tokens, n_tok, qo, nb, q0 == 0, q0 + nb == nq, q_k ? q_k + q0 : nullptr, kmax,
                N, ix->s0, ix->idf, ix->indptr, ix->vocab, lazy ? -1 : g.dense_max, ws->shift,
                ws->qkp, ws->lrec, ws->lpost, ws->thresh, ws->sq, ws->ctr, ix->status,
                lazy ? ix->variant : -1, lazy ? qp->k1 : 0.0, lazy ? qp->delta : 0.0);
        }
        count_launch();
        BM25_LAUNCH_CHECK();
        {
            const int g2 = (int)std::min<int64_t>((int64_t)nb * n_tiles,
                                                  (int64_t)di.sm_count * per_sm);
            ProfileScope ps_("k_tile_staged", s);
            tile_kernel<<<g2, tile_threads, smem, s>>>(
                N, lazy ? ix->posts_lazy : ix->posts, reinterpret_cast<const uint32_t*>(ws->seg),
                W, n_tiles, kstride,
                ws->lrec, ws->lpost, ws->ctr, ws->ctr + 3, ws->thresh, ws->tcount, ws->cand,
                ix->status,
                handshake_polls(), plan.stages, plan.stage_entries, tl_cap, lz);
        }
        count_launch();
        BM25_LAUNCH_CHECK();
        tstride = 1;
        for (int l = 0; l < levels; l++) {
            const int64_t n_v = ((int64_t)n_tiles + tstride - 1) / tstride;
            const int64_t n_groups = (n_v + fan - 1) / fan;
            ProfileScope ps_("k_merge_level", s);
            k_merge_level<<<(unsigned)(n_groups * nb), kMergeThreads, tsmem, s>>>(
                ws->cand, ws->tcount, ws->lrec, ws->ctr, n_tiles, tstride, fan, kstride, nb);
            count_launch();
            BM25_LAUNCH_CHECK();
            tstride *= fan;
        }
        {
            ProfileScope ps_("k_merge", s);
            k_merge<<<nb, kMergeThreads, msmem, s>>>(ws->cand, ws->tcount, ws->lrec, ws->ctr,
                                                     n_tiles, tstride, kstride, kmax, ws->shift,
                                                     ids, scores, buf_cap,
                                                     (int32_t)ix->doc_offset);
        }
        count_launch();
        BM25_LAUNCH_CHECK();
        if (g.dense_ctas > 0 && !lazy) {
            const int g4 = std::min(g.dense_ctas, nb);
            ProfileScope ps_("k_dense_topk", s);
            k_dense_topk<<<g4, kDenseThreads, g.dense_smem, s>>>(
                q_tokens, n_tok, qo, ws->qkp, ws->shift, ix->indptr, ix->indices, ix->data,
                ix->vocab, N, ws->sq, ws->ctr, ws->dslots, ws->dlists, g.list_cap, kstride, kmax,
                ids, scores, (int32_t)ix->doc_offset);
            count_launch();
            BM25_LAUNCH_CHECK();
        }
    }
    return BM25_OK;
}

}  // namespace bm25
