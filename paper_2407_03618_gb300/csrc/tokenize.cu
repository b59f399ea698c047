// Tokenizer front end on the device (arXiv 2407.03618 Sec. 2 "Tokenization":
// split with the pattern (?u)\b\w\w+\b, remove stopwords, map every distinct
// word to an integer id).
//
// Read on UTF-8 bytes: ASCII letters, digits and '_' and every byte of a
// non-ASCII character (0x80-0xFF) are word characters; ASCII letters are
// lowercased; a token is a maximal run of word bytes inside one text with at
// least two characters (bytes other than UTF-8 continuation bytes
// 0x80-0xBF); a token equal to a stopword is dropped.  Corpus ids follow the
// first occurrence of each word (text order, then position); a query keeps
// the tokens the vocabulary knows, with their ids.
//
// Launches (all on the caller's stream):
//   T1 k_mark_texts    bit per byte: a text starts here
//   T2 k_starts        bit per byte: a run of word bytes starts here (a word
//                      byte after a non-word byte or at a text start)
//   T3 k_emit_starts   the start position of every run, in order (prefix sum
//                      of the per-word bit counts)
//   T4 k_measure       per run: its end, its character count, a 64-bit hash
//                      of its lowercased bytes (FNV-1a, then the splitmix64
//                      finaliser), kept if >= 2 characters and not a stopword
//   T5 k_compact       the kept tokens in order (prefix sum of the flags)
//   T6 k_text_offsets  per text, its first kept token (a lower bound)
//   corpus:  T7 k_insert       open-addressing table hash -> first token
//            T8 k_first_flags  flag the first occurrence of every word
//            T9 k_assign       id = rank of its first occurrence; every
//                              token's id, its bytes checked against the
//                              first occurrence's (a hash collision is an error)
//   queries: T10 k_lookup      id from the table, bytes checked against the
//                              vocabulary's copy of the word; unknown -> dropped
#include <algorithm>
#include <cstring>
#include <vector>

#include "device.cuh"
#include "internal.h"

struct bm25_vocab {
    int device = 0;
    int64_t n_words = 0, n_bytes = 0;
    uint64_t* keys = nullptr;      // [cap] word hash, 0 = empty slot
    int32_t* ids = nullptr;        // [cap] word id of the slot
    int64_t cap = 0;               // power of two
    uint8_t* words = nullptr;      // [n_bytes] the words' bytes (lowercased), in id order
    int64_t* word_off = nullptr;   // [n_words + 1]
    // stopwords, lowercased: table and bytes
    uint64_t* stop_keys = nullptr; // [stop_cap]
    int32_t* stop_ids = nullptr;   // [stop_cap]
    int64_t stop_cap = 0;
    uint8_t* stop_bytes = nullptr;
    int64_t* stop_off = nullptr;   // [n_stop + 1]
    int32_t n_stop = 0;
};

namespace bm25 {
namespace {

constexpr int kTokThreads = 256;
constexpr int kMaxProbes = 1 << 16;  // probes before an insert or lookup gives up

__device__ __forceinline__ bool is_word(uint32_t c)
{
    return (c >= '0' && c <= '9') || (c >= 'a' && c <= 'z') || (c >= 'A' && c <= 'Z') || c == '_' ||
           c >= 0x80u;
}

__device__ __forceinline__ uint32_t lower(uint32_t c) { return (c >= 'A' && c <= 'Z') ? c + 32u : c; }

__device__ __forceinline__ bool is_cont(uint32_t c) { return c >= 0x80u && c <= 0xBFu; }

// FNV-1a over the lowercased bytes (offset basis 14695981039346656037,
// prime 1099511628211), then the splitmix64 finaliser to spread the bits
// over the table's low bits; never 0 (the empty-slot key).
__device__ __forceinline__ uint64_t hash_step(uint64_t h, uint32_t c)
{
    return (h ^ (uint64_t)c) * 1099511628211ull;
}
__device__ __forceinline__ uint64_t hash_final(uint64_t h)
{
    h ^= h >> 30;
    h *= 0xbf58476d1ce4e5b9ull;
    h ^= h >> 27;
    h *= 0x94d049bb133111ebull;
    h ^= h >> 31;
    return h ? h : 1ull;
}
constexpr uint64_t kFnvBasis = 14695981039346656037ull;

__device__ __forceinline__ bool bit(const uint32_t* bits, int64_t i)
{
    return (bits[i >> 5] >> (i & 31)) & 1u;
}

// T1: texts [0, n) start at off[t]; a text's start is a run boundary.
__global__ void k_mark_texts(const int64_t* __restrict__ off, int64_t n, int64_t n_bytes,
                             uint32_t* __restrict__ tstart, int* status)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = off[t], b = off[t + 1];
        if (a < 0 || b < a || b > n_bytes || (t == 0 && a != 0) || (t == n - 1 && b != n_bytes)) {
            set_status(status, BM25_E_TOKEN_RANGE);
            continue;
        }
        if (a < n_bytes)
            atomicOr(&tstart[a >> 5], 1u << (a & 31));
    }
}

// T2: one warp per 32 bytes (lane = byte): start bit and per-word count.
__global__ void k_starts(const uint8_t* __restrict__ text, int64_t n_bytes,
                         const uint32_t* __restrict__ tstart, uint32_t* __restrict__ sbits,
                         uint32_t* __restrict__ wcount)
{
    const int lane = threadIdx.x & 31;
    const int64_t n_words = (n_bytes + 31) >> 5;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n_words;
         w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t i = (w << 5) + lane;
        bool s = false;
        if (i < n_bytes) {
            const bool wd = is_word(text[i]);
            const bool prev = i > 0 && is_word(text[i - 1]);
            s = wd && (bit(tstart, i) || !prev);
        }
        const uint32_t b = __ballot_sync(0xffffffffu, s);
        if (lane == 0) {
            sbits[w] = b;
            wcount[w] = (uint32_t)__popc(b);
        }
    }
}

// T3: the start positions in order (wbase = exclusive prefix sum of wcount).
__global__ void k_emit_starts(const uint32_t* __restrict__ sbits, const uint32_t* __restrict__ wbase,
                              int64_t n_words, int64_t* __restrict__ run_start)
{
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n_words;
         w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t b = sbits[w];
        uint32_t o = wbase[w];
        while (b) {
            const int k = __ffs(b) - 1;
            b &= b - 1u;
            run_start[o++] = (w << 5) + k;
        }
    }
}

// The table slot of hash h (-1 if absent).
__device__ __forceinline__ int64_t table_find(const uint64_t* __restrict__ keys, int64_t mask,
                                              uint64_t h)
{
    int64_t s = (int64_t)(h & (uint64_t)mask);
    for (int p = 0; p < kMaxProbes; p++) {
        const uint64_t k = keys[s];
        if (k == h)
            return s;
        if (k == 0ull)
            return -1;
        s = (s + 1) & mask;
    }
    return -1;
}

__device__ __forceinline__ bool same_bytes(const uint8_t* __restrict__ text, int64_t a, int32_t len,
                                           const uint8_t* __restrict__ w, int64_t wa, int64_t wlen)
{
    if ((int64_t)len != wlen)
        return false;
    for (int32_t i = 0; i < len; i++)
        if (lower(text[a + i]) != (uint32_t)w[wa + i])
            return false;
    return true;
}

// T4: per run r: end, characters, hash; keep[r] = 1 if >= 2 characters and
// not a stopword.
__global__ void k_measure(const uint8_t* __restrict__ text, int64_t n_bytes,
                          const uint32_t* __restrict__ tstart, const int64_t* __restrict__ run_start,
                          int64_t n_runs, const uint64_t* __restrict__ stop_keys,
                          const int32_t* __restrict__ stop_ids, int64_t stop_mask,
                          const uint8_t* __restrict__ stop_bytes, const int64_t* __restrict__ stop_off,
                          uint64_t* __restrict__ run_hash, int32_t* __restrict__ run_len,
                          uint32_t* __restrict__ keep)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_runs;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = run_start[r];
        int64_t e = a;
        uint32_t chars = 0;
        uint64_t h = kFnvBasis;
        while (e < n_bytes) {
            const uint32_t c = text[e];
            if (!is_word(c) || (e > a && bit(tstart, e)))
                break;
            h = hash_step(h, lower(c));
            chars += is_cont(c) ? 0u : 1u;
            e++;
        }
        h = hash_final(h);
        const int32_t len = (int32_t)(e - a);
        bool k = chars >= 2u;
        if (k && stop_keys) {
            const int64_t s = table_find(stop_keys, stop_mask, h);
            if (s >= 0) {
                const int32_t sid = stop_ids[s];
                k = !same_bytes(text, a, len, stop_bytes, stop_off[sid],
                                stop_off[sid + 1] - stop_off[sid]);
            }
        }
        run_hash[r] = h;
        run_len[r] = len;
        keep[r] = k ? 1u : 0u;
    }
}

// T5: kept runs in order.
__global__ void k_compact(const int64_t* __restrict__ run_start, const uint64_t* __restrict__ run_hash,
                          const int32_t* __restrict__ run_len, const uint32_t* __restrict__ keep,
                          const uint32_t* __restrict__ kpos, int64_t n_runs,
                          int64_t* __restrict__ tok_start, uint64_t* __restrict__ tok_hash,
                          int32_t* __restrict__ tok_len)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_runs;
         r += (int64_t)gridDim.x * blockDim.x) {
        if (keep[r]) {
            const uint32_t j = kpos[r];
            tok_start[j] = run_start[r];
            tok_hash[j] = run_hash[r];
            tok_len[j] = run_len[r];
        }
    }
}

// T6: out[t] = number of kept tokens starting before off[t] (t = 0..n).
__global__ void k_text_offsets(const int64_t* __restrict__ off, int64_t n,
                               const int64_t* __restrict__ tok_start, int64_t n_tok,
                               int64_t* __restrict__ out)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = off[t];
        int64_t lo = 0, hi = n_tok;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (tok_start[mid] < x)
                lo = mid + 1;
            else
                hi = mid;
        }
        out[t] = lo;
    }
}

// T7: insert every token's hash; first[slot] = smallest token index.
__global__ void k_insert(const uint64_t* __restrict__ tok_hash, int64_t n_tok,
                         unsigned long long* __restrict__ keys, int64_t mask,
                         int64_t* __restrict__ first, int* status)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_tok;
         j += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long h = tok_hash[j];
        int64_t s = (int64_t)(h & (uint64_t)mask);
        bool done = false;
        for (int p = 0; p < kMaxProbes; p++) {
            const unsigned long long k = atomicCAS(&keys[s], 0ull, h);
            if (k == 0ull || k == h) {
                atomicMin(reinterpret_cast<long long*>(&first[s]), (long long)j);
                done = true;
                break;
            }
            s = (s + 1) & mask;
        }
        if (!done)
            set_status(status, BM25_E_INVALID);  // table full
    }
}

// T8: flag[j] = 1 where token j is the first occurrence of its word.
__global__ void k_first_flags(const int64_t* __restrict__ first, const unsigned long long* __restrict__ keys,
                              int64_t cap, uint32_t* __restrict__ flag)
{
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < cap;
         s += (int64_t)gridDim.x * blockDim.x)
        if (keys[s] != 0ull)
            flag[first[s]] = 1u;
}

// T9: slot ids (rank of the first occurrence), every token's id, the
// collision check, and the words' lengths in id order.
__global__ void k_slot_ids(const int64_t* __restrict__ first, const unsigned long long* __restrict__ keys,
                           int64_t cap, const uint32_t* __restrict__ rank,
                           const int32_t* __restrict__ tok_len, int32_t* __restrict__ ids,
                           int64_t* __restrict__ word_len)
{
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < cap;
         s += (int64_t)gridDim.x * blockDim.x) {
        if (keys[s] != 0ull) {
            const int32_t id = (int32_t)rank[first[s]];
            ids[s] = id;
            word_len[id] = tok_len[first[s]];
        }
    }
}

__global__ void k_assign(const uint8_t* __restrict__ text, const int64_t* __restrict__ tok_start,
                         const uint64_t* __restrict__ tok_hash, const int32_t* __restrict__ tok_len,
                         int64_t n_tok, const unsigned long long* __restrict__ keys, int64_t mask,
                         const int64_t* __restrict__ first, const int32_t* __restrict__ ids,
                         int32_t* __restrict__ out, int* status)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_tok;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = table_find(reinterpret_cast<const uint64_t*>(keys), mask, tok_hash[j]);
        if (s < 0) {
            set_status(status, BM25_E_INVALID);
            out[j] = 0;
            continue;
        }
        const int64_t f = first[s];
        const int64_t a = tok_start[j], fa = tok_start[f];
        const int32_t len = tok_len[j];
        bool same = len == tok_len[f];
        for (int32_t i = 0; same && i < len; i++)
            same = lower(text[a + i]) == lower(text[fa + i]);
        if (!same)
            set_status(status, BM25_E_INVALID);  // two words with one hash
        out[j] = ids[s];
    }
}

// The words' bytes in id order (lowercased), from their first occurrences.
__global__ void k_gather_words(const uint8_t* __restrict__ text, const int64_t* __restrict__ tok_start,
                               const int64_t* __restrict__ first, const unsigned long long* __restrict__ keys,
                               int64_t cap, const int32_t* __restrict__ ids,
                               const int64_t* __restrict__ word_off, uint8_t* __restrict__ words)
{
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < cap;
         s += (int64_t)gridDim.x * blockDim.x) {
        if (keys[s] != 0ull) {
            const int32_t id = ids[s];
            const int64_t a = tok_start[first[s]];
            for (int64_t i = word_off[id]; i < word_off[id + 1]; i++)
                words[i] = (uint8_t)lower(text[a + (i - word_off[id])]);
        }
    }
}

// T10: a query token's id (or -1 when the vocabulary does not know it).
__global__ void k_lookup(const uint8_t* __restrict__ text, const int64_t* __restrict__ tok_start,
                         const uint64_t* __restrict__ tok_hash, const int32_t* __restrict__ tok_len,
                         int64_t n_tok, const uint64_t* __restrict__ keys, int64_t mask,
                         const int32_t* __restrict__ ids, const uint8_t* __restrict__ words,
                         const int64_t* __restrict__ word_off, int32_t* __restrict__ out,
                         uint32_t* __restrict__ known)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_tok;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = table_find(keys, mask, tok_hash[j]);
        int32_t id = -1;
        if (s >= 0) {
            const int32_t c = ids[s];
            if (same_bytes(text, tok_start[j], tok_len[j], words, word_off[c],
                           word_off[c + 1] - word_off[c]))
                id = c;
        }
        out[j] = id;
        known[j] = id >= 0 ? 1u : 0u;
    }
}

__global__ void k_keep_known(const int32_t* __restrict__ in, const uint32_t* __restrict__ known,
                             const uint32_t* __restrict__ pos, int64_t n, int32_t* __restrict__ out,
                             const int64_t* __restrict__ tok_start, int64_t* __restrict__ start_out)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x)
        if (known[j]) {
            out[pos[j]] = in[j];
            start_out[pos[j]] = tok_start[j];
        }
}

// Stopword table: hashes of the lowercased stopwords (one thread each).
__global__ void k_stop_hash(const uint8_t* __restrict__ bytes, const int64_t* __restrict__ off,
                            int32_t n, unsigned long long* __restrict__ keys, int32_t* __restrict__ ids,
                            int64_t mask, int* status)
{
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint64_t h = kFnvBasis;
        for (int64_t p = off[i]; p < off[i + 1]; p++)
            h = hash_step(h, lower(bytes[p]));
        h = hash_final(h);
        int64_t s = (int64_t)(h & (uint64_t)mask);
        bool done = false;
        for (int p = 0; p < kMaxProbes && !done; p++) {
            const unsigned long long k = atomicCAS(&keys[s], 0ull, (unsigned long long)h);
            if (k == 0ull) {
                ids[s] = i;
                done = true;
            } else if (k == h) {
                done = true;  // the same word twice, or a collision: the first one kept
            } else {
                s = (s + 1) & mask;
            }
        }
        if (!done)
            set_status(status, BM25_E_INVALID);
    }
}

__global__ void k_lower_bytes(uint8_t* __restrict__ b, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (uint8_t)lower(b[i]);
}

// ---- host side -------------------------------------------------------------

int grid(int64_t n, int max_blocks)
{
    const int64_t b = (n + kTokThreads - 1) / kTokThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, max_blocks));
}

struct Tmp {
    cudaMemPool_t pool = nullptr;
    cudaStream_t s = nullptr;
    std::vector<void*> ptrs;
    template <typename T>
    int alloc(T** p, int64_t n)
    {
        *p = nullptr;
        const size_t bytes = (size_t)std::max<int64_t>(n, 1) * sizeof(T);
        if (forced_alloc_failure())
            return set_error(BM25_E_OOM, "device allocation of %zu bytes failed (forced by "
                             "bm25_debug_fail_allocs)", bytes);
        cudaError_t e = cudaMallocFromPoolAsync((void**)p, bytes, pool, s);
        if (e != cudaSuccess) {
            *p = nullptr;
            return set_error(e == cudaErrorMemoryAllocation ? BM25_E_OOM : BM25_E_CUDA,
                             "device allocation of %zu bytes failed: %s", bytes,
                             cudaGetErrorString(e));
        }
        ptrs.push_back((void*)*p);
        return BM25_OK;
    }
    void release(void* p)  // keep p: it leaves with the result
    {
        ptrs.erase(std::remove(ptrs.begin(), ptrs.end(), p), ptrs.end());
    }
    ~Tmp()
    {
        for (void* p : ptrs)
            cudaFreeAsync(p, s);
    }
};

int64_t pow2_at_least(int64_t n)
{
    int64_t c = 1;
    while (c < n)
        c <<= 1;
    return c;
}

// T1-T6 over `n` texts: the kept tokens (start, hash, length) and the
// per-text token offsets.  Synchronises once (the token count).
struct Split {
    int64_t n_tok = 0;
    int64_t* tok_start = nullptr;
    uint64_t* tok_hash = nullptr;
    int32_t* tok_len = nullptr;
};

int split_texts(const uint8_t* text, int64_t n_bytes, const int64_t* off, int64_t n,
                const bm25_vocab* stops, int64_t* text_tok_off, Tmp& tmp, Split* out)
{
    DeviceInfo di;
    BM25_TRY(device_info(&di));
    const int mb = di.sm_count * 16;
    cudaStream_t s = tmp.s;
    const int64_t n_words = (n_bytes + 31) >> 5;
    uint32_t *tstart = nullptr, *sbits = nullptr, *wcount = nullptr, *d_total = nullptr,
             *scan_tmp = nullptr;
    int* status = nullptr;
    BM25_TRY(tmp.alloc(&tstart, n_words));
    BM25_TRY(tmp.alloc(&sbits, n_words));
    BM25_TRY(tmp.alloc(&wcount, n_words));
    BM25_TRY(tmp.alloc(&d_total, 2));
    BM25_TRY(tmp.alloc(&status, 1));
    BM25_CUDA_TRY(cudaMemsetAsync(tstart, 0, sizeof(uint32_t) * (size_t)std::max<int64_t>(n_words, 1), s));
    BM25_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
    k_mark_texts<<<grid(n, mb), kTokThreads, 0, s>>>(off, n, n_bytes, tstart, status);
    k_starts<<<grid(n_words * 32, mb), kTokThreads, 0, s>>>(text, n_bytes, tstart, sbits, wcount);
    count_launch(2);
    BM25_LAUNCH_CHECK();
    const int64_t scan_elems = scan_tmp_elems(std::max<int64_t>(n_words, 1) * 32);
    BM25_TRY(tmp.alloc(&scan_tmp, scan_elems));
    BM25_TRY(exclusive_scan_u32(wcount, wcount, n_words, d_total, scan_tmp, s));
    uint32_t h_runs = 0;
    int h_status = 0;
    BM25_CUDA_TRY(cudaMemcpyAsync(&h_runs, d_total, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    BM25_CUDA_TRY(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    BM25_CUDA_TRY(cudaStreamSynchronize(s));
    if (h_status)
        return set_error(BM25_E_TOKEN_RANGE, "text offsets are malformed");
    const int64_t n_runs = h_runs;
    int64_t* run_start = nullptr;
    uint64_t* run_hash = nullptr;
    int32_t* run_len = nullptr;
    uint32_t *keep = nullptr, *kpos = nullptr;
    BM25_TRY(tmp.alloc(&run_start, n_runs));
    BM25_TRY(tmp.alloc(&run_hash, n_runs));
    BM25_TRY(tmp.alloc(&run_len, n_runs));
    BM25_TRY(tmp.alloc(&keep, n_runs));
    BM25_TRY(tmp.alloc(&kpos, n_runs));
    k_emit_starts<<<grid(n_words, mb), kTokThreads, 0, s>>>(sbits, wcount, n_words, run_start);
    k_measure<<<grid(n_runs, mb), kTokThreads, 0, s>>>(
        text, n_bytes, tstart, run_start, n_runs, stops ? stops->stop_keys : nullptr,
        stops ? stops->stop_ids : nullptr, stops ? stops->stop_cap - 1 : 0,
        stops ? stops->stop_bytes : nullptr, stops ? stops->stop_off : nullptr, run_hash, run_len,
        keep);
    count_launch(2);
    BM25_LAUNCH_CHECK();
    BM25_TRY(exclusive_scan_u32(keep, kpos, n_runs, d_total, scan_tmp, s));
    uint32_t h_tok = 0;
    BM25_CUDA_TRY(cudaMemcpyAsync(&h_tok, d_total, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    BM25_CUDA_TRY(cudaStreamSynchronize(s));
    out->n_tok = h_tok;
    BM25_TRY(tmp.alloc(&out->tok_start, out->n_tok));
    BM25_TRY(tmp.alloc(&out->tok_hash, out->n_tok));
    BM25_TRY(tmp.alloc(&out->tok_len, out->n_tok));
    k_compact<<<grid(n_runs, mb), kTokThreads, 0, s>>>(run_start, run_hash, run_len, keep, kpos,
                                                       n_runs, out->tok_start, out->tok_hash,
                                                       out->tok_len);
    k_text_offsets<<<grid(n + 1, mb), kTokThreads, 0, s>>>(off, n, out->tok_start, out->n_tok,
                                                           text_tok_off);
    count_launch(2);
    BM25_LAUNCH_CHECK();
    return BM25_OK;
}

int check_texts(const uint8_t* text, int64_t n_bytes, const int64_t* off, int64_t n)
{
    if (n < 1 || !off || n_bytes < 0 || n_bytes > (int64_t)INT32_MAX - 1 || (n_bytes > 0 && !text))
        return set_error(BM25_E_INVALID, "need n_texts >= 1, 0 <= n_bytes < 2^31 - 1 and "
                         "non-NULL arrays");
    return BM25_OK;
}

}  // namespace
}  // namespace bm25

using namespace bm25;

extern "C" {

int bm25_tokenize_corpus(const uint8_t* text, int64_t n_bytes, const int64_t* doc_offsets,
                         int64_t n_docs, const uint8_t* stopwords, const int64_t* stop_offsets,
                         int32_t n_stopwords, int32_t* token_ids, int64_t capacity,
                         int64_t* token_offsets, int64_t* n_tokens, bm25_vocab** vocab,
                         void* cuda_stream)
{
    clear_error();
    if (!vocab || !n_tokens || !token_offsets)
        return set_error(BM25_E_INVALID, "NULL argument");
    *vocab = nullptr;
    BM25_TRY(check_texts(text, n_bytes, doc_offsets, n_docs));
    if (n_stopwords < 0 || (n_stopwords > 0 && (!stopwords || !stop_offsets)))
        return set_error(BM25_E_INVALID, "bad stopword list");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    DeviceInfo di;
    BM25_TRY(device_info(&di));
    const int mb = di.sm_count * 16;
    Tmp tmp;
    tmp.s = s;
    BM25_TRY(pool_for_current_device(&tmp.pool));
    bm25_vocab* v = new bm25_vocab();
    v->device = di.device;
    auto fail = [&](int rc) {
        bm25_vocab_free(v);
        return rc;
    };
    // stopwords (host) -> device, lowercased, and their table
    int* status = nullptr;
    if (tmp.alloc(&status, 1) != BM25_OK)
        return fail(BM25_E_OOM);
    BM25_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
    if (n_stopwords > 0) {
        const int64_t nb = stop_offsets[n_stopwords];
        v->n_stop = n_stopwords;
        v->stop_cap = pow2_at_least(2 * (int64_t)n_stopwords);
        int r = BM25_OK;
        if (r == BM25_OK) r = tmp.alloc(&v->stop_bytes, nb);
        if (r == BM25_OK) r = tmp.alloc(&v->stop_off, n_stopwords + 1);
        if (r == BM25_OK) r = tmp.alloc(&v->stop_keys, v->stop_cap);
        if (r == BM25_OK) r = tmp.alloc(&v->stop_ids, v->stop_cap);
        if (r != BM25_OK)
            return fail(r);
        tmp.release(v->stop_bytes);
        tmp.release(v->stop_off);
        tmp.release(v->stop_keys);
        tmp.release(v->stop_ids);
        BM25_CUDA_TRY(cudaMemcpyAsync(v->stop_bytes, stopwords, (size_t)nb, cudaMemcpyHostToDevice, s));
        BM25_CUDA_TRY(cudaMemcpyAsync(v->stop_off, stop_offsets, sizeof(int64_t) * (n_stopwords + 1),
                                      cudaMemcpyHostToDevice, s));
        BM25_CUDA_TRY(cudaMemsetAsync(v->stop_keys, 0, sizeof(uint64_t) * v->stop_cap, s));
        k_lower_bytes<<<grid(nb, mb), kTokThreads, 0, s>>>(v->stop_bytes, nb);
        k_stop_hash<<<grid(n_stopwords, mb), kTokThreads, 0, s>>>(
            v->stop_bytes, v->stop_off, n_stopwords,
            reinterpret_cast<unsigned long long*>(v->stop_keys), v->stop_ids, v->stop_cap - 1,
            status);
        count_launch(2);
        BM25_LAUNCH_CHECK();
    }
    Split sp;
    {
        int r = split_texts(text, n_bytes, doc_offsets, n_docs, n_stopwords > 0 ? v : nullptr,
                            token_offsets, tmp, &sp);
        if (r != BM25_OK)
            return fail(r);
    }
    *n_tokens = sp.n_tok;
    if (sp.n_tok > capacity || (sp.n_tok > 0 && !token_ids))
        return fail(set_error(BM25_E_INVALID, "%lld tokens do not fit the capacity %lld",
                              (long long)sp.n_tok, (long long)capacity));
    // vocabulary: hash table of the corpus words, ids by first occurrence
    v->cap = pow2_at_least(std::max<int64_t>(2 * sp.n_tok, 16));
    int64_t* first = nullptr;
    uint32_t *flag = nullptr, *rank = nullptr, *d_total = nullptr, *scan_tmp = nullptr;
    int64_t* word_len = nullptr;
    {
        int r = BM25_OK;
        if (r == BM25_OK) r = tmp.alloc(&v->keys, v->cap);
        if (r == BM25_OK) r = tmp.alloc(&v->ids, v->cap);
        if (r == BM25_OK) r = tmp.alloc(&first, v->cap);
        if (r == BM25_OK) r = tmp.alloc(&flag, sp.n_tok);
        if (r == BM25_OK) r = tmp.alloc(&rank, sp.n_tok);
        if (r == BM25_OK) r = tmp.alloc(&d_total, 2);
        if (r == BM25_OK) r = tmp.alloc(&scan_tmp, scan_tmp_elems(std::max<int64_t>(sp.n_tok, 1)));
        if (r != BM25_OK)
            return fail(r);
        tmp.release(v->keys);
        tmp.release(v->ids);
    }
    BM25_CUDA_TRY(cudaMemsetAsync(v->keys, 0, sizeof(uint64_t) * v->cap, s));
    BM25_CUDA_TRY(cudaMemsetAsync(first, 0x7f, sizeof(int64_t) * v->cap, s));
    BM25_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(uint32_t) * std::max<int64_t>(sp.n_tok, 1), s));
    const int64_t mask = v->cap - 1;
    auto* ukeys = reinterpret_cast<unsigned long long*>(v->keys);
    k_insert<<<grid(sp.n_tok, mb), kTokThreads, 0, s>>>(sp.tok_hash, sp.n_tok, ukeys, mask, first,
                                                        status);
    k_first_flags<<<grid(v->cap, mb), kTokThreads, 0, s>>>(first, ukeys, v->cap, flag);
    count_launch(2);
    BM25_LAUNCH_CHECK();
    BM25_TRY(exclusive_scan_u32(flag, rank, sp.n_tok, d_total, scan_tmp, s));
    uint32_t h_words = 0;
    BM25_CUDA_TRY(cudaMemcpyAsync(&h_words, d_total, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    BM25_CUDA_TRY(cudaStreamSynchronize(s));
    v->n_words = sp.n_tok > 0 ? h_words : 0;
    if (tmp.alloc(&word_len, v->n_words + 1) != BM25_OK ||
        tmp.alloc(&v->word_off, v->n_words + 1) != BM25_OK)
        return fail(BM25_E_OOM);
    tmp.release(v->word_off);
    k_slot_ids<<<grid(v->cap, mb), kTokThreads, 0, s>>>(first, ukeys, v->cap, rank, sp.tok_len,
                                                        v->ids, word_len);
    k_assign<<<grid(sp.n_tok, mb), kTokThreads, 0, s>>>(text, sp.tok_start, sp.tok_hash,
                                                        sp.tok_len, sp.n_tok, ukeys, mask, first,
                                                        v->ids, token_ids, status);
    count_launch(2);
    BM25_LAUNCH_CHECK();
    // word offsets: exclusive prefix sum of the lengths (host: one pass over n_words)
    std::vector<int64_t> h_len((size_t)v->n_words + 1, 0);
    if (v->n_words > 0)
        BM25_CUDA_TRY(cudaMemcpyAsync(h_len.data(), word_len, sizeof(int64_t) * v->n_words,
                                      cudaMemcpyDeviceToHost, s));
    int h_status = 0;
    BM25_CUDA_TRY(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    BM25_CUDA_TRY(cudaStreamSynchronize(s));
    if (h_status)
        return fail(set_error(BM25_E_INVALID, "tokenizer: hash table full or two words with one "
                              "64-bit hash"));
    int64_t acc = 0;
    for (int64_t i = 0; i < v->n_words; i++) {
        const int64_t l = h_len[i];
        h_len[i] = acc;
        acc += l;
    }
    h_len[v->n_words] = acc;
    v->n_bytes = acc;
    BM25_CUDA_TRY(cudaMemcpyAsync(v->word_off, h_len.data(), sizeof(int64_t) * (v->n_words + 1),
                                  cudaMemcpyHostToDevice, s));
    if (tmp.alloc(&v->words, acc) != BM25_OK)
        return fail(BM25_E_OOM);
    tmp.release(v->words);
    k_gather_words<<<grid(v->cap, mb), kTokThreads, 0, s>>>(text, sp.tok_start, first, ukeys,
                                                            v->cap, v->ids, v->word_off, v->words);
    count_launch();
    BM25_LAUNCH_CHECK();
    BM25_CUDA_TRY(cudaStreamSynchronize(s));
    *vocab = v;
    return BM25_OK;
}

int bm25_tokenize_queries(const bm25_vocab* v, const uint8_t* text, int64_t n_bytes,
                          const int64_t* offsets, int64_t n_texts, int32_t* token_ids,
                          int64_t capacity, int64_t* token_offsets, int64_t* n_tokens,
                          void* cuda_stream)
{
    clear_error();
    if (!v || !n_tokens || !token_offsets)
        return set_error(BM25_E_INVALID, "NULL argument");
    BM25_TRY(check_texts(text, n_bytes, offsets, n_texts));
    int dev = 0;
    BM25_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != v->device)
        return set_error(BM25_E_INVALID, "current device %d is not the vocabulary's device %d", dev,
                         v->device);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    DeviceInfo di;
    BM25_TRY(device_info(&di));
    const int mb = di.sm_count * 16;
    Tmp tmp;
    tmp.s = s;
    BM25_TRY(pool_for_current_device(&tmp.pool));
    Split sp;
    int64_t* raw_off = nullptr;
    BM25_TRY(tmp.alloc(&raw_off, n_texts + 1));
    BM25_TRY(split_texts(text, n_bytes, offsets, n_texts, v->n_stop > 0 ? v : nullptr, raw_off, tmp,
                         &sp));
    int32_t* ids = nullptr;
    uint32_t *known = nullptr, *pos = nullptr, *d_total = nullptr, *scan_tmp = nullptr;
    int64_t* kept_start = nullptr;
    BM25_TRY(tmp.alloc(&ids, sp.n_tok));
    BM25_TRY(tmp.alloc(&known, sp.n_tok));
    BM25_TRY(tmp.alloc(&pos, sp.n_tok));
    BM25_TRY(tmp.alloc(&d_total, 2));
    BM25_TRY(tmp.alloc(&scan_tmp, scan_tmp_elems(std::max<int64_t>(sp.n_tok, 1))));
    BM25_TRY(tmp.alloc(&kept_start, sp.n_tok));
    if (sp.n_tok > 0) {
        k_lookup<<<grid(sp.n_tok, mb), kTokThreads, 0, s>>>(
            text, sp.tok_start, sp.tok_hash, sp.tok_len, sp.n_tok, v->keys, v->cap - 1, v->ids,
            v->words, v->word_off, ids, known);
        count_launch();
        BM25_LAUNCH_CHECK();
    }
    BM25_TRY(exclusive_scan_u32(known, pos, sp.n_tok, d_total, scan_tmp, s));
    uint32_t h_kept = 0;
    BM25_CUDA_TRY(cudaMemcpyAsync(&h_kept, d_total, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    BM25_CUDA_TRY(cudaStreamSynchronize(s));
    *n_tokens = sp.n_tok > 0 ? h_kept : 0;
    if (*n_tokens > capacity || (*n_tokens > 0 && !token_ids))
        return set_error(BM25_E_INVALID, "%lld tokens do not fit the capacity %lld",
                         (long long)*n_tokens, (long long)capacity);
    if (sp.n_tok > 0) {
        k_keep_known<<<grid(sp.n_tok, mb), kTokThreads, 0, s>>>(ids, known, pos, sp.n_tok, token_ids,
                                                                sp.tok_start, kept_start);
        count_launch();
        BM25_LAUNCH_CHECK();
    }
    k_text_offsets<<<grid(n_texts + 1, mb), kTokThreads, 0, s>>>(offsets, n_texts, kept_start,
                                                                 *n_tokens, token_offsets);
    count_launch();
    BM25_LAUNCH_CHECK();
    BM25_CUDA_TRY(cudaStreamSynchronize(s));
    return BM25_OK;
}

int bm25_vocab_info(const bm25_vocab* v, int64_t* n_words, int64_t* n_bytes)
{
    clear_error();
    if (!v)
        return set_error(BM25_E_INVALID, "vocabulary is NULL");
    if (n_words) *n_words = v->n_words;
    if (n_bytes) *n_bytes = v->n_bytes;
    return BM25_OK;
}

int bm25_vocab_export(const bm25_vocab* v, uint8_t* words, int64_t* word_offsets)
{
    clear_error();
    if (!v)
        return set_error(BM25_E_INVALID, "vocabulary is NULL");
    if (words && v->n_bytes > 0)
        BM25_CUDA_TRY(cudaMemcpy(words, v->words, (size_t)v->n_bytes, cudaMemcpyDeviceToHost));
    if (word_offsets)
        BM25_CUDA_TRY(cudaMemcpy(word_offsets, v->word_off, sizeof(int64_t) * (v->n_words + 1),
                                 cudaMemcpyDeviceToHost));
    return BM25_OK;
}

void bm25_vocab_free(bm25_vocab* v)
{
    if (!v)
        return;
    void* ps[] = {v->keys, v->ids, v->words, v->word_off, v->stop_keys, v->stop_ids,
                  v->stop_bytes, v->stop_off};
    for (void* p : ps)
        if (p)
            cudaFreeAsync(p, nullptr);
    cudaDeviceSynchronize();
    delete v;
}

}  // extern "C"
