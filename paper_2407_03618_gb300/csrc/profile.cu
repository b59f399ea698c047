// Opt-in per-kernel timing: while enabled, every kernel launch of the library
// is bracketed by a pair of CUDA events recorded on the launching stream.
// bm25_profile_end() waits for them and aggregates per kernel name.  Off by
// default; never active while a stream is being captured into a graph.
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace bm25 {
namespace {

struct Rec {
    const char* name;
    cudaEvent_t a, b;
};

struct Agg {
    std::string name;
    int64_t launches = 0;
    double ms = 0.0;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_free;
std::vector<Agg> g_agg;

cudaEvent_t take_event()
{
    if (!g_free.empty()) {
        cudaEvent_t e = g_free.back();
        g_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

}  // namespace

ProfileScope::ProfileScope(const char* name, cudaStream_t s) : name_(name), s_(s)
{
    if (!g_on)
        return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return;
    std::lock_guard<std::mutex> g(g_mu);
    a_ = take_event();
    if (a_)
        cudaEventRecord((cudaEvent_t)a_, s);
}

ProfileScope::~ProfileScope()
{
    if (!a_)
        return;
    std::lock_guard<std::mutex> g(g_mu);
    cudaEvent_t b = take_event();
    if (!b)
        return;
    cudaEventRecord(b, s_);
    g_recs.push_back({name_, (cudaEvent_t)a_, b});
}

}  // namespace bm25

using namespace bm25;

extern "C" {

int bm25_profile_begin(void)
{
    std::lock_guard<std::mutex> g(g_mu);
    g_agg.clear();
    g_recs.clear();
    g_on = true;
    return BM25_OK;
}

int bm25_profile_end(void)
{
    clear_error();
    std::vector<Rec> recs;
    {
        std::lock_guard<std::mutex> g(g_mu);
        g_on = false;
        recs.swap(g_recs);
    }
    std::vector<Agg> agg;
    int rc = BM25_OK;
    for (const Rec& r : recs) {
        float ms = 0.0f;
        if (cudaEventSynchronize(r.b) != cudaSuccess ||
            cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess)
            rc = set_error(BM25_E_CUDA, "profile event failed");
        Agg* slot = nullptr;
        for (Agg& x : agg)
            if (x.name == r.name)
                slot = &x;
        if (!slot) {
            agg.push_back(Agg());
            slot = &agg.back();
            slot->name = r.name;
        }
        slot->launches++;
        slot->ms += ms;
    }
    std::lock_guard<std::mutex> g(g_mu);
    for (const Rec& r : recs) {
        g_free.push_back(r.a);
        g_free.push_back(r.b);
    }
    g_agg.swap(agg);
    return rc;
}

int bm25_profile_count(void)
{
    std::lock_guard<std::mutex> g(g_mu);
    return (int)g_agg.size();
}

int bm25_profile_get(int i, char* name, int name_cap, int64_t* launches, double* total_ms)
{
    std::lock_guard<std::mutex> g(g_mu);
    if (i < 0 || i >= (int)g_agg.size())
        return set_error(BM25_E_INVALID, "profile entry %d out of range", i);
    const Agg& a = g_agg[i];
    if (name && name_cap > 0) {
        strncpy(name, a.name.c_str(), (size_t)name_cap - 1);
        name[name_cap - 1] = 0;
    }
    if (launches)
        *launches = a.launches;
    if (total_ms)
        *total_ms = a.ms;
    return BM25_OK;
}

}  // extern "C"
