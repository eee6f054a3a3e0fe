// Batched execution of independent plans (many 3D transforms per call).
//
// A batch spreads its plans over a few internal streams: the caller's
// stream records a fork event that every internal stream waits for, each
// plan's stage launches go to the stream it was assigned, and the caller's
// stream waits for a join event of every internal stream.  Small grids leave
// most of the GPU idle one launch at a time; side by side on several
// streams their launches overlap.  The fork/join uses only events, so a
// batch call can be captured into a CUDA graph (the internal streams join
// the capture through the fork event).
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "p3dfft_gb300.h"

namespace p3 {
p3_status run_direction(p3_plan plan, int dir, const void* in, void* out, void* ws, void* stream);
size_t plan_workspace(p3_plan plan);
double plan_work(p3_plan plan);
int plan_device(p3_plan plan);
}  // namespace p3

struct p3_batch_s {
    std::vector<p3_plan> plans;
    std::vector<int> stream_of;        // internal stream of each plan
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> join;     // one per internal stream
    cudaEvent_t fork;
    int device;
};

static void destroy_batch(p3_batch b)
{
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != b->device) cudaSetDevice(b->device);
    for (cudaEvent_t e : b->join)
        if (e) cudaEventDestroy(e);
    for (cudaStream_t s : b->streams)
        if (s) cudaStreamDestroy(s);
    if (b->fork) cudaEventDestroy(b->fork);
    if (cur >= 0 && cur != b->device) cudaSetDevice(cur);
    cudaGetLastError();
    delete b;
}

extern "C" {

p3_status p3_batch_create(p3_batch* out, int nplans, const p3_plan* plans, int nstreams)
{
    if (!out) return P3_ERR_INVALID;
    *out = NULL;
    if (nplans < 1 || !plans || nstreams < 1) return P3_ERR_INVALID;
    for (int i = 0; i < nplans; ++i)
        if (!plans[i]) return P3_ERR_INVALID;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return P3_ERR_CUDA;
    }
    for (int i = 0; i < nplans; ++i)
        if (p3::plan_device(plans[i]) != dev) return P3_ERR_INVALID;
    if (nstreams > nplans) nstreams = nplans;
    p3_batch b = new (std::nothrow) p3_batch_s();
    if (!b) return P3_ERR_NOMEM;
    b->device = dev;
    b->fork = NULL;
    b->plans.assign(plans, plans + nplans);
    // longest-processing-time assignment: largest plans first, each to the
    // stream with the least work so far
    std::vector<int> order((size_t)nplans);
    for (int i = 0; i < nplans; ++i) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return p3::plan_work(plans[x]) > p3::plan_work(plans[y]); });
    std::vector<double> load((size_t)nstreams, 0.0);
    b->stream_of.assign((size_t)nplans, 0);
    for (int i : order) {
        const int s = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        b->stream_of[(size_t)i] = s;
        load[(size_t)s] += p3::plan_work(plans[i]);
    }
    b->streams.assign((size_t)nstreams, NULL);
    b->join.assign((size_t)nstreams, NULL);
    bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int s = 0; ok && s < nstreams; ++s) {
        ok = cudaStreamCreateWithFlags(&b->streams[(size_t)s], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->join[(size_t)s], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        destroy_batch(b);
        return P3_ERR_CUDA;
    }
    *out = b;
    return P3_OK;
}

p3_status p3_batch_destroy(p3_batch batch)
{
    if (batch) destroy_batch(batch);
    return P3_OK;
}

static p3_status batch_run(p3_batch b, int dir, const void* const* in, void* const* out, void* const* ws,
                           void* stream)
{
    if (!b || !in || !out) return P3_ERR_INVALID;
    const size_t n = b->plans.size();
    for (size_t i = 0; i < n; ++i) {
        if (!in[i] || !out[i]) return P3_ERR_INVALID;
        if (p3::plan_workspace(b->plans[i]) > 0 && (!ws || !ws[i])) return P3_ERR_WORKSPACE;
    }
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        return P3_ERR_CUDA;
    }
    if (cur != b->device) return P3_ERR_INVALID;
    cudaStream_t s0 = (cudaStream_t)stream;
    if (cudaEventRecord(b->fork, s0) != cudaSuccess) return P3_ERR_CUDA;
    for (cudaStream_t s : b->streams)
        if (cudaStreamWaitEvent(s, b->fork, 0) != cudaSuccess) return P3_ERR_CUDA;
    p3_status rc = P3_OK;
    for (size_t i = 0; i < n && rc == P3_OK; ++i)
        rc = p3::run_direction(b->plans[i], dir, in[i], out[i], ws ? ws[i] : NULL,
                               (void*)b->streams[(size_t)b->stream_of[i]]);
    // join even after an error, so the caller's stream never runs ahead of
    // work already enqueued on the internal streams
    for (size_t s = 0; s < b->streams.size(); ++s) {
        if (cudaEventRecord(b->join[s], b->streams[s]) != cudaSuccess ||
            cudaStreamWaitEvent(s0, b->join[s], 0) != cudaSuccess)
            return P3_ERR_CUDA;
    }
    return rc;
}

p3_status p3_batch_ftran_r2c(p3_batch batch, const void* const* in, void* const* out, void* const* ws, void* stream)
{
    return batch_run(batch, 0, in, out, ws, stream);
}

p3_status p3_batch_btran_c2r(p3_batch batch, const void* const* in, void* const* out, void* const* ws, void* stream)
{
    return batch_run(batch, 1, in, out, ws, stream);
}

}  // extern "C"
