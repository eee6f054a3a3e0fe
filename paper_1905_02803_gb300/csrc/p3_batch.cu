// Batched execution of independent plans (many 3D transforms per call).
//
// Persistent mode (nstreams = 0): every stage of every plan of a direction
// becomes a task of the generic stage kernel, and one launch runs them all:
// its CTAs take (task, tile) tickets in order, level by level (each plan's
// first stage, then each plan's second, ...), a tile waiting (bounded) only
// for the plan's previous stage.  One launch per call, whatever the number
// of plans; the call's buffers travel in the launch's parameters, so calls
// never race on them, and the launch can be captured into a CUDA graph.
//
// Stream mode (nstreams >= 1): the batch spreads its plans over internal
// streams: the caller's
// stream records a fork event that every internal stream waits for, each
// plan's stage launches go to the stream it was assigned, and the caller's
// stream waits for a join event of every internal stream.  Small grids leave
// most of the GPU idle one launch at a time; side by side on several
// streams their launches overlap.  The fork/join uses only events, so a
// batch call can be captured into a CUDA graph (the internal streams join
// the capture through the fork event).
#include <cuda_runtime.h>

#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "p3dfft_gb300.h"

#include "p3_internal.h"

namespace p3 {
p3_status run_direction(p3_plan plan, int dir, const void* in, void* out, void* ws, void* stream);
size_t plan_workspace(p3_plan plan);
double plan_work(p3_plan plan);
int plan_device(p3_plan plan);
p3_status generic_stages(p3_plan plan, int dir, std::vector<GenericStage>& out);
p3_status check_generic_call(p3_plan plan, int dir, const void* in, void* out, void* ws);
bool plan_batchable(p3_plan plan);
}  // namespace p3

struct p3_batch_s {
    std::vector<p3_plan> plans;
    std::vector<int> stream_of;        // internal stream of each plan
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> join;     // one per internal stream
    cudaEvent_t fork;
    int device;
    // persistent mode, per direction
    bool persistent;
    p3::BatchTask* dtasks[2];
    int ntasks[2];
    unsigned total[2];
    size_t smem[2];
    int grid[2];
    unsigned* dctr[2];
    unsigned* derr;
    unsigned spin_limit, wait_extra;
};

static void destroy_batch(p3_batch b)
{
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != b->device) cudaSetDevice(b->device);
    for (int d = 0; d < 2; ++d) {
        if (b->dtasks[d]) cudaFree(b->dtasks[d]);
        if (b->dctr[d]) cudaFree(b->dctr[d]);
    }
    if (b->derr) cudaFree(b->derr);
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

// Builds the task table of direction d: plans largest first within each
// level, tickets numbered level by level.
static p3_status build_tasks(p3_batch b, int d)
{
    const int n = (int)b->plans.size();
    std::vector<std::vector<p3::GenericStage>> st((size_t)n);
    size_t levels = 0;
    for (int i = 0; i < n; ++i) {
        const p3_status rc = p3::generic_stages(b->plans[(size_t)i], d, st[(size_t)i]);
        if (rc != P3_OK) return rc;
        levels = std::max(levels, st[(size_t)i].size());
    }
    std::vector<int> order((size_t)n);
    for (int i = 0; i < n; ++i) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return p3::plan_work(b->plans[(size_t)x]) > p3::plan_work(b->plans[(size_t)y]);
    });
    std::vector<p3::BatchTask> tasks;
    std::vector<int> last((size_t)n, -1);  // task index of each plan's previous stage
    long long next = 0;
    size_t smem = 0;
    for (size_t lv = 0; lv < levels; ++lv) {
        for (int i : order) {
            if (lv >= st[(size_t)i].size()) continue;
            const p3::GenericStage& g = st[(size_t)i][lv];
            p3::BatchTask t;
            memset(&t, 0, sizeof(t));
            t.a = g.a;
            t.a.err = b->derr;
            const long long nl = t.a.nrows > t.a.nlines ? t.a.nrows : t.a.nlines;  // pair ops index rows
            p3::line_magic(t.a.in, nl);
            p3::line_magic(t.a.out, nl);
            p3::generic_consts(t.a);
            t.first = next;
            t.ntiles = g.a.nlines > 0 ? (g.a.nlines + g.a.B - 1) / g.a.B : 0;
            t.plan = i;
            t.src = g.src;
            t.dst = g.dst;
            t.dep = last[(size_t)i];
            last[(size_t)i] = (int)tasks.size();
            next += t.ntiles;
            smem = std::max(smem, g.a.smem);
            tasks.push_back(t);
        }
    }
    if (next >= (1LL << 31)) return P3_ERR_UNSUPPORTED;
    b->ntasks[d] = (int)tasks.size();
    b->total[d] = (unsigned)next;
    b->smem[d] = smem;
    b->grid[d] = p3::batch_grid(smem);
    if (b->grid[d] < 1) return P3_ERR_CUDA;
    // the tasks, then their compact scheduling fields
    const size_t tb = sizeof(p3::BatchTask) * std::max<size_t>(1, tasks.size());
    std::vector<p3::BatchMeta> meta(tasks.size());
    for (size_t i = 0; i < tasks.size(); ++i) {
        meta[i].first = (unsigned)tasks[i].first;
        meta[i].ntiles = (unsigned)tasks[i].ntiles;
        meta[i].dep = tasks[i].dep;
        meta[i].plan = tasks[i].plan;
        meta[i].src = tasks[i].src;
        meta[i].dst = tasks[i].dst;
    }
    const size_t mb = sizeof(p3::BatchMeta) * std::max<size_t>(1, tasks.size());
    if (cudaMalloc(&b->dtasks[d], tb + mb) != cudaSuccess ||
        cudaMalloc(&b->dctr[d], sizeof(unsigned) * (size_t)(1 + b->ntasks[d])) != cudaSuccess) {
        cudaGetLastError();
        return P3_ERR_NOMEM;
    }
    if (!tasks.empty() && (cudaMemcpy(b->dtasks[d], tasks.data(), sizeof(p3::BatchTask) * tasks.size(),
                                      cudaMemcpyHostToDevice) != cudaSuccess ||
                           cudaMemcpy(reinterpret_cast<unsigned char*>(b->dtasks[d]) + tb, meta.data(),
                                      sizeof(p3::BatchMeta) * meta.size(), cudaMemcpyHostToDevice) != cudaSuccess)) {
        cudaGetLastError();
        return P3_ERR_CUDA;
    }
    return P3_OK;
}

p3_status p3_batch_create(p3_batch* out, int nplans, const p3_plan* plans, int nstreams)
{
    if (!out) return P3_ERR_INVALID;
    *out = NULL;
    if (nplans < 1 || !plans || nstreams < 0) return P3_ERR_INVALID;
    for (int i = 0; i < nplans; ++i)
        if (!plans[i]) return P3_ERR_INVALID;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return P3_ERR_CUDA;
    }
    for (int i = 0; i < nplans; ++i)
        if (p3::plan_device(plans[i]) != dev) return P3_ERR_INVALID;
    if (nstreams == 0) {
        if (nplans > p3::kBatchMaxPlans) return P3_ERR_UNSUPPORTED;
        for (int i = 0; i < nplans; ++i)
            if (!p3::plan_batchable(plans[i])) return P3_ERR_UNSUPPORTED;
    }
    if (nstreams > nplans) nstreams = nplans;
    p3_batch b = new (std::nothrow) p3_batch_s();
    if (!b) return P3_ERR_NOMEM;
    b->device = dev;
    b->fork = NULL;
    b->persistent = nstreams == 0;
    for (int d = 0; d < 2; ++d) {
        b->dtasks[d] = NULL;
        b->dctr[d] = NULL;
        b->ntasks[d] = 0;
        b->total[d] = 0;
        b->smem[d] = 0;
        b->grid[d] = 0;
    }
    b->derr = NULL;
    b->spin_limit = 1u << 23;
    b->wait_extra = 0;
    b->plans.assign(plans, plans + nplans);
    if (b->persistent) {
        if (cudaMalloc(&b->derr, 256) != cudaSuccess || cudaMemset(b->derr, 0, 256) != cudaSuccess) {
            cudaGetLastError();
            destroy_batch(b);
            return P3_ERR_NOMEM;
        }
        for (int d = 0; d < 2; ++d) {
            const p3_status rc = build_tasks(b, d);
            if (rc != P3_OK) {
                destroy_batch(b);
                return rc;
            }
        }
        *out = b;
        return P3_OK;
    }
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

static p3_status batch_run_persistent(p3_batch b, int dir, const void* const* in, void* const* out,
                                      void* const* ws, void* stream)
{
    const size_t n = b->plans.size();
    p3::BatchLaunch L;
    memset(&L, 0, sizeof(L));
    for (size_t i = 0; i < n; ++i) {
        const p3_status rc = p3::check_generic_call(b->plans[i], dir, in[i], out[i], ws ? ws[i] : NULL);
        if (rc != P3_OK) return rc;
        L.buf[i][0] = const_cast<void*>(in[i]);
        L.buf[i][1] = out[i];
        L.buf[i][2] = ws ? ws[i] : NULL;
    }
    L.tasks = b->dtasks[dir];
    L.meta = reinterpret_cast<const p3::BatchMeta*>(reinterpret_cast<const unsigned char*>(b->dtasks[dir]) +
                                                    sizeof(p3::BatchTask) * std::max<size_t>(1, (size_t)b->ntasks[dir]));
    L.ntasks = b->ntasks[dir];
    L.total = b->total[dir];
    L.ctr = b->dctr[dir];
    L.err = b->derr;
    L.spin_limit = b->spin_limit;
    L.extra = b->wait_extra;
    return p3::batch_launch(L, b->grid[dir], b->smem[dir], (cudaStream_t)stream) == cudaSuccess ? P3_OK
                                                                                                  : P3_ERR_CUDA;
}

static p3_status batch_run(p3_batch b, int dir, const void* const* in, void* const* out, void* const* ws,
                           void* stream)
{
    if (!b || !in || !out) return P3_ERR_INVALID;
    const size_t n = b->plans.size();
    if (b->persistent) {
        for (size_t i = 0; i < n; ++i)
            if (!in[i] || !out[i]) return P3_ERR_INVALID;
        int cur = -1;
        if (cudaGetDevice(&cur) != cudaSuccess) {
            cudaGetLastError();
            return P3_ERR_CUDA;
        }
        if (cur != b->device) return P3_ERR_INVALID;
        for (size_t i = 0; i < n; ++i)
            if (!p3::plan_batchable(b->plans[i])) return P3_ERR_UNSUPPORTED;  // a Z hook set since
        return batch_run_persistent(b, dir, in, out, ws, stream);
    }
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

p3_status p3_batch_wait_status(p3_batch batch)
{
    if (!batch) return P3_ERR_INVALID;
    if (!batch->derr) return P3_OK;
    unsigned v = 0;
    if (cudaMemcpy(&v, batch->derr, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return P3_ERR_CUDA;
    }
    if (!v) return P3_OK;
    if (cudaMemset(batch->derr, 0, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return P3_ERR_CUDA;
    }
    return P3_ERR_TIMEOUT;
}

p3_status p3_batch_set_wait_limits(p3_batch batch, unsigned spin_limit, unsigned extra)
{
    if (!batch || spin_limit == 0) return P3_ERR_INVALID;
    batch->spin_limit = spin_limit;
    batch->wait_extra = extra;
    return P3_OK;
}

p3_status p3_batch_launches(p3_batch batch, int dir, int* launches)
{
    if (!batch || !launches || (dir != 0 && dir != 1)) return P3_ERR_INVALID;
    if (batch->persistent) {
        *launches = batch->total[dir] > 0 ? 1 : 0;
        return P3_OK;
    }
    int n = 0;
    for (p3_plan p : batch->plans) {
        int k = 0;
        if (p3_plan_launches(p, dir, &k) != P3_OK) return P3_ERR_INVALID;
        n += k;
    }
    *launches = n;
    return P3_OK;
}

}  // extern "C"
