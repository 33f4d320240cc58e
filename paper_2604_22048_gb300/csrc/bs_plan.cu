// Ragged batches of the image sampling phase: one launch plan over galaxies of
// mixed stamp sizes and per-galaxy PSFs, replayed as a CUDA graph.
//
// Galaxies are split by the number of 32-column slots their side needs
// (<= 31, <= 63, <= 95, <= 127 px) and ordered largest first within each
// class (longest-processing-time order for the persistent CTAs' work queue).
// Each class gets its own persistent launch, sized for the largest stamp of
// the class: shared memory, grid, and the kernel instance (column slots per
// lane, register budget).  With capture the class launches are recorded once
// as parallel branches of a CUDA graph (fork/join on the plan's streams); the
// graph is replayed by bs_fit_plan_launch on any stream.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "bs_internal.h"

struct bs_fit_plan_s {
    struct Launch {
        bs::FitParams p;
        int grid;
        unsigned int *queue;
    };
    std::vector<Launch> launches;
    cudaStream_t streams[4] = {};
    cudaEvent_t fork = nullptr, join[4] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int32_t *status = nullptr;
    int n_gal = 0;
};

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

size_t plan_bytes(int n_gal) { return align_up((size_t)n_gal * sizeof(int32_t)) + 4 * kAlign; }

bs_status enqueue(bs_fit_plan_s *pl, cudaStream_t s0, bool forked)
{
    cudaError_t e;
    if (pl->status) {
        e = cudaMemsetAsync(pl->status, 0, sizeof(int32_t) * (size_t)pl->n_gal, s0);
        if (e != cudaSuccess) return bs::set_error(BS_ERR_CUDA, "bs_fit_plan: status reset: %s", cudaGetErrorString(e));
    }
    if (forked) {
        e = cudaEventRecord(pl->fork, s0);
        if (e != cudaSuccess) return bs::set_error(BS_ERR_CUDA, "bs_fit_plan: fork: %s", cudaGetErrorString(e));
    }
    for (size_t i = 0; i < pl->launches.size(); ++i) {
        auto &L = pl->launches[i];
        cudaStream_t s = forked ? pl->streams[i] : s0;
        if (forked) cudaStreamWaitEvent(s, pl->fork, 0);
        e = cudaMemsetAsync(L.queue, 0, sizeof(unsigned int), s);
        if (e == cudaSuccess) e = bs::launch_fit(L.p, L.grid, s);
        if (e != cudaSuccess) return bs::set_error(BS_ERR_CUDA, "bs_fit_plan: launch: %s", cudaGetErrorString(e));
        if (forked) {
            cudaEventRecord(pl->join[i], s);
            cudaStreamWaitEvent(s0, pl->join[i], 0);
        }
    }
    return BS_OK;
}

void release(bs_fit_plan_s *pl)
{
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    for (int i = 0; i < 4; ++i) {
        if (pl->streams[i]) cudaStreamDestroy(pl->streams[i]);
        if (pl->join[i]) cudaEventDestroy(pl->join[i]);
    }
    if (pl->fork) cudaEventDestroy(pl->fork);
    delete pl;
}

}  // namespace

extern "C" {

size_t bs_fit_plan_workspace_bytes(const bs_fit_args *args)
{
    return args ? plan_bytes(args->n_gal) : 0;
}

bs_status bs_fit_plan_create(const bs_fit_args *a, const bs_fit_out *o, const int32_t *side_host,
                             int32_t capture, void *workspace, size_t workspace_bytes, void *stream,
                             bs_fit_plan *plan)
{
    if (!plan) return bs::set_error(BS_ERR_INVALID_ARG, "bs_fit_plan_create: NULL plan");
    *plan = nullptr;
    bs::FitParams base;
    bs_status st = bs::fit_params_from_args(a, o, base, "bs_fit_plan_create");
    if (st != BS_OK) return st;
    if (!side_host) return bs::set_error(BS_ERR_INVALID_ARG, "bs_fit_plan_create: NULL side_host");
    const int n = a->n_gal;
    if (!workspace || workspace_bytes < plan_bytes(n))
        return bs::set_error(BS_ERR_OUT_OF_MEMORY, "bs_fit_plan_create: workspace of %zu bytes needed",
                             plan_bytes(n));
    for (int i = 0; i < n; ++i)
        if (side_host[i] < 3 || side_host[i] > a->max_side || !(side_host[i] & 1))
            return bs::set_error(BS_ERR_INVALID_ARG, "bs_fit_plan_create: side[%d] = %d", i, side_host[i]);
    // classes by 32-column slots, largest first inside each class
    std::vector<int32_t> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t x, int32_t y) { return side_host[x] > side_host[y]; });
    int count[4] = {0, 0, 0, 0}, maxs[4] = {0, 0, 0, 0};
    for (int i = 0; i < n; ++i) {
        const int c = (side_host[i] + 31) / 32 - 1;
        ++count[c];
        maxs[c] = std::max(maxs[c], (int)side_host[i]);
    }
    // work lists grouped by class (descending sides keep classes contiguous)
    int32_t *dev_work = static_cast<int32_t *>(workspace);
    unsigned char *counters = static_cast<unsigned char *>(workspace) + align_up((size_t)n * sizeof(int32_t));
    cudaStream_t s0 = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (n > 0) e = cudaMemcpyAsync(dev_work, order.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s0);
    if (e != cudaSuccess) return bs::set_error(BS_ERR_CUDA, "bs_fit_plan_create: work list: %s", cudaGetErrorString(e));

    bs_fit_plan_s *pl = new bs_fit_plan_s();
    pl->status = o->status;
    pl->n_gal = n;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int start = 0;   // classes appear from the largest in `order`
    for (int c = 3; c >= 0; --c) {
        if (count[c] == 0) continue;
        bs_fit_plan_s::Launch L;
        L.p = base;
        L.p.max_side = maxs[c];
        L.p.h_max = (maxs[c] + 1) / 2;
        L.p.npad = 32 * (c + 1);
        L.p.work = dev_work + start;
        L.p.n_work = count[c];
        L.queue = reinterpret_cast<unsigned int *>(counters + kAlign * c);
        L.p.queue = L.queue;
        const int per_sm = bs::fit_blocks_per_sm(a->n_chains, maxs[c]);
        L.grid = std::min(count[c], sms * per_sm);
        pl->launches.push_back(L);
        start += count[c];
    }
    if (capture && !pl->launches.empty()) {
        for (size_t i = 0; i < pl->launches.size() && e == cudaSuccess; ++i) {
            e = cudaStreamCreateWithFlags(&pl->streams[i], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->join[i], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->fork, cudaEventDisableTiming);
        cudaStream_t cap = nullptr;
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            if (cap) cudaStreamDestroy(cap);
            release(pl);
            return bs::set_error(BS_ERR_CUDA, "bs_fit_plan_create: streams: %s", cudaGetErrorString(e));
        }
        // kernel attributes are set outside the capture
        for (auto &L : pl->launches) bs::fit_blocks_per_sm(a->n_chains, L.p.max_side);
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            st = enqueue(pl, cap, true);
            cudaError_t e2 = cudaStreamEndCapture(cap, &pl->graph);
            if (st == BS_OK && e2 != cudaSuccess) {
                e = e2;
            }
        }
        if (e == cudaSuccess && st == BS_OK) e = cudaGraphInstantiate(&pl->exec, pl->graph, 0);
        cudaStreamDestroy(cap);
        if (st != BS_OK || e != cudaSuccess) {
            release(pl);
            if (st != BS_OK) return st;
            return bs::set_error(BS_ERR_CUDA, "bs_fit_plan_create: graph: %s", cudaGetErrorString(e));
        }
    }
    *plan = pl;
    return BS_OK;
}

bs_status bs_fit_plan_launch(bs_fit_plan plan, void *stream)
{
    if (!plan) return bs::set_error(BS_ERR_INVALID_ARG, "bs_fit_plan_launch: NULL plan");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (plan->exec) {
        cudaError_t e = cudaGraphLaunch(plan->exec, s);
        return e == cudaSuccess ? BS_OK
                                : bs::set_error(BS_ERR_CUDA, "bs_fit_plan_launch: %s", cudaGetErrorString(e));
    }
    return enqueue(plan, s, false);
}

bs_status bs_fit_plan_destroy(bs_fit_plan plan)
{
    if (plan) release(plan);
    return BS_OK;
}

}  // extern "C"
