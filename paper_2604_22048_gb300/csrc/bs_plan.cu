// Ragged batches of the image sampling phase: one launch plan over galaxies of
// mixed stamp sizes and per-galaxy PSFs, replayed as a CUDA graph.
//
// Galaxies are split by the number of 32-column slots their side needs
// (<= 31, <= 63, <= 95, <= 127 px) and ordered largest first within each
// class (longest-processing-time order for the persistent CTAs' work queue).
// Each class gets its own persistent launch, sized for the largest stamp of
// the class: shared memory, grid, and the kernel instance (column slots per
// lane, register budget).  With BS_PLAN_AUTOTUNE the register cap of each
// class -- 128 (4 CTAs = 16 warps of 4-chain galaxies per SM), 96 (5 CTAs) or
// 80 (6 CTAs, some spills), as far as shared memory allows -- is chosen by
// timing the three instances on the class's first galaxies (two waves of the
// largest grid, the second of two runs timed); the instances do the same
// arithmetic, so the choice changes only the speed.  With BS_PLAN_CAPTURE the class launches are recorded once as
// parallel branches of a CUDA graph (fork/join on the plan's streams); the
// graph is replayed by bs_fit_plan_launch on any stream.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <memory>
#include <new>
#include <vector>

#include "bs_internal.h"

struct bs_fit_plan_s {
    struct Launch {
        bs::FitParams p;
        int grid;
        unsigned int *queue;
        int slot_class;
        float trial_ms[3];   // autotune: time of the 128-, 96- and 80-register instance (0 = not timed)
        float trial_half[3]; // the same instances with half the chains per CTA
    };
    std::vector<Launch> launches;
    cudaStream_t streams[4] = {};
    cudaEvent_t fork = nullptr, join[4] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long graph_kernels = 0;   // kernels one replay of the graph launches
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

// Time one launch of L on its first n_trial galaxies with register cap regs
// (a private stream; outputs of those galaxies are overwritten by the plan's
// own launches later).
cudaError_t time_variant(const bs_fit_plan_s::Launch &L, int regs, int n_trial, int sms, cudaStream_t st,
                         cudaEvent_t e0, cudaEvent_t e1, float &ms)
{
    bs::FitParams p = L.p;
    p.regs = regs;
    p.n_work = n_trial;
    const int per_sm = bs::fit_blocks_per_sm(bs::cta_chains(p), p.max_side, regs, p.profile);
    const int grid = std::min(n_trial * bs::cta_groups(p), sms * per_sm);
    cudaError_t e = cudaSuccess;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        e = cudaMemsetAsync(L.queue, 0, sizeof(unsigned int), st);
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = bs::launch_fit(p, grid, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    return e;
}

constexpr int kRegVariants[3] = {128, 96, 80};

// Half the chains per CTA is a candidate layout where a CTA's results do not
// depend on how many threads staged the galaxy: the one-exposure white-noise
// spectral path of the exponential profile.
bool half_layout_ok(const bs::FitParams &p)
{
    return p.profile == 0 && p.n_exp == 1 && !p.noise_corr && !p.done && p.n_chains >= 2 && p.n_chains % 2 == 0;
}

cudaError_t autotune(bs_fit_plan_s *pl, int sms)
{
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (auto &L : pl->launches) {
        if (e != cudaSuccess) break;
        int waves = 1;
        for (int r : kRegVariants) waves = std::max(waves, bs::fit_blocks_per_sm(L.p.n_chains, L.p.max_side, r, L.p.profile));
        const int n_trial = std::min(L.p.n_work, 2 * sms * waves);
        float best = 0.f;
        int best_regs = 128, best_cpc = 0;
        // Candidates: the 128-, 96- and 80-register instances, with all of a
        // galaxy's chains in one CTA or half of them (two CTAs per galaxy,
        // each staging it).  All give the same chains bit for bit (the library
        // is built without implicit multiply-add contraction, so every budget
        // rounds alike), so the choice changes speed only.
        for (int v = 0; v < 3 && e == cudaSuccess; ++v) {
            if (kRegVariants[v] == 96 && L.p.n_chains > 4) continue;   // that instance takes <= 128 threads
            float ms = 0.f;
            L.p.cpc = 0;
            e = time_variant(L, kRegVariants[v], n_trial, sms, st, e0, e1, ms);
            L.trial_ms[v] = ms;
            if (e == cudaSuccess && (v == 0 || ms < best)) {
                best = ms;
                best_regs = kRegVariants[v];
                best_cpc = 0;
            }
            if (e == cudaSuccess && half_layout_ok(L.p)) {
                L.p.cpc = L.p.n_chains / 2;
                e = time_variant(L, kRegVariants[v], n_trial, sms, st, e0, e1, ms);
                L.trial_half[v] = ms;
                L.p.cpc = 0;
                if (e == cudaSuccess && ms < best) {
                    best = ms;
                    best_regs = kRegVariants[v];
                    best_cpc = L.p.n_chains / 2;
                }
            }
        }
        L.p.regs = best_regs;
        L.p.cpc = best_cpc;
        const int groups = bs::cta_groups(L.p);
        L.grid = std::min(L.p.n_work * groups,
                          sms * bs::fit_blocks_per_sm(bs::cta_chains(L.p), L.p.max_side, best_regs, L.p.profile));
    }
    if (st) cudaStreamDestroy(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return e;
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

}  // extern "C"

namespace {

bs_status plan_create(const bs_fit_args *a, const bs_fit_out *o, const int32_t *side_host, int32_t flags,
                      void *workspace, size_t workspace_bytes, void *stream, bs_fit_plan *plan)
{
    if (!plan) return bs::set_error(BS_ERR_INVALID_ARG, "bs_fit_plan_create: NULL plan");
    if (flags & ~(BS_PLAN_CAPTURE | BS_PLAN_AUTOTUNE))
        return bs::set_error(BS_ERR_INVALID_ARG, "bs_fit_plan_create: unknown flags 0x%x", (unsigned)flags);
    const bool capture = (flags & BS_PLAN_CAPTURE) != 0;
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

    // owned until handed out; released (CUDA objects included) on every failure
    std::unique_ptr<bs_fit_plan_s, void (*)(bs_fit_plan_s *)> owner(new bs_fit_plan_s(), release);
    bs_fit_plan_s *pl = owner.get();
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
        L.slot_class = c + 1;
        L.trial_ms[0] = L.trial_ms[1] = L.trial_ms[2] = 0.f;
        L.trial_half[0] = L.trial_half[1] = L.trial_half[2] = 0.f;
        const int per_sm = bs::fit_blocks_per_sm(a->n_chains, maxs[c], L.p.regs, L.p.profile);
        L.grid = std::min(count[c], sms * per_sm);
        pl->launches.push_back(L);
        start += count[c];
    }
    if ((flags & BS_PLAN_AUTOTUNE) && n > 0) {
        e = autotune(pl, sms);
        if (e != cudaSuccess)
            return bs::set_error(BS_ERR_CUDA, "bs_fit_plan_create: autotune: %s", cudaGetErrorString(e));
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
            return bs::set_error(BS_ERR_CUDA, "bs_fit_plan_create: streams: %s", cudaGetErrorString(e));
        }
        // kernel attributes are set outside the capture
        for (auto &L : pl->launches) bs::fit_blocks_per_sm(bs::cta_chains(L.p), L.p.max_side, L.p.regs, L.p.profile);
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            bs::capture_launches(&pl->graph_kernels);   // recorded, not launched
            st = enqueue(pl, cap, true);
            bs::capture_launches(nullptr);
            cudaError_t e2 = cudaStreamEndCapture(cap, &pl->graph);
            if (st == BS_OK && e2 != cudaSuccess) {
                e = e2;
            }
        }
        if (e == cudaSuccess && st == BS_OK) e = cudaGraphInstantiate(&pl->exec, pl->graph, 0);
        cudaStreamDestroy(cap);
        if (st != BS_OK || e != cudaSuccess) {
            if (st != BS_OK) return st;
            return bs::set_error(BS_ERR_CUDA, "bs_fit_plan_create: graph: %s", cudaGetErrorString(e));
        }
    }
    *plan = owner.release();
    return BS_OK;
}

}  // namespace

extern "C" {

bs_status bs_fit_plan_create(const bs_fit_args *a, const bs_fit_out *o, const int32_t *side_host,
                             int32_t flags, void *workspace, size_t workspace_bytes, void *stream,
                             bs_fit_plan *plan)
{
    // no C++ exception crosses the C ABI: a failed host allocation is reported
    try {
        return plan_create(a, o, side_host, flags, workspace, workspace_bytes, stream, plan);
    } catch (const std::bad_alloc &) {
        return bs::set_error(BS_ERR_OUT_OF_MEMORY, "bs_fit_plan_create: host allocation failed");
    } catch (const std::exception &ex) {
        return bs::set_error(BS_ERR_CUDA, "bs_fit_plan_create: %s", ex.what());
    }
}

bs_status bs_fit_plan_launch(bs_fit_plan plan, void *stream)
{
    if (!plan) return bs::set_error(BS_ERR_INVALID_ARG, "bs_fit_plan_launch: NULL plan");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (plan->exec) {
        cudaError_t e = cudaGraphLaunch(plan->exec, s);
        if (e != cudaSuccess) return bs::set_error(BS_ERR_CUDA, "bs_fit_plan_launch: %s", cudaGetErrorString(e));
        bs::count_launches(plan->graph_kernels);
        return BS_OK;
    }
    return enqueue(plan, s, false);
}

bs_status bs_fit_plan_info(bs_fit_plan plan, int32_t i, bs_fit_plan_launch_info *info)
{
    if (!plan || !info) return bs::set_error(BS_ERR_INVALID_ARG, "bs_fit_plan_info: NULL argument");
    if (i < 0 || i >= (int32_t)plan->launches.size())
        return bs::set_error(BS_ERR_INVALID_ARG, "bs_fit_plan_info: launch %d of %zu", i, plan->launches.size());
    const auto &L = plan->launches[i];
    info->slot_class = L.slot_class;
    info->max_side = L.p.max_side;
    info->n_gal = L.p.n_work;
    info->grid = L.grid;
    info->registers = L.p.regs ? L.p.regs : 128;
    info->trial_ms_128 = L.trial_ms[0];
    info->trial_ms_96 = L.trial_ms[1];
    info->trial_ms_80 = L.trial_ms[2];
    info->chains_per_cta = bs::cta_chains(L.p);
    info->trial_ms_128_half = L.trial_half[0];
    info->trial_ms_96_half = L.trial_half[1];
    info->trial_ms_80_half = L.trial_half[2];
    return BS_OK;
}

int32_t bs_fit_plan_num_launches(bs_fit_plan plan) { return plan ? (int32_t)plan->launches.size() : 0; }

bs_status bs_fit_plan_destroy(bs_fit_plan plan)
{
    if (plan) release(plan);
    return BS_OK;
}

}  // extern "C"
