// Serving engine: galaxy fit requests admitted while others run.
//
// Host side only; the device work is the fit kernel of bs_fit.cu with its
// serving fields set (each CTA publishes its galaxy's outputs to a pinned
// mirror and raises a flag there).  One engine thread per server:
//
//   submit()  -> pending FIFO (mutex)
//   engine    -> reap: done flags of in-flight requests -> ready queue
//             -> admit: the FIFO prefix that fits the arena and the in-flight
//                cap becomes one "tick": one arena block holding, per
//                32-column slot class, the launch's inputs (stamps, PSFs,
//                noise, starts) followed by its outputs; the inputs are
//                written to the pinned mirror of the block and copied to the
//                device with one cudaMemcpyAsync, and each class is launched
//                (one CTA per galaxy) on a stream with no work left, so the
//                launches of different ticks never wait on one another
//   poll()    -> ready queue; the completions handed out by the previous poll
//                are released, and a tick's block returns to the arena when
//                all its requests are released
//
// Every wait is on the host (flags in pinned memory, events); the device
// never waits for the host.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <stdexcept>
#include <mutex>
#include <thread>
#include <vector>

#include "bs_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// First-fit allocator over [0, cap) with a coalescing free list.
class Arena {
public:
    explicit Arena(size_t cap) : cap_(cap)
    {
        if (cap) free_[0] = cap;
    }
    bool alloc(size_t n, size_t *off)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            const size_t o = it->first, rest = it->second - n;
            free_.erase(it);
            if (rest) free_[o + n] = rest;
            used_ += n;
            high_ = std::max(high_, used_);
            *off = o;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n)
    {
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t largest() const
    {
        size_t m = 0;
        for (const auto &f : free_) m = std::max(m, f.second);
        return m;
    }
    size_t used() const { return used_; }
    size_t high_water() const { return high_; }
    size_t capacity() const { return cap_; }

private:
    size_t cap_, used_ = 0, high_ = 0;
    std::map<size_t, size_t> free_;
};

// Byte layout of one class launch inside a tick block.  Inputs of all the
// tick's classes come first (one copy), outputs after them.
struct SubLayout {
    int cls = 0, n = 0, max_side = 0;
    size_t queue, offsets, side, psf, sigma, gal_id, init, status, stamps;   // inputs
    size_t samples, logp, accepted, accept_rate, step, inv_mass, n_div, n_grad, done;  // outputs
};

struct Req {
    bs_serve_request r;
    int64_t t_submit;
};

struct Tick;

struct Inflight {
    bs_serve_request r;
    int64_t t_submit, t_admit;
    Tick *tick;
    int sub, j;     // class launch within the tick, position in it
};

struct Tick {
    size_t off, bytes;
    std::vector<SubLayout> subs;
    int unreleased;  // requests whose completion has not been released yet
};

constexpr size_t kA = 16;   // alignment of every array in a block

size_t req_in_bytes(int C, int side)
{
    // offsets, side, psf, sigma, gal_id, init, status, stamp
    return 8 + 4 + sizeof(bs_psf) + 4 + 8 + 24 * (size_t)C + 4 + 4 * (size_t)side * side;
}

size_t req_out_bytes(int C, int S)
{
    const size_t cs = (size_t)C * S;
    return 24 * cs + 4 * cs + cs + 4 * (size_t)C * 2 + 24 * (size_t)C + 8 * (size_t)C + 4;
}

}  // namespace

struct bs_server_s {
    bs_serve_cfg cfg;
    int device = 0;
    bs::FitParams base;         // configuration part of every launch
    unsigned char *arena_dev = nullptr;
    unsigned char *mirror = nullptr;       // pinned, host view
    unsigned char *mirror_dev = nullptr;   // the same memory, device view
    Arena arena{0};
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> stream_idle;  // recorded after each use
    std::vector<cudaEvent_t> copy_done;    // one per stream that issued a copy
    size_t rr = 0;
    int resident = 0;           // galaxies of side 63 the GPU holds at once
    Clock::time_point t0;

    std::mutex mu;
    std::condition_variable cv_work, cv_ready;
    std::deque<Req> pending;
    std::vector<Inflight> inflight;
    std::deque<bs_serve_completion> ready;
    std::deque<Tick *> ready_ticks;       // tick of each ready completion (parallel to `ready`)
    std::vector<Tick *> returned;         // ticks of the completions handed out by the last poll
    bool stop = false;
    bs_status error = BS_OK;
    char error_msg[256] = {0};
    int64_t last_admit = 0;
    bs_serve_stats st{};
    std::thread engine;

    int64_t now() const
    {
        return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - t0).count();
    }
};

namespace {

void engine_fail(bs_server_s *s, cudaError_t e, const char *what)
{
    if (s->error != BS_OK) return;
    s->error = BS_ERR_CUDA;
    snprintf(s->error_msg, sizeof s->error_msg, "bs_serve engine: %s: %s", what, cudaGetErrorString(e));
}

// Lay out the tick's class launches; returns the block size.
size_t layout_tick(std::vector<SubLayout> &subs, int C, int S, const std::vector<size_t> &stamp_floats)
{
    size_t cur = 0;
    for (size_t k = 0; k < subs.size(); ++k) {
        SubLayout &L = subs[k];
        const size_t n = L.n;
        L.queue = cur;              cur = align_up(cur + 4, kA);
        L.offsets = cur;            cur = align_up(cur + 8 * n, kA);
        L.side = cur;               cur = align_up(cur + 4 * n, kA);
        L.psf = cur;                cur = align_up(cur + sizeof(bs_psf) * n, kA);
        L.sigma = cur;              cur = align_up(cur + 4 * n, kA);
        L.gal_id = cur;             cur = align_up(cur + 8 * n, kA);
        L.init = cur;               cur = align_up(cur + 24 * (size_t)C * n, kA);
        L.status = cur;             cur = align_up(cur + 4 * n, kA);
        L.stamps = cur;             cur = align_up(cur + 4 * stamp_floats[k], kA);
    }
    const size_t cs = (size_t)C * S;
    for (auto &L : subs) {
        const size_t n = L.n;
        L.samples = cur;            cur = align_up(cur + 24 * cs * n, kA);
        L.logp = cur;               cur = align_up(cur + 4 * cs * n, kA);
        L.accepted = cur;           cur = align_up(cur + cs * n, kA);
        L.accept_rate = cur;        cur = align_up(cur + 4 * (size_t)C * n, kA);
        L.step = cur;               cur = align_up(cur + 4 * (size_t)C * n, kA);
        L.inv_mass = cur;           cur = align_up(cur + 24 * (size_t)C * n, kA);
        L.n_div = cur;              cur = align_up(cur + 4 * (size_t)C * n, kA);
        L.n_grad = cur;             cur = align_up(cur + 4 * (size_t)C * n, kA);
        L.done = cur;               cur = align_up(cur + 4 * n, kA);
    }
    return align_up(cur, 256);
}

int slot_class(int side) { return (side + 31) / 32 - 1; }   // 0..3

// Reap: move the requests whose done flag is up to the ready queue.
void reap(bs_server_s *s)
{
    const int C = s->cfg.n_chains, S = s->cfg.n_samples;
    const int64_t t = s->now();
    size_t w = 0;
    for (size_t i = 0; i < s->inflight.size(); ++i) {
        Inflight &f = s->inflight[i];
        const SubLayout &L = f.tick->subs[f.sub];
        unsigned char *base = s->mirror + f.tick->off;
        const uint32_t *done = reinterpret_cast<const uint32_t *>(base + L.done);
        if (__atomic_load_n(done + f.j, __ATOMIC_ACQUIRE) == 0u) {
            if (w != i) s->inflight[w] = f;
            ++w;
            continue;
        }
        const size_t cs = (size_t)C * S, j = f.j;
        bs_serve_completion c;
        std::memset(&c, 0, sizeof c);
        c.tag = f.r.tag;
        c.side = f.r.side;
        c.status = reinterpret_cast<const int32_t *>(base + L.status)[j];
        c.t_arrival_ns = f.r.t_arrival_ns;
        c.t_submit_ns = f.t_submit;
        c.t_admit_ns = f.t_admit;
        c.t_done_ns = t;
        c.samples = reinterpret_cast<const float *>(base + L.samples) + j * cs;
        c.plane_stride = (int64_t)(L.n * cs);
        c.logp = reinterpret_cast<const float *>(base + L.logp) + j * cs;
        c.accepted = base + L.accepted + j * cs;
        c.accept_rate = reinterpret_cast<const float *>(base + L.accept_rate) + j * C;
        c.step_size = reinterpret_cast<const float *>(base + L.step) + j * C;
        c.inv_mass = reinterpret_cast<const float *>(base + L.inv_mass) + j * C * 6;
        c.n_divergent = reinterpret_cast<const int32_t *>(base + L.n_div) + j * C;
        c.n_grad = reinterpret_cast<const int32_t *>(base + L.n_grad) + j * C;
        s->ready.push_back(c);
        s->ready_ticks.push_back(f.tick);
        ++s->st.completed;
    }
    s->inflight.resize(w);
}

// Find a stream with no work left (round robin from the last one used).
int idle_stream(bs_server_s *s, const std::vector<int> &taken)
{
    const size_t n = s->streams.size();
    for (size_t k = 0; k < n; ++k) {
        const int i = (int)((s->rr + k) % n);
        if (std::find(taken.begin(), taken.end(), i) != taken.end()) continue;
        const cudaError_t q = cudaEventQuery(s->stream_idle[i]);
        if (q == cudaSuccess) {
            s->rr = (size_t)i + 1;
            return i;
        }
        if (q != cudaErrorNotReady) {
            engine_fail(s, q, "cudaEventQuery");
            return -1;
        }
    }
    return -1;
}

// Admit the FIFO prefix of pending requests that fits; launch it.
void admit(bs_server_s *s)
{
    const int C = s->cfg.n_chains, S = s->cfg.n_samples;
    const int cap = s->cfg.max_inflight - (int)s->inflight.size();
    if (cap <= 0) {
        ++s->st.waits_inflight;
        return;
    }
    // choose the prefix: per-class counts and stamp sizes, bounded by the
    // largest free extent of the arena (alignment slack included)
    const size_t room = s->arena.largest();
    const size_t slack = 4 * (18 * kA + 256);
    size_t need = 0;
    int take = 0;
    const int npend = (int)s->pending.size();
    while (take < npend && take < cap) {
        const int side = s->pending[take].r.side;
        const size_t b = req_in_bytes(C, side) + req_out_bytes(C, S) + 18 * kA;
        if (need + b + slack > room) break;
        need += b;
        ++take;
    }
    if (take == 0) {
        ++s->st.waits_memory;
        return;
    }
    if (take < npend && take < cap) ++s->st.waits_memory;
    // classes present and a stream for each
    int count[4] = {0, 0, 0, 0}, mside[4] = {0, 0, 0, 0};
    std::vector<size_t> stamp_floats;
    for (int i = 0; i < take; ++i) {
        const int side = s->pending[i].r.side, c = slot_class(side);
        ++count[c];
        mside[c] = std::max(mside[c], side);
    }
    std::vector<SubLayout> subs;
    std::vector<int> sub_of_class(4, -1);
    for (int c = 0; c < 4; ++c) {
        if (!count[c]) continue;
        SubLayout L;
        L.cls = c;
        L.n = 0;
        L.max_side = mside[c];
        sub_of_class[c] = (int)subs.size();
        subs.push_back(L);
        stamp_floats.push_back(0);
    }
    std::vector<int> strm;
    for (size_t k = 0; k < subs.size(); ++k) {
        const int i = idle_stream(s, strm);
        if (i < 0) {
            if (s->error == BS_OK) ++s->st.waits_streams;
            return;
        }
        strm.push_back(i);
    }
    for (int i = 0; i < take; ++i) {
        const int side = s->pending[i].r.side, k = sub_of_class[slot_class(side)];
        subs[k].n += 1;
        stamp_floats[k] += (size_t)side * side;
    }
    const size_t bytes = layout_tick(subs, C, S, stamp_floats);
    size_t off = 0;
    if (!s->arena.alloc(bytes, &off)) {   // the slack covers the layout; not expected
        ++s->st.waits_memory;
        return;
    }
    Tick *tick = new Tick{off, bytes, subs, take};
    unsigned char *hb = s->mirror + off;
    // fill the inputs in the mirror, in FIFO order within each class
    std::vector<int> pos(subs.size(), 0);
    std::vector<int64_t> stamp_at(subs.size(), 0);
    const int64_t t_admit = s->now();
    for (int i = 0; i < take; ++i) {
        const Req &q = s->pending[i];
        const int k = sub_of_class[slot_class(q.r.side)];
        const SubLayout &L = subs[k];
        const int j = pos[k]++;
        const int N = q.r.side;
        reinterpret_cast<int64_t *>(hb + L.offsets)[j] = stamp_at[k];
        reinterpret_cast<int32_t *>(hb + L.side)[j] = N;
        reinterpret_cast<bs_psf *>(hb + L.psf)[j] = q.r.psf;
        reinterpret_cast<float *>(hb + L.sigma)[j] = q.r.noise_sigma;
        reinterpret_cast<uint64_t *>(hb + L.gal_id)[j] = q.r.gal_id;
        std::memcpy(hb + L.init + (size_t)j * 24 * C, q.r.init, 24 * (size_t)C);
        reinterpret_cast<int32_t *>(hb + L.status)[j] = 0;
        std::memcpy(hb + L.stamps + 4 * (size_t)stamp_at[k], q.r.stamp, 4 * (size_t)N * N);
        stamp_at[k] += (int64_t)N * N;
        reinterpret_cast<uint32_t *>(hb + L.done)[j] = 0u;
        s->inflight.push_back(Inflight{q.r, q.t_submit, t_admit, tick, k, j});
    }
    for (auto &L : subs) *reinterpret_cast<uint32_t *>(hb + L.queue) = 0u;
    const size_t in_bytes = subs.back().stamps + 4 * stamp_floats.back();
    unsigned char *db = s->arena_dev + off;
    const long long shift = (long long)((s->mirror_dev + off) - db);
    cudaStream_t s0 = s->streams[strm[0]];
    cudaError_t e = cudaMemcpyAsync(db, hb, in_bytes, cudaMemcpyHostToDevice, s0);
    if (e != cudaSuccess) return engine_fail(s, e, "input copy");
    if (subs.size() > 1) {
        e = cudaEventRecord(s->copy_done[strm[0]], s0);
        if (e != cudaSuccess) return engine_fail(s, e, "cudaEventRecord");
    }
    for (size_t k = 0; k < subs.size(); ++k) {
        const SubLayout &L = subs[k];
        cudaStream_t sk = s->streams[strm[k]];
        if (k > 0) {
            e = cudaStreamWaitEvent(sk, s->copy_done[strm[0]], 0);
            if (e != cudaSuccess) return engine_fail(s, e, "cudaStreamWaitEvent");
        }
        bs::FitParams p = s->base;
        p.data = db + L.stamps;
        p.data_f64 = 0;
        p.offsets = reinterpret_cast<const int64_t *>(db + L.offsets);
        p.side = reinterpret_cast<const int32_t *>(db + L.side);
        p.psf = reinterpret_cast<const bs_psf *>(db + L.psf);
        p.n_psf = L.n;
        p.sigma = reinterpret_cast<const float *>(db + L.sigma);
        p.gal_id = reinterpret_cast<const uint64_t *>(db + L.gal_id);
        p.init = reinterpret_cast<const float *>(db + L.init);
        p.n_gal = L.n;
        p.samples = reinterpret_cast<float *>(db + L.samples);
        p.logp = reinterpret_cast<float *>(db + L.logp);
        p.accepted = db + L.accepted;
        p.accept_rate = reinterpret_cast<float *>(db + L.accept_rate);
        p.step_size = reinterpret_cast<float *>(db + L.step);
        p.inv_mass = reinterpret_cast<float *>(db + L.inv_mass);
        p.n_div = reinterpret_cast<int32_t *>(db + L.n_div);
        p.status = reinterpret_cast<int32_t *>(db + L.status);
        p.n_grad = reinterpret_cast<int32_t *>(db + L.n_grad);
        p.work = nullptr;
        p.n_work = L.n;
        p.queue = reinterpret_cast<unsigned int *>(db + L.queue);
        p.max_side = L.max_side;
        p.h_max = (L.max_side + 1) / 2;
        p.npad = 32 * ((L.max_side + 31) / 32);
        p.regs = s->cfg.registers[L.cls];
        p.done = reinterpret_cast<uint32_t *>(s->mirror_dev + off + L.done);
        p.pub_shift = shift;
        e = bs::launch_fit(p, L.n, sk);
        if (e != cudaSuccess) return engine_fail(s, e, "fit launch");
        e = cudaEventRecord(s->stream_idle[strm[k]], sk);
        if (e != cudaSuccess) return engine_fail(s, e, "cudaEventRecord");
        ++s->st.launches;
    }
    s->pending.erase(s->pending.begin(), s->pending.begin() + take);
    s->st.admitted += take;
    ++s->st.ticks;
    s->last_admit = s->now();
}

void release_returned(bs_server_s *s)
{
    for (Tick *t : s->returned) {
        if (--t->unreleased == 0) {
            s->arena.release(t->off, t->bytes);
            delete t;
        }
    }
    s->returned.clear();
}

void engine_main(bs_server_s *s)
{
    cudaSetDevice(s->device);
    const int64_t tick_ns = (int64_t)s->cfg.batch_us * 1000;
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        if (s->error == BS_OK) {
            try {
                const size_t before = s->ready.size();
                reap(s);
                if (s->ready.size() != before) s->cv_ready.notify_all();
                const bool starving = (int)s->inflight.size() < s->resident;
                if (!s->pending.empty() && (starving || s->now() - s->last_admit >= tick_ns)) admit(s);
            } catch (const std::exception &ex) {
                s->error = BS_ERR_OUT_OF_MEMORY;
                snprintf(s->error_msg, sizeof s->error_msg, "bs_serve engine: %s", ex.what());
            }
        }
        if (s->error != BS_OK) s->cv_ready.notify_all();
        if (s->inflight.empty() && (s->pending.empty() || s->error != BS_OK)) {
            s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
        } else {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
    }
}

bs_status serve_fail(bs_status st, const char *msg) { return bs::set_error(st, "%s", msg); }

}  // namespace

extern "C" {

size_t bs_serve_request_bytes(const bs_serve_cfg *cfg, int32_t side)
{
    if (!cfg || side < 1) return 0;
    return req_in_bytes(cfg->n_chains, side) + req_out_bytes(cfg->n_chains, cfg->n_samples);
}

bs_status bs_serve_create(const bs_serve_cfg *cfg, void *arena, size_t arena_bytes, bs_server *out)
{
    if (!cfg || !out) return serve_fail(BS_ERR_INVALID_ARG, "bs_serve_create: NULL argument");
    *out = nullptr;
    if (!arena || arena_bytes < ((size_t)1 << 20))
        return serve_fail(BS_ERR_INVALID_ARG, "bs_serve_create: arena must be >= 1 MiB of device memory");
    if (cfg->n_streams != 0 && (cfg->n_streams < 4 || cfg->n_streams > 128))
        return serve_fail(BS_ERR_INVALID_ARG, "bs_serve_create: n_streams must be 0 or 4..128");
    if (cfg->max_inflight < 0 || cfg->batch_us < 0)
        return serve_fail(BS_ERR_INVALID_ARG, "bs_serve_create: max_inflight / batch_us < 0");
    for (int c = 0; c < 4; ++c) {
        const int r = cfg->registers[c];
        if (r != 0 && r != 128 && r != 96 && r != 80)
            return serve_fail(BS_ERR_INVALID_ARG, "bs_serve_create: registers must be 0, 128, 96 or 80");
    }
    // validate the sampler configuration through the fit path's checks
    bs_fit_args a;
    std::memset(&a, 0, sizeof a);
    static const float dummy = 0.f;
    a.n_gal = 0;
    a.data_dtype = BS_F32;
    a.data = &dummy;
    a.offsets = reinterpret_cast<const int64_t *>(&dummy);
    a.side = reinterpret_cast<const int32_t *>(&dummy);
    a.max_side = cfg->max_side;
    a.psf = reinterpret_cast<const bs_psf *>(&dummy);
    a.n_psf = 0;
    a.noise_sigma = &dummy;
    a.init = &dummy;
    a.pixel_scale = cfg->pixel_scale;
    a.prior = cfg->prior;
    a.n_chains = cfg->n_chains;
    a.n_warmup = cfg->n_warmup;
    a.n_samples = cfg->n_samples;
    a.n_leapfrog = cfg->n_leapfrog;
    a.target_accept = cfg->target_accept;
    a.jitter = cfg->jitter;
    a.adapt_mass = cfg->adapt_mass;
    a.random_steps = cfg->random_steps;
    a.seed = cfg->seed;
    bs_fit_out o;
    std::memset(&o, 0, sizeof o);
    o.samples = const_cast<float *>(&dummy);
    std::unique_ptr<bs_server_s> s(new (std::nothrow) bs_server_s);
    if (!s) return serve_fail(BS_ERR_OUT_OF_MEMORY, "bs_serve_create: out of host memory");
    bs_status st = bs::fit_params_from_args(&a, &o, s->base, "bs_serve_create");
    if (st != BS_OK) return st;
    s->cfg = *cfg;
    if (s->cfg.batch_us == 0) s->cfg.batch_us = 500;
    if (s->cfg.n_streams == 0) s->cfg.n_streams = 128;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) return bs::set_error(BS_ERR_CUDA, "bs_serve_create: %s", cudaGetErrorString(e));
    s->resident = bs_fit_resident_galaxies(cfg->n_chains, 63 < cfg->max_side ? 63 : cfg->max_side,
                                           cfg->max_side > 31 ? cfg->registers[1] : cfg->registers[0]);
    if (s->resident <= 0) s->resident = 1;
    if (s->cfg.max_inflight == 0) s->cfg.max_inflight = 2 * s->resident;
    e = cudaHostAlloc(reinterpret_cast<void **>(&s->mirror), arena_bytes, cudaHostAllocMapped | cudaHostAllocPortable);
    if (e != cudaSuccess) return bs::set_error(BS_ERR_CUDA, "bs_serve_create: pinned mirror: %s", cudaGetErrorString(e));
    e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&s->mirror_dev), s->mirror, 0);
    if (e != cudaSuccess) {
        cudaFreeHost(s->mirror);
        return bs::set_error(BS_ERR_CUDA, "bs_serve_create: mirror device pointer: %s", cudaGetErrorString(e));
    }
    s->arena_dev = static_cast<unsigned char *>(arena);
    s->arena = Arena(arena_bytes);
    for (int i = 0; i < s->cfg.n_streams; ++i) {
        cudaStream_t q;
        cudaEvent_t ev, cp;
        e = cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&cp, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (size_t k = 0; k < s->streams.size(); ++k) {
                cudaStreamDestroy(s->streams[k]);
                cudaEventDestroy(s->stream_idle[k]);
                cudaEventDestroy(s->copy_done[k]);
            }
            cudaFreeHost(s->mirror);
            return bs::set_error(BS_ERR_CUDA, "bs_serve_create: streams: %s", cudaGetErrorString(e));
        }
        s->streams.push_back(q);
        s->stream_idle.push_back(ev);
        s->copy_done.push_back(cp);
    }
    s->st.arena_bytes = (int64_t)arena_bytes;
    s->t0 = Clock::now();
    s->last_admit = -(int64_t)1 << 60;
    try {
        s->engine = std::thread(engine_main, s.get());
    } catch (const std::exception &ex) {
        for (size_t k = 0; k < s->streams.size(); ++k) {
            cudaStreamDestroy(s->streams[k]);
            cudaEventDestroy(s->stream_idle[k]);
            cudaEventDestroy(s->copy_done[k]);
        }
        cudaFreeHost(s->mirror);
        return bs::set_error(BS_ERR_INVALID_ARG, "bs_serve_create: engine thread: %s", ex.what());
    }
    *out = s.release();
    return BS_OK;
}

bs_status bs_serve_submit(bs_server s, const bs_serve_request *req, int32_t n)
{
    if (!s || (n > 0 && !req) || n < 0) return serve_fail(BS_ERR_INVALID_ARG, "bs_serve_submit: bad arguments");
    const int C = s->cfg.n_chains, S = s->cfg.n_samples;
    for (int i = 0; i < n; ++i) {
        const bs_serve_request &r = req[i];
        if (r.side < 3 || r.side > s->cfg.max_side || !(r.side & 1))
            return bs::set_error(BS_ERR_INVALID_ARG, "bs_serve_submit: request %d: side %d", i, r.side);
        if (!r.stamp || !r.init)
            return bs::set_error(BS_ERR_INVALID_ARG, "bs_serve_submit: request %d: NULL stamp/init", i);
        if (!(r.noise_sigma > 0.f) || !(r.psf.fwhm > 0.f) ||
            (r.psf.kind != BS_PSF_GAUSSIAN && !(r.psf.kind == BS_PSF_MOFFAT && r.psf.beta > 1.f)))
            return bs::set_error(BS_ERR_INVALID_ARG, "bs_serve_submit: request %d: noise or PSF", i);
        const size_t b = req_in_bytes(C, r.side) + req_out_bytes(C, S) + 4 * (18 * kA + 256) + 18 * kA;
        if (b > s->arena.capacity())
            return bs::set_error(BS_ERR_INVALID_ARG, "bs_serve_submit: request %d needs more than the arena", i);
    }
    try {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->error != BS_OK) return bs::set_error(s->error, "%s", s->error_msg);
        const int64_t t = s->now();
        for (int i = 0; i < n; ++i) {
            Req q{req[i], t};
            if (q.r.t_arrival_ns < 0) q.r.t_arrival_ns = t;
            s->pending.push_back(q);
        }
        s->st.submitted += n;
    } catch (const std::exception &ex) {
        return bs::set_error(BS_ERR_OUT_OF_MEMORY, "bs_serve_submit: %s", ex.what());
    }
    s->cv_work.notify_one();
    return BS_OK;
}

bs_status bs_serve_poll(bs_server s, bs_serve_completion *out, int32_t max, int32_t timeout_us, int32_t *n_out)
{
    if (!s || !n_out || max < 0 || (max > 0 && !out)) return serve_fail(BS_ERR_INVALID_ARG, "bs_serve_poll: bad arguments");
    *n_out = 0;
    std::unique_lock<std::mutex> lk(s->mu);
    release_returned(s);
    if (s->ready.empty() && timeout_us > 0 && s->error == BS_OK)
        s->cv_ready.wait_for(lk, std::chrono::microseconds(timeout_us),
                             [s] { return !s->ready.empty() || s->error != BS_OK; });
    int k = 0;
    try {
        s->returned.reserve((size_t)max);
    } catch (const std::exception &ex) {
        return bs::set_error(BS_ERR_OUT_OF_MEMORY, "bs_serve_poll: %s", ex.what());
    }
    while (k < max && !s->ready.empty()) {
        out[k++] = s->ready.front();
        s->ready.pop_front();
        s->returned.push_back(s->ready_ticks.front());   // within the reserved capacity
        s->ready_ticks.pop_front();
    }
    *n_out = k;
    if (s->error != BS_OK && k == 0) return bs::set_error(s->error, "%s", s->error_msg);
    return BS_OK;
}

bs_status bs_serve_get_stats(bs_server s, bs_serve_stats *out)
{
    if (!s || !out) return serve_fail(BS_ERR_INVALID_ARG, "bs_serve_get_stats: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    out->arena_used = (int64_t)s->arena.used();
    out->arena_high_water = (int64_t)s->arena.high_water();
    out->pending = (int32_t)s->pending.size();
    out->inflight = (int32_t)s->inflight.size();
    return BS_OK;
}

int64_t bs_serve_now_ns(bs_server s) { return s ? s->now() : -1; }

bs_status bs_serve_destroy(bs_server s)
{
    if (!s) return BS_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->pending.clear();
    }
    s->cv_work.notify_all();
    s->engine.join();
    cudaSetDevice(s->device);
    cudaError_t first = cudaSuccess;
    for (size_t k = 0; k < s->streams.size(); ++k) {
        const cudaError_t e = cudaStreamSynchronize(s->streams[k]);
        if (first == cudaSuccess) first = e;
        cudaStreamDestroy(s->streams[k]);
        cudaEventDestroy(s->stream_idle[k]);
        cudaEventDestroy(s->copy_done[k]);
    }
    std::vector<Tick *> ticks;
    for (auto &f : s->inflight) ticks.push_back(f.tick);
    for (Tick *t : s->ready_ticks) ticks.push_back(t);
    for (Tick *t : s->returned) ticks.push_back(t);
    std::sort(ticks.begin(), ticks.end());
    ticks.erase(std::unique(ticks.begin(), ticks.end()), ticks.end());
    for (Tick *t : ticks) delete t;
    cudaFreeHost(s->mirror);
    delete s;
    return first == cudaSuccess ? BS_OK : bs::set_error(BS_ERR_CUDA, "bs_serve_destroy: %s", cudaGetErrorString(first));
}

}  // extern "C"
