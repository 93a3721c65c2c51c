// Continuous-batching request server over a pool of device-resident
// generators (mtgp_server_* in include/mtgp.h).  Built on the public pool and
// graph calls: each tick is one replay of the pool's captured persistent
// launch, advancing every active request by up to `chunk` numbers.
#include "mtgp.h"
#include "mtgp_graph.h"
#include "mtgp_internal.h"

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <deque>
#include <exception>
#include <map>
#include <new>
#include <unordered_map>
#include <vector>

namespace {

struct Req {
    uint32_t gen = 0, dtype = 0;
    uint64_t n = 0, done = 0;        // numbers requested / already launched
    uint64_t off = 0, bytes = 0;     // output range in the arena
    double submit_s = 0, done_s = 0;
    bool admitted = false, finished = false;
};

struct Tick {
    cudaEvent_t ev = nullptr;
    std::vector<uint64_t> finishing;   // tickets whose last numbers this tick generates
};

mtgp_status fail(mtgp_status st, const char *msg) { return (mtgp_status)mtgp::report_error(st, msg); }

mtgp_status fail_cuda(cudaError_t e, const char *what)
{
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s (%d)", what, cudaGetErrorString(e), (int)e);
    return fail(MTGP_ECUDA, buf);
}

// Entry points return MTGP_ENOMEM instead of letting a container's
// allocation failure cross the C ABI.
template <class F>
mtgp_status guarded(F &&f)
{
    try {
        return f();
    } catch (const std::bad_alloc &) {
        return fail(MTGP_ENOMEM, "server: host allocation failed");
    } catch (const std::exception &e) {
        return fail(MTGP_EINVAL, e.what());
    }
}

constexpr uint64_t kAlign = 256;

}  // namespace

struct mtgp_server {
    mtgp_pool *pool = nullptr;
    mtgp_graph *graph = nullptr;
    cudaStream_t stream = nullptr;
    mtgp_server_config cfg{};
    uint32_t count = 0;
    char *arena = nullptr;
    std::map<uint64_t, uint64_t> free_list;        // offset -> size, coalesced
    std::deque<uint64_t> pending;                  // submission order
    std::unordered_map<uint64_t, Req> reqs;
    std::vector<uint64_t> active;
    std::vector<uint8_t> gen_busy;                 // a request of the generator is being generated
    std::deque<Tick> inflight;
    std::vector<cudaEvent_t> spare_events;
    std::deque<mtgp_completion> done_q;
    cudaEvent_t ev_ref = nullptr;
    std::chrono::steady_clock::time_point t0;
    uint64_t next_ticket = 1;
    uint64_t numbers_done = 0, ticks = 0;
    std::vector<mtgp_request> tick_reqs;
    std::vector<uint32_t> held_mark;               // == held_stamp: generator held back this pass
    uint32_t held_stamp = 0;

    double now_s() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }

    bool alloc(uint64_t bytes, uint64_t *off)
    {
        bytes = (bytes + kAlign - 1) / kAlign * kAlign;
        for (auto it = free_list.begin(); it != free_list.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const uint64_t rest = it->second - bytes, at = it->first + bytes;
                free_list.erase(it);
                if (rest) free_list[at] = rest;
                return true;
            }
        }
        return false;
    }

    void release_range(uint64_t off, uint64_t bytes)
    {
        bytes = (bytes + kAlign - 1) / kAlign * kAlign;
        auto it = free_list.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_list.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_list.erase(next);
        }
        if (it != free_list.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_list.erase(it);
            }
        }
    }
};

extern "C" {

mtgp_status mtgp_server_create(mtgp_pool *pool, const mtgp_server_config *cfg, void *stream, mtgp_server **out)
{
    return guarded([&]() -> mtgp_status {
        if (!pool || !out) return fail(MTGP_EINVAL, "server: NULL pool or out");
        *out = nullptr;
        mtgp_server *s = new (std::nothrow) mtgp_server;
        if (!s) return fail(MTGP_ENOMEM, "host allocation");
        s->pool = pool;
        s->stream = (cudaStream_t)stream;
        if (cfg) s->cfg = *cfg;
        if (!s->cfg.arena_bytes) s->cfg.arena_bytes = 1ull << 32;
        if (!s->cfg.chunk) s->cfg.chunk = 1ull << 20;
        if (!s->cfg.max_active) s->cfg.max_active = 4096;
        if (!s->cfg.max_inflight) s->cfg.max_inflight = 2;
        s->cfg.arena_bytes = s->cfg.arena_bytes / kAlign * kAlign;
        uint64_t dev_bytes = 0;
        mtgp_status st = mtgp_pool_info(pool, &s->count, &dev_bytes);
        if (st != MTGP_OK) {
            delete s;
            return st;
        }
        s->gen_busy.assign(s->count, 0);
        cudaError_t e = cudaMalloc(&s->arena, s->cfg.arena_bytes);
        if (e != cudaSuccess) {
            delete s;
            return e == cudaErrorMemoryAllocation ? fail(MTGP_ENOMEM, "server: arena allocation")
                                                  : fail_cuda(e, "server: cudaMalloc arena");
        }
        s->free_list[0] = s->cfg.arena_bytes;
        // ticks never split a request into jump-ahead pieces: that would need the
        // annihilating polynomial of every generator a request may name
        st = mtgp::graph_create(pool, std::min<uint32_t>(s->cfg.max_active, s->count), stream, false, &s->graph);
        if (st != MTGP_OK) {
            mtgp_server_destroy(s);
            return st;
        }
        e = cudaEventCreate(&s->ev_ref);
        if (e == cudaSuccess) e = cudaEventRecord(s->ev_ref, s->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(s->ev_ref);
        if (e != cudaSuccess) {
            mtgp_server_destroy(s);
            return fail_cuda(e, "server: reference event");
        }
        s->t0 = std::chrono::steady_clock::now();
        *out = s;
        return MTGP_OK;
    });
}

mtgp_status mtgp_server_submit(mtgp_server *s, uint32_t gen, uint32_t dtype, uint64_t n, uint64_t *ticket)
{
    return guarded([&]() -> mtgp_status {
        if (!s || !ticket) return fail(MTGP_EINVAL, "server: NULL argument");
        if (gen >= s->count) return fail(MTGP_EINVAL, "server: generator out of range");
        if (dtype > 2u) return fail(MTGP_EINVAL, "server: unknown dtype");
        if (n == 0) return fail(MTGP_EINVAL, "server: empty request");
        if (4u * n > s->cfg.arena_bytes) return fail(MTGP_EINVAL, "server: request larger than the arena");
        Req r;
        r.gen = gen;
        r.dtype = dtype;
        r.n = n;
        r.bytes = 4u * n;
        r.submit_s = s->now_s();
        const uint64_t t = s->next_ticket++;
        s->reqs[t] = r;
        s->pending.push_back(t);
        *ticket = t;
        return MTGP_OK;
    });
}

}  // extern "C"

namespace {

// Moves finished ticks (oldest first) to the completion queue.  If `wait`,
// blocks on the oldest tick first.
mtgp_status retire(mtgp_server *s, bool wait)
{
    while (!s->inflight.empty()) {
        Tick &t = s->inflight.front();
        cudaError_t e = wait ? cudaEventSynchronize(t.ev) : cudaEventQuery(t.ev);
        if (e == cudaErrorNotReady) break;
        if (e != cudaSuccess) return fail_cuda(e, "server: tick event");
        wait = false;
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, s->ev_ref, t.ev);
        if (e != cudaSuccess) return fail_cuda(e, "server: cudaEventElapsedTime");
        for (uint64_t tk : t.finishing) {
            Req &r = s->reqs[tk];
            r.finished = true;
            r.done_s = ms * 1e-3;
            mtgp_completion c{};
            c.ticket = tk;
            c.gen = r.gen;
            c.dtype = r.dtype;
            c.n = r.n;
            c.dev_out = s->arena + r.off;
            c.submit_s = r.submit_s;
            c.done_s = r.done_s;
            s->done_q.push_back(c);
            s->numbers_done += r.n;
        }
        s->spare_events.push_back(t.ev);
        s->inflight.pop_front();
    }
    return MTGP_OK;
}

// Admits pending requests in submission order: a free slot, no other request
// of the same generator in generation, room in the arena.  A request that
// cannot be admitted holds back the later requests of its generator.
void admit(mtgp_server *s)
{
    if (s->held_mark.size() != s->count) s->held_mark.assign(s->count, 0);
    if (++s->held_stamp == 0) {                   // stamp wrapped: clear the marks once
        std::fill(s->held_mark.begin(), s->held_mark.end(), 0u);
        s->held_stamp = 1;
    }
    const uint32_t stamp = s->held_stamp;
    for (auto it = s->pending.begin(); it != s->pending.end();) {
        if (s->active.size() >= s->cfg.max_active) break;
        Req &r = s->reqs[*it];
        if (s->gen_busy[r.gen] || s->held_mark[r.gen] == stamp || !s->alloc(r.bytes, &r.off)) {
            s->held_mark[r.gen] = stamp;
            ++it;
            continue;
        }
        r.admitted = true;
        s->gen_busy[r.gen] = 1;
        s->active.push_back(*it);
        it = s->pending.erase(it);
    }
}

// Launches one tick: every active request advances by up to cfg.chunk.
mtgp_status launch_tick(mtgp_server *s)
{
    s->tick_reqs.clear();
    Tick t;
    std::vector<uint64_t> still;
    for (uint64_t tk : s->active) {
        Req &r = s->reqs[tk];
        const uint64_t take = std::min<uint64_t>(s->cfg.chunk, r.n - r.done);
        mtgp_request q{r.gen, r.dtype, take, r.off / 4u + r.done};
        s->tick_reqs.push_back(q);
        r.done += take;
        if (r.done == r.n) {
            t.finishing.push_back(tk);
            s->gen_busy[r.gen] = 0;      // later requests of the generator follow in stream order
        } else {
            still.push_back(tk);
        }
    }
    mtgp_status st = mtgp_graph_set_requests(s->graph, s->tick_reqs.data(), (uint32_t)s->tick_reqs.size(),
                                             s->arena, MTGP_LAYOUT_BLOCKED, s->stream);
    if (st != MTGP_OK) return st;
    st = mtgp_graph_launch(s->graph, s->stream);
    if (st != MTGP_OK) return st;
    if (s->spare_events.empty()) {
        cudaEvent_t ev;
        cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return fail_cuda(e, "server: cudaEventCreate");
        s->spare_events.push_back(ev);
    }
    t.ev = s->spare_events.back();
    s->spare_events.pop_back();
    cudaError_t e = cudaEventRecord(t.ev, s->stream);
    if (e != cudaSuccess) return fail_cuda(e, "server: cudaEventRecord");
    s->inflight.push_back(t);
    s->active.swap(still);
    ++s->ticks;
    return MTGP_OK;
}

}  // namespace

extern "C" {

mtgp_status mtgp_server_poll(mtgp_server *s, mtgp_completion *done, uint32_t max, uint32_t *ndone, int block)
{
    return guarded([&]() -> mtgp_status {
        if (!s || !ndone || (max && !done)) return fail(MTGP_EINVAL, "server: NULL argument");
        *ndone = 0;
        mtgp_status st = retire(s, false);
        if (st != MTGP_OK) return st;
        admit(s);
        bool launched = false;
        if (!s->active.empty() && s->inflight.size() < s->cfg.max_inflight) {
            st = launch_tick(s);
            if (st != MTGP_OK) return st;
            launched = true;
        }
        if (block && !launched && s->done_q.empty() && !s->inflight.empty()) {
            st = retire(s, true);
            if (st != MTGP_OK) return st;
            admit(s);
        }
        while (*ndone < max && !s->done_q.empty()) {
            done[(*ndone)++] = s->done_q.front();
            s->done_q.pop_front();
        }
        return MTGP_OK;
    });
}

mtgp_status mtgp_server_release(mtgp_server *s, uint64_t ticket)
{
    return guarded([&]() -> mtgp_status {
        if (!s) return fail(MTGP_EINVAL, "server: NULL server");
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return fail(MTGP_EINVAL, "server: unknown ticket");
        if (!it->second.finished) return fail(MTGP_EBUSY, "server: request not completed yet");
        s->release_range(it->second.off, it->second.bytes);
        s->reqs.erase(it);
        return MTGP_OK;
    });
}

mtgp_status mtgp_server_stats(const mtgp_server *s, mtgp_server_stats_t *out)
{
    if (!s || !out) return fail(MTGP_EINVAL, "server: NULL argument");
    out->pending = (uint32_t)s->pending.size();
    out->active = (uint32_t)s->active.size();
    out->inflight_ticks = (uint32_t)s->inflight.size();
    out->ticks = s->ticks;
    out->numbers_completed = s->numbers_done;
    uint64_t free_bytes = 0;
    for (const auto &kv : s->free_list) free_bytes += kv.second;
    out->arena_free_bytes = free_bytes;
    out->now_s = s->now_s();
    return MTGP_OK;
}

void mtgp_server_destroy(mtgp_server *s)
{
    if (!s) return;
    for (Tick &t : s->inflight) {
        cudaEventSynchronize(t.ev);
        cudaEventDestroy(t.ev);
    }
    for (cudaEvent_t ev : s->spare_events) cudaEventDestroy(ev);
    if (s->ev_ref) cudaEventDestroy(s->ev_ref);
    mtgp_graph_destroy(s->graph);
    cudaFree(s->arena);
    delete s;
    (void)cudaGetLastError();      // the statuses above are ignored: leave none behind
}

}  // extern "C"

extern "C" mtgp_status mtgp_server_run_trace(mtgp_server *s, const double *arrival_s, const uint32_t *gens,
                                             const uint32_t *dtypes, const uint64_t *ns, uint32_t count,
                                             double *latency_s, double *done_s)
{
    return guarded([&]() -> mtgp_status {
        if (!s || (count && (!arrival_s || !gens || !dtypes || !ns || !latency_s))) return fail(MTGP_EINVAL, "trace: NULL argument");
        std::unordered_map<uint64_t, uint32_t> index;     // ticket -> position in the trace
        index.reserve(count * 2u + 1u);
        std::vector<mtgp_completion> buf(1024);
        const double start = s->now_s();
        uint32_t next = 0, finished = 0;
        for (uint32_t i = 0; i < count; ++i)
            if (i && arrival_s[i] < arrival_s[i - 1]) return fail(MTGP_EINVAL, "trace: arrival times must not decrease");
        while (finished < count) {
            const double now = s->now_s() - start;
            while (next < count && arrival_s[next] <= now) {
                uint64_t t = 0;
                mtgp_status st = mtgp_server_submit(s, gens[next], dtypes[next], ns[next], &t);
                if (st != MTGP_OK) return st;
                index[t] = next++;
            }
            uint32_t nd = 0;
            mtgp_status st = mtgp_server_poll(s, buf.data(), (uint32_t)buf.size(), &nd, next == count ? 1 : 0);
            if (st != MTGP_OK) return st;
            for (uint32_t j = 0; j < nd; ++j) {
                const uint32_t i = index[buf[j].ticket];
                latency_s[i] = buf[j].done_s - buf[j].submit_s;
                if (done_s) done_s[i] = buf[j].done_s - start;
                index.erase(buf[j].ticket);
                st = mtgp_server_release(s, buf[j].ticket);
                if (st != MTGP_OK) return st;
                ++finished;
            }
        }
        return MTGP_OK;
    });
}
