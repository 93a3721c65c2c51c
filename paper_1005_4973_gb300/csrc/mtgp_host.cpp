// Host side of libmtgp: parameter sets, device-resident generator pools, work
// lists and launches.  Implements the C ABI declared in include/mtgp.h.
#include "mtgp.h"
#include "mtgp_graph.h"
#include "mtgp_internal.h"
#include "mtgp_jump.h"

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <exception>
#include <new>
#include <string>
#include <vector>

using namespace mtgp;

namespace {

thread_local std::string g_err;

mtgp_status fail(mtgp_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

}  // namespace

namespace mtgp {
int report_error(int status, const char *msg)
{
    g_err = msg;
    return status;
}
}  // namespace mtgp

namespace {

mtgp_status cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation)
        return fail(MTGP_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return fail(MTGP_ECUDA, "%s: %s (%d)", what, cudaGetErrorString(e), (int)e);
}

#define CU(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// ---- SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) -------------------------
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

uint64_t splitmix_next(uint64_t &s)
{
    s += kGamma;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint32_t pow2_floor(uint32_t x)
{
    uint32_t p = 1;
    while (p <= x / 2u) p <<= 1;
    return p;
}

uint32_t pow2_ceil(uint32_t x)
{
    uint32_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Table of a 4x32 matrix: entry b = (4-bit row vector b) x matrix, where the
// leftmost component of b (its bit 3) multiplies row 0 (Sec. 3.6, 3.7, 5).
void rows_to_table(const uint32_t rows[4], uint32_t tbl[16])
{
    for (uint32_t b = 0; b < 16u; ++b) {
        uint32_t v = 0;
        if (b & 8u) v ^= rows[0];
        if (b & 4u) v ^= rows[1];
        if (b & 2u) v ^= rows[2];
        if (b & 1u) v ^= rows[3];
        tbl[b] = v;
    }
}

// v -> (v ^ rec[v]) restricted to the four LSBs is a bijection iff the 4x4
// LSB block of R plus the identity is invertible (Sec. 5).
bool lsb_block_bijective(const uint32_t rec[16])
{
    unsigned seen = 0;
    for (uint32_t v = 0; v < 16u; ++v) seen |= 1u << ((v ^ rec[v]) & 15u);
    return seen == 0xFFFFu;
}

bool table_linear(const uint32_t t[16])
{
    for (uint32_t a = 0; a < 16u; ++a)
        for (uint32_t b = 0; b < 16u; ++b)
            if (t[a ^ b] != (t[a] ^ t[b])) return false;
    return true;
}

void mexp_derive(uint32_t mexp, uint32_t *N, uint32_t *r, uint32_t *mask)
{
    *N = (mexp + 31u) / 32u;
    *r = 32u * *N - mexp;
    *mask = *r >= 32u ? 0u : (0xFFFFFFFFu << *r);
}

// M range: Sec. 5 draws 2 < M < N - [N]_2; Sec. 3.5 (M >= 2, N - M >= [N-2]_2)
// is used for states too small for that range.
void pos_range(uint32_t N, uint32_t *lo, uint32_t *hi)
{
    const uint32_t f = pow2_floor(N);
    if (N >= f + 4u) {
        *lo = 3u;
        *hi = N - f - 1u;
    } else {
        *lo = 2u;
        *hi = N - pow2_floor(N - 2u);
    }
}

struct Slice {        // piece of a request routed to a staging buffer
    uint32_t gen, dtype;
    uint64_t n, host_off;
};

}  // namespace

// --------------------------------------------------------------------------
// objects
// --------------------------------------------------------------------------
struct mtgp_pool {
    uint32_t count = 0;
    uint32_t max_N = 0;
    int device = 0;
    int sm_count = 0;
    std::vector<DevGen> host_gens;         // parameters + offsets (count field stale)
    DevGen *d_gens = nullptr;
    uint32_t *d_state = nullptr;
    uint64_t state_words = 0;
    unsigned *d_ctl = nullptr;             // [0] work counter, [1] error flags
    // work-list upload
    void *h_stage = nullptr;               // pinned
    size_t h_stage_bytes = 0;
    void *d_work = nullptr;
    size_t d_work_bytes = 0;
    cudaEvent_t ev_upload = nullptr;       // upload out of h_stage done
    bool upload_pending = false;
    // in-flight tracking
    cudaEvent_t ev_done = nullptr;
    cudaStream_t last_stream = nullptr;
    bool used = false;
    // end-to-end staging
    void *d_e2e[2] = {nullptr, nullptr};
    size_t e2e_bytes = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_gen[2] = {nullptr, nullptr};
    cudaEvent_t ev_copy[2] = {nullptr, nullptr};
    mtgp_config cfg{};
    uint64_t launches = 0;                 // kernels launched by generation calls
    // jump-ahead (Sec. 7): polynomials, piece start states, walk scratch
    JumpCache jc;
    uint32_t *d_jstate = nullptr;
    uint64_t jstate_words = 0;
    uint32_t *d_seq = nullptr;
    uint64_t seq_words = 0;
    // graphs whose work lists may hold jump jobs, which point at polynomials
    // in jc: emptied before those polynomials are freed
    std::vector<mtgp_graph *> jump_graphs;
    // per-kernel timing (mtgp_pool_set_timing): a ring of timing_n entries of
    // three events (before the jump launch, before and after the generation
    // launch) recorded by the last calls
    std::vector<cudaEvent_t> tev;
    std::vector<uint8_t> tjump;
    uint32_t timing_n = 0, timing_next = 0, timing_count = 0;
    uint32_t spin_limit = 0;               // flow form: polls per bounded wait (0: default)
};

struct mtgp_state {
    mtgp_pool *pool = nullptr;
};

// A captured persistent launch (see mtgp_graph_create).  Device buffer layout:
// [0] work counter, [4] error word, [8] work-item count, [16] output base
// pointer, [24] jump-job count, [256 ..) DevWork[max_items], then
// DevSeg[max_items], then (with pieces) DevJump[max_items].
struct mtgp_graph {
    mtgp_pool *pool = nullptr;
    uint32_t max_items = 0;
    void *d_buf = nullptr;
    size_t d_bytes = 0;
    void *h_stage[2] = {nullptr, nullptr};   // pinned, alternating per upload
    cudaEvent_t ev_stage[2] = {nullptr, nullptr};
    bool stage_used[2] = {false, false};
    int slot = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint32_t B = 0;
    uint32_t form = 0;                       // form of the captured kernel (3: blocked layouts only)
    // jump-ahead pieces (Sec. 7): the capture holds a jump launch over up to
    // max_items jobs before the generation launch, writing the pieces' start
    // states to d_jstate
    bool jump = false;
    uint32_t *d_jstate = nullptr;
    uint64_t jstate_cap = 0;                 // words
    uint32_t j_max_N = 0, j_max_nseq = 0, j_max_ncoef = 0;
};

namespace {

// Empties the work lists of the pool's graphs that may hold jump jobs (their
// replays then generate nothing until the next set_requests): called, after
// the pool's work finished, before cached jump polynomials are freed.
mtgp_status empty_graph_lists(mtgp_pool *p)
{
    for (mtgp_graph *g : p->jump_graphs) {
        CU(cudaMemsetAsync((char *)g->d_buf + 8u, 0, sizeof(uint32_t), nullptr), "empty graph work list");
        CU(cudaMemsetAsync((char *)g->d_buf + 24u, 0, sizeof(uint32_t), nullptr), "empty graph jump list");
    }
    if (!p->jump_graphs.empty()) CU(cudaStreamSynchronize(nullptr), "cudaStreamSynchronize");
    return MTGP_OK;
}

}  // namespace

namespace {

const mtgp_config kDefaultConfig = {128u, 1u, 0u, 256u, 0u, 0u, 0u, 0u, 0u};   // plain, persistent, auto
constexpr size_t kJumpStoreCap = (size_t)1 << 30;   // device bytes of cached jump polynomials
constexpr uint64_t kSeqCap = 256ull << 20;           // walk scratch words per launch

mtgp_status check_config(const mtgp_config &c)
{
    if (c.form > 5u)
        return fail(MTGP_EINVAL, "form must be 0 (plain), 1 (split), 2 (flow), 3 (wide), 4 (pairs) or 5 (dual)");
    if (!threads_supported(c.threads, c.form))
        return fail(MTGP_EINVAL, "no kernel of form %u with %u threads per block", c.form, c.threads);
    if (c.persistent > 1u) return fail(MTGP_EINVAL, "persistent must be 0 or 1");
    if (c.blocks_per_sm > 32u) return fail(MTGP_EINVAL, "blocks_per_sm must be <= 32");
    if (c.chunk < 32u || (c.chunk & (c.chunk - 1u)))
        return fail(MTGP_EINVAL, "chunk must be a power of two >= 32, got %u", c.chunk);
    if (c.buffer_words > 57344u) return fail(MTGP_EINVAL, "buffer_words must be <= 57344 (224 KiB)");
    if (c.pieces > 256u) return fail(MTGP_EINVAL, "pieces must be <= 256");
    if (c.piece_log2 != 0u && (c.piece_log2 < 10u || c.piece_log2 > 40u))
        return fail(MTGP_EINVAL, "piece_log2 must be 0 or in [10, 40]");
    if (c.round_words != 0u && (c.round_words < 8u || (c.round_words & 3u) || c.round_words > 65536u))
        return fail(MTGP_EINVAL, "round_words must be 0 or a multiple of 4 in [8, 65536]");
    return MTGP_OK;
}

// Entry points that allocate host memory (containers) return MTGP_ENOMEM
// instead of letting an exception cross the C ABI.
template <class F>
mtgp_status guarded(F &&f)
{
    try {
        return f();
    } catch (const std::bad_alloc &) {
        return fail(MTGP_ENOMEM, "host allocation failed");
    } catch (const std::exception &e) {
        return fail(MTGP_EINVAL, "%s", e.what());
    }
}

// Waits until the pool's last work finished (for synchronous calls).
mtgp_status pool_sync(mtgp_pool *p)
{
    if (p->used) CU(cudaEventSynchronize(p->ev_done), "cudaEventSynchronize");
    if (p->upload_pending) {
        CU(cudaEventSynchronize(p->ev_upload), "cudaEventSynchronize");
        p->upload_pending = false;
    }
    return MTGP_OK;
}

// A pool call copies its work list out of the pool's pinned staging buffer,
// which the next call overwrites, and records the pool's completion events;
// captured into a caller's CUDA graph, a replay would read whatever the buffer
// then holds.  Calls on a stream under capture are therefore refused:
// mtgp_graph_* is the captured form.
mtgp_status refuse_capture(cudaStream_t s)
{
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CU(cudaStreamIsCapturing(s, &cap), "cudaStreamIsCapturing");
    if (cap != cudaStreamCaptureStatusNone)
        return fail(MTGP_EINVAL, "the stream is being captured into a CUDA graph: pool calls cannot be "
                                 "captured (mtgp_graph_create captures a pool launch)");
    return MTGP_OK;
}

mtgp_status pool_busy_check(mtgp_pool *p, cudaStream_t s)
{
    mtgp_status st = refuse_capture(s);
    if (st != MTGP_OK) return st;
    if (!p->used || s == p->last_stream) return MTGP_OK;
    const cudaError_t e = cudaEventQuery(p->ev_done);
    if (e == cudaErrorNotReady)
        return fail(MTGP_EBUSY, "pool has work in flight on another stream");
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventQuery");
    return MTGP_OK;
}

mtgp_status ensure_upload_space(mtgp_pool *p, size_t bytes)
{
    if (p->upload_pending) {
        CU(cudaEventSynchronize(p->ev_upload), "cudaEventSynchronize");
        p->upload_pending = false;
    }
    if (bytes > p->h_stage_bytes) {
        if (p->h_stage) CU(cudaFreeHost(p->h_stage), "cudaFreeHost");
        p->h_stage = nullptr;
        const size_t nb = std::max(bytes, (size_t)1 << 16);
        CU(cudaHostAlloc(&p->h_stage, nb, cudaHostAllocDefault), "cudaHostAlloc");
        p->h_stage_bytes = nb;
    }
    if (bytes > p->d_work_bytes) {
        if (p->used) CU(cudaEventSynchronize(p->ev_done), "cudaEventSynchronize");
        if (p->d_work) CU(cudaFree(p->d_work), "cudaFree");
        p->d_work = nullptr;
        const size_t nb = std::max(bytes, (size_t)1 << 16);
        CU(cudaMalloc(&p->d_work, nb), "cudaMalloc work list");
        p->d_work_bytes = nb;
    }
    return MTGP_OK;
}

// Builds the work list of a request batch into the pool's upload buffers.
struct Plan {
    std::vector<DevWork> work;
    std::vector<DevSeg> segs;
    std::vector<DevJump> jobs;             // jump-ahead jobs starting the pieces
    uint64_t jstate_words = 0, seq_words = 0;
    uint32_t jmax_N = 0, jmax_nseq = 0, jmax_ncoef = 0;
    uint32_t wmax = 0;
    uint32_t nmax = 0;
    uint64_t total = 0;
};

mtgp_status build_plan(const mtgp_pool *p, const mtgp_request *reqs, uint32_t nreq, mtgp_layout layout,
                       Plan *plan)
{
    if (nreq && !reqs) return fail(MTGP_EINVAL, "reqs is NULL");
    if (layout != MTGP_LAYOUT_BLOCKED && layout != MTGP_LAYOUT_INTERLEAVED)
        return fail(MTGP_EINVAL, "unknown layout %d", (int)layout);
    const mtgp_config &c = p->cfg;
    std::vector<int32_t> slot(p->count, -1);
    std::vector<std::vector<DevSeg>> per;
    std::vector<uint32_t> gens;
    const uint32_t clog = (uint32_t)__builtin_ctz(c.chunk);
    for (uint32_t j = 0; j < nreq; ++j) {
        const mtgp_request &r = reqs[j];
        if (r.gen >= p->count) return fail(MTGP_EINVAL, "request %u: generator %u out of range", j, r.gen);
        if (r.dtype > 2u) return fail(MTGP_EINVAL, "request %u: unknown dtype %u", j, r.dtype);
        if (layout == MTGP_LAYOUT_INTERLEAVED && r.n != reqs[0].n)
            return fail(MTGP_EINVAL, "interleaved layout needs equal n in every request");
        if (r.n == 0) continue;
        DevSeg s{};
        s.n = r.n;
        s.dtype = r.dtype;
        if (layout == MTGP_LAYOUT_BLOCKED) {
            s.out_off = r.out_offset;
            s.stride = 0;
            s.chunk_log2 = kBlocked;
        } else {
            s.out_off = (uint64_t)j * c.chunk;
            s.stride = (uint64_t)nreq * c.chunk;
            s.chunk_log2 = clog;
        }
        if (slot[r.gen] < 0) {
            slot[r.gen] = (int32_t)per.size();
            per.emplace_back();
            gens.push_back(r.gen);
        } else if (layout == MTGP_LAYOUT_INTERLEAVED) {
            return fail(MTGP_EINVAL, "interleaved layout needs distinct generators");
        }
        per[(size_t)slot[r.gen]].push_back(s);
    }
    plan->work.clear();
    plan->segs.clear();
    for (size_t w = 0; w < per.size(); ++w) {
        DevWork dw{};
        dw.gen = gens[w];
        dw.seg_begin = (uint32_t)plan->segs.size();
        dw.seg_count = (uint32_t)per[w].size();
        for (const DevSeg &s : per[w]) {
            dw.total += s.n;
            plan->segs.push_back(s);
        }
        plan->total += dw.total;
        const DevGen &g = p->host_gens[dw.gen];
        plan->nmax = std::max(plan->nmax, g.N);
        plan->work.push_back(dw);
    }
    if (c.persistent)   // longest first, so the tail of the persistent grid is short work
        std::stable_sort(plan->work.begin(), plan->work.end(),
                         [](const DevWork &a, const DevWork &b) { return a.total > b.total; });
    return MTGP_OK;
}

// Kernel shape for a launch running the generators gens[0 .. n): slot count
// qmax and shared buffer words B under configuration c (items = work items
// expected, which sets how many blocks per SM the buffer is sized for).
// Wide form: a round of S words spans at most (S + 6) / 4 + 1 groups of 4
// columns, QW = ceil(groups / threads) per thread.  The buffer is four
// sub-buffers of P words with P = 8 mod 32 (stride-1 copies stay free of bank
// conflicts), at least 2N + S + 24 words in all.
mtgp_status launch_shape_wide(const mtgp_pool *p, const mtgp_config &c, const uint32_t *gens, size_t n,
                              size_t items, uint32_t nmax, uint32_t smax, uint32_t *qmax_out, uint32_t *B_out)
{
    const uint32_t groups = (smax + 6u) / 4u + 1u;
    const uint32_t qmax = kernel_slots(c.threads, 3u, (groups + c.threads - 1u) / c.threads);
    if (!qmax)
        return fail(MTGP_EINVAL, "no compiled wide kernel runs rounds of %u words with %u threads", smax, c.threads);
    uint32_t need = 0;
    for (size_t i = 0; i < n; ++i) {
        const DevGen &g = p->host_gens[gens[i]];
        need = std::max(need, 2u * g.N + (g.N - g.M) + 24u);
    }
    uint32_t B = c.buffer_words;
    if (!B) {
        uint32_t per_sm = c.persistent ? (c.blocks_per_sm ? c.blocks_per_sm : 10u)
                                       : (uint32_t)std::min<size_t>(12, (items + p->sm_count - 1) / (size_t)p->sm_count);
        per_sm = std::max(per_sm, 1u);
        const uint32_t budget = std::min(57344u, (uint32_t)((227u * 1024u / per_sm - 1024u) / 4u));
        B = std::min(2u * nmax + 32u * smax + 32u, budget);
        B = std::max(B, need);
        uint32_t P = B / 4u;
        P = P < 8u ? 8u : ((P - 8u) & ~31u) + 8u;                 // 8 mod 32, not above B / 4
        if (4u * P < need) P += 32u;
        B = 4u * P;
    }
    if (B / 4u * 4u < need)
        return fail(MTGP_EINVAL, "buffer_words %u below the minimum %u for this launch", B, (need + 3u) & ~3u);
    if (B > 57344u) return fail(MTGP_EINVAL, "state too large for shared memory (%u words)", B);
    *qmax_out = qmax;
    *B_out = B;
    return MTGP_OK;
}

mtgp_status launch_shape(const mtgp_pool *p, mtgp_config &c, const uint32_t *gens, size_t n, size_t items,
                         uint32_t *qmax_out, uint32_t *B_out)
{
    uint32_t nmax = 0, smax = 0;
    for (size_t i = 0; i < n; ++i) {
        const DevGen &g = p->host_gens[gens[i]];
        nmax = std::max(nmax, g.N);
        smax = std::max(smax, g.N - g.M);
    }
    // plain form: rounds longer than the configured block size has a kernel
    // for (exponents above 44497) run with the smallest larger block size that
    // has one
    if (c.form == 0u && !kernel_slots(c.threads, 0u, (smax + c.threads - 1u) / c.threads))
        for (uint32_t t : {256u, 512u})
            if (t > c.threads && kernel_slots(t, 0u, (smax + t - 1u) / t)) {
                c.threads = t;
                break;
            }
    if (c.form == 3u) return launch_shape_wide(p, c, gens, n, items, nmax, smax, qmax_out, B_out);
    // columns a slot covers: one per thread (plain, dual), one per thread of
    // the recursion half (split, flow), two per thread (pairs)
    const uint32_t owners = c.form == 4u ? 2u * c.threads : (c.form == 0u || c.form == 5u) ? c.threads : c.threads / 2u;
    const uint32_t qmax = kernel_slots(c.threads, c.form, (smax + owners - 1u) / owners);
    if (!qmax)
        return fail(MTGP_EINVAL, "no compiled kernel runs rounds of %u words with %u threads (form %u)", smax,
                    c.threads, c.form);
    // shared buffer: at least the form's minimum; up to 32 rounds between
    // compactions if the blocks wanted per SM fit
    uint32_t need = 0;
    for (size_t i = 0; i < n; ++i) {
        const DevGen &g = p->host_gens[gens[i]];
        const uint32_t S = g.N - g.M, nq = (S + owners - 1u) / owners;
        if (c.form == 5u && nq != qmax)   // dual: every item runs the compiled slot count
            return fail(MTGP_EINVAL, "form 5 runs rounds of %u .. %u words with %u threads; generator %u has %u",
                        (qmax - 1u) * c.threads + 1u, qmax * c.threads, c.threads, gens[i], S);
        if (c.form == 2u)   // flow: epochs of at least N + S words between compactions
            need = std::max(need, 2u * g.N + 2u * S + 32u * nq + 32u);
        else if (c.form == 5u)   // dual: two halves, each as the plain form's buffer
            need = std::max(need, 2u * (2u * g.N + nq * owners + 32u));
        else                // plain / split: reads of the last column slot stay inside
            need = std::max(need, 2u * g.N + nq * owners + 32u);
    }
    uint32_t B = c.buffer_words;
    if (!B) {
        uint32_t per_sm = c.persistent ? c.blocks_per_sm
                                       : (uint32_t)std::min<size_t>(8, (items + p->sm_count - 1) / (size_t)p->sm_count);
        if (c.persistent && !per_sm) {
            // as many blocks as the kernel's registers and threads allow, with
            // buffers sized for them (measured: C2 +1 %, C3 and C4 level)
            int occ = 0;
            if (generate_occupancy(c.threads, c.form, qmax, need, &occ) != cudaSuccess || occ < 1) occ = 6;
            per_sm = (uint32_t)occ;
        }
        per_sm = std::max(per_sm, 1u);
        const uint32_t budget = std::min(57344u, (uint32_t)((227u * 1024u / per_sm - 1024u) / 4u));
        const uint32_t halves = c.form == 5u ? 2u : 1u;
        B = std::min(halves * (2u * nmax + 32u * smax + 32u), budget);
        B = std::max(B, std::min(need + halves * smax, 57344u));
        B = std::max(B, need);
    }
    if (c.form == 4u && !c.buffer_words) {
        // two halves of H words, H = 16 (mod 32): the copies between the
        // halves stay free of bank conflicts
        uint32_t H = B / 2u;
        H = H < 16u ? 16u : ((H - 16u) & ~31u) + 16u;
        if (2u * H < need) H += 32u;
        B = 2u * H;
    }
    if (c.form == 4u || c.form == 5u) B &= ~1u;               // the kernel uses 2 floor(B / 2) words
    if (B < need) return fail(MTGP_EINVAL, "buffer_words %u below the minimum %u for this launch", B, need);
    if (B > 57344u) return fail(MTGP_EINVAL, "state too large for shared memory (%u words)", B);
    *qmax_out = qmax;
    *B_out = B;
    return MTGP_OK;
}

// Grows the piece-state and walk scratch buffers (waiting for queued work
// that may still read the old ones).
mtgp_status ensure_jump_space(mtgp_pool *p, uint64_t jstate_words, uint64_t seq_words)
{
    if (jstate_words <= p->jstate_words && seq_words <= p->seq_words) return MTGP_OK;
    if (p->used) CU(cudaEventSynchronize(p->ev_done), "cudaEventSynchronize");
    if (jstate_words > p->jstate_words) {
        if (p->d_jstate) CU(cudaFree(p->d_jstate), "cudaFree");
        p->d_jstate = nullptr;
        p->jstate_words = 0;
        CU(cudaMalloc(&p->d_jstate, 4u * jstate_words), "cudaMalloc piece states");
        p->jstate_words = jstate_words;
    }
    if (seq_words > p->seq_words) {
        if (p->d_seq) CU(cudaFree(p->d_seq), "cudaFree");
        p->d_seq = nullptr;
        p->seq_words = 0;
        const uint64_t w = std::max<uint64_t>(seq_words, seq_words + seq_words / 4u);
        CU(cudaMalloc(&p->d_seq, 4u * w), "cudaMalloc walk scratch");
        p->seq_words = w;
    }
    return MTGP_OK;
}

// Splits long blocked work items into pieces that run on separate blocks
// (Sec. 7): piece m of an item of length n starts m L numbers into the
// generator's stream, from the state F^(m L) s that the jump kernels compute
// before the launch; the last piece writes the generator's state back.  The
// pieces' outputs are exactly the item's, in the same places.
mtgp_status split_plan(mtgp_pool *p, Plan *plan, cudaStream_t s)
{
    const mtgp_config &c = p->cfg;
    if (c.pieces == 1u || plan->work.empty()) return MTGP_OK;
    const uint64_t min_piece = 1ull << (c.piece_log2 ? c.piece_log2 : 20u);
    // auto: pieces of about Lt = total / (16 SMs) numbers, so that the launch
    // has about 16 equal shares of work per SM and long items stop setting its
    // tail; explicit: up to `pieces` per item
    const uint64_t kt = c.pieces ? c.pieces : 64u;
    const uint64_t Lt = c.pieces ? 0u : (plan->total + 16ull * (uint64_t)std::max(p->sm_count, 1) - 1u) /
                                           (16ull * (uint64_t)std::max(p->sm_count, 1));
    if (kt < 2u) return MTGP_OK;
    const uint64_t sms = (uint64_t)std::max(p->sm_count, 1);
    const bool few = plan->work.size() < sms;
    // auto, fewer items than SMs: at most 1 + 2 SMs / items pieces per item, so
    // that the jumps run in one wave (two jump blocks fit on an SM)
    const uint64_t kfew = 1u + 2u * sms / (uint64_t)plan->work.size();
    struct Cut {
        uint32_t k;
        uint64_t L;
    };
    std::vector<Cut> cut(plan->work.size(), Cut{0u, 0u});
    std::vector<uint32_t> gl;
    std::vector<std::pair<uint32_t, uint64_t>> need;
    uint64_t seq_est = 0;
    for (size_t w = 0; w < plan->work.size(); ++w) {
        const DevWork &dw = plan->work[w];
        const DevGen &g = p->host_gens[dw.gen];
        // auto: a piece at least mexp N / 4 numbers long, so that its jump
        // (about 0.7 mexp N word operations) stays a few per cent of its work;
        // when the work items do not fill the SMs, also pieces down to 2^14
        // numbers, at most kfew per item (jumps then run on SMs that would
        // otherwise idle, and a launch's time is one jump plus one piece) --
        // whichever rule gives more pieces (long items in a launch of few
        // items, 2^26 numbers of MTGP23209 each: 15 pieces, not 3)
        const uint64_t lmin = c.piece_log2 ? min_piece : std::max<uint64_t>(min_piece, (uint64_t)g.mexp * g.N / 4u);
        const uint64_t lfew = c.piece_log2 ? min_piece : (uint64_t)1u << 14;
        const bool few_rule = !c.pieces && few;
        if (dw.total < 2u * (few_rule ? std::min(lmin, lfew) : lmin)) continue;
        bool blocked = true;
        for (uint32_t q = 0; q < dw.seg_count; ++q)
            blocked = blocked && plan->segs[dw.seg_begin + q].chunk_log2 == kBlocked;
        if (!blocked) continue;
        const uint64_t kLt = Lt ? (dw.total + Lt - 1u) / Lt : ~0ull;
        uint64_t k = std::min<uint64_t>({kt, dw.total / lmin, kLt});
        if (few_rule) {
            const uint64_t kf = std::min<uint64_t>({kt, dw.total / lfew, kLt, kfew});
            k = c.piece_log2 ? std::min(k, kfew) : std::max(k, kf);
        }
        if (k < 2u) continue;
        uint64_t L = (dw.total + k - 1u) / k;
        L = (L + 63u) & ~63ull;
        k = (dw.total + L - 1u) / L;
        if (k < 2u) continue;
        const uint64_t walk = (k - 1u) * (uint64_t)jump_seq_words(g.N, g.mexp + 1u) + jump_seq_words(g.N, 0u);
        if (seq_est + walk > kSeqCap) continue;
        seq_est += walk;
        cut[w] = Cut{(uint32_t)k, L};
        gl.push_back(dw.gen);
        for (uint64_t m = 1; m < k; ++m) need.emplace_back(dw.gen, m * L);
    }
    if (gl.empty()) return MTGP_OK;
    int st = jump_annihilate(p->jc, p->host_gens.data(), p->d_gens, p->d_state, gl.data(), gl.size(), s);
    if (st != MTGP_OK) return (mtgp_status)st;
    if (p->jc.dev_bytes > kJumpStoreCap) {
        mtgp_status r = pool_sync(p);
        if (r == MTGP_OK) r = empty_graph_lists(p);
        if (r != MTGP_OK) return r;
        jump_clear(p->jc, false);
    }
    st = jump_polys(p->jc, need);
    if (st != MTGP_OK) return (mtgp_status)st;
    std::vector<DevWork> work;
    std::vector<DevSeg> segs;
    uint64_t jst = 0, seq = 0;
    for (size_t w = 0; w < plan->work.size(); ++w) {
        const DevWork &dw = plan->work[w];
        if (!cut[w].k) {
            DevWork o = dw;
            o.seg_begin = (uint32_t)segs.size();
            segs.insert(segs.end(), plan->segs.begin() + dw.seg_begin,
                        plan->segs.begin() + dw.seg_begin + dw.seg_count);
            work.push_back(o);
            continue;
        }
        const DevGen &g = p->host_gens[dw.gen];
        const uint64_t L = cut[w].L;
        for (uint32_t m = 0; m < cut[w].k; ++m) {
            const uint64_t a = (uint64_t)m * L, b = std::min(a + L, dw.total);
            DevWork pw{};
            pw.gen = dw.gen;
            pw.seg_begin = (uint32_t)segs.size();
            pw.flags = kItemPiece | (m + 1u == cut[w].k ? kItemLast : 0u);
            pw.total = b - a;
            pw.src = jst;
            uint64_t c0 = 0;
            for (uint32_t q = 0; q < dw.seg_count; ++q) {
                const DevSeg &sg = plan->segs[dw.seg_begin + q];
                const uint64_t lo = std::max(a, c0), hi = std::min(b, c0 + sg.n);
                if (lo < hi) {
                    DevSeg o = sg;
                    o.n = hi - lo;
                    o.out_off = sg.out_off + (lo - c0);
                    segs.push_back(o);
                }
                c0 += sg.n;
            }
            pw.seg_count = (uint32_t)(segs.size() - pw.seg_begin);
            work.push_back(pw);
            DevJump jb{};
            if (m && !p->jc.polys.count({dw.gen, a})) return fail(MTGP_EINVAL, "jump polynomial missing");
            const JumpPoly jp = m ? jump_poly(p->jc, dw.gen, a) : JumpPoly{};
            jb.poly = jp.d;
            jb.ncoef = jp.ncoef;
            jb.src = g.state_off;
            jb.dst = jst;
            jb.seq = seq;
            jb.gen = dw.gen;
            jb.nseq = jump_seq_words(g.N, jb.ncoef);
            jb.mode = kJumpStep;
            plan->jobs.push_back(jb);
            plan->jmax_N = std::max(plan->jmax_N, g.N);
            plan->jmax_nseq = std::max(plan->jmax_nseq, jb.nseq);
            plan->jmax_ncoef = std::max(plan->jmax_ncoef, jb.ncoef);
            jst += (g.N + 3u) & ~3u;
            seq += jb.nseq;
        }
    }
    plan->work.swap(work);
    plan->segs.swap(segs);
    plan->jstate_words = jst;
    plan->seq_words = seq;
    if (c.persistent)
        std::stable_sort(plan->work.begin(), plan->work.end(),
                         [](const DevWork &x, const DevWork &y) { return x.total > y.total; });
    return MTGP_OK;
}

mtgp_status launch_plan(mtgp_pool *p, const Plan &plan, void *dev_out, cudaStream_t s)
{
    if (plan.work.empty()) return MTGP_OK;
    mtgp_config c = p->cfg;
    if (c.form == 3u)   // the wide form writes blocked segments only: interleaved launches run plain
        for (const DevSeg &sg : plan.segs)
            if (sg.chunk_log2 != kBlocked) {
                c.form = 0u;
                c.threads = 128u;
                break;
            }
    std::vector<uint32_t> gens(plan.work.size());
    for (size_t i = 0; i < plan.work.size(); ++i) gens[i] = plan.work[i].gen;
    uint32_t qmax = 0, B = 0;
    mtgp_status st0 = launch_shape(p, c, gens.data(), gens.size(), plan.work.size(), &qmax, &B);
    if (st0 != MTGP_OK) return st0;
    // upload
    const size_t wbytes = plan.work.size() * sizeof(DevWork);
    const size_t sbytes = plan.segs.size() * sizeof(DevSeg);
    const size_t jbytes = plan.jobs.size() * sizeof(DevJump);
    mtgp_status st = ensure_upload_space(p, wbytes + sbytes + jbytes);
    if (st != MTGP_OK) return st;
    const bool fused = jump_fused_fits(plan.jmax_N, plan.jmax_nseq, plan.jmax_ncoef);
    if (!plan.jobs.empty()) {
        st = ensure_jump_space(p, plan.jstate_words, fused ? 0u : plan.seq_words);
        if (st != MTGP_OK) return st;
    }
    std::memcpy(p->h_stage, plan.work.data(), wbytes);
    std::memcpy((char *)p->h_stage + wbytes, plan.segs.data(), sbytes);
    std::memcpy((char *)p->h_stage + wbytes + sbytes, plan.jobs.data(), jbytes);
    CU(cudaMemcpyAsync(p->d_work, p->h_stage, wbytes + sbytes + jbytes, cudaMemcpyHostToDevice, s),
       "upload work list");
    CU(cudaEventRecord(p->ev_upload, s), "cudaEventRecord");
    p->upload_pending = true;
    cudaEvent_t *tev = nullptr;                       // this call's timing entry
    if (p->timing_n) {
        tev = &p->tev[3u * p->timing_next];
        p->tjump[p->timing_next] = plan.jobs.empty() ? 0u : 1u;
        p->timing_next = (p->timing_next + 1u) % p->timing_n;
        p->timing_count = std::min(p->timing_count + 1u, p->timing_n);
        CU(cudaEventRecord(tev[0], s), "cudaEventRecord");
    }
    if (!plan.jobs.empty()) {   // start states of the pieces (Sec. 7)
        const DevJump *jobs = (const DevJump *)((char *)p->d_work + wbytes + sbytes);
        const uint32_t nj = (uint32_t)plan.jobs.size();
        if (fused) {
            CU(launch_jump_fused(p->d_gens, p->d_state, p->d_jstate, jobs, nj, plan.jmax_N, plan.jmax_nseq,
                                 plan.jmax_ncoef, s),
               "jump kernel launch");
            p->launches += 1u;
        } else {
            CU(launch_walk(p->d_gens, p->d_state, p->d_seq, jobs, nj, plan.jmax_N, s), "walk kernel launch");
            CU(launch_jump_sum(p->d_gens, p->d_seq, p->d_jstate, jobs, nj, plan.jmax_N, s), "jump kernel launch");
            p->launches += 2u;
        }
    }
    uint32_t grid = (uint32_t)plan.work.size();
    // fewer work items than SMs: each block's round latency is the time, so
    // the kernel with interleaved round tails (where compiled)
    const bool interleave = plan.work.size() < (size_t)std::max(p->sm_count, 1);
    bool persistent = c.persistent != 0u || c.form == 5u;   // the dual form always pulls items
    if (persistent) {
        int occ = 0;
        CU(generate_occupancy(c.threads, c.form, qmax, B, &occ, interleave), "occupancy");
        if (occ < 1) return fail(MTGP_EINVAL, "configuration does not fit on an SM");
        const int per_sm = c.blocks_per_sm ? std::min<int>((int)c.blocks_per_sm, occ) : occ;
        // every item resident at once: one block per item, no work counter
        if (!c.blocks_per_sm && c.form != 5u && plan.work.size() <= (size_t)per_sm * (size_t)p->sm_count)
            persistent = false;
        else {
            CU(cudaMemsetAsync(p->d_ctl, 0, sizeof(unsigned), s), "reset work counter");
            if (c.form == 5u) grid = (grid + 1u) / 2u;      // two items per block
            grid = std::min<uint32_t>(grid, (uint32_t)(per_sm * p->sm_count));
        }
    }
    LaunchArgs a{};
    a.gens = p->d_gens;
    a.state = p->d_state;
    a.work = (const DevWork *)p->d_work;
    a.segs = (const DevSeg *)((char *)p->d_work + wbytes);
    a.out = (uint32_t *)dev_out;
    a.counter = p->d_ctl;
    a.err = p->d_ctl + 1;
    a.nwork = (uint32_t)plan.work.size();
    a.buf_words = B;
    a.persistent = persistent ? 1u : 0u;
    a.jstate = p->d_jstate;
    a.interleave = interleave ? 1u : 0u;
    a.spin_limit = p->spin_limit;
    a.round_words = c.round_words;
    if (tev) CU(cudaEventRecord(tev[1], s), "cudaEventRecord");
    CU(launch_generate(a, c.threads, c.form, qmax, grid, s), "generate kernel launch");
    if (tev) CU(cudaEventRecord(tev[2], s), "cudaEventRecord");
    p->launches += 1u;
    CU(cudaEventRecord(p->ev_done, s), "cudaEventRecord");
    p->last_stream = s;
    p->used = true;
    return MTGP_OK;
}

mtgp_status pool_run(mtgp_pool *p, const mtgp_request *reqs, uint32_t nreq, void *dev_out,
                     mtgp_layout layout, cudaStream_t s)
{
    mtgp_status st = pool_busy_check(p, s);
    if (st != MTGP_OK) return st;
    Plan plan;
    st = build_plan(p, reqs, nreq, layout, &plan);
    if (st != MTGP_OK) return st;
    if (plan.total && !dev_out) return fail(MTGP_EINVAL, "dev_out is NULL");
    if (((uintptr_t)dev_out & 3u) != 0) return fail(MTGP_EINVAL, "dev_out must be 4-byte aligned");
    st = split_plan(p, &plan, s);
    if (st != MTGP_OK) return st;
    return launch_plan(p, plan, dev_out, s);
}

}  // namespace

// --------------------------------------------------------------------------
// C ABI
// --------------------------------------------------------------------------
extern "C" {

const char *mtgp_version(void) { return "libmtgp 0.1 (sm_103a)"; }

const char *mtgp_last_error(void) { return g_err.c_str(); }

mtgp_status mtgp_params_draw(uint32_t mexp, uint64_t param_seed, uint32_t id, mtgp_params *out)
{
    if (!out) return fail(MTGP_EINVAL, "out is NULL");
    if (mexp < 65u) return fail(MTGP_EINVAL, "mexp %u too small (N must be >= 3)", mexp);
    mtgp_params p{};
    mexp_derive(mexp, &p.N, &p.r, &p.mask);
    if (p.N > MTGP_MAX_N) return fail(MTGP_EINVAL, "mexp %u gives N = %u > %u", mexp, p.N, MTGP_MAX_N);
    uint32_t lo, hi;
    pos_range(p.N, &lo, &hi);
    uint64_t s = param_seed;
    p.mexp = mexp;
    p.id = id;
    p.pos = lo + (uint32_t)(splitmix_next(s) % (uint64_t)(hi - lo + 1u));
    uint32_t R[4], T[4];
    for (uint32_t &row : R) row = (uint32_t)splitmix_next(s);
    R[0] = (R[0] & 0x0000FFFFu) | (id & 0xFFFF0000u);               // ID[31:16]
    R[1] = (R[1] & ~0x000FFFF0u) | ((id & 0x0000FFFFu) << 4);        // ID[15:0]
    for (;;) {
        rows_to_table(R, p.rec_tbl);
        if (lsb_block_bijective(p.rec_tbl)) break;
        for (uint32_t &row : R) row = (row & ~0xFu) | ((uint32_t)splitmix_next(s) & 0xFu);
    }
    for (uint32_t &row : T) row = (uint32_t)splitmix_next(s);
    rows_to_table(T, p.tmp_tbl);
    p.sh1 = 13u;
    p.sh2 = 4u;
    *out = p;
    return MTGP_OK;
}

mtgp_status mtgp_params_validate(const mtgp_params *p)
{
    if (!p) return fail(MTGP_EINVAL, "params is NULL");
    if (p->mexp < 65u) return fail(MTGP_EINVAL, "mexp %u too small", p->mexp);
    uint32_t N, r, mask;
    mexp_derive(p->mexp, &N, &r, &mask);
    if (p->N != N || p->r != r || p->mask != mask)
        return fail(MTGP_EINVAL, "N/r/mask (%u/%u/%08x) inconsistent with mexp %u", p->N, p->r, p->mask, p->mexp);
    if (N > MTGP_MAX_N) return fail(MTGP_EINVAL, "N = %u exceeds %u", N, MTGP_MAX_N);
    if (p->pos < 2u || p->pos >= N) return fail(MTGP_EINVAL, "pos %u outside [2, N)", p->pos);
    if (p->sh1 < 1u || p->sh1 > 31u || p->sh2 < 1u || p->sh2 > 31u)
        return fail(MTGP_EINVAL, "shifts must be in [1, 31]");
    if (!table_linear(p->rec_tbl) || !table_linear(p->tmp_tbl))
        return fail(MTGP_EINVAL, "look-up tables are not F2-linear");
    if (!lsb_block_bijective(p->rec_tbl))
        return fail(MTGP_EINVAL, "LSB block of R plus identity is singular");
    return MTGP_OK;
}

mtgp_status mtgp_pool_create(const mtgp_params *ps, const uint32_t *gen_ids, const uint64_t *seeds,
                             uint32_t count, void *stream, mtgp_pool **out)
{
    return guarded([&]() -> mtgp_status {
        if (!out) return fail(MTGP_EINVAL, "out is NULL");
        *out = nullptr;
        if (!ps || !gen_ids || !seeds || count == 0) return fail(MTGP_EINVAL, "empty or NULL pool arguments");
        for (uint32_t i = 0; i < count; ++i) {
            mtgp_status st = mtgp_params_validate(&ps[i]);
            if (st != MTGP_OK) {
                std::string m = g_err;
                return fail(st, "parameter set %u: %s", i, m.c_str());
            }
        }
        cudaStream_t s = (cudaStream_t)stream;
        mtgp_status cs = refuse_capture(s);
        if (cs != MTGP_OK) return cs;
        mtgp_pool *p = new (std::nothrow) mtgp_pool;
        if (!p) return fail(MTGP_ENOMEM, "host allocation");
        p->count = count;
        p->cfg = kDefaultConfig;
        try {
            p->host_gens.resize(count);
            p->jc.ann.resize(count);
        } catch (const std::exception &) {
            delete p;
            return fail(MTGP_ENOMEM, "host allocation");
        }
        uint64_t off = 0;
        for (uint32_t i = 0; i < count; ++i) {
            DevGen &g = p->host_gens[i];
            std::memset(&g, 0, sizeof g);
            g.N = ps[i].N;
            g.M = ps[i].pos;
            g.mask = ps[i].mask;
            g.sh1 = ps[i].sh1;
            g.sh2 = ps[i].sh2;
            g.mexp = ps[i].mexp;
            g.id = ps[i].id;
            g.state_off = off;
            std::memcpy(g.rec, ps[i].rec_tbl, sizeof g.rec);
            std::memcpy(g.tmp, ps[i].tmp_tbl, sizeof g.tmp);
            off += (g.N + 3u) & ~3u;                   // 16-byte aligned states
            p->max_N = std::max(p->max_N, g.N);
        }
        p->state_words = off;
        auto cleanup = [&](mtgp_status st) { mtgp_pool_destroy(p); return st; };
        cudaError_t e;
    #define CUP(call, what)                                           \
        do {                                                          \
            e = (call);                                               \
            if (e != cudaSuccess) return cleanup(cuda_fail(e, what)); \
        } while (0)
        CUP(cudaGetDevice(&p->device), "cudaGetDevice");
        CUP(cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device), "SM count");
        CUP(cudaEventCreateWithFlags(&p->ev_done, cudaEventDisableTiming), "cudaEventCreate");
        CUP(cudaEventCreateWithFlags(&p->ev_upload, cudaEventDisableTiming), "cudaEventCreate");
        CUP(cudaMalloc(&p->d_gens, sizeof(DevGen) * count), "cudaMalloc generators");
        CUP(cudaMalloc(&p->d_state, sizeof(uint32_t) * off), "cudaMalloc states");
        CUP(cudaMalloc(&p->d_ctl, 4 * sizeof(unsigned)), "cudaMalloc control");
        CUP(cudaMemsetAsync(p->d_ctl, 0, 4 * sizeof(unsigned), s), "cudaMemsetAsync");
        // upload parameters and seeding inputs through one pinned staging buffer
        const size_t gbytes = sizeof(DevGen) * count, ibytes = sizeof(uint32_t) * count,
                     sbytes = sizeof(uint64_t) * count;
        const size_t ioff = gbytes, soff = (gbytes + ibytes + 15u) & ~(size_t)15u;
        mtgp_status st = ensure_upload_space(p, soff + sbytes);
        if (st != MTGP_OK) return cleanup(st);
        std::memcpy(p->h_stage, p->host_gens.data(), gbytes);
        std::memcpy((char *)p->h_stage + ioff, gen_ids, ibytes);
        std::memcpy((char *)p->h_stage + soff, seeds, sbytes);
        CUP(cudaMemcpyAsync(p->d_gens, p->h_stage, gbytes, cudaMemcpyHostToDevice, s), "upload generators");
        CUP(cudaMemcpyAsync(p->d_work, (char *)p->h_stage + ioff, soff + sbytes - ioff, cudaMemcpyHostToDevice, s),
            "upload seeds");
        CUP(launch_seed(p->d_gens, p->d_state, (const uint32_t *)p->d_work,
                        (const uint64_t *)((char *)p->d_work + (soff - ioff)), 0, count, s),
            "seed kernel launch");
        CUP(cudaEventRecord(p->ev_upload, s), "cudaEventRecord");
        p->upload_pending = true;
        CUP(cudaEventRecord(p->ev_done, s), "cudaEventRecord");
        p->last_stream = s;
        p->used = true;
    #undef CUP
        *out = p;
        return MTGP_OK;
    });
}

mtgp_status mtgp_pool_info(const mtgp_pool *p, uint32_t *count, uint64_t *device_bytes)
{
    if (!p) return fail(MTGP_EINVAL, "pool is NULL");
    if (count) *count = p->count;
    if (device_bytes)
        *device_bytes = sizeof(DevGen) * (uint64_t)p->count + 4ull * p->state_words + p->d_work_bytes +
                        2ull * p->e2e_bytes + p->jc.dev_bytes + 4ull * (p->jstate_words + p->seq_words);
    return MTGP_OK;
}

mtgp_status mtgp_pool_get_config(const mtgp_pool *p, mtgp_config *cfg)
{
    if (!p || !cfg) return fail(MTGP_EINVAL, "NULL argument");
    *cfg = p->cfg;
    return MTGP_OK;
}

mtgp_status mtgp_pool_set_config(mtgp_pool *p, const mtgp_config *cfg)
{
    if (!p || !cfg) return fail(MTGP_EINVAL, "NULL argument");
    mtgp_status st = check_config(*cfg);
    if (st != MTGP_OK) return st;
    p->cfg = *cfg;
    return MTGP_OK;
}

mtgp_status mtgp_pool_generate(mtgp_pool *p, const mtgp_request *reqs, uint32_t nreq, void *dev_out,
                               mtgp_layout layout, void *stream)
{
    return guarded([&]() -> mtgp_status {
        if (!p) return fail(MTGP_EINVAL, "pool is NULL");
        return pool_run(p, reqs, nreq, dev_out, layout, (cudaStream_t)stream);
    });
}

mtgp_status mtgp_pool_generate_host(mtgp_pool *p, const mtgp_request *reqs, uint32_t nreq, void *host_out,
                                    mtgp_layout layout, uint64_t staging_bytes, void *stream)
{
    return guarded([&]() -> mtgp_status {
        if (!p) return fail(MTGP_EINVAL, "pool is NULL");
        if (layout != MTGP_LAYOUT_BLOCKED) return fail(MTGP_EINVAL, "host output supports the blocked layout only");
        if (nreq && !reqs) return fail(MTGP_EINVAL, "reqs is NULL");
        cudaStream_t s = (cudaStream_t)stream;
        mtgp_status st = pool_busy_check(p, s);
        if (st != MTGP_OK) return st;
        uint64_t total = 0;
        for (uint32_t j = 0; j < nreq; ++j) {
            if (reqs[j].gen >= p->count || reqs[j].dtype > 2u) return fail(MTGP_EINVAL, "request %u invalid", j);
            total += reqs[j].n;
        }
        if (!total) return MTGP_OK;
        if (!host_out) return fail(MTGP_EINVAL, "host_out is NULL");
        if (!staging_bytes) staging_bytes = 1ull << 30;
        staging_bytes &= ~15ull;
        if (staging_bytes < 4096u) return fail(MTGP_EINVAL, "staging_bytes too small");
        if (staging_bytes > p->e2e_bytes) {
            st = pool_sync(p);
            if (st != MTGP_OK) return st;
            for (int b = 0; b < 2; ++b) {
                if (p->d_e2e[b]) CU(cudaFree(p->d_e2e[b]), "cudaFree");
                p->d_e2e[b] = nullptr;
            }
            p->e2e_bytes = 0;
            for (int b = 0; b < 2; ++b) CU(cudaMalloc(&p->d_e2e[b], staging_bytes), "cudaMalloc staging");
            p->e2e_bytes = staging_bytes;
        }
        if (!p->copy_stream) {
            CU(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking), "cudaStreamCreate");
            for (int b = 0; b < 2; ++b) {
                CU(cudaEventCreateWithFlags(&p->ev_gen[b], cudaEventDisableTiming), "cudaEventCreate");
                CU(cudaEventCreateWithFlags(&p->ev_copy[b], cudaEventDisableTiming), "cudaEventCreate");
                CU(cudaEventRecord(p->ev_copy[b], p->copy_stream), "cudaEventRecord");
            }
        }
        const uint64_t cap = p->e2e_bytes / 4u;
        std::vector<Slice> slices;
        std::vector<mtgp_request> batch;
        int buf = 0;
        auto flush = [&]() -> mtgp_status {
            if (slices.empty()) return MTGP_OK;
            CU(cudaStreamWaitEvent(s, p->ev_copy[buf], 0), "cudaStreamWaitEvent");
            batch.clear();
            uint64_t off = 0;
            for (const Slice &sl : slices) {
                batch.push_back(mtgp_request{sl.gen, sl.dtype, sl.n, off});
                off += sl.n;
            }
            mtgp_status r = pool_run(p, batch.data(), (uint32_t)batch.size(), p->d_e2e[buf], MTGP_LAYOUT_BLOCKED, s);
            if (r != MTGP_OK) return r;
            CU(cudaEventRecord(p->ev_gen[buf], s), "cudaEventRecord");
            CU(cudaStreamWaitEvent(p->copy_stream, p->ev_gen[buf], 0), "cudaStreamWaitEvent");
            off = 0;
            for (const Slice &sl : slices) {
                CU(cudaMemcpyAsync((char *)host_out + 4u * sl.host_off, (char *)p->d_e2e[buf] + 4u * off, 4u * sl.n,
                                   cudaMemcpyDeviceToHost, p->copy_stream),
                   "copy to host");
                off += sl.n;
            }
            CU(cudaEventRecord(p->ev_copy[buf], p->copy_stream), "cudaEventRecord");
            slices.clear();
            buf ^= 1;
            return MTGP_OK;
        };
        uint64_t used = 0;
        for (uint32_t j = 0; j < nreq; ++j) {
            uint64_t left = reqs[j].n, host_off = reqs[j].out_offset;
            while (left) {
                if (used == cap) {
                    st = flush();
                    if (st != MTGP_OK) return st;
                    used = 0;
                }
                const uint64_t take = std::min(left, cap - used);
                slices.push_back(Slice{reqs[j].gen, reqs[j].dtype, take, host_off});
                used += take;
                left -= take;
                host_off += take;
            }
        }
        st = flush();
        if (st != MTGP_OK) return st;
        CU(cudaStreamSynchronize(p->copy_stream), "cudaStreamSynchronize");
        return MTGP_OK;
    });
}

mtgp_status mtgp_pool_position(mtgp_pool *p, uint32_t i, uint64_t *pos)
{
    if (!p || !pos || i >= p->count) return fail(MTGP_EINVAL, "bad pool, index or NULL pos");
    mtgp_status st = pool_sync(p);
    if (st != MTGP_OK) return st;
    CU(cudaMemcpy(pos, (const char *)p->d_gens + sizeof(DevGen) * i + offsetof(DevGen, count), sizeof(uint64_t),
                  cudaMemcpyDeviceToHost),
       "read position");
    return MTGP_OK;
}

mtgp_status mtgp_pool_read_state(mtgp_pool *p, uint32_t i, uint32_t *host_state)
{
    if (!p || !host_state || i >= p->count) return fail(MTGP_EINVAL, "bad pool, index or NULL buffer");
    mtgp_status st = pool_sync(p);
    if (st != MTGP_OK) return st;
    const DevGen &g = p->host_gens[i];
    CU(cudaMemcpy(host_state, p->d_state + g.state_off, 4u * g.N, cudaMemcpyDeviceToHost), "read state");
    return MTGP_OK;
}

// Checkpoint format: "MTGP" magic, version, count, state_words, then the
// DevGen records, then the state buffer.
mtgp_status mtgp_pool_save(mtgp_pool *p, void *host_buf, size_t *bytes)
{
    if (!p || !bytes) return fail(MTGP_EINVAL, "NULL argument");
    const size_t need = 16u + sizeof(DevGen) * p->count + 4u * p->state_words;
    if (!host_buf) {
        *bytes = need;
        return MTGP_OK;
    }
    if (*bytes < need) return fail(MTGP_EINVAL, "buffer of %zu bytes, need %zu", *bytes, need);
    mtgp_status st = pool_sync(p);
    if (st != MTGP_OK) return st;
    uint32_t hdr[4] = {0x5047544Du, MTGP_PARAMS_VERSION, p->count, (uint32_t)p->state_words};
    std::memcpy(host_buf, hdr, 16);
    CU(cudaMemcpy((char *)host_buf + 16, p->d_gens, sizeof(DevGen) * p->count, cudaMemcpyDeviceToHost),
       "save generators");
    CU(cudaMemcpy((char *)host_buf + 16 + sizeof(DevGen) * p->count, p->d_state, 4u * p->state_words,
                  cudaMemcpyDeviceToHost),
       "save states");
    *bytes = need;
    return MTGP_OK;
}

mtgp_status mtgp_pool_load(mtgp_pool *p, const void *host_buf, size_t bytes)
{
    return guarded([&]() -> mtgp_status {
        if (!p || !host_buf) return fail(MTGP_EINVAL, "NULL argument");
        const size_t need = 16u + sizeof(DevGen) * p->count + 4u * p->state_words;
        if (bytes != need) return fail(MTGP_EINVAL, "checkpoint of %zu bytes, expected %zu", bytes, need);
        uint32_t hdr[4];
        std::memcpy(hdr, host_buf, 16);
        if (hdr[0] != 0x5047544Du || hdr[1] != MTGP_PARAMS_VERSION || hdr[2] != p->count ||
            hdr[3] != (uint32_t)p->state_words)
            return fail(MTGP_EINVAL, "checkpoint header does not match this pool");
        const DevGen *gs = (const DevGen *)((const char *)host_buf + 16);
        for (uint32_t i = 0; i < p->count; ++i) {
            DevGen a = gs[i], b = p->host_gens[i];
            a.count = b.count = 0;
            if (std::memcmp(&a, &b, sizeof a) != 0)
                return fail(MTGP_EINVAL, "checkpoint generator %u has other parameters", i);
        }
        mtgp_status st = pool_sync(p);
        if (st != MTGP_OK) return st;
        CU(cudaMemcpy(p->d_gens, gs, sizeof(DevGen) * p->count, cudaMemcpyHostToDevice), "load generators");
        CU(cudaMemcpy(p->d_state, (const char *)host_buf + 16 + sizeof(DevGen) * p->count, 4u * p->state_words,
                      cudaMemcpyHostToDevice),
           "load states");
        st = empty_graph_lists(p);   // their jump jobs were planned for the replaced states
        if (st != MTGP_OK) return st;
        jump_clear(p->jc, true);   // annihilators belong to the replaced states
        return MTGP_OK;
    });
}

void mtgp_pool_destroy(mtgp_pool *p)
{
    if (!p) return;
    for (mtgp_graph *g : p->jump_graphs) g->pool = nullptr;   // graphs destroyed late must not reach back
    if (p->used && p->ev_done) cudaEventSynchronize(p->ev_done);
    if (p->copy_stream) cudaStreamSynchronize(p->copy_stream);
    if (p->upload_pending && p->ev_upload) cudaEventSynchronize(p->ev_upload);
    jump_clear(p->jc, true);
    cudaFree(p->d_jstate);
    cudaFree(p->d_seq);
    cudaFree(p->d_gens);
    cudaFree(p->d_state);
    cudaFree(p->d_ctl);
    cudaFree(p->d_work);
    for (int b = 0; b < 2; ++b) {
        cudaFree(p->d_e2e[b]);
        if (p->ev_gen[b]) cudaEventDestroy(p->ev_gen[b]);
        if (p->ev_copy[b]) cudaEventDestroy(p->ev_copy[b]);
    }
    if (p->h_stage) cudaFreeHost(p->h_stage);
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    if (p->ev_done) cudaEventDestroy(p->ev_done);
    if (p->ev_upload) cudaEventDestroy(p->ev_upload);
    for (cudaEvent_t e : p->tev) cudaEventDestroy(e);
    delete p;
    (void)cudaGetLastError();      // the statuses above are ignored: leave none behind
}

// ---- single generator: a pool of one ---------------------------------------
mtgp_status mtgp_state_create(const mtgp_params *params, uint32_t gen_id, uint64_t seed, void *stream,
                              mtgp_state **out)
{
    return guarded([&]() -> mtgp_status {
        if (!out) return fail(MTGP_EINVAL, "out is NULL");
        *out = nullptr;
        mtgp_state *s = new (std::nothrow) mtgp_state;
        if (!s) return fail(MTGP_ENOMEM, "host allocation");
        mtgp_status st = mtgp_pool_create(params, &gen_id, &seed, 1u, stream, &s->pool);
        if (st != MTGP_OK) {
            delete s;
            return st;
        }
        *out = s;
        return MTGP_OK;
    });
}

mtgp_status mtgp_generate(mtgp_state *s, mtgp_dtype dt, void *dev_out, uint64_t n, void *stream)
{
    if (!s) return fail(MTGP_EINVAL, "state is NULL");
    if ((uint32_t)dt > 2u) return fail(MTGP_EINVAL, "unknown dtype %d", (int)dt);
    mtgp_request r{0u, (uint32_t)dt, n, 0u};
    return pool_run(s->pool, &r, 1u, dev_out, MTGP_LAYOUT_BLOCKED, (cudaStream_t)stream);
}

mtgp_status mtgp_state_save(const mtgp_state *s, void *host_buf, size_t *bytes)
{
    if (!s) return fail(MTGP_EINVAL, "state is NULL");
    return mtgp_pool_save(s->pool, host_buf, bytes);
}

mtgp_status mtgp_state_load(mtgp_state *s, const void *host_buf, size_t bytes)
{
    if (!s) return fail(MTGP_EINVAL, "state is NULL");
    return mtgp_pool_load(s->pool, host_buf, bytes);
}

mtgp_status mtgp_state_position(const mtgp_state *s, uint64_t *pos)
{
    if (!s) return fail(MTGP_EINVAL, "state is NULL");
    return mtgp_pool_position(s->pool, 0u, pos);
}

void mtgp_state_destroy(mtgp_state *s)
{
    if (!s) return;
    mtgp_pool_destroy(s->pool);
    delete s;
}

mtgp_status mtgp_fill_probe(void *dev_buf, uint64_t words, uint32_t pattern, void *stream)
{
    if (!dev_buf || ((uintptr_t)dev_buf & 15u) || (words & 3u))
        return fail(MTGP_EINVAL, "fill probe needs a 16-byte aligned buffer and a multiple of 4 words");
    CU(launch_fill((uint32_t *)dev_buf, words, pattern, (cudaStream_t)stream), "fill kernel launch");
    return MTGP_OK;
}

// ---- autotuner ---------------------------------------------------------------
mtgp_status mtgp_autotune(mtgp_pool *p, const mtgp_request *reqs, uint32_t nreq, void *dev_scratch,
                          uint32_t layouts, void *stream, mtgp_config *best, mtgp_layout *best_layout,
                          float *best_ms)
{
    return guarded([&]() -> mtgp_status {
        if (!p) return fail(MTGP_EINVAL, "pool is NULL");
        if (!(layouts & 3u)) return fail(MTGP_EINVAL, "layouts: bit 0 (blocked) and/or bit 1 (interleaved)");
        cudaStream_t s = (cudaStream_t)stream;
        mtgp_status st = pool_busy_check(p, s);
        if (st != MTGP_OK) return st;
        // the interleaved layout needs equal lengths and distinct generators;
        // chunks that divide the length leave no gaps in the output
        bool inter = (layouts & 2u) && nreq > 0;
        for (uint32_t j = 0; inter && j < nreq; ++j) inter = reqs[j].n == reqs[0].n && reqs[j].n > 0;
        if (inter) {
            std::vector<uint8_t> seen(p->count, 0);
            for (uint32_t j = 0; inter && j < nreq; ++j) {
                inter = reqs[j].gen < p->count && !seen[reqs[j].gen];
                if (inter) seen[reqs[j].gen] = 1;
            }
        }
        if (!(layouts & 1u) && !inter)
            return fail(MTGP_EINVAL, "autotune: the interleaved layout needs equal lengths and distinct generators");
        size_t bytes = 0;
        st = mtgp_pool_save(p, nullptr, &bytes);
        if (st != MTGP_OK) return st;
        std::vector<char> ckpt(bytes);
        st = mtgp_pool_save(p, ckpt.data(), &bytes);
        if (st != MTGP_OK) return st;
        const mtgp_config orig = p->cfg;
        // stage 1: form, block size, words per round (wide form), persistence
        // and occupancy, jump-ahead pieces -- blocked layout (or the
        // interleaved one, with the default chunk, if blocked is not allowed)
        std::vector<mtgp_config> cands;
        for (uint32_t pieces : {0u, 1u})
            for (uint32_t form : {0u, 1u, 2u, 3u, 4u, 5u})
                for (uint32_t threads : {32u, 64u, 96u, 128u, 192u, 256u, 512u, 1024u})
                    for (uint32_t rw : {0u, 128u, 256u})
                        for (uint32_t pers : {0u, 1u})
                            for (uint32_t bps : {0u, 2u, 4u, 8u}) {
                                if (!pers && bps) continue;
                                if (rw && form != 3u) continue;
                                if (!threads_supported(threads, form)) continue;
                                mtgp_config c{threads, pers, bps, orig.chunk, 0u, form, pieces, 0u, rw};
                                cands.push_back(c);
                            }
        cudaEvent_t e0, e1;
        CU(cudaEventCreate(&e0), "cudaEventCreate");
        CU(cudaEventCreate(&e1), "cudaEventCreate");
        auto time_one = [&](const mtgp_config &c, mtgp_layout lay, float *ms) -> bool {
            p->cfg = c;
            if (pool_run(p, reqs, nreq, dev_scratch, lay, s) != MTGP_OK) return false;   // warm-up
            if (cudaEventRecord(e0, s) != cudaSuccess) return false;
            const mtgp_status r = pool_run(p, reqs, nreq, dev_scratch, lay, s);
            if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return false;
            return r == MTGP_OK && cudaEventElapsedTime(ms, e0, e1) == cudaSuccess;
        };
        const mtgp_layout lay1 = (layouts & 1u) ? MTGP_LAYOUT_BLOCKED : MTGP_LAYOUT_INTERLEAVED;
        float best_t = 1e30f;
        mtgp_config best_c = orig;
        mtgp_layout best_l = lay1;
        for (const mtgp_config &c : cands) {
            float ms = 0.f;
            if (time_one(c, lay1, &ms) && ms < best_t) {
                best_t = ms;
                best_c = c;
            }
        }
        // stage 2: the interleaved layout with chunks of 2^8, 2^12, 2^16 words
        // (those dividing the length), for the best configuration of stage 1
        if (inter && best_t < 1e30f) {
            for (uint32_t chunk : {256u, 4096u, 65536u}) {
                if (reqs[0].n % chunk) continue;
                mtgp_config c = best_c;
                c.chunk = chunk;
                if (c.form == 3u) {                           // the wide form writes blocked layouts only
                    c.form = 0u;
                    c.threads = 128u;
                    c.round_words = 0u;
                }
                float ms = 0.f;
                if (time_one(c, MTGP_LAYOUT_INTERLEAVED, &ms) && ms < best_t) {
                    best_t = ms;
                    best_c = c;
                    best_l = MTGP_LAYOUT_INTERLEAVED;
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        (void)cudaGetLastError();                             // failed candidates leave nothing behind
        p->cfg = best_c;
        // psi found while tuning annihilates the restored (earlier) states as well:
        // psi(F) F^k s = 0 and F is invertible (R4 + I invertible, Sec. 5)
        const std::vector<f2::Poly> ann = p->jc.ann;
        st = mtgp_pool_load(p, ckpt.data(), bytes);
        if (st != MTGP_OK) return st;
        p->jc.ann = ann;
        if (best_t >= 1e30f) return fail(MTGP_EINVAL, "autotune: no candidate configuration ran");
        if (best) *best = best_c;
        if (best_layout) *best_layout = best_l;
        if (best_ms) *best_ms = best_t;
        return MTGP_OK;
    });
}

}  // extern "C"

// ---- graph-captured batched launch -------------------------------------------
namespace {

// Device buffer of a graph: control words [0, 256) (work counter, error word,
// item count at 8, output base at 16, job count at 24), then max_items work
// items, max_items segments and, with pieces, max_items jump jobs.
size_t graph_job_offset(uint32_t max_items)
{
    return 256u + (size_t)max_items * (sizeof(DevWork) + sizeof(DevSeg));
}

}  // namespace

// The graph of mtgp_graph_create; allow_pieces = false keeps every work item
// whole (the server: its generators' annihilating polynomials are not known).
mtgp_status mtgp::graph_create(mtgp_pool *p, uint32_t max_items, void *stream, bool allow_pieces, mtgp_graph **out)
{
    return guarded([&]() -> mtgp_status {
        if (!p || !out || max_items == 0) return fail(MTGP_EINVAL, "graph: NULL pool/out or max_items == 0");
        *out = nullptr;
        cudaStream_t s = (cudaStream_t)stream;
        mtgp_status st = refuse_capture(s);
        if (st != MTGP_OK) return st;
        st = pool_sync(p);
        if (st != MTGP_OK) return st;
        mtgp_config c = p->cfg;
        c.persistent = 1u;                                   // a fixed grid pulls however many items there are
        std::vector<uint32_t> all(p->count);
        for (uint32_t i = 0; i < p->count; ++i) all[i] = i;  // any generator of the pool may appear
        uint32_t qmax = 0, B = 0;
        st = launch_shape(p, c, all.data(), all.size(), max_items, &qmax, &B);
        if (st != MTGP_OK) return st;
        int occ = 0;
        CU(generate_occupancy(c.threads, c.form, qmax, B, &occ), "occupancy");
        if (occ < 1) return fail(MTGP_EINVAL, "graph: configuration does not fit on an SM");
        const int per_sm = c.blocks_per_sm ? std::min<int>((int)c.blocks_per_sm, occ) : occ;
        const uint32_t grid = std::min<uint32_t>(max_items, (uint32_t)(per_sm * p->sm_count));
        mtgp_graph *g = new (std::nothrow) mtgp_graph;
        if (!g) return fail(MTGP_ENOMEM, "host allocation");
        g->pool = p;
        g->max_items = max_items;
        g->B = B;
        g->form = c.form;
        // pieces when the pool's configuration allows them and every generator's
        // jump fits the fused kernel (polynomials of degree up to mexp)
        g->jump = allow_pieces && c.pieces != 1u;
        for (uint32_t i = 0; g->jump && i < p->count; ++i) {
            const DevGen &hg = p->host_gens[i];
            g->j_max_N = std::max(g->j_max_N, hg.N);
            g->j_max_ncoef = std::max(g->j_max_ncoef, hg.mexp + 1u);
            g->j_max_nseq = std::max(g->j_max_nseq, jump_seq_words(hg.N, hg.mexp + 1u));
        }
        if (g->jump) g->jump = jump_fused_fits(g->j_max_N, g->j_max_nseq, g->j_max_ncoef);
        g->d_bytes = graph_job_offset(max_items) + (g->jump ? (size_t)max_items * sizeof(DevJump) : 0u);
        auto bail = [&](mtgp_status r) { mtgp_graph_destroy(g); return r; };
        cudaError_t e;
    #define CUG(call, what)                                       \
        do {                                                      \
            e = (call);                                           \
            if (e != cudaSuccess) return bail(cuda_fail(e, what)); \
        } while (0)
        CUG(cudaMalloc(&g->d_buf, g->d_bytes), "cudaMalloc graph work list");
        if (g->jump) {
            g->jstate_cap = (uint64_t)max_items * ((g->j_max_N + 3u) & ~3u);
            CUG(cudaMalloc(&g->d_jstate, 4u * g->jstate_cap), "cudaMalloc graph piece states");
            CUG(prepare_jump_fused(g->j_max_N, g->j_max_nseq, g->j_max_ncoef), "jump kernel shared memory");
        }
        CUG(cudaMemsetAsync(g->d_buf, 0, 256u, s), "cudaMemsetAsync");
        for (int k = 0; k < 2; ++k) {
            CUG(cudaHostAlloc(&g->h_stage[k], g->d_bytes, cudaHostAllocDefault), "cudaHostAlloc");
            CUG(cudaEventCreateWithFlags(&g->ev_stage[k], cudaEventDisableTiming), "cudaEventCreate");
        }
        CUG(cudaStreamSynchronize(s), "cudaStreamSynchronize");
        CUG(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking), "cudaStreamCreate");
        char *b = (char *)g->d_buf;
        LaunchArgs a{};
        a.gens = p->d_gens;
        a.state = p->d_state;
        a.work = (const DevWork *)(b + 256u);
        a.segs = (const DevSeg *)(b + 256u + (size_t)max_items * sizeof(DevWork));
        a.out = nullptr;
        a.counter = (unsigned *)b;
        a.err = (unsigned *)(b + 4u);
        a.nwork = 0;
        a.nwork_dev = (const uint32_t *)(b + 8u);
        a.out_dev = (uint32_t *const *)(b + 16u);
        a.buf_words = B;
        a.persistent = 1u;
        a.jstate = g->d_jstate;
        a.spin_limit = p->spin_limit;                         // fixed in the capture
        a.round_words = c.round_words;
        CUG(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
        cudaError_t e1 = cudaMemsetAsync(b, 0, sizeof(unsigned), g->cap_stream);
        if (e1 == cudaSuccess && g->jump)
            e1 = launch_jump_fused(p->d_gens, p->d_state, g->d_jstate,
                                   (const DevJump *)(b + graph_job_offset(max_items)), max_items, g->j_max_N,
                                   g->j_max_nseq, g->j_max_ncoef, g->cap_stream, (const uint32_t *)(b + 24u),
                                   2u * (uint32_t)std::max(p->sm_count, 1));   // two blocks fit on an SM
        cudaError_t e2 = e1 == cudaSuccess ? launch_generate(a, c.threads, c.form, qmax, grid, g->cap_stream) : e1;
        e = cudaStreamEndCapture(g->cap_stream, &g->graph);
        if (e2 != cudaSuccess) return bail(cuda_fail(e2, "graph: capture of the generation launch"));
        if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamEndCapture"));
        CUG(cudaGraphInstantiate(&g->exec, g->graph, 0), "cudaGraphInstantiate");
    #undef CUG
        if (g->jump) p->jump_graphs.push_back(g);
        *out = g;
        return MTGP_OK;
    });
}

extern "C" {

mtgp_status mtgp_graph_create(mtgp_pool *p, uint32_t max_items, void *stream, mtgp_graph **out)
{
    return mtgp::graph_create(p, max_items, stream, true, out);
}

mtgp_status mtgp_graph_set_requests(mtgp_graph *g, const mtgp_request *reqs, uint32_t nreq, void *dev_out,
                                    mtgp_layout layout, void *stream)
{
    return guarded([&]() -> mtgp_status {
        if (!g) return fail(MTGP_EINVAL, "graph is NULL");
        mtgp_pool *p = g->pool;
        cudaStream_t s = (cudaStream_t)stream;
        mtgp_status st = pool_busy_check(p, s);
        if (st != MTGP_OK) return st;
        // on an error the work list in place is emptied: it may refer to jump
        // polynomials that planning evicted from the cache
        auto invalidate = [&](mtgp_status r) {
            (void)cudaMemsetAsync((char *)g->d_buf + 8u, 0, sizeof(uint32_t), s);
            (void)cudaMemsetAsync((char *)g->d_buf + 24u, 0, sizeof(uint32_t), s);
            return r;
        };
        if (((uintptr_t)dev_out & 3u) != 0) return invalidate(fail(MTGP_EINVAL, "dev_out must be 4-byte aligned"));
        if (g->form == 3u && layout != MTGP_LAYOUT_BLOCKED)
            return invalidate(fail(MTGP_EINVAL, "graph: the wide form (3) it captured writes blocked layouts only"));
        const mtgp_config saved = p->cfg;
        p->cfg.persistent = 1u;                              // longest-first order for the fixed grid
        Plan plan;
        st = build_plan(p, reqs, nreq, layout, &plan);
        if (st == MTGP_OK && g->jump) {
            // pieces (Sec. 7) as in a pool call, when they fit the captured
            // capacity and the captured jump kernel; otherwise whole items
            Plan pieces = plan;
            st = split_plan(p, &pieces, s);
            const bool fits = pieces.work.size() <= g->max_items && pieces.segs.size() <= g->max_items &&
                              pieces.jobs.size() <= g->max_items && pieces.jstate_words <= g->jstate_cap &&
                              pieces.jmax_N <= g->j_max_N && pieces.jmax_nseq <= g->j_max_nseq &&
                              pieces.jmax_ncoef <= g->j_max_ncoef;
            if (st == MTGP_OK && fits) plan = std::move(pieces);
        }
        p->cfg = saved;
        if (st != MTGP_OK) return invalidate(st);
        if (plan.work.size() > g->max_items || plan.segs.size() > g->max_items)
            return invalidate(fail(MTGP_EINVAL, "graph: %zu work items / %zu segments exceed its capacity %u",
                                   plan.work.size(), plan.segs.size(), g->max_items));
        if (plan.total && !dev_out) return invalidate(fail(MTGP_EINVAL, "dev_out is NULL"));
        const int k = g->slot;
        if (g->stage_used[k]) CU(cudaEventSynchronize(g->ev_stage[k]), "cudaEventSynchronize");
        char *h = (char *)g->h_stage[k];
        const uint32_t nwork = (uint32_t)plan.work.size(), njobs = (uint32_t)plan.jobs.size();
        std::memset(h, 0, 256u);
        std::memcpy(h + 8u, &nwork, sizeof nwork);
        std::memcpy(h + 16u, &dev_out, sizeof dev_out);
        std::memcpy(h + 24u, &njobs, sizeof njobs);
        std::memcpy(h + 256u, plan.work.data(), plan.work.size() * sizeof(DevWork));
        const size_t seg_off = 256u + (size_t)g->max_items * sizeof(DevWork);
        std::memcpy(h + seg_off, plan.segs.data(), plan.segs.size() * sizeof(DevSeg));
        const size_t job_off = graph_job_offset(g->max_items);
        if (njobs) std::memcpy(h + job_off, plan.jobs.data(), plan.jobs.size() * sizeof(DevJump));
        // control words from [8, 256), then the work items, the segments, the jobs
        CU(cudaMemcpyAsync((char *)g->d_buf + 8u, h + 8u, 248u + plan.work.size() * sizeof(DevWork),
                           cudaMemcpyHostToDevice, s),
           "graph: upload work list");
        if (!plan.segs.empty())
            CU(cudaMemcpyAsync((char *)g->d_buf + seg_off, h + seg_off, plan.segs.size() * sizeof(DevSeg),
                               cudaMemcpyHostToDevice, s),
               "graph: upload segments");
        if (njobs)
            CU(cudaMemcpyAsync((char *)g->d_buf + job_off, h + job_off, plan.jobs.size() * sizeof(DevJump),
                               cudaMemcpyHostToDevice, s),
               "graph: upload jump jobs");
        CU(cudaEventRecord(g->ev_stage[k], s), "cudaEventRecord");
        g->stage_used[k] = true;
        g->slot ^= 1;
        p->last_stream = s;
        CU(cudaEventRecord(p->ev_done, s), "cudaEventRecord");
        p->used = true;
        return MTGP_OK;
    });
}

mtgp_status mtgp_graph_launch(mtgp_graph *g, void *stream)
{
    if (!g) return fail(MTGP_EINVAL, "graph is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    mtgp_status st = pool_busy_check(g->pool, s);
    if (st != MTGP_OK) return st;
    CU(cudaGraphLaunch(g->exec, s), "cudaGraphLaunch");
    g->pool->launches += g->jump ? 2u : 1u;                 // jump (whatever its job count) and generation
    CU(cudaEventRecord(g->pool->ev_done, s), "cudaEventRecord");
    g->pool->last_stream = s;
    g->pool->used = true;
    return MTGP_OK;
}

mtgp_status mtgp_graph_errors(mtgp_graph *g, uint32_t *flags)
{
    if (!g || !flags) return fail(MTGP_EINVAL, "NULL argument");
    mtgp_status st = pool_sync(g->pool);
    if (st != MTGP_OK) return st;
    CU(cudaMemcpy(flags, (char *)g->d_buf + 4u, sizeof(uint32_t), cudaMemcpyDeviceToHost), "read error word");
    CU(cudaMemset((char *)g->d_buf + 4u, 0, sizeof(uint32_t)), "clear error word");
    return MTGP_OK;
}

void mtgp_graph_destroy(mtgp_graph *g)
{
    if (!g) return;
    if (g->pool) {
        auto &v = g->pool->jump_graphs;
        v.erase(std::remove(v.begin(), v.end(), g), v.end());
    }
    if (g->pool && g->pool->used) cudaEventSynchronize(g->pool->ev_done);
    for (int k = 0; k < 2; ++k) {
        if (g->stage_used[k]) cudaEventSynchronize(g->ev_stage[k]);
        if (g->ev_stage[k]) cudaEventDestroy(g->ev_stage[k]);
        if (g->h_stage[k]) cudaFreeHost(g->h_stage[k]);
    }
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    cudaFree(g->d_buf);
    cudaFree(g->d_jstate);
    delete g;
    (void)cudaGetLastError();      // the statuses above are ignored: leave none behind
}

// ---- error words -----------------------------------------------------------------
mtgp_status mtgp_pool_errors(mtgp_pool *p, uint32_t *flags)
{
    if (!p || !flags) return fail(MTGP_EINVAL, "NULL argument");
    mtgp_status st = pool_sync(p);
    if (st != MTGP_OK) return st;
    CU(cudaMemcpy(flags, p->d_ctl + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost), "read error word");
    CU(cudaMemset(p->d_ctl + 1, 0, sizeof(uint32_t)), "clear error word");
    return MTGP_OK;
}

mtgp_status mtgp_pool_launch_count(const mtgp_pool *p, uint64_t *launches)
{
    if (!p || !launches) return fail(MTGP_EINVAL, "NULL argument");
    *launches = p->launches;
    return MTGP_OK;
}

mtgp_status mtgp_pool_set_spin_limit(mtgp_pool *p, uint32_t polls)
{
    if (!p) return fail(MTGP_EINVAL, "NULL pool");
    mtgp_status st = pool_sync(p);
    if (st != MTGP_OK) return st;
    p->spin_limit = polls;
    return MTGP_OK;
}

mtgp_status mtgp_pool_set_timing(mtgp_pool *p, uint32_t entries)
{
    return guarded([&]() -> mtgp_status {
        if (!p) return fail(MTGP_EINVAL, "NULL pool");
        if (entries > 65536u) return fail(MTGP_EINVAL, "at most 65536 timing entries");
        mtgp_status st = pool_sync(p);
        if (st != MTGP_OK) return st;
        for (cudaEvent_t e : p->tev) CU(cudaEventDestroy(e), "cudaEventDestroy");
        p->tev.clear();
        p->tjump.assign(entries, 0u);
        p->timing_n = p->timing_next = p->timing_count = 0;
        for (uint32_t i = 0; i < 3u * entries; ++i) {
            cudaEvent_t e = nullptr;
            CU(cudaEventCreate(&e), "cudaEventCreate");
            p->tev.push_back(e);
        }
        p->timing_n = entries;
        return MTGP_OK;
    });
}

mtgp_status mtgp_pool_kernel_times(mtgp_pool *p, uint32_t count, float *jump_ms, float *gen_ms)
{
    if (!p || (count && (!jump_ms || !gen_ms))) return fail(MTGP_EINVAL, "NULL argument");
    if (count > p->timing_count)
        return fail(MTGP_EINVAL, "%u timed calls requested, %u recorded", count, p->timing_count);
    for (uint32_t k = 0; k < count; ++k) {      // oldest first
        const uint32_t e = (p->timing_next + p->timing_n - count + k) % p->timing_n;
        cudaEvent_t *t = &p->tev[3u * e];
        CU(cudaEventSynchronize(t[2]), "cudaEventSynchronize");
        float a = 0.f, b = 0.f;
        if (p->tjump[e]) CU(cudaEventElapsedTime(&a, t[0], t[1]), "cudaEventElapsedTime");
        CU(cudaEventElapsedTime(&b, t[1], t[2]), "cudaEventElapsedTime");
        jump_ms[k] = a;
        gen_ms[k] = b;
    }
    return MTGP_OK;
}

mtgp_status mtgp_pool_jump(mtgp_pool *p, uint32_t i, uint64_t steps, void *stream)
{
    return guarded([&]() -> mtgp_status {
        if (!p || i >= p->count) return fail(MTGP_EINVAL, "bad pool or generator index");
        cudaStream_t s = (cudaStream_t)stream;
        mtgp_status st = pool_busy_check(p, s);
        if (st != MTGP_OK) return st;
        if (steps == 0) return MTGP_OK;
        int r = jump_annihilate(p->jc, p->host_gens.data(), p->d_gens, p->d_state, &i, 1u, s);
        if (r != MTGP_OK) return (mtgp_status)r;
        if (p->jc.dev_bytes > kJumpStoreCap) {
            st = pool_sync(p);
            if (st == MTGP_OK) st = empty_graph_lists(p);
            if (st != MTGP_OK) return st;
            jump_clear(p->jc, false);
        }
        r = jump_polys(p->jc, {{i, steps}});
        if (r != MTGP_OK) return (mtgp_status)r;
        const JumpPoly jp = jump_poly(p->jc, i, steps);
        const DevGen &g = p->host_gens[i];
        DevJump jb{};
        jb.poly = jp.d;
        jb.ncoef = jp.ncoef;
        jb.src = g.state_off;
        jb.dst = g.state_off;                 // in place: the walk reads the state first
        jb.gen = i;
        jb.nseq = jump_seq_words(g.N, jb.ncoef);
        jb.mode = kJumpStep;
        st = ensure_upload_space(p, sizeof jb);
        if (st != MTGP_OK) return st;
        const bool fused = jump_fused_fits(g.N, jb.nseq, jb.ncoef);
        st = ensure_jump_space(p, 0u, fused ? 0u : jb.nseq);
        if (st != MTGP_OK) return st;
        std::memcpy(p->h_stage, &jb, sizeof jb);
        CU(cudaMemcpyAsync(p->d_work, p->h_stage, sizeof jb, cudaMemcpyHostToDevice, s), "upload jump job");
        if (fused) {                          // in place: the block reads the whole state before writing
            CU(launch_jump_fused(p->d_gens, p->d_state, p->d_state, (const DevJump *)p->d_work, 1u, g.N, jb.nseq,
                                 jb.ncoef, s),
               "jump kernel launch");
        } else {
            CU(launch_walk(p->d_gens, p->d_state, p->d_seq, (const DevJump *)p->d_work, 1u, g.N, s),
               "walk kernel launch");
            CU(launch_jump_sum(p->d_gens, p->d_seq, p->d_state, (const DevJump *)p->d_work, 1u, g.N, s),
               "jump kernel launch");
        }
        CU(cudaStreamSynchronize(s), "jump");
        uint64_t pos = 0;
        char *cnt = (char *)p->d_gens + sizeof(DevGen) * i + offsetof(DevGen, count);
        CU(cudaMemcpy(&pos, cnt, sizeof pos, cudaMemcpyDeviceToHost), "read position");
        pos += steps;
        CU(cudaMemcpy(cnt, &pos, sizeof pos, cudaMemcpyHostToDevice), "write position");
        return MTGP_OK;
    });
}

mtgp_status mtgp_state_jump(mtgp_state *s, uint64_t steps, void *stream)
{
    if (!s) return fail(MTGP_EINVAL, "state is NULL");
    return mtgp_pool_jump(s->pool, 0u, steps, stream);
}

mtgp_status mtgp_pool_annihilator(mtgp_pool *p, uint32_t i, uint64_t *poly, uint32_t poly_words,
                                  uint32_t *degree, void *stream)
{
    return guarded([&]() -> mtgp_status {
        if (!p || i >= p->count || !degree) return fail(MTGP_EINVAL, "bad pool, index or NULL degree");
        cudaStream_t s = (cudaStream_t)stream;
        mtgp_status st = pool_busy_check(p, s);
        if (st != MTGP_OK) return st;
        const int r = jump_annihilate(p->jc, p->host_gens.data(), p->d_gens, p->d_state, &i, 1u, s);
        if (r != MTGP_OK) return (mtgp_status)r;
        const f2::Poly &a = p->jc.ann[i];
        const int64_t d = f2::degree(a);
        *degree = (uint32_t)std::max<int64_t>(d, 0);
        if (!poly) return MTGP_OK;
        const size_t need = (size_t)(*degree / 64u) + 1u;
        if (poly_words < need) return fail(MTGP_EINVAL, "poly has %u words, need %zu", poly_words, need);
        std::memset(poly, 0, sizeof(uint64_t) * poly_words);
        std::copy(a.begin(), a.end(), poly);
        return MTGP_OK;
    });
}

}  // extern "C"

namespace {

mtgp_status poly_out(const f2::Poly &r, uint64_t *out, uint32_t out_words, int64_t *deg)
{
    *deg = f2::degree(r);
    const size_t need = *deg < 0 ? 1u : (size_t)(*deg / 64) + 1u;
    if (out_words < need) return fail(MTGP_EINVAL, "output has %u words, need %zu", out_words, need);
    std::memset(out, 0, sizeof(uint64_t) * out_words);
    std::copy(r.begin(), r.end(), out);
    return MTGP_OK;
}

}  // namespace

extern "C" {

mtgp_status mtgp_f2_minpoly(const uint64_t *bits, uint64_t n, uint64_t *out, uint32_t out_words, int64_t *deg)
{
    if ((!bits && n) || !out || !deg) return fail(MTGP_EINVAL, "NULL argument");
    try {
        return poly_out(n ? f2::minpoly(bits, n) : f2::Poly{1u}, out, out_words, deg);
    } catch (const std::exception &) {
        return fail(MTGP_ENOMEM, "host allocation");
    }
}

mtgp_status mtgp_f2_mulmod(const uint64_t *a, uint32_t a_words, const uint64_t *b, uint32_t b_words,
                           const uint64_t *m, uint32_t m_words, uint64_t *out, uint32_t out_words, int64_t *deg)
{
    if ((!a && a_words) || (!b && b_words) || !m || !out || !deg) return fail(MTGP_EINVAL, "NULL argument");
    try {
        const f2::Poly mp(m, m + m_words);
        if (f2::degree(mp) < 1) return fail(MTGP_EINVAL, "modulus of degree < 1");
        const f2::Modulus M = f2::make_modulus(mp);
        f2::Poly x(a, a + a_words), y(b, b + b_words);
        f2::reduce(x, M);
        f2::reduce(y, M);
        return poly_out(f2::mulmod(x, y, M), out, out_words, deg);
    } catch (const std::exception &) {
        return fail(MTGP_ENOMEM, "host allocation");
    }
}

mtgp_status mtgp_f2_xpow_mod(uint64_t e, const uint64_t *m, uint32_t m_words, uint64_t *out, uint32_t out_words,
                             int64_t *deg)
{
    if (!m || !out || !deg) return fail(MTGP_EINVAL, "NULL argument");
    try {
        const f2::Poly mp(m, m + m_words);
        if (f2::degree(mp) < 1) return fail(MTGP_EINVAL, "modulus of degree < 1");
        return poly_out(f2::xpow_mod(e, f2::make_modulus(mp)), out, out_words, deg);
    } catch (const std::exception &) {
        return fail(MTGP_ENOMEM, "host allocation");
    }
}

}  // extern "C"
