// Allocation-free generation: mtgp_generate_noalloc.
//
// Everything the generation kernel needs besides the caller's buffers (the
// generators' parameter records, the work list, the segment list and the
// error word) lives in one file-scope device array, g_noalloc_scratch, that
// every GPU loading this library keeps until the process exits.  No device
// memory is allocated or freed on this path.
#include "mtgp.h"
#include "mtgp_internal.h"

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <exception>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

using namespace mtgp;

namespace {

static_assert(sizeof(DevGen) * MTGP_NOALLOC_MAX_GENS + sizeof(DevWork) * MTGP_NOALLOC_MAX_REQS +
                      sizeof(DevSeg) * MTGP_NOALLOC_MAX_REQS + 256u <=
                  MTGP_NOALLOC_SCRATCH_BYTES,
              "scratch too small for its limits");

// Layout: [0, 256) control words (error flags), then DevGen[count],
// DevWork[nwork], DevSeg[nreq], each 16-byte aligned.
static __device__ __align__(256) unsigned char g_noalloc_scratch[MTGP_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
// Held from the copy of a call's records into the array through the launch
// of its kernel, so that calls from several host threads on one stream queue
// as copy, kernel, copy, kernel: each kernel then reads its own records.
std::mutex g_call_mu;
void *g_scratch_addr[kMaxDevices] = {};   // device address of g_noalloc_scratch per device

mtgp_status fail(mtgp_status st, const char *msg) { return (mtgp_status)report_error(st, msg); }

mtgp_status fail_cuda(cudaError_t e, const char *what)
{
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s (%d)", what, cudaGetErrorString(e), (int)e);
    return fail(MTGP_ECUDA, buf);
}

// Set-up, once per device, with that device current: the host-side name of
// the array is only a stand-in, so its device address is looked up here.
mtgp_status scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(MTGP_EINVAL, "device ordinal out of range for the scratch table");
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return fail_cuda(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return MTGP_OK;
}

size_t align16(size_t x) { return (x + 15u) & ~(size_t)15u; }

}  // namespace

namespace {

mtgp_status generate_noalloc(const mtgp_params *ps, uint32_t count, uint32_t *dev_states,
                             const uint64_t *state_offsets, const mtgp_request *reqs, uint32_t nreq,
                             void *dev_out, void *stream)
{
    if (!ps || !state_offsets || !dev_states || count == 0)
        return fail(MTGP_EINVAL, "noalloc: NULL parameters, states or offsets, or count == 0");
    if (count > MTGP_NOALLOC_MAX_GENS) {
        char buf[160];
        snprintf(buf, sizeof buf, "noalloc: %u generators exceed the scratch limit of %u per call", count,
                 MTGP_NOALLOC_MAX_GENS);
        return fail(MTGP_EINVAL, buf);
    }
    if (nreq > MTGP_NOALLOC_MAX_REQS) {
        char buf[160];
        snprintf(buf, sizeof buf, "noalloc: %u requests exceed the scratch limit of %u per call", nreq,
                 MTGP_NOALLOC_MAX_REQS);
        return fail(MTGP_EINVAL, buf);
    }
    if (nreq && !reqs) return fail(MTGP_EINVAL, "noalloc: reqs is NULL");
    if (((uintptr_t)dev_states & 3u) || ((uintptr_t)dev_out & 3u))
        return fail(MTGP_EINVAL, "noalloc: buffers must be 4-byte aligned");
    // host-side records (ordinary host memory; nothing on the device is allocated)
    std::vector<DevGen> gens(count);
    uint32_t nmax = 0, smax = 0;
    for (uint32_t i = 0; i < count; ++i) {
        mtgp_status st = mtgp_params_validate(&ps[i]);
        if (st != MTGP_OK) return st;
        DevGen &g = gens[i];
        std::memset(&g, 0, sizeof g);
        g.N = ps[i].N;
        g.M = ps[i].pos;
        g.mask = ps[i].mask;
        g.sh1 = ps[i].sh1;
        g.sh2 = ps[i].sh2;
        g.mexp = ps[i].mexp;
        g.id = ps[i].id;
        g.state_off = state_offsets[i];
        std::memcpy(g.rec, ps[i].rec_tbl, sizeof g.rec);
        std::memcpy(g.tmp, ps[i].tmp_tbl, sizeof g.tmp);
        nmax = g.N > nmax ? g.N : nmax;
        smax = g.N - g.M > smax ? g.N - g.M : smax;
    }
    // two generators whose state ranges overlap would run in two blocks that
    // read and write the same words at once: refused
    {
        std::vector<std::pair<uint64_t, uint64_t>> rng(count);
        for (uint32_t i = 0; i < count; ++i) rng[i] = {state_offsets[i], state_offsets[i] + gens[i].N};
        std::sort(rng.begin(), rng.end());
        for (uint32_t i = 1; i < count; ++i)
            if (rng[i].first < rng[i - 1].second)
                return fail(MTGP_EINVAL, "noalloc: the state ranges of two generators overlap");
    }
    // requests grouped per generator, in array order (blocked layout)
    std::vector<DevWork> work;
    std::vector<DevSeg> segs;
    std::vector<std::vector<uint32_t>> per(count);
    uint64_t total = 0;
    for (uint32_t j = 0; j < nreq; ++j) {
        if (reqs[j].gen >= count || reqs[j].dtype > 2u) return fail(MTGP_EINVAL, "noalloc: request out of range");
        if (reqs[j].n) per[reqs[j].gen].push_back(j);
        total += reqs[j].n;
    }
    if (!total) return MTGP_OK;
    if (!dev_out) return fail(MTGP_EINVAL, "noalloc: dev_out is NULL");
    for (uint32_t g = 0; g < count; ++g) {
        if (per[g].empty()) continue;
        DevWork w{};
        w.gen = g;
        w.seg_begin = (uint32_t)segs.size();
        w.seg_count = (uint32_t)per[g].size();
        for (uint32_t j : per[g]) {
            DevSeg s{};
            s.n = reqs[j].n;
            s.out_off = reqs[j].out_offset;
            s.dtype = reqs[j].dtype;
            s.chunk_log2 = kBlocked;
            w.total += s.n;
            segs.push_back(s);
        }
        work.push_back(w);
    }
    // launch shape: 128 threads per block, the smallest slot count covering S
    const uint32_t threads = 128u;
    const uint32_t qmax = kernel_slots(threads, 0u, (smax + threads - 1u) / threads);
    if (!qmax) return fail(MTGP_EINVAL, "noalloc: round size too large for 128 threads");
    const uint32_t span = (smax + threads - 1u) / threads * threads;
    uint32_t B = 2u * nmax + 32u * smax + 32u;
    const uint32_t need = 2u * nmax + span + 32u;
    if (B > 12288u) B = 12288u;                      // 48 KiB of shared memory per block
    if (B < need) B = need;
    // The kernel raises its buffer error (and skips the item) only when a
    // generator's slot count exceeds qmax or its buffer minimum exceeds B.
    // Both hold here for every generator, so the kernel's error word, which
    // no call reads back, cannot be set on this path.
    for (uint32_t i = 0; i < count; ++i) {
        const uint32_t S = gens[i].N - gens[i].M, nq = (S + threads - 1u) / threads;
        if (nq > qmax || 2u * gens[i].N + nq * threads + 32u > B)
            return fail(MTGP_EINVAL, "noalloc: internal launch shape does not fit a generator");
    }
    // one image of the scratch: control words zeroed, then the records
    const size_t gb = align16(sizeof(DevGen) * count), wb = align16(sizeof(DevWork) * work.size());
    const size_t bytes = 256u + gb + wb + sizeof(DevSeg) * segs.size();
    std::vector<unsigned char> image(bytes, 0u);
    std::memcpy(image.data() + 256u, gens.data(), sizeof(DevGen) * count);
    std::memcpy(image.data() + 256u + gb, work.data(), sizeof(DevWork) * work.size());
    std::memcpy(image.data() + 256u + gb + wb, segs.data(), sizeof(DevSeg) * segs.size());
    cudaStream_t s = (cudaStream_t)stream;
    // the records are copied out of this call's own host memory, which is gone
    // by the time a captured graph would replay the copy: no capture
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(s, &cap);
    if (ce != cudaSuccess) return fail_cuda(ce, "cudaStreamIsCapturing");
    if (cap != cudaStreamCaptureStatusNone)
        return fail(MTGP_EINVAL, "noalloc: the stream is being captured into a CUDA graph; calls cannot be captured");
    void *base = nullptr;
    mtgp_status st = scratch_address(&base);
    if (st != MTGP_OK) return st;
    std::lock_guard<std::mutex> lock(g_call_mu);
    cudaError_t e = cudaMemcpyAsync(base, image.data(), bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail_cuda(e, "noalloc: copy records to scratch");
    unsigned char *b = (unsigned char *)base;
    LaunchArgs a{};
    a.gens = (DevGen *)(b + 256u);
    a.state = dev_states;
    a.work = (const DevWork *)(b + 256u + gb);
    a.segs = (const DevSeg *)(b + 256u + gb + wb);
    a.out = (uint32_t *)dev_out;
    a.counter = (unsigned *)b;
    a.err = (unsigned *)(b + 4u);
    a.nwork = (uint32_t)work.size();
    a.buf_words = B;
    a.persistent = 0u;
    e = launch_generate(a, threads, 0u, qmax, (uint32_t)work.size(), s);
    if (e != cudaSuccess) return fail_cuda(e, "noalloc: generate kernel launch");
    return MTGP_OK;
}

}  // namespace

// The records are built in host containers; a failed host allocation comes
// back as MTGP_ENOMEM instead of an exception crossing the C ABI.
extern "C" mtgp_status mtgp_generate_noalloc(const mtgp_params *ps, uint32_t count, uint32_t *dev_states,
                                             const uint64_t *state_offsets, const mtgp_request *reqs,
                                             uint32_t nreq, void *dev_out, void *stream)
{
    try {
        return generate_noalloc(ps, count, dev_states, state_offsets, reqs, nreq, dev_out, stream);
    } catch (const std::bad_alloc &) {
        return fail(MTGP_ENOMEM, "noalloc: host allocation failed");
    } catch (const std::exception &e) {
        return fail(MTGP_EINVAL, e.what());
    }
}
