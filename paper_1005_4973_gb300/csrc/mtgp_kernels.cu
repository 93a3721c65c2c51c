// MTGP kernels for sm_103a other than the generation kernel (which lives in
// mtgp_device.cuh and the per-block-size units mtgp_gen_t*.cu): state seeding,
// the write-only bandwidth probe, and the launchers.
#include "mtgp_internal.h"

#include <map>
#include <mutex>
#include <utility>

namespace mtgp {

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;   // SplitMix64 Weyl increment

// SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Seeds generator `first + blockIdx.x`: word j of the state is the low half of
// SplitMix64 output j+1 from (seed ^ key), key = SplitMix64 output 1 from the
// generator ID.  A state whose p effective bits are all zero (a fixed point of
// the linear recursion) gets x_{N-1} = 1.
__global__ void k_seed(DevGen *gens, uint32_t *state, const uint32_t *gen_ids,
                       const uint64_t *seeds, uint32_t first)
{
    const uint32_t g = first + blockIdx.x;
    const uint32_t N = gens[g].N, mask = gens[g].mask;
    const uint64_t s0 = seeds[g] ^ mix64((uint64_t)gen_ids[g] + kGamma);
    uint32_t *st = state + gens[g].state_off;
    uint32_t any = 0;
    for (uint32_t j = threadIdx.x; j < N; j += blockDim.x) {
        const uint32_t w = (uint32_t)mix64(s0 + (uint64_t)(j + 1u) * kGamma);
        st[j] = w;
        any |= (j == 0u) ? (w & mask) : w;
    }
    const int nonzero = __syncthreads_or(any != 0u);
    if (threadIdx.x == 0) {
        if (!nonzero) st[N - 1u] = 1u;
        gens[g].count = 0;
    }
}

// Write-only bandwidth probe: 16-byte streaming stores over a grid-stride loop.
__global__ void k_fill(uint4 *buf, uint64_t n16, uint32_t pattern)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
        const uint32_t v = pattern ^ (uint32_t)i;
        __stcs(buf + i, make_uint4(v, v + 1u, v + 2u, v + 3u));
    }
}

GenKernel pick(uint32_t threads, uint32_t form, uint32_t qmax, bool interleave = false)
{
    if (interleave && form == 0u && threads == 128u) {
        GenKernel k = gen_kernel_t128_il(qmax);
        if (k) return k;
    }
    if (form == 3u) return wide_kernel(threads, qmax);
    if (form == 5u) return threads == 128u && qmax == 3u ? dual_kernel_t128_q3() : nullptr;
    if (form == 4u) {
        if (threads == 128u) {
            switch (qmax) {
            case 2: return pair_kernel_t128_q2();
            case 3: return pair_kernel_t128_q3();
            case 6: return pair_kernel_t128_q6();
            default: return nullptr;
            }
        }
        return nullptr;
    }
    if (form == 2u) {
        switch (threads) {
        case 128: return flow_kernel_w2(qmax);
        case 256: return flow_kernel_w4(qmax);
        case 512: return flow_kernel_w8(qmax);
        case 1024: return flow_kernel_w16(qmax);
        default: return nullptr;
        }
    }
    if (form == 1u) {
        switch (threads) {
        case 128: return split_kernel_rt64(qmax);
        case 256: return split_kernel_rt128(qmax);
        case 512: return split_kernel_rt256(qmax);
        case 1024: return split_kernel_rt512(qmax);
        default: return nullptr;
        }
    }
    switch (threads) {
    case 32: return gen_kernel_t32(qmax);
    case 64: return gen_kernel_t64(qmax);
    case 128: return gen_kernel_t128(qmax);
    case 256: return gen_kernel_t256(qmax);
    case 512: return gen_kernel_t512(qmax);
    default: return nullptr;
    }
}

}  // namespace

// A kernel's dynamic shared-memory limit is a function attribute that captured
// graphs rely on at replay: it is only ever raised, never lowered below what an
// earlier launch or capture used.
cudaError_t raise_smem_limit(const void *kernel, size_t dyn_bytes)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> set;  // (device, kernel) -> limit set
    if (dyn_bytes + 1024u <= 48u * 1024u) return cudaSuccess;   // within the default (static words aside)
    int dev = 0;
    const cudaError_t de = cudaGetDevice(&dev);
    if (de != cudaSuccess) return de;
    std::lock_guard<std::mutex> lock(mu);
    size_t &cur = set[{dev, kernel}];
    if (dyn_bytes <= cur) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_bytes);
    if (e == cudaSuccess) cur = dyn_bytes;
    return e;
}

// Slot counts compiled: MTGP_QMAX_LIST for forms 0-2, 1..4 groups for form 3.
static const uint32_t kSlots[] = {MTGP_QMAX_LIST};
static const uint32_t kWideSlots[] = {1, 2, 3, 4};

bool threads_supported(uint32_t threads, uint32_t form)
{
    if (form == 3u) {
        for (uint32_t q : kWideSlots)
            if (pick(threads, form, q)) return true;
        return false;
    }
    for (uint32_t q : kSlots)
        if (pick(threads, form, q)) return true;
    return false;
}

uint32_t kernel_slots(uint32_t threads, uint32_t form, uint32_t nq)
{
    if (form == 3u) {
        for (uint32_t q : kWideSlots)
            if (q >= nq && pick(threads, form, q)) return q;
        return 0;
    }
    for (uint32_t q : kSlots)
        if (q >= nq && pick(threads, form, q)) return q;
    return 0;
}

cudaError_t launch_seed(DevGen *gens, uint32_t *state, const uint32_t *gen_ids,
                        const uint64_t *seeds, uint32_t first, uint32_t count, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    clear_stale_error();
    k_seed<<<count, 256, 0, s>>>(gens, state, gen_ids, seeds, first);
    return cudaGetLastError();
}

cudaError_t launch_generate(const LaunchArgs &a, uint32_t threads, uint32_t form, uint32_t qmax, uint32_t grid,
                            cudaStream_t s)
{
    GenKernel k = pick(threads, form, qmax, a.interleave != 0u);
    if (!k) return cudaErrorInvalidValue;
    const size_t smem = (size_t)a.buf_words * sizeof(uint32_t);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return e;
    // dynamic words past the default limit (raised before a capture by
    // generate_occupancy; a function attribute is not captured)
    if (cap == cudaStreamCaptureStatusNone) {
        e = raise_smem_limit((const void *)k, smem);
        if (e != cudaSuccess) return e;
    }
    clear_stale_error();
    k<<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t generate_occupancy(uint32_t threads, uint32_t form, uint32_t qmax, uint32_t buf_words,
                               int *blocks_per_sm, bool interleave)
{
    GenKernel k = pick(threads, form, qmax, interleave);
    if (!k) return cudaErrorInvalidValue;
    const size_t smem = (size_t)buf_words * sizeof(uint32_t);
    cudaError_t e = raise_smem_limit((const void *)k, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, threads, smem);
}

cudaError_t launch_fill(uint32_t *buf, uint64_t words, uint32_t pattern, cudaStream_t s)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    clear_stale_error();
    k_fill<<<(unsigned)sms * 8u, 512, 0, s>>>(reinterpret_cast<uint4 *>(buf), words / 4u, pattern);
    return cudaGetLastError();
}

}  // namespace mtgp
