// Host side of jump-ahead (Sec. 7).  See mtgp_jump.h.
//
// psi for a state s: walk the recursion from s on the GPU, take the parity of
// a mask of the second state word along the walk (a linear functional of the
// state, Sec. 3.3), and find that bit sequence's minimal polynomial phi by
// Berlekamp-Massey.  phi divides the annihilator of s; to make sure nothing
// was missed, the GPU computes V = phi(F) s.  If V = 0, psi = phi; otherwise
// the same steps run on V (with another mask) and psi is the product of the
// factors found, since each V is the previous one with the found factor
// applied.
#include "mtgp_jump.h"

#include "mtgp.h"

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <exception>
#include <map>
#include <thread>

namespace mtgp {

namespace {

int jfail(int st, const char *what)
{
    return report_error(st, what);
}

int jcuda(cudaError_t e, const char *what)
{
    char buf[256];
    snprintf(buf, sizeof buf, "jump-ahead: %s: %s (%d)", what, cudaGetErrorString(e), (int)e);
    return report_error(e == cudaErrorMemoryAllocation ? MTGP_ENOMEM : MTGP_ECUDA, buf);
}

#define JCU(call, what)                                 \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return jcuda(e_, what);  \
    } while (0)

// Runs f(i) for i in [0, n) on the host cores.
template <class F>
void parallel_for(size_t n, F f)
{
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const size_t nt = std::min<size_t>(n, hw);
    if (nt <= 1) {
        for (size_t i = 0; i < n; ++i) f(i);
        return;
    }
    std::atomic<size_t> next{0};
    std::vector<std::thread> th;
    th.reserve(nt);
    for (size_t t = 0; t < nt; ++t)
        th.emplace_back([&] {
            for (size_t i; (i = next.fetch_add(1)) < n;) f(i);
        });
    for (auto &t : th) t.join();
}

// Device buffer freed on scope exit.
struct DevBuf {
    void *p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
};

// Mask of the functional of pass k: parities of mixes first, then every
// single bit of the word.  A pass leaves a remainder whose sequence under its
// functional is zero, and later passes keep it zero (they apply polynomials in
// F to the remainder), so after the 32 single-bit passes every coordinate of
// every state on the remainder's orbit is zero -- the state words x_1 ..
// x_{N-1} directly, and the masked bits of x_0 through x_N, which the
// recursion maps injectively (R4 + I invertible) -- and the remainder is 0.
constexpr uint32_t kMixMasks[] = {0xFFFFFFFFu, 0x55555555u, 0x33333333u, 0x0F0F0F0Fu, 0x00FF00FFu, 0x0000FFFFu};
constexpr int kMixes = (int)(sizeof kMixMasks / sizeof kMixMasks[0]);
constexpr int kPasses = kMixes + 32;

uint32_t pass_mask(int k)
{
    return k < kMixes ? kMixMasks[k] : 1u << (k - kMixes);
}

}  // namespace

int jump_annihilate(JumpCache &jc, const DevGen *hg, const DevGen *d_gens, const uint32_t *d_state,
                    const uint32_t *gens, size_t n, cudaStream_t s)
{
    std::vector<uint32_t> todo;
    for (size_t k = 0; k < n; ++k) {
        const uint32_t g = gens[k];
        if (g >= jc.ann.size()) return jfail(MTGP_EINVAL, "jump-ahead: generator out of range");
        if (jc.ann[g].empty()) todo.push_back(g);
    }
    std::sort(todo.begin(), todo.end());
    todo.erase(std::unique(todo.begin(), todo.end()), todo.end());
    // batches of at most 64 MiB of walked sequence
    size_t b0 = 0;
    while (b0 < todo.size()) {
        size_t b1 = b0;
        uint64_t words = 0;
        while (b1 < todo.size()) {
            const uint64_t w = (2ull * hg[todo[b1]].mexp + 3u + 3u) & ~3ull;
            if (b1 > b0 && words + w > (16ull << 20)) break;
            words += w;
            ++b1;
        }
        const size_t nb = b1 - b0;
        std::vector<uint64_t> seq_off(nb), v_off(nb), nseq(nb);
        uint64_t vwords = 0;
        uint32_t max_N = 3;
        for (size_t k = 0, so = 0; k < nb; ++k) {
            const DevGen &g = hg[todo[b0 + k]];
            nseq[k] = (2ull * g.mexp + 3u + 3u) & ~3ull;
            seq_off[k] = so;
            so += nseq[k];
            v_off[k] = vwords;
            vwords += (g.N + 3u) & ~3u;
            max_N = std::max(max_N, g.N);
        }
        uint64_t poly_words_max = 0;
        for (size_t k = 0; k < nb; ++k) poly_words_max += (hg[todo[b0 + k]].mexp + 2u) / 64u + 4u;
        DevBuf d_seq, d_v[2], d_jobs, d_poly;
        JCU(cudaMalloc(&d_seq.p, 4ull * words), "sequence scratch");
        JCU(cudaMalloc(&d_v[0].p, 4ull * vwords), "state scratch");
        JCU(cudaMalloc(&d_v[1].p, 4ull * vwords), "state scratch");
        JCU(cudaMalloc(&d_jobs.p, sizeof(DevJump) * nb), "job list");
        JCU(cudaMalloc(&d_poly.p, 8ull * poly_words_max), "polynomials");
        std::vector<f2::Poly> psi(nb, f2::Poly{1u});
        std::vector<uint8_t> done(nb, 0);
        std::vector<uint32_t> host_seq(words);
        std::vector<DevJump> jobs(nb);
        std::vector<uint32_t> hv(vwords);
        int cur = -1;                         // -1: sources are the generator states
        for (int pass = 0;; ++pass) {
            std::vector<size_t> act;
            for (size_t k = 0; k < nb; ++k)
                if (!done[k]) act.push_back(k);
            if (act.empty()) break;
            if (pass >= kPasses) return jfail(MTGP_EINVAL, "jump-ahead: annihilating polynomial did not converge");
            // walk 2 mexp + 3 words from each source
            for (size_t a = 0; a < act.size(); ++a) {
                const size_t k = act[a];
                const uint32_t g = todo[b0 + k];
                DevJump j{};
                j.gen = g;
                j.src = cur < 0 ? hg[g].state_off : v_off[k];
                j.seq = seq_off[k];
                j.nseq = (uint32_t)nseq[k];
                jobs[a] = j;
            }
            JCU(cudaMemcpyAsync(d_jobs.p, jobs.data(), sizeof(DevJump) * act.size(), cudaMemcpyHostToDevice, s),
                "upload jobs");
            JCU(launch_walk(d_gens, cur < 0 ? d_state : (const uint32_t *)d_v[cur].p, (uint32_t *)d_seq.p,
                            (const DevJump *)d_jobs.p, (uint32_t)act.size(), max_N, s),
                "walk kernel");
            JCU(cudaMemcpyAsync(host_seq.data(), d_seq.p, 4ull * words, cudaMemcpyDeviceToHost, s), "read walk");
            JCU(cudaStreamSynchronize(s), "walk");
            // minimal polynomial of the functional's sequence, per generator
            const uint32_t fmask = pass_mask(pass);
            std::vector<f2::Poly> phi(act.size());
            std::atomic<bool> oom{false};
            parallel_for(act.size(), [&](size_t a) {
                try {
                    const size_t k = act[a];
                    const uint64_t nbits = 2ull * hg[todo[b0 + k]].mexp + 2u;
                    std::vector<uint64_t> bits((size_t)(nbits / 64u) + 1u, 0u);
                    const uint32_t *x = host_seq.data() + seq_off[k];
                    for (uint64_t i = 0; i < nbits; ++i)
                        bits[i >> 6] |= (uint64_t)__builtin_parity(x[i + 1u] & fmask) << (i & 63u);
                    phi[a] = f2::minpoly(bits.data(), nbits);
                } catch (const std::exception &) {
                    oom = true;
                }
            });
            if (oom) return jfail(MTGP_ENOMEM, "jump-ahead: host allocation");
            // V = phi(F) source, from the same walk
            std::vector<uint64_t> hpoly;
            std::vector<uint64_t> poff(act.size());
            for (size_t a = 0; a < act.size(); ++a) {
                poff[a] = hpoly.size();
                hpoly.insert(hpoly.end(), phi[a].begin(), phi[a].end());
                hpoly.push_back(0u);
                hpoly.push_back(0u);
            }
            for (size_t a = 0; a < act.size(); ++a) {
                const size_t k = act[a];
                jobs[a].poly = (const uint64_t *)d_poly.p + poff[a];
                jobs[a].ncoef = (uint32_t)(f2::degree(phi[a]) + 1);
                jobs[a].dst = v_off[k];
                jobs[a].mode = kJumpSum;
                if (jobs[a].ncoef == 0u) return jfail(MTGP_EINVAL, "jump-ahead: zero polynomial");
            }
            const int nxt = cur == 0 ? 1 : 0;
            JCU(cudaMemcpyAsync(d_poly.p, hpoly.data(), 8ull * hpoly.size(), cudaMemcpyHostToDevice, s),
                "upload polynomials");
            JCU(cudaMemcpyAsync(d_jobs.p, jobs.data(), sizeof(DevJump) * act.size(), cudaMemcpyHostToDevice, s),
                "upload jobs");
            JCU(launch_jump_sum(d_gens, (const uint32_t *)d_seq.p, (uint32_t *)d_v[nxt].p,
                                (const DevJump *)d_jobs.p, (uint32_t)act.size(), max_N, s),
                "sum kernel");
            JCU(cudaMemcpyAsync(hv.data(), d_v[nxt].p, 4ull * vwords, cudaMemcpyDeviceToHost, s), "read sums");
            JCU(cudaStreamSynchronize(s), "sum");
            // the next pass reads the sums from d_v[nxt]; generators that are
            // done keep their (zero) sums there, which is harmless
            for (size_t a = 0; a < act.size(); ++a) {
                const size_t k = act[a];
                const DevGen &g = hg[todo[b0 + k]];
                psi[k] = f2::mul(psi[k], phi[a]);
                const uint32_t *v = hv.data() + v_off[k];
                bool zero = (v[0] & g.mask) == 0u;
                for (uint32_t j = 1; zero && j < g.N; ++j) zero = v[j] == 0u;
                if (zero) done[k] = 1;
                if (f2::degree(psi[k]) > (int64_t)g.mexp)
                    return jfail(MTGP_EINVAL, "jump-ahead: annihilating polynomial above the state dimension");
            }
            cur = nxt;
        }
        for (size_t k = 0; k < nb; ++k) jc.ann[todo[b0 + k]] = std::move(psi[k]);
        b0 = b1;
    }
    return MTGP_OK;
}

int jump_polys(JumpCache &jc, const std::vector<std::pair<uint32_t, uint64_t>> &need)
{
    // missing (gen, J), grouped by generator, J ascending
    std::map<uint32_t, std::vector<uint64_t>> miss;
    for (const auto &k : need) {
        if (k.second == 0u) continue;
        if (k.first >= jc.ann.size() || jc.ann[k.first].empty())
            return jfail(MTGP_EINVAL, "jump-ahead: annihilating polynomial not computed");
        if (!jc.polys.count(k)) miss[k.first].push_back(k.second);
    }
    if (miss.empty()) return MTGP_OK;
    std::vector<uint32_t> gl;
    std::vector<std::vector<uint64_t>> jl;
    for (auto &kv : miss) {
        std::sort(kv.second.begin(), kv.second.end());
        kv.second.erase(std::unique(kv.second.begin(), kv.second.end()), kv.second.end());
        gl.push_back(kv.first);
        jl.push_back(kv.second);
    }
    // g_J = x^(J-1) mod psi; consecutive J with a repeated gap share x^gap
    std::vector<std::vector<f2::Poly>> res(gl.size());
    std::atomic<bool> oom{false};
    parallel_for(gl.size(), [&](size_t t) {
        try {
            const f2::Modulus M = f2::make_modulus(jc.ann[gl[t]]);
            std::vector<f2::Poly> &out = res[t];
            uint64_t Jp = 1, gap = 0;
            f2::Poly gp{1u}, xgap;
            for (uint64_t J : jl[t]) {
                const uint64_t d = J - Jp;
                f2::Poly g;
                if (d == 0) {
                    g = gp;
                } else if (d == gap) {
                    g = f2::mulmod(gp, xgap, M);
                } else if (Jp == 1u) {
                    g = f2::xpow_mod(d, M);
                    xgap = f2::mulx_mod(g, M);            // x^J = x^gap when the next gap is J
                    gap = J;
                } else {
                    xgap = f2::xpow_mod(d, M);
                    gap = d;
                    g = f2::mulmod(gp, xgap, M);
                }
                f2::trim(g);
                out.push_back(g);
                gp = g;
                Jp = J;
            }
            if (M.D == 0u)                                  // psi = 1: the state is zero
                for (auto &g : out) g.clear();
        } catch (const std::exception &) {
            oom = true;
        }
    });
    if (oom) return jfail(MTGP_ENOMEM, "jump-ahead: host allocation");
    std::vector<uint64_t> host;
    std::vector<std::pair<size_t, uint32_t>> at;     // word offset, ncoef
    for (size_t t = 0; t < gl.size(); ++t)
        for (const f2::Poly &g : res[t]) {
            at.emplace_back(host.size(), (uint32_t)(f2::degree(g) + 1));
            host.insert(host.end(), g.begin(), g.end());
            host.push_back(0u);
            host.push_back(0u);
        }
    void *chunk = nullptr;
    JCU(cudaMalloc(&chunk, 8ull * host.size()), "polynomial store");
    cudaError_t e = cudaMemcpy(chunk, host.data(), 8ull * host.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(chunk);
        return jcuda(e, "upload polynomials");
    }
    jc.chunks.push_back(chunk);
    jc.dev_bytes += 8ull * host.size();
    size_t q = 0;
    for (size_t t = 0; t < gl.size(); ++t)
        for (size_t u = 0; u < jl[t].size(); ++u, ++q) {
            JumpPoly jp;
            jp.d = (const uint64_t *)chunk + at[q].first;
            jp.ncoef = at[q].second;
            jc.polys[{gl[t], jl[t][u]}] = jp;
        }
    return MTGP_OK;
}

JumpPoly jump_poly(const JumpCache &jc, uint32_t gen, uint64_t J)
{
    auto it = jc.polys.find({gen, J});
    return it == jc.polys.end() ? JumpPoly{} : it->second;
}

void jump_clear(JumpCache &jc, bool all)
{
    for (void *c : jc.chunks) cudaFree(c);
    jc.chunks.clear();
    jc.polys.clear();
    jc.dev_bytes = 0;
    if (all)
        for (auto &a : jc.ann) a.clear();
}

}  // namespace mtgp
