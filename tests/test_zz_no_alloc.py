"""GPU test of mtgp_generate_noalloc, the entry point for callers that must not
allocate device memory themselves or through this library: code running inside
a framework whose own allocator already reserves the GPU's memory, loops that
cannot afford the device-wide synchronisation cudaMalloc and cudaFree may
cause, and programs under a fixed memory budget.  Such a caller passes its own
state and output buffers; this test checks that the result is exactly what the
allocating pool path (mtgp_pool_generate) produces, over two calls in a row
that continue the same generator streams.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _lib():
    from paper_1005_4973_gb300 import build
    build.build()
    import paper_1005_4973_gb300 as M
    from paper_1005_4973_gb300 import _lib as L
    return M, L


def _noalloc(L, ps, states, offsets, reqs, out, stream):
    parr = (L.mtgp_params * len(ps))(*ps)
    offs = (ctypes.c_uint64 * len(offsets))(*offsets)
    rarr = L.requests_array(reqs)
    return L.LIB.mtgp_generate_noalloc(parr, len(ps), states.data_ptr(), offs, rarr, len(reqs),
                                       out.data_ptr(), stream)


@pytest.mark.gpu
def test_noalloc_matches_pool_path_over_two_calls():
    M, L = _lib()
    assert torch.cuda.is_available()
    specs = [(11213, 1, 0, 1234), (23209, 2, 1, 99), (44497, 3, 2, 7), (521, 4, 3, 5)]
    ps = [M.mtgp_params_draw(m, s, i) for m, s, i, _ in specs]
    pool = M.Pool(ps, [i for _, _, i, _ in specs], [sd for *_, sd in specs])   # reference path
    # caller-owned state buffer, each state 16-byte aligned, filled with the seeded states
    offsets, off = [], 0
    for p in ps:
        offsets.append(off)
        off += (p.N + 3) // 4 * 4
    states = torch.zeros(off, dtype=torch.int32, device="cuda")
    for i, p in enumerate(ps):
        states[offsets[i]:offsets[i] + p.N] = torch.from_numpy(pool.read_state(i).view(np.int32)).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    calls = [
        [(0, 0, 100003, 0), (1, 2, 5000, 100003), (2, 1, 70001, 105003), (0, 1, 777, 175004),
         (3, 0, 20000, 175781)],
        [(2, 0, 1, 0), (0, 2, 333333, 1), (1, 0, 4097, 333334), (3, 1, 12345, 337431), (2, 2, 64, 349776)],
    ]
    for reqs in calls:
        total = sum(r[2] for r in reqs)
        got = torch.full((total,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
        ref = torch.full((total,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
        assert _noalloc(L, ps, states, offsets, reqs, got, stream) == L.MTGP_OK, L.last_error()
        pool.generate(reqs, ref)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)                     # bit-exact: every output is an exact pattern
    for i, p in enumerate(ps):                           # both paths advanced the streams alike
        assert np.array_equal(states[offsets[i]:offsets[i] + p.N].cpu().numpy().view(np.uint32),
                              pool.read_state(i))
    pool.close()


@pytest.mark.gpu
def test_noalloc_rejects_calls_beyond_its_scratch():
    M, L = _lib()
    p = M.mtgp_params_draw(11213, 1, 0)
    n = L.MTGP_NOALLOC_MAX_GENS + 1
    ps = [p] * n
    states = torch.zeros(n * 352, dtype=torch.int32, device="cuda")
    out = torch.zeros(16, dtype=torch.int32, device="cuda")
    st = _noalloc(L, ps, states, [352 * i for i in range(n)], [(0, 0, 16, 0)], out,
                  torch.cuda.current_stream().cuda_stream)
    assert st == L.MTGP_EINVAL and "scratch limit" in L.last_error()
    reqs = [(0, 0, 1, k) for k in range(L.MTGP_NOALLOC_MAX_REQS + 1)]
    st = _noalloc(L, ps[:1], states, [0], reqs, out, torch.cuda.current_stream().cuda_stream)
    assert st == L.MTGP_EINVAL and "scratch limit" in L.last_error()


@pytest.mark.gpu
def test_noalloc_refuses_a_stream_under_capture():
    # the records are copied out of the call's own host memory, so a captured
    # copy would replay from memory that is gone: the call is refused before it
    # touches the stream, and the next call on that stream runs normally
    M, L = _lib()
    p = M.mtgp_params_draw(11213, 1, 0)
    pool = M.Pool([p], [0], [1234])
    states = torch.zeros(352, dtype=torch.int32, device="cuda")
    states[:p.N] = torch.from_numpy(pool.read_state(0).view(np.int32)).cuda()
    out = torch.zeros(4096, dtype=torch.int32, device="cuda")
    ref = torch.zeros(4096, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        st = _noalloc(L, [p], states, [0], [(0, 0, 4096, 0)], out, s.cuda_stream)
        torch.zeros(4, device="cuda").add_(1)        # keeps the captured graph non-empty
    assert st == L.MTGP_EINVAL and "captur" in L.last_error()
    assert _noalloc(L, [p], states, [0], [(0, 0, 4096, 0)], out, s.cuda_stream) == L.MTGP_OK
    pool.generate([(0, 0, 4096, 0)], ref)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    pool.close()


def test_noalloc_refuses_overlapping_state_ranges():
    # Two generators whose N-word states overlap would run in two blocks that
    # read and write the same words at once.  The call refuses them on the
    # host, before it touches the device, so this runs without a GPU (the
    # buffer addresses below are never dereferenced).
    from paper_1005_4973_gb300 import build
    build.build()
    from paper_1005_4973_gb300 import _lib as L
    import paper_1005_4973_gb300 as M
    p = M.mtgp_params_draw(11213, 1, 0)
    q = M.mtgp_params_draw(11213, 2, 1)
    fake_states, fake_out = 0x10000, 0x20000
    parr = (L.mtgp_params * 2)(p, q)
    rarr = L.requests_array([(0, 0, 16, 0), (1, 0, 16, 16)])
    for offs in ([0, 100], [350, 0], [0, 0], [400, 50]):
        o = (ctypes.c_uint64 * 2)(*offs)
        st = L.LIB.mtgp_generate_noalloc(parr, 2, fake_states, o, rarr, 2, fake_out, None)
        assert st == L.MTGP_EINVAL and "overlap" in L.last_error(), offs
