"""Shared test plumbing: builds the same workload on both sides from a recipe.

The CUDA side draws its parameter sets with the library's mtgp_params_draw and
the oracle side with the oracle's own drawer; nothing computed by one side is
fed to the other.
"""
import numpy as np

import oracle as O


def oracle_params(spec):
    return O.params_draw(spec.mexp, spec.param_seed, spec.id)


def oracle_state(spec):
    p = oracle_params(spec)
    return p, O.seed_state(p, spec.gen_id, spec.seed)


def oracle_stream(spec, segments):
    """Outputs of consecutive (dtype, n) segments of one generator, and its final state."""
    p, st = oracle_state(spec)
    outs = [O.generate(p, st, n, dt) for dt, n in segments]
    return outs, st


def lib_pool(gens, stream=None):
    import paper_1005_4973_gb300 as M
    ps = [M.mtgp_params_draw(g.mexp, g.param_seed, g.id) for g in gens]
    return M.Pool(ps, [g.gen_id for g in gens], [g.seed for g in gens], stream=stream)


def as_u32(t):
    return t.view(dtype=__import__("torch").int32).cpu().numpy().view(np.uint32)
