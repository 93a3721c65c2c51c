"""Seeded synthetic workloads: which generators, parameter seeds, lengths and
dtypes each benchmark configuration uses.  Recipes only -- no part of the
MTGP arithmetic lives here; tests feed the same recipe to the CUDA library and
to the CPU oracle.

Configurations (MTGP32; every output is 4 bytes):
  C1  mexp 11213, parameter set drawn from seed 1 (ID 0), one generator
      (gen_id 0, seed 1234), 2^20 uint32 outputs.
  C2  mexp 11213, 128 parameter sets drawn from seeds 1..128 (IDs 0..127), one
      generator per set (gen_id = ID, seed 1234), 2^24 outputs each in uint32,
      float [1,2) and float [0,1); each dtype run starts from the seeded state;
      blocked layout.
  C3  mexp 23209 and 44497, 128 sets each (seeds 1..128, IDs 0..127), 2^26
      float [0,1) outputs per generator, blocked.
  C4  8192 generators, IDs 0..8191, parameter seed ID + 1, mexp uniform over
      {11213, 23209, 44497} (numpy seed 7), length floor(2^U(10, 24)),
      dtype alternating uint32 / float [0,1), blocked at prefix-sum offsets.
  C5  served: 65536 resident generators (mexp mix as C4, numpy seed 11),
      Poisson arrivals, length floor(2^U(8, 26)), dtype uint32 / float [0,1)
      50/50, generator uniform.
  paper  Sec. 4.4: 5e7 numbers of one dtype from 108 MTGP11213 generators
      (parameter seeds 1..108, IDs 0..107, seed 1234), 462,963 each (the last
      462,959), blocked.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

U32, F12, F01 = 0, 1, 2
MEXPS = (11213, 23209, 44497)
SEED = 1234


@dataclass
class GenSpec:
    """One generator: parameter set (mexp, param_seed, id) and state seeding."""
    mexp: int
    param_seed: int
    id: int
    gen_id: int
    seed: int = SEED


@dataclass
class Workload:
    name: str
    gens: list[GenSpec]
    requests: list[tuple[int, int, int, int]] = field(default_factory=list)  # (gen, dtype, n, out_offset)

    @property
    def total_numbers(self) -> int:
        return int(sum(r[2] for r in self.requests))

    @property
    def out_bytes(self) -> int:
        return 4 * self.total_numbers


def _blocked(reqs):
    out, off = [], 0
    for g, dt, n in reqs:
        out.append((g, dt, int(n), off))
        off += int(n)
    return out


def c1(n: int = 1 << 20, dtype: int = U32) -> Workload:
    return Workload("C1", [GenSpec(11213, 1, 0, 0)], _blocked([(0, dtype, n)]))


def c2(n: int = 1 << 24, dtypes=(U32, F12, F01), count: int = 128) -> Workload:
    """Each (set, dtype) pair is its own generator instance seeded identically,
    so all dtype runs start from the seeded state."""
    gens, reqs = [], []
    for dt in dtypes:
        for i in range(count):
            gens.append(GenSpec(11213, i + 1, i, i))
            reqs.append((len(gens) - 1, dt, n))
    return Workload("C2", gens, _blocked(reqs))


def paper(dtype: int = F01, total: int = 50_000_000, count: int = 108) -> Workload:
    """Sec. 4.4's speed measurement: 5e7 numbers of one dtype from 108
    MTGP11213 generators with distinct parameter sets, split as evenly as
    whole numbers allow."""
    per = -(-total // count)
    gens, reqs = [], []
    for i in range(count):
        gens.append(GenSpec(11213, i + 1, i, i))
        reqs.append((i, dtype, min(per, total - i * per)))
    return Workload("paper", gens, _blocked(reqs))


def c3(mexps=(23209, 44497), n: int = 1 << 26, count: int = 128) -> Workload:
    gens, reqs = [], []
    for mexp in mexps:
        for i in range(count):
            gens.append(GenSpec(mexp, i + 1, i, i))
            reqs.append((len(gens) - 1, F01, n))
    return Workload("C3", gens, _blocked(reqs))


def c4(count: int = 8192, lo: float = 10.0, hi: float = 24.0, seed: int = 7) -> Workload:
    rng = np.random.default_rng(seed)
    mexp = rng.choice(MEXPS, size=count)
    lens = np.floor(2.0 ** rng.uniform(lo, hi, size=count)).astype(np.int64)
    gens = [GenSpec(int(mexp[i]), i + 1, i, i) for i in range(count)]
    reqs = [(i, U32 if i % 2 == 0 else F01, int(lens[i])) for i in range(count)]
    return Workload("C4", gens, _blocked(reqs))


def c5_pool(count: int = 65536, seed: int = 11) -> list[GenSpec]:
    rng = np.random.default_rng(seed)
    mexp = rng.choice(MEXPS, size=count)
    return [GenSpec(int(mexp[i]), i + 1, i, i) for i in range(count)]


def c5_arrivals(rate_per_s: float, count: int, pool_size: int = 65536, lo: float = 8.0, hi: float = 26.0,
                seed: int = 13):
    """Poisson arrivals: (arrival_time_s, gen, dtype, n) sorted by time."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    t = np.cumsum(gaps)
    gens = rng.integers(0, pool_size, size=count)
    lens = np.floor(2.0 ** rng.uniform(lo, hi, size=count)).astype(np.int64)
    dts = np.where(rng.random(count) < 0.5, U32, F01)
    return [(float(t[i]), int(gens[i]), int(dts[i]), int(lens[i])) for i in range(count)]


def expected_log_uniform_len(lo: float, hi: float) -> float:
    """E[2^U(lo, hi)] = (2^hi - 2^lo) / ((hi - lo) ln 2)."""
    return (2.0 ** hi - 2.0 ** lo) / ((hi - lo) * np.log(2.0))
