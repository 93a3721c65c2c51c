"""Writes the stored expected values under tests/golden/ from the oracle only.

  full_period_sets.json   parameter sets of reduced exponent found by the small
                          MTGPDC recursion search (Sec. 5): the Berlekamp-Massey
                          minimal polynomial has degree p and is irreducible.
  oracle_digests.json     SHA-256 of oracle outputs for the 2^20-output
                          MTGP11213 workload (param seed 1, id 0, generator 0,
                          seed 1234) and the first state words of two seeds.
                          These are project-defined values (the paper prints no
                          output); they guard the oracle against accidental change.

Run:  python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402

SEARCH = [(89, 1000, 7), (107, 1000, 7), (127, 1000, 7), (521, 1000, 7), (607, 1000, 7),
          (1279, 1000, 7), (521, 5000, 0x12345678), (607, 9000, 0xCAFEF00D)]


def main():
    sets = []
    for mexp, seed0, gid in SEARCH:
        p, seed, tries = O.search_full_period(mexp, seed0, gid)
        sets.append(dict(mexp=mexp, N=p.N, r=p.r, pos=p.pos, sh1=p.sh1, sh2=p.sh2, id=p.id,
                         R=[int(x) for x in p.R], T=[int(x) for x in p.T],
                         param_seed=seed, tries=tries))
        print(mexp, seed, tries)
    with open(os.path.join(HERE, "full_period_sets.json"), "w") as f:
        json.dump({"source": "oracle.search_full_period (Sec. 5 search at reduced size)",
                   "sets": sets}, f, indent=1)

    p = O.params_draw(11213, 1, 0)
    dig = {}
    for name, dt in (("u32", O.U32), ("f12", O.F12), ("f01", O.F01)):
        st = O.seed_state(p, 0, 1234)
        out = O.generate(p, st, 1 << 20, dt)
        dig[name] = hashlib.sha256(out.tobytes()).hexdigest()
        dig[name + "_state_after"] = hashlib.sha256(st.tobytes()).hexdigest()
    first = {str(s): [int(x) for x in O.seed_state(p, 0, s)[:8]] for s in (1, 1234)}
    with open(os.path.join(HERE, "oracle_digests.json"), "w") as f:
        json.dump({"source": "oracle (project-defined; no printed outputs exist in the paper)",
                   "workload": "mexp 11213, param_seed 1, id 0, gen_id 0, seed 1234, n 2^20",
                   "sha256": dig, "seed_state_first8": first}, f, indent=1)


if __name__ == "__main__":
    main()
