"""Writes the oracle regression fixtures in this folder (calls only the oracle).

Run from the repository root:  python tests/golden/make_golden.py
A change to any stored value must come with a change to the oracle's
arithmetic that names the passage or reading that justifies it.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def pin_cell_small(strict=False):
    pb = W.pin_cell_mg(n=1000, inactive=2, active=3)
    o = oracle.Oracle(pb, strict=strict).run(threads=1)
    ktl, kc, m = o.cycle_k(5)
    h = o.histories()
    b = o.bank()
    mode = "strict" if strict else "plain"
    return {
        "what": f"oracle ({mode} arithmetic), multigroup pin cell (seed 1), 1000 particles/cycle, "
                "2+3 cycles, 1 thread",
        "bank_size": m.tolist(), "k_tl": ktl.tolist(), "k_col": kc.tolist(),
        "rng_end_first16": [int(v) for v in h["rng_end"][:16]],
        "n_coll_first16": h["n_coll"][:16].tolist(), "n_cross_first16": h["n_cross"][:16].tolist(),
        "bank_xyz_first4": b["xyz"][:4].tolist(),
    }


def rng_words():
    out = []
    for sid in [0, 1, 2, 1000, (7 << 32) + 3]:
        s = oracle.rng_stream(1, sid)
        words = []
        for _ in range(4):
            s = oracle.rng_next(s)
            words.append(int(s))
        out.append({"stream": sid, "words": words})
    return {"what": "oracle stream words, seed 1, first 4 draws", "streams": out}


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_pin_cell_small.json"), "w") as f:
        json.dump(pin_cell_small(), f, indent=1)
    with open(os.path.join(HERE, "oracle_pin_cell_small_strict.json"), "w") as f:
        json.dump(pin_cell_small(strict=True), f, indent=1)
    with open(os.path.join(HERE, "oracle_rng_words.json"), "w") as f:
        json.dump(rng_words(), f, indent=1)
