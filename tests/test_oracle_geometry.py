"""Pins of the oracle's geometry: located cells and distances to the nearest
boundary against brute-force classification and ray marching (csg_brute)."""
import numpy as np
import pytest

import workloads as W
from oracle import Oracle
from tests.csg_brute import brute_distance, classify


def _problems():
    return {
        "pin": (W.pin_cell_mg(n=10), [-0.63, 0.63, -0.63, 0.63, -5, 5], 1e-4, 3.0),
        "lattice": (W.c5g7_like_lattice(n=10), [0, 64.26, 0, 64.26, -5, 5], 1e-4, 4.0),
        "slab": (W.diff_slab(n=10), [0, 30, -1, 1, -1, 1], 2e-4, 8.0),
        "box0": (W.batch_boxes(nproblems=3)[0], None, 5e-4, None),
        "box2": (W.batch_boxes(nproblems=3)[2], None, 5e-4, None),
    }


@pytest.mark.parametrize("name", ["pin", "lattice", "slab", "box0", "box2"])
def test_locate_and_distance_vs_brute_force(orc, name):
    pb, box, h, tcap = _problems()[name]
    if box is None:
        xs = [s["coef"][0] for s in pb["surfaces"] if s["type"] == "px"]
        ys = [s["coef"][0] for s in pb["surfaces"] if s["type"] == "py"]
        zs = [s["coef"][0] for s in pb["surfaces"] if s["type"] == "pz"]
        box = [min(xs), max(xs), min(ys), max(ys), min(zs), max(zs)]
    o = Oracle(pb)
    rng = np.random.default_rng(abs(hash(name)) % 2**32)
    nc = len(pb["cells"])
    checked = 0
    for _ in range(60):
        pos = np.array([rng.uniform(box[0], box[1]), rng.uniform(box[2], box[3]),
                        rng.uniform(box[4], box[5])])
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        code = classify(pb, pos[None, :])[0]
        path, dist, kind = o.probe(pos, d)
        # located path equals brute-force classification
        root = int(path[0])
        path = [int(v) for v in path]
        if pb["cells"][root]["fill_kind"] == "lattice":
            expect = (root * (nc + 1) + path[3] + 1) * 10**7 + path[1] * 3000 + path[2]
        else:
            expect = root * (nc + 1) * 10**7
        assert code == expect
        tmax = min(dist * 1.2 + 10 * h, tcap if tcap else dist * 1.2 + 10 * h)
        bd = brute_distance(pb, pos, d, tmax, h)
        if np.isinf(bd):
            assert dist > tmax - 10 * h
        else:
            assert abs(bd - dist) < 1e-9 * max(1.0, dist), (pos, d, bd, dist, kind)
        checked += 1
    assert checked == 60
