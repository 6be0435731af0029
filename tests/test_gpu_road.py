"""GPU road-network cost matrix (lbdd_road_cm) against the oracle's Dijkstra,
and ASRAL on such a matrix against the oracle."""
import numpy as np
import pytest

import lbdd_inputs as L
import oracle

pytestmark = pytest.mark.gpu


def gpu_cm(lb, g):
    import torch
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()
    k, n = len(g.centers), len(g.demand)
    out = torch.zeros((n, k), dtype=torch.int32, device="cuda")
    lb.road_cm(t(g.row_ptr), t(g.col), t(g.w), t(g.centers), t(g.demand), out)
    return out.cpu().numpy()


@pytest.mark.parametrize("shape", [(9, 7, 3), (40, 30, 12), (96, 80, 40), (256, 256, 109)])
def test_road_cm_matches_dijkstra(gpu_lib, shape):
    W, H, k = shape
    g = L.road_network(400 + W, W, H, k)
    rc, ref = oracle.road_cm(g.row_ptr, g.col, g.w, g.centers, g.demand)
    assert rc == 0
    assert np.array_equal(gpu_cm(gpu_lib, g), ref)


def test_road_cm_rejects_bad_input(gpu_lib):
    g = L.road_network(7, 8, 8, 3)
    w = g.w.copy()
    w[5] = 0
    bad = L.RoadNetwork(g.V, g.row_ptr, g.col, w, g.xy, g.centers, g.demand)
    with pytest.raises(gpu_lib.LbddError):
        gpu_cm(gpu_lib, bad)
    # a node with no roads cannot be reached
    row_ptr = np.append(g.row_ptr, g.row_ptr[-1]).astype(np.int32)
    iso = L.RoadNetwork(g.V + 1, row_ptr, g.col, g.w, g.xy, g.centers,
                        np.append(g.demand, g.V).astype(np.int32))
    with pytest.raises(gpu_lib.LbddError):
        gpu_cm(gpu_lib, iso)


def test_asral_on_road_cm(gpu_lib):
    """The paper's pipeline on a small road network: CM from shortest paths,
    then ASRAL (capacities 0.7 n split at random, penalties in [1, 200])."""
    g = L.road_network(21, 48, 40, 16)
    cm = gpu_cm(gpu_lib, g)
    k, n = cm.shape[1], cm.shape[0]
    inst = L.random_small(21, n=n, k=k, cap_frac=0.7, pen=(1, 200))   # capacities and penalties
    ref = oracle.asral(cm, inst.cap, inst.pen)
    with gpu_lib.Solver(cm, inst.cap, inst.pen) as s:
        s.solve()
        assert s.objective == ref.delta
        assert np.array_equal(s.assignment(), ref.assign)
