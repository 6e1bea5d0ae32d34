"""Host-side serving statistics (no GPU): requests that were never finished count as not served
and as infinitely late in the latency percentiles."""
import numpy as np


def _req(i, kind, t_arr, t_done, W=640, H=480, iters=0):
    from paper_2605_31419_gb300.serve import Request
    r = Request(i, kind, np.array([525.0, 525.0, W / 2, H / 2, W, H]), np.zeros(12), t_arr)
    r.t_done = t_done
    r.iters_done = iters
    return r


def test_latency_stats_counts_not_served_requests():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2605_31419_gb300.serve import latency_stats
    renders = [_req(i, "render", 0.01 * i, 0.01 * i + 0.005) for i in range(98)]
    renders += [_req(98, "render", 0.98, -1.0), _req(99, "render", 0.99, -1.0)]  # never finished
    tracks = [_req(100 + i, "track", 0.02 * i, 0.02 * i + 0.05, iters=10) for i in range(50)]
    st = latency_stats(renders + tracks, seconds=2.0)
    r = st["render"]
    assert (r["n"], r["not_served"], r["submitted"]) == (98, 2, 100)
    assert abs(r["p50_ms"] - 5.0) < 1e-6
    assert r["p99_ms"] is None and r["p99_not_served"]  # 2 % of the renders were not served
    t = st["track"]
    assert t["not_served"] == 0 and abs(t["p99_ms"] - 50.0) < 1e-6
    assert st["not_served"] == 2 and st["completed"] == 148 and st["submitted"] == 150
    px = 98 * 640 * 480 + 50 * 10 * 640 * 480
    assert abs(st["mpix_s"] - px / 2.0 / 1e6) < 1e-9
