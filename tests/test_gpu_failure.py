"""Failure detection without a GPU fault: a bounded device wait that runs out reports
TS_ERR_TIMEOUT through ts_sync_status, the context stays usable, and ts_workspace_init clears it."""
import numpy as np
import pytest

from harness import assert_images, gpu_run, oracle_run, params_pair
from ts_synth.scenes import random_triangles_scene

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_recovers(oracle):
    import paper_2605_31419_gb300 as ts
    sc = random_triangles_scene(seed=1)
    rast = ts.Rasterizer(sc.cams, sc.n_faces)
    ts.ts_debug_timeout_probe(rast.plan, rast.ws, 2000)  # a 2 ms limit on a phase nothing completes
    st = rast.counters(raise_on_error=False)
    assert st["status"] == "TS_ERR_TIMEOUT" and st["error_bits"] & 2
    with pytest.raises(ts.TsError):
        rast.counters()
    ts.ts_workspace_init(rast.plan, rast.ws)
    assert rast.counters(raise_on_error=False)["status"] == "TS_OK"
    # the same process renders correctly afterwards
    p, po = params_pair()
    g = gpu_run(sc, p, backward=False)
    r = oracle_run(oracle, sc, po, backward=False)
    assert_images(g["color"], r["color"], "color")
