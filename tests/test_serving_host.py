"""Host-side serving logic without a GPU: the horizon route sends each request
to its model's server with the smallest horizon that holds it; the request-loop
entry points reject a missing server before touching the device."""
import pytest

import workloads as W
from paper_2603_10711_gb300 import serving


def test_horizon_route_picks_the_smallest_bucket_that_holds_the_request():
    route = serving.horizon_route({1: (40, 72, 120), 2: (100, 200)})
    for N, key in ((30, (1, 40)), (40, (1, 40)), (41, (1, 72)), (72, (1, 72)), (73, (1, 120)), (120, (1, 120))):
        assert route(W.quad_box(1, seed=1, N_range=(N, N), obs_range=(5, 5))) == key
    for N, key in ((50, (2, 100)), (100, (2, 100)), (101, (2, 200)), (200, (2, 200))):
        assert route(W.mars_batch(1, seed=1, N=N)) == key
    with pytest.raises(ValueError):                       # no bucket holds it
        route(W.mars_batch(1, seed=1, N=201))


def test_loop_entry_points_reject_a_null_server():
    from paper_2603_10711_gb300 import build, ucn
    build.build()
    L = serving._setup(ucn.lib())
    assert L.ucn_serve_loop_start(None, 0, 1.0) == ucn.UCN_EINVAL
    assert "null server" in ucn.ucn_last_error()
    assert L.ucn_serve_loop_stop(None) == ucn.UCN_EINVAL
    assert L.ucn_serve_loop_launches(None) == -1
    assert L.ucn_serve_loop_capacity(None) == -1


def test_device_use_counts_the_solves_running_at_once():
    # spans in ns: two overlap, a third starts when the first has ended (an end at the
    # same instant as a start does not count as overlap)
    d = serving.device_use([(0, 10), (5, 15), (10, 20)])
    assert d["max_running"] == 2
    assert abs(d["span_s"] - 20e-9) < 1e-15
    assert abs(d["mean_running"] - 30.0 / 20.0) < 1e-12
    assert serving.device_use([(3, 4)])["max_running"] == 1


def test_server_names_of_stream_keys():
    assert serving.server_name((1, 40)) == "1/40"
    assert serving.server_name(2) == "2"
