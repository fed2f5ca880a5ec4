"""Host-side serving logic without a GPU: the horizon route sends each request
to its model's server with the smallest horizon that holds it."""
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
