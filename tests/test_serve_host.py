"""Host-side request checks of the serving loop (no GPU: a server with no
slots never touches the device)."""

import types

import pytest
import torch

from paper_1902_09465_gb300 import serve


def _server(method="adaptive"):
    ds = types.SimpleNamespace(n=1000, m=16)
    return serve.Server([ds], [serve.DatasetConfig(method=method)], slots=0)


def test_well_formed_requests_are_queued():
    s = _server()
    s.submit(serve.Request(rid=0, dataset=0, Q=torch.zeros(3, 16), k=10))
    s.submit(serve.Request(rid=1, dataset=0, Q=torch.zeros(1, 16), k=512))
    assert len(s.queue) == 2 and s.queue[0].t_arrival > 0


@pytest.mark.parametrize("bad", [
    dict(dataset=1),                                   # no such dataset
    dict(Q=torch.zeros(3, 15)),                        # wrong dimension
    dict(Q=torch.zeros(0, 16)),                        # no query
    dict(Q=torch.zeros(3, 16, dtype=torch.float64)),   # wrong dtype
    dict(Q=torch.zeros(16)),                           # not 2-D
    dict(k=0), dict(k=513), dict(k=1001),              # k outside [1, min(n, 512)]
])
def test_malformed_requests_are_refused_at_submit(bad):
    s = _server()
    req = dict(rid=7, dataset=0, Q=torch.zeros(3, 16), k=10)
    req.update(bad)
    with pytest.raises(ValueError):
        s.submit(serve.Request(**req))
    assert not s.queue


def test_exact_engine_allows_the_full_candidate_limit():
    s = _server("exact")
    s.submit(serve.Request(rid=0, dataset=0, Q=torch.zeros(1, 16), k=1000))
    with pytest.raises(ValueError):
        s.submit(serve.Request(rid=1, dataset=0, Q=torch.zeros(1, 16), k=1001))


def test_dataset_options_reach_the_launch():
    ds = types.SimpleNamespace(n=1000, m=16)
    s = serve.Server([ds, ds], [serve.DatasetConfig(c_alpha=3e-4, B0=16, threads=1024),
                                serve.DatasetConfig(replace=False)], slots=0)
    o0, o1 = s._opts(0), s._opts(1)
    assert o0["c_alpha"] == 3e-4 and o0["B0"] == 16 and o0["threads"] == 1024 and "replace" not in o0
    assert o1["replace"] is False and "share_points" not in o1
