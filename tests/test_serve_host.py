"""The serving loop's admission policy, on the host alone: streams are
stand-ins and launches are recorded instead of run, so no GPU is needed.
Batches take requests of the head's kind in arrival order, up to max_batch,
while their memory estimate fits the budget; a request that does not fit
waits for memory to free up unless nothing is in flight (then it runs
alone, so the server always makes progress); without a free stream nothing
is admitted; the segment estimate learns from observed statistics."""
import types

import numpy as np
import pytest
import torch

from paper_2603_00413_gb300 import serve


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_00413_gb300 import build
    build.build()


def _server(monkeypatch, budget, max_batch=8, streams=2):
    monkeypatch.setattr(torch.cuda, "Stream", lambda device=None: object())
    scenes = [types.SimpleNamespace(V=torch.zeros(500, 3)), types.SimpleNamespace(V=torch.zeros(2000, 3))]
    srv = serve.Server(scenes, budget, max_batch=max_batch, streams=streams, device=torch.device("cpu"))
    launched = []

    def fake_launch(reqs, mem):
        srv.free_streams.popleft()
        srv.mem_used += mem
        srv.inflight.append((reqs, mem))
        launched.append(([r.rid for r in reqs], mem))

    srv._launch = fake_launch
    return srv, launched


def _req(rid, kind="render", side=128, depth=6, scene=0):
    return serve.Request(rid=rid, scene=scene, cam=np.zeros(10, np.float32), width=side, height=side, depth=depth,
                         kind=kind, arrival=0.001 * rid)


def test_batches_group_the_head_kind_in_arrival_order(monkeypatch):
    srv, launched = _server(monkeypatch, budget=1 << 40)
    kinds = ["render", "grad", "render", "render", "grad"]
    srv.pending.extend(_req(i, k) for i, k in enumerate(kinds))
    srv._admit()
    assert [ids for ids, _ in launched] == [[0, 2, 3], [1, 4]]
    assert not srv.pending and not srv.free_streams


def test_max_batch_caps_a_batch(monkeypatch):
    srv, launched = _server(monkeypatch, budget=1 << 40, max_batch=4, streams=3)
    srv.pending.extend(_req(i) for i in range(6))
    srv._admit()
    assert [ids for ids, _ in launched] == [[0, 1, 2, 3], [4, 5]]


def test_memory_budget_splits_batches_and_waits(monkeypatch):
    srv, _ = _server(monkeypatch, budget=1 << 40)
    m = srv._mem_estimate(_req(0))
    srv, launched = _server(monkeypatch, budget=int(2.5 * m))
    srv.pending.extend(_req(i) for i in range(5))
    srv._admit()
    # two fit; the third waits for memory although a stream is free
    assert [ids for ids, _ in launched] == [[0, 1]]
    assert [r.rid for r in srv.pending] == [2, 3, 4] and srv.free_streams
    assert launched[0][1] == 2 * m and srv.mem_used == 2 * m
    # memory freed: the next two go
    srv.inflight.clear()
    srv.mem_used = 0
    srv.free_streams.append(object())
    srv._admit()
    assert [ids for ids, _ in launched] == [[0, 1], [2, 3]]


def test_an_oversized_request_runs_alone_when_nothing_is_in_flight(monkeypatch):
    srv, _ = _server(monkeypatch, budget=1 << 40)
    big = srv._mem_estimate(_req(0, side=1024))
    srv, launched = _server(monkeypatch, budget=big // 4)
    srv.pending.extend([_req(0, side=1024), _req(1, side=64)])
    srv._admit()
    assert [ids for ids, _ in launched] == [[0]]
    assert [r.rid for r in srv.pending] == [1]  # waits behind the oversized batch


def test_nothing_is_admitted_without_a_free_stream(monkeypatch):
    srv, launched = _server(monkeypatch, budget=1 << 40, streams=1)
    srv.pending.extend([_req(0, "grad"), _req(1, "render")])
    srv._admit()
    assert [ids for ids, _ in launched] == [[0]]
    assert [r.rid for r in srv.pending] == [1]


def test_gradient_requests_are_charged_more_and_estimates_learn(monkeypatch):
    srv, _ = _server(monkeypatch, budget=1 << 40)
    r, g = _req(0, "render", scene=1), _req(1, "grad", scene=1)
    assert srv._mem_estimate(g) > srv._mem_estimate(r)
    # before any statistics: 2 depth + 3 segments per pixel (at most 24)
    assert srv._seg_estimate(r) == 128 * 128 * 15 + 1024
    assert srv._seg_estimate(_req(2, depth=20)) == 128 * 128 * 24 + 1024
    # an observed 4 segments per pixel for (scene, depth) sizes later arenas with a 25 % margin
    srv.seg_per_pixel[(1, 6)] = 4.0
    assert srv._seg_estimate(r) == 128 * 128 * 5 + 1024
    assert srv._seg_estimate(_req(3, scene=0)) == 128 * 128 * 15 + 1024
