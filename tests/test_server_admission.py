"""The server's admission policy, on the host (no GPU): RHServer._admit run on a
stand-in object with grids, an arena and a queue of sized requests.

* a round opens with the oldest waiting request and takes, in arrival order, the
  requests of grids whose n_x is within mix_ratio of it, while they fit;
* requests of other size classes, and those that no longer fit, keep their
  places at the front of the queue;
* a request larger than an arena is refused on its future; mix_ratio = 0 mixes any.
"""
import collections
import concurrent.futures as cf
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")
from paper_2201_00241_gb300.server import RHServer, _Req  # noqa: E402


def stand_in(mix_ratio=2.0, max_batch=8, io=1000, work=10_000):
    grids = {"small": types.SimpleNamespace(n_x=181, n_p=107), "mid": types.SimpleNamespace(n_x=300, n_p=107),
             "big": types.SimpleNamespace(n_x=17036, n_p=2889)}
    srv = types.SimpleNamespace(grids=grids, max_batch=max_batch, mix_ratio=mix_ratio, waited_for_budget=0,
                                _q=collections.deque())
    arena = types.SimpleNamespace(io=io, work=work)
    return srv, arena


def req(name, n_io, n_work, tag):
    r = _Req(name, np.zeros((1, 1)), cf.Future(), float(tag))
    r.n_io, r.n_work = n_io, n_work
    return r


def admit(srv, arena):
    return RHServer._admit(srv, arena)


def test_round_takes_one_size_class_in_arrival_order():
    srv, a = stand_in()
    q = [req("small", 10, 10, 0), req("big", 100, 100, 1), req("mid", 10, 10, 2), req("small", 10, 10, 3),
         req("big", 100, 100, 4)]
    srv._q.extend(q)
    b1 = admit(srv, a)
    assert [r.t_arrival for r in b1] == [0, 2, 3]            # small and mid (n_x within 2x), in order
    assert [r.t_arrival for r in srv._q] == [1, 4]           # the big ones keep their order
    b2 = admit(srv, a)
    assert [r.t_arrival for r in b2] == [1, 4] and not srv._q


def test_budget_and_batch_limits_keep_the_rest_in_place():
    srv, a = stand_in(io=25, max_batch=8)
    srv._q.extend([req("small", 10, 10, k) for k in range(5)])
    b = admit(srv, a)
    assert [r.t_arrival for r in b] == [0, 1] and srv.waited_for_budget == 1
    assert [r.t_arrival for r in srv._q] == [2, 3, 4]
    srv, a = stand_in(max_batch=2)
    srv._q.extend([req("small", 10, 10, k) for k in range(5)])
    assert [r.t_arrival for r in admit(srv, a)] == [0, 1] and len(srv._q) == 3


def test_oversize_request_is_refused_and_any_mix_when_ratio_is_zero():
    srv, a = stand_in(mix_ratio=0.0)
    too_big = req("big", 5000, 10, 0)
    srv._q.extend([too_big, req("small", 10, 10, 1), req("big", 100, 100, 2)])
    b = admit(srv, a)
    assert too_big.future.done() and isinstance(too_big.future.exception(), ValueError)
    assert [r.t_arrival for r in b] == [1, 2] and not srv._q
