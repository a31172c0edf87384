"""The autotuner's configurations against rh_hessvec.

Every configuration the autotuner can choose (interleave width x CTA shape x
narrow-level k-split cap x dense-tail bound) computes every item of a batched
launch equal to rh_hessvec on the same grid and W within 1e-12 of max |HW|: the
configurations change only which lanes, CTAs and dense triangles do the work, so
they differ by rounding alone.  tune() returns and caches all four choices, and
the server launches with them.
"""
import json

import numpy as np
import pytest

from paper_2201_00241_gb300 import gridgen as gg

pytestmark = pytest.mark.gpu


def _ready(name, k=None):
    from paper_2201_00241_gb300 import rh
    g = gg.make_grid(30, 41, 6, 4) if name == "tiny30" else gg.make_case(name)
    lg = rh.Grid(g, device=0)
    st = lg.plant()
    pd, qd = st.pd, st.qd
    if k is not None:
        s = gg.load_scales(g.n_bus, k + 1, g.seed)[k]
        pd, qd = pd * s, qd * s
    lg.set_state(st.p, pd, qd)
    lg.powerflow(st.x)
    lg.adjoint()
    return lg


def _items(grids_n, seed=0):
    import torch
    from paper_2201_00241_gb300 import rh
    items, refs = [], []
    for i, (lg, N) in enumerate(grids_n):
        W = gg.random_directions(lg.n_p, N, seed + i)
        Wd = torch.from_numpy(np.ascontiguousarray(W.T)).cuda().t()
        HW = torch.full((N, lg.n_p), np.nan, dtype=torch.float64, device="cuda").t()
        work = torch.empty(rh.work_doubles(lg, N), dtype=torch.float64, device="cuda")
        items.append((lg, Wd, HW, work))
        refs.append(lg.hessvec(W))
    return items, refs


def _check(items, refs, tag):
    import torch
    torch.cuda.synchronize()
    for (lg, _, HW, _), ref in zip(items, refs):
        got = HW.cpu().numpy()
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= 1e-12, (tag, lg.n_bus, err)


@pytest.fixture(scope="module")
def batch():
    grids_n = [(_ready("case1354", k), 40 + 7 * k) for k in range(3)] + [(_ready("case118"), 7),
                                                                         (_ready("tiny30"), 3),
                                                                         (_ready("case9241"), 5)]
    return grids_n


def test_every_configuration_equals_rh_hessvec(batch):
    from paper_2201_00241_gb300 import autotune
    items, refs = _items(batch)
    grids = [lg for lg, _, _, _ in items]
    for t in autotune.TAILS:
        tg = autotune.with_tail(grids, t)
        titems = [(g2,) + tuple(it[1:]) for g2, it in zip(tg, items)]
        try:
            for w in autotune.WIDTHS:
                for th in autotune.SHAPES:
                    for sp in (1, 2, 4, 8, 16, 32):
                        for _, _, HW, _ in titems:
                            HW.fill_(np.nan)
                        autotune.launch(titems, {"width": w, "threads": th, "split_lanes": sp})
                        _check(titems, refs, (t, w, th, sp))
        finally:
            for g2, g in zip(tg, grids):
                if g2 is not g:
                    g2.close()


def test_tail_bounds_change_only_rounding():
    """rh_hessvec on the same state with dense-tail bounds 2 .. 512 (tails of 0 to
    several hundred variables) against the oracle."""
    from oracle import OracleGrid
    from paper_2201_00241_gb300 import rh
    g = gg.make_case("case1354")
    base = _ready("case1354")
    o = OracleGrid(g)
    so = o.plant()
    W = gg.random_directions(base.n_p, 9, 3)
    Ho = o.hessvec(so.x, so.p, so.pd, so.qd, W)
    for t in (2, 16, 64, 256, 512):
        lg = base.clone(max_tail=t)
        HW = lg.hessvec(W)
        assert np.abs(HW - Ho).max() <= 1e-10 * np.abs(Ho).max(), t
        Hf = lg.hessian_columns(0, 11)
        E = np.zeros((lg.n_p, 11))
        E[np.arange(11), np.arange(11)] = 1.0
        assert np.abs(Hf - o.hessvec(so.x, so.p, so.pd, so.qd, E)).max() <= 1e-10 * np.abs(Ho).max(), t
        lg.close()
    with pytest.raises(rh.RHError):
        base.clone(max_tail=1)


def test_tune_returns_and_caches_every_choice(batch, tmp_path):
    from paper_2201_00241_gb300 import autotune
    items, refs = _items(batch[:3], seed=10)
    path = str(tmp_path / "tune.json")
    res = autotune.tune(items, widths=(0, 4), shapes=(128, 384), splits=(1, 32), tails=(64, 128), cache_path=path)
    for k in ("width", "threads", "ctas_per_sm", "split_lanes", "max_tail", "ms", "table"):
        assert k in res
    n_tails = len({64, 128} | {int(items[0][0].dims.max_tail)})
    assert not res["cached"] and len(res["table"]) == 2 * 2 * 2 * n_tails
    assert res["ctas_per_sm"] == autotune.CTAS_PER_SM[res["threads"]]
    assert res["ms"] == min(r["ms"] for r in res["table"])
    again = autotune.tune(items, widths=(0, 4), shapes=(128, 384), splits=(1, 32), tails=(64, 128), cache_path=path)
    assert again["cached"] and {k: again[k] for k in ("width", "threads", "split_lanes", "max_tail")} == \
        {k: res[k] for k in ("width", "threads", "split_lanes", "max_tail")}
    autotune._memo.clear()
    from_file = autotune.tune(items, widths=(0, 4), shapes=(128, 384), splits=(1, 32), tails=(64, 128),
                              cache_path=path)
    assert from_file["cached"] and from_file["threads"] == res["threads"]
    assert len(json.load(open(path))) == 1
    # the tuned configuration, with its tail, equals rh_hessvec
    tg = autotune.with_tail([lg for lg, _, _, _ in items], res["max_tail"])
    titems = [(g2,) + tuple(it[1:]) for g2, it in zip(tg, items)]
    for _, _, HW, _ in titems:
        HW.fill_(np.nan)
    autotune.launch(titems, res)
    _check(titems, refs, "tuned")


def test_server_launches_with_tuned_configuration(batch):
    from paper_2201_00241_gb300 import autotune
    from paper_2201_00241_gb300.server import RHServer
    grids = {f"s{k}": lg for k, (lg, _) in enumerate(batch)}
    srv = RHServer(device=0, budget_bytes=2 << 30, max_batch=8, n_streams=2)
    try:
        for n, lg in grids.items():
            srv.register(n, lg)
        res = srv.tune([("s0", 32), ("s1", 32), ("s3", 8), ("s5", 4)], tails=autotune.TAILS)
        assert srv.config == {k: res[k] for k in ("width", "threads", "split_lanes")}
        assert all(int(srv.grids[n].dims.max_tail) == res["max_tail"] for n in ("s0", "s1", "s3", "s5"))
        reqs = [(n, gg.random_directions(lg.n_p, N, 50 + i)) for i, (n, lg, N) in
                enumerate([(n, lg, N) for n, lg in grids.items() for N in (1, 17, 64)])]
        refs = [grids[n].hessvec(W) for n, W in reqs]          # rh_hessvec before serving starts
        futs = [srv.submit(n, W) for n, W in reqs]
        for (n, _), f, ref in zip(reqs, futs, refs):
            assert np.abs(f.result(timeout=120) - ref).max() <= 1e-12 * np.abs(ref).max(), n
        assert srv.stats()["config"] == srv.config
    finally:
        srv.close()
