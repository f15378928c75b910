"""Continuous-batching server: each request's result is the same alone and
in the mix, admission respects the device-memory cap, cancellation and
failed set-ups leave the other requests untouched."""
import numpy as np
import pytest

from paper_1901_07374_gb300 import serve
from paper_1901_07374_gb300 import specimen as S

pytestmark = pytest.mark.gpu


def _requests():
    ws = [S.taylor_impact(4000, v_impact=220.0, seed=1),
          S.tensile_bar_jc(nx=8, ny=8, nz=30, seed=2),
          S.failure_variant(S.tensile_bar_cl(nx=7, ny=7, nz=24)),
          S.taylor_impact(2500, v_impact=160.0, seed=3)]
    steps = (60, 95, 130, 45)
    return [serve.Request(k, 0.0, w, n) for k, (w, n) in enumerate(zip(ws, steps))]


def test_result_is_the_same_alone_and_in_the_mix():
    mix = serve.Server(chunk_steps=25).run(_requests(), realtime=False)
    assert all(r.status == "done" for r in mix)
    for r in _requests():
        alone = serve.Server(chunk_steps=40).run([r], realtime=False)[0]
        ref = next(m for m in mix if m.id == r.id)
        for k, v in alone.result.items():
            assert np.array_equal(v, ref.result[k]), (r.id, k)


def test_admission_respects_the_memory_cap():
    reqs = _requests()
    need = sorted(serve.memory_estimate(r.workload) for r in reqs)
    cap = need[-1] + need[-2]          # room for about two requests at once
    srv = serve.Server(mem_cap_bytes=cap, chunk_steps=20)
    srv.run(reqs, realtime=False)
    assert all(r.status == "done" for r in reqs)
    assert srv.peak_used <= cap
    assert max(n for _, n, _ in srv.timeline) < len(reqs)
    # first come, first served
    adm = [r.admitted for r in sorted(reqs, key=lambda r: r.id)]
    assert adm == sorted(adm)


def test_cancel_and_failed_setup():
    reqs = _requests()
    bad = S.tensile_bar_cl(nx=4, ny=4, nz=6)
    bad.specimen.vol = -bad.specimen.vol          # rejected by tlsph_create
    reqs.append(serve.Request(9, 0.0, bad, 10))
    srv = serve.Server(chunk_steps=20)
    srv.cancel(2)
    srv.run(reqs, realtime=False)
    st = {r.id: r.status for r in reqs}
    assert st[2] == "cancelled" and st[9] == "failed"
    assert all(st[k] == "done" for k in (0, 1, 3))
    assert srv.used == 0


def test_realtime_arrivals_and_summary():
    reqs = _requests()
    for k, r in enumerate(reqs):
        r.arrival = 0.05 * k
    srv = serve.Server(chunk_steps=30)
    import time
    t0 = time.perf_counter()
    srv.run(reqs, realtime=True)
    summ = serve.summarize(reqs, time.perf_counter() - t0)
    assert summ["done"] == len(reqs)
    assert 0 < summ["p50_s"] <= summ["p95_s"] <= summ["p99_s"]
    assert all(r.admitted >= r.arrival for r in reqs)
