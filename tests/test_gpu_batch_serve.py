"""Batched and served PT2: many uneven instances in one captured launch, and
continuous batching of submitted requests.

Energies and set statistics are accumulated exactly, so an instance's result
must be bit-identical alone (pt2_run), inside a batch and inside a served
mix.  Every instance is also checked against the oracle, batched and served,
on one constraint class (alpha % 11 == 5: the oracle drops the other classes'
terms before computing their matrix elements, so it stays quick); the two
smallest instances in full.
"""

import concurrent.futures as cf
import os

import numpy as np
import pytest

import oracle
from paper_1808_02049_gb300 import inputs, pt2

pytestmark = pytest.mark.gpu

SAME = ("e2", "n_terms", "n_unique", "n_in_ref", "n_external", "digest_sum", "digest_xor", "n_pos_denom",
        "min_abs_denom")


def same(a, b):
    return all(a[k] == b[k] for k in SAME)


@pytest.fixture(scope="module")
def fleet():
    from paper_1808_02049_gb300 import build

    build.build_library()
    c = pt2.Context(0)
    refs = []
    for k in range(10):
        prm = inputs.batch_instance_params(k)
        prm["n_det"] = min(prm["n_det"], 600 + 150 * k)  # keep the test quick
        s, r = inputs.make_instance(prm)
        sid = c.load_system(s.h, s.eri)
        e0 = float(c.diagonal(sid, r.keys).min() - 0.1)
        rid = c.load_reference(sid, r.keys, r.coef, e0)
        refs.append(dict(sid=sid, rid=rid, s=s, r=r, e0=e0, alone=c.run(rid)))
    yield c, refs
    c.close()


def test_batch_matches_single_runs_and_oracle(fleet):
    c, refs = fleet
    ids = [x["rid"] for x in refs]
    bid = c.batch_create(ids)
    try:
        info = c.batch_info(bid)
        assert info["steps"] >= 1 and info["n_terms"] == sum(x["alone"]["n_terms"] for x in refs)
        res = c.batch_run(bid, len(ids))
        again = c.batch_run(bid, len(ids))  # graph replay
    finally:
        c.batch_destroy(bid)
    for x, got, rep in zip(refs, res, again):
        assert same(got, x["alone"]), (got, x["alone"])
        assert same(rep, got)
    small = sorted(refs, key=lambda x: x["alone"]["n_terms"])[:2]
    for x in small:
        ref = oracle.pt2(x["s"].h, x["s"].eri, x["r"].keys, x["r"].coef, x["e0"])
        assert x["alone"]["n_external"] == ref["n_external"]
        assert (x["alone"]["digest_sum"], x["alone"]["digest_xor"]) == (ref["digest_sum"], ref["digest_xor"])
        assert abs(x["alone"]["e2"] - ref["e2"]) <= max(1e-10, 1e-10 * abs(ref["e2"]))


CLASS = (11, 5)


@pytest.fixture(scope="module")
def oracle_class(fleet):
    # the oracle on one constraint class of every instance, on the host cores
    _, refs = fleet
    oracle.build()
    with cf.ThreadPoolExecutor(max_workers=min(len(refs), os.cpu_count() or 1)) as ex:
        return list(ex.map(lambda x: oracle.pt2(x["s"].h, x["s"].eri, x["r"].keys, x["r"].coef, x["e0"],
                                                constraint=CLASS), refs))


def same_as_oracle(got, ref):
    assert got["n_terms"] == ref["n_terms"]
    assert got["n_external"] == ref["n_external"]
    assert got["n_in_ref"] == ref["n_in_ref"]
    assert (got["digest_sum"], got["digest_xor"]) == (ref["digest_sum"], ref["digest_xor"])
    assert abs(got["e2"] - ref["e2"]) <= max(1e-10, 1e-10 * abs(ref["e2"]))


def test_every_batched_instance_matches_oracle_on_a_class(fleet, oracle_class):
    c, refs = fleet
    bid = c.batch_create([x["rid"] for x in refs], constraint=CLASS)
    try:
        res = c.batch_run(bid, len(refs))
    finally:
        c.batch_destroy(bid)
    for got, ref in zip(res, oracle_class):
        assert ref["n_terms"] > 0
        same_as_oracle(got, ref)


def test_every_served_instance_matches_oracle_on_a_class(fleet, oracle_class):
    c, refs = fleet
    tickets = [c.submit(x["rid"], constraint=CLASS) for x in refs]
    for t, ref in zip(tickets, oracle_class):
        same_as_oracle(c.wait(t, timeout_s=600), ref)


def test_profiled_batch_matches_graph_replay(fleet):
    c, refs = fleet
    ids = [x["rid"] for x in refs]
    bid = c.batch_create(ids, profile=True)  # steps launched one by one, with phase events
    try:
        res = c.batch_run(bid, len(ids))
        ph, launches = c.phase_times()
    finally:
        c.batch_destroy(bid)
    for x, got in zip(refs, res):
        assert same(got, x["alone"])
    assert ph["emit"] > 0 and ph["tile_sort_reduce"] > 0 and launches > 0


def test_batch_with_small_step_budget_and_autotune(fleet):
    c, refs = fleet
    ids = [x["rid"] for x in refs]
    best = c.autotune(refs[3]["rid"])
    assert best in (704, 768, 832, 896)
    # a small pass budget splits instances into many passes packed into steps
    bid = c.batch_create(ids, pass_budget_bytes=200 << 20, autotune=True)
    try:
        assert c.batch_info(bid)["steps"] > 1
        res = c.batch_run(bid, len(ids))
    finally:
        c.batch_destroy(bid)
    for x, got in zip(refs, res):
        assert same(got, x["alone"])


def test_served_mix_matches_single_runs(fleet):
    c, refs = fleet
    order = [3, 1, 4, 1, 5, 9, 2, 6, 5, 3, 5, 8, 9, 7, 0]
    tickets = [(c.submit(refs[i]["rid"]), i) for i in order]
    for t, i in tickets:
        got = c.wait(t, timeout_s=600)
        assert same(got, refs[i]["alone"]), (i, got, refs[i]["alone"])
        assert got["seconds"] > 0
    st = c.server_stats()
    assert st["pending"] == 0 and st["active"] == 0 and st["steps"] >= 1
    with pytest.raises(pt2.Pt2Error) as e:  # a finished ticket is reported once
        c.poll(tickets[0][0])
    assert e.value.code == pt2.PT2_ERR_NOT_FOUND


def test_served_request_timeout_and_busy_reference():
    from paper_1808_02049_gb300 import build

    build.build_library()
    s, r = inputs.make_workload("large", n_det=40000)  # ~5e9 terms: runs for a while
    with pt2.Context(0) as c:
        sid = c.load_system(s.h, s.eri)
        e0 = float(c.diagonal(sid, r.keys).min() - 0.1)
        rid = c.load_reference(sid, r.keys, r.coef, e0)
        t = c.submit(rid)
        try:
            early = pt2.pt2_wait(c.handle, t, 0.0)
        except pt2.Pt2Error as e:
            assert e.code == pt2.PT2_ERR_TIMEOUT, str(e)
        else:
            pytest.fail(f"the request was done at once: {early}")
        with pytest.raises(pt2.Pt2Error) as e:
            c.unload(rid)  # still in flight
        assert e.value.code == pt2.PT2_ERR_BUSY
        got = c.wait(t, timeout_s=600)
        assert same(got, c.run(rid))
