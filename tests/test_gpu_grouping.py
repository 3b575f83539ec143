"""The in-tile grouping, its rarely taken paths, and the term arithmetic,
checked against the oracle through the C ABI.

A tile's records are ordered by one counting-sort pass on the top bits of a
32-bit key hash and then grouped by full key inside each thread's buckets; a
bucket too long for one thread is grouped by a warp, and keys that share the
hash are told apart by the 128-bit comparison.  On ordinary inputs two keys of
one tile share the hash with probability about 2e-5, so the run option
PT2_DEBUG_NARROW_SORT_HASH keeps only 4 bits of it: then nearly every key of a
tile meets others with the same hash and bucket.  Every such run must give the
oracle's result (the set bit-exactly, numerators to 1e-13, E2 to 1e-10), for
small tiles (serial grouping), the default and the largest tile target (warp
grouping, and the oversize chunked path).

The term num^2 / (E0 - H_aa) uses a hardware reciprocal estimate refined by
one Newton-Raphson step (Eq. 3's division, done without an FP64 divide); its
relative error is bounded here against exact rational arithmetic over the
whole range of denominators the library accepts.
"""

import math
from fractions import Fraction

import numpy as np
import pytest

import brute
import oracle
from paper_1808_02049_gb300 import inputs, pt2

pytestmark = pytest.mark.gpu

E2_TOL = 1e-10


def e2_close(a, b):
    return abs(a - b) <= max(E2_TOL, E2_TOL * abs(b))


@pytest.fixture(scope="module")
def ctx():
    from paper_1808_02049_gb300 import build

    build.build_library()
    c = pt2.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def small(ctx):
    s, r = inputs.make_workload("small")
    e0 = oracle.e0_of(s.h, s.eri, r.keys)
    sid = ctx.load_system(s.h, s.eri)
    rid = ctx.load_reference(sid, r.keys, r.coef, e0)
    ref = oracle.pt2(s.h, s.eri, r.keys, r.coef, e0)
    dump = oracle.dump_external(s.h, s.eri, r.keys, r.coef, e0)
    return dict(s=s, r=r, e0=e0, sid=sid, rid=rid, ref=ref, dump=dump)


def sort_keys(k, *vals):
    order = np.lexsort((k[:, 1], k[:, 0]))
    return (k[order],) + tuple(v[order] for v in vals)


def assert_same_result(got, ref):
    for f in ("n_terms", "n_external", "n_in_ref", "n_unique", "digest_sum", "digest_xor", "n_pos_denom"):
        assert got[f] == ref[f], f
    assert e2_close(got["e2"], ref["e2"]), (got["e2"], ref["e2"])


@pytest.mark.parametrize("tile_target", [16, 0, 1024])
def test_narrow_sort_hash_matches_oracle(ctx, small, tile_target):
    got = ctx.run(small["rid"], tile_target=tile_target, narrow_sort_hash=True)
    assert got["n_hash_collisions"] > 0
    assert_same_result(got, small["ref"])
    if tile_target == 1024:
        assert got["n_oversize"] > 0  # the chunked path grouped with the narrow hash too
    # the same energy, bit for bit, as the ordinary grouping
    assert got["e2"] == ctx.run(small["rid"], tile_target=tile_target)["e2"]
    k, num, haa = ctx.dump_external(small["rid"], small["ref"]["n_external"] + 10, tile_target=tile_target,
                                    narrow_sort_hash=True)
    ok, onum, ohaa, _ = small["dump"]
    k, num, haa = sort_keys(k, num, haa)
    assert np.array_equal(k, ok)
    np.testing.assert_allclose(num, onum, rtol=0, atol=1e-13)
    np.testing.assert_allclose(haa, ohaa, rtol=0, atol=1e-11)


def test_ordinary_runs_meet_no_collision_on_the_small_workload(ctx, small):
    # 3,800 tiles of ~450 keys: the expected number of equal 32-bit hashes
    # among different keys of a tile is ~0.1 over the whole run
    got = ctx.run(small["rid"])
    assert got["n_hash_collisions"] <= 2
    assert_same_result(got, small["ref"])


@pytest.mark.parametrize("tile_target", [16, 1024])
def test_narrow_sort_hash_on_a_brute_force_system(ctx, tile_target):
    from test_oracle_pins import strong_integrals

    n_orb, na, nb, n_ref, seed = 6, 3, 3, 5, 5
    h, eri = strong_integrals(n_orb, seed)
    dets = brute.basis(n_orb, na, nb)
    H = brute.hamiltonian(h, eri, dets)
    rng = np.random.default_rng(100 + seed)
    idx = sorted(rng.choice(len(dets), size=n_ref, replace=False).tolist())
    coef = rng.normal(0, 1, n_ref)
    e0 = float(min(H[i, i] for i in idx) - 0.37)
    bf = brute.pt2(h, eri, dets, H, idx, coef, e0)
    keys = np.empty(2 * n_ref, dtype=np.uint64)
    keys[0::2] = [dets[i][0] for i in idx]
    keys[1::2] = [dets[i][1] for i in idx]
    sid = ctx.load_system(h, eri)
    rid = ctx.load_reference(sid, keys, coef, e0)
    try:
        got = ctx.run(rid, tile_target=tile_target, narrow_sort_hash=True)
        k, num, haa = ctx.dump_external(rid, len(dets), tile_target=tile_target, narrow_sort_hash=True)
    finally:
        ctx.unload(rid)
        ctx.unload(sid)
    assert got["n_hash_collisions"] > 0
    k, num, haa = sort_keys(k, num, haa)
    assert np.array_equal(k, bf["keys"])
    np.testing.assert_allclose(num, bf["num"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(haa, bf["haa"], rtol=0, atol=1e-12)
    assert e2_close(got["e2"], bf["e2"])


def test_short_copy_wait_reports_timeout_and_context_survives(ctx, small):
    # every tile CTA gives up on its first bulk copy after 64 cycles (the copy
    # still lands through the second bounded wait); the run reports the timeout
    with pytest.raises(pt2.Pt2Error) as e:
        ctx.run(small["rid"], short_copy_wait=True)
    assert e.value.code == pt2.PT2_ERR_TIMEOUT
    # the error word is cleared by the next run, which is correct
    assert_same_result(ctx.run(small["rid"]), small["ref"])


def _exact_term(num, den):
    dfx = round(Fraction(den) * 2 ** 48)  # nearest integer, ties to even, like the device conversion
    return Fraction(num) ** 2 * 2 ** 48 / dfx


def test_term_arithmetic_error_bound(ctx):
    rng = np.random.default_rng(20181806)
    n = 20000
    mag = 10.0 ** rng.uniform(-8, math.log10(32767.0), n)
    den = mag * rng.choice([-1.0, 1.0], n)
    num = 10.0 ** rng.uniform(-15, 1, n) * rng.choice([-1.0, 1.0], n)
    # edges: the smallest and largest accepted denominators, powers of two
    # (exact reciprocal estimates) and their neighbours, zero numerators
    edge = [2.0 ** -48, -(2.0 ** -48), 3 * 2.0 ** -48, 32767.99, -32767.99, 1e-8, -1e-8]
    for k in range(-20, 15):
        for d in (2.0 ** k, np.nextafter(2.0 ** k, 0), np.nextafter(2.0 ** k, 2.0 ** 16)):
            edge += [d, -d]
    den = np.concatenate([den, np.array(edge)])
    num = np.concatenate([num, rng.uniform(-1, 1, len(edge))])
    num[:5] = 0.0
    got = ctx.eval_terms(num, den)
    worst = 0.0
    for x, d, g in zip(num.tolist(), den.tolist(), got.tolist()):
        ex = _exact_term(x, d)
        if ex == 0:
            assert g == 0.0
            continue
        worst = max(worst, float(abs(Fraction(g) - ex) / abs(ex)))
    assert worst < 2.0 ** -43, worst


def test_term_arithmetic_rejects_out_of_range_denominators(ctx):
    for d in (0.0, 1e-16, 40000.0, float("nan")):
        with pytest.raises(pt2.Pt2Error) as e:
            ctx.eval_terms(np.array([0.5]), np.array([d]))
        assert e.value.code == pt2.PT2_ERR_INVALID


@pytest.mark.parametrize("tile_target", [16, 0, 1024])
def test_hashed_keys_equal_the_exact_grouping(ctx, small, tile_target):
    # the hashing section's compression: keys of a tile identified by a
    # 54-bit hash; with no merge of different keys (reported as 0) the run is
    # the ordinary one bit for bit, and the oracle's
    got = ctx.run(small["rid"], tile_target=tile_target, hashed_keys=True)
    assert got["n_hash_collisions"] == 0
    assert_same_result(got, small["ref"])
    exact = ctx.run(small["rid"], tile_target=tile_target)
    assert got["e2"] == exact["e2"]
    assert (got["digest_sum"], got["digest_xor"]) == (exact["digest_sum"], exact["digest_xor"])
    k, num, haa = ctx.dump_external(small["rid"], small["ref"]["n_external"] + 10, tile_target=tile_target,
                                    hashed_keys=True)
    ok, onum, ohaa, _ = small["dump"]
    k, num, haa = sort_keys(k, num, haa)
    assert np.array_equal(k, ok)
    np.testing.assert_allclose(num, onum, rtol=0, atol=1e-13)


def test_hashed_keys_on_the_large_system(ctx):
    s, r = inputs.make_workload("large", n_det=2000)
    e0 = oracle.e0_of(s.h, s.eri, r.keys)
    sid = ctx.load_system(s.h, s.eri)
    rid = ctx.load_reference(sid, r.keys, r.coef, e0)
    try:
        a = ctx.run(rid)
        b = ctx.run(rid, hashed_keys=True)
    finally:
        ctx.unload(rid)
        ctx.unload(sid)
    assert b["n_hash_collisions"] == 0
    assert a["e2"] == b["e2"]
    for f in ("n_terms", "n_unique", "n_in_ref", "n_external", "digest_sum", "digest_xor", "n_oversize"):
        assert a[f] == b[f], f
