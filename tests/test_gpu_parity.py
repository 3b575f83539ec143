"""Parity of the CUDA path (through the C ABI) against the CPU oracle.

Tolerance: |dE2| <= 1e-10 Ha absolute or 1e-10 relative; the connected
external set (count and order-independent digest, and the full key list where
the oracle can enumerate it) must match bit-exactly; per-key numerators agree
to 1e-13 absolute (they are sums of FP64 products, summed in a different
order) and diagonals to 1e-11 absolute (incremental on the GPU, direct in the
oracle).
"""

import math

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
    return dict(s=s, r=r, e0=e0, sid=sid, rid=rid, ref=ref)


def assert_same_result(got, ref):
    assert got["n_terms"] == ref["n_terms"]
    assert got["n_external"] == ref["n_external"]
    assert got["n_in_ref"] == ref["n_in_ref"]
    assert got["n_unique"] == ref["n_unique"]
    assert (got["digest_sum"], got["digest_xor"]) == (ref["digest_sum"], ref["digest_xor"])
    assert got["n_pos_denom"] == ref["n_pos_denom"]
    if ref["n_external"]:
        assert abs(got["min_abs_denom"] - ref["min_abs_denom"]) < 1e-10
    assert e2_close(got["e2"], ref["e2"]), (got["e2"], ref["e2"])


def sort_keys(k, *vals):
    order = np.lexsort((k[:, 1], k[:, 0]))
    return (k[order],) + tuple(v[order] for v in vals)


def test_diagonal_matches_oracle(ctx, small):
    s, r = small["s"], small["r"]
    got = ctx.diagonal(small["sid"], r.keys)
    np.testing.assert_allclose(got, oracle.diagonals(s.h, s.eri, r.keys), rtol=0, atol=1e-12)


@pytest.mark.parametrize("det", [0, 1, 123, 999])
def test_det_terms_match_oracle(ctx, small, det):
    s, r = small["s"], small["r"]
    k, v, d = ctx.det_terms(small["rid"], det, 4000)
    ok, ov, od = oracle.det_terms(s.h, s.eri, r.keys[2 * det], r.keys[2 * det + 1], r.coef[det])
    assert k.shape == ok.shape == (3192, 2)
    k, v, d = sort_keys(k, v, d)
    ok, ov, od = sort_keys(ok, ov, od)
    assert np.array_equal(k, ok)
    np.testing.assert_allclose(v, ov, rtol=0, atol=1e-14)
    np.testing.assert_allclose(d, od, rtol=0, atol=1e-11)


def test_e2_small_workload_matches_oracle(ctx, small):
    got = ctx.run(small["rid"])
    assert_same_result(got, small["ref"])


def test_external_set_dump_matches_oracle(ctx, small):
    s, r, e0 = small["s"], small["r"], small["e0"]
    k, num, haa = ctx.dump_external(small["rid"], small["ref"]["n_external"] + 10)
    ok, onum, ohaa, _ = oracle.dump_external(s.h, s.eri, r.keys, r.coef, e0)
    k, num, haa = sort_keys(k, num, haa)
    assert np.array_equal(k, ok)
    np.testing.assert_allclose(num, onum, rtol=0, atol=1e-13)
    np.testing.assert_allclose(haa, ohaa, rtol=0, atol=1e-11)


def test_run_is_bit_identical_across_runs(ctx, small):
    a = ctx.run(small["rid"])
    b = ctx.run(small["rid"])
    assert a["e2"] == b["e2"]
    assert a == {**b, "seconds": a["seconds"]}


@pytest.mark.parametrize("tile_target", [16, 256, 1024])
def test_tile_sizes_and_oversize_path(ctx, small, tile_target):
    got = ctx.run(small["rid"], tile_target=tile_target)
    assert_same_result(got, small["ref"])
    if tile_target == 1024:
        assert got["n_oversize"] > 0  # tiles above shared-memory capacity took the chunked path


def test_oversize_tiles_with_mostly_distinct_keys(ctx):
    # Three determinants of the large system: almost every one of the ~3.9e5
    # terms is a distinct key, so at the largest tile target about half of the
    # tiles exceed shared memory with more distinct keys than one chunk holds;
    # their partials are split by hash before the final reduction.
    s, r = inputs.make_workload("large", n_det=3)
    e0 = oracle.e0_of(s.h, s.eri, r.keys)
    sid = ctx.load_system(s.h, s.eri)
    rid = ctx.load_reference(sid, r.keys, r.coef, e0)
    try:
        ref = oracle.pt2(s.h, s.eri, r.keys, r.coef, e0)
        assert ref["n_unique"] > 0.95 * ref["n_terms"]
        got = ctx.run(rid, tile_target=1024)
        assert got["n_oversize"] > 0.2 * got["n_tiles"]
        assert_same_result(got, ref)
        assert ctx.run(rid)["e2"] == got["e2"]
    finally:
        ctx.unload(rid)
        ctx.unload(sid)


def test_e2_is_bit_identical_for_any_tiling_and_pass_plan(ctx, small):
    # numerators and the energy are summed exactly in fixed point, so the
    # result cannot depend on how terms are split into passes and tiles
    base = ctx.run(small["rid"])
    for kw in [dict(tile_target=16), dict(tile_target=1024), dict(pass_budget_bytes=12 << 20),
               dict(pass_budget_bytes=40 << 20, tile_target=100)]:
        got = ctx.run(small["rid"], **kw)
        assert got["e2"] == base["e2"], kw
        assert (got["digest_sum"], got["digest_xor"], got["n_external"]) == \
            (base["digest_sum"], base["digest_xor"], base["n_external"])


def test_heavy_alpha_class_is_split_by_beta_class(ctx, small):
    # 288 of the 1000 determinants share the Hartree-Fock alpha string, so its
    # alpha class holds at least 288 * (4*12 + 6*66) = 127,872 terms; a 1 MB
    # pass budget holds about 32,000, so that class must be split into passes
    # by beta class (the run fails otherwise) and give the same result
    alpha = small["r"].keys[0::2]
    assert np.unique(alpha, return_counts=True)[1].max() == 288
    base = ctx.run(small["rid"])
    got = ctx.run(small["rid"], pass_budget_bytes=1 << 20)
    assert got["n_passes"] > 90
    assert_same_result(got, small["ref"])
    assert got["e2"] == base["e2"]
    assert (got["digest_sum"], got["digest_xor"]) == (base["digest_sum"], base["digest_xor"])


def test_many_passes(ctx, small):
    # a 12 MB pass budget forces several memory-bounded passes
    got = ctx.run(small["rid"], pass_budget_bytes=12 << 20)
    assert got["n_passes"] >= 5
    assert_same_result(got, small["ref"])


def test_grouped_tile_counts(ctx, small):
    # consecutive passes over whole alpha classes are counted by one launch
    # per group of at most 64 passes; a 1 MB budget makes about 100 passes,
    # so more than one group, and splits the heavy alpha class by beta class
    # between them.  The run must equal the oracle and, bit for bit, the same
    # plan run as a batch, whose steps count their own tiles
    kw = dict(pass_budget_bytes=1 << 20, tile_target=256)
    got = ctx.run(small["rid"], **kw)
    assert got["n_passes"] > 90
    assert_same_result(got, small["ref"])
    bid = ctx.batch_create([small["rid"]], **kw)
    try:
        (b,) = ctx.batch_run(bid, 1)
    finally:
        ctx.batch_destroy(bid)
    for f in ("e2", "n_terms", "n_unique", "n_external", "digest_sum", "digest_xor", "n_tiles", "n_passes"):
        assert b[f] == got[f], f


def test_constraint_classes(ctx, small):
    s, r, e0 = small["s"], small["r"], small["e0"]
    m = 5
    tot = 0.0
    for k in range(m):
        got = ctx.run(small["rid"], constraint=(m, k))
        ref = oracle.pt2(s.h, s.eri, r.keys, r.coef, e0, constraint=(m, k))
        assert_same_result(got, ref)
        tot += got["e2"]
    assert e2_close(tot, small["ref"]["e2"])


def test_permutation_invariance_is_bit_exact(ctx, small):
    s, r, e0 = small["s"], small["r"], small["e0"]
    perm = np.random.default_rng(11).permutation(r.n_det)
    pk = np.empty_like(r.keys)
    pk[0::2], pk[1::2] = r.keys[0::2][perm], r.keys[1::2][perm]
    rid = ctx.load_reference(small["sid"], pk, r.coef[perm], e0)
    try:
        a = ctx.run(small["rid"])
        b = ctx.run(rid)
    finally:
        ctx.unload(rid)
    assert a["e2"] == b["e2"]
    assert (a["digest_sum"], a["digest_xor"]) == (b["digest_sum"], b["digest_xor"])


def test_scaling_and_spin_swap(ctx, small):
    s, r, e0 = small["s"], small["r"], small["e0"]
    base = ctx.run(small["rid"])["e2"]
    rid = ctx.load_reference(small["sid"], r.keys, 2.0 * r.coef, e0)
    try:
        dbl = ctx.run(rid)["e2"]
    finally:
        ctx.unload(rid)
    assert abs(dbl - 4.0 * base) <= 1e-14 * abs(base)
    sw = r.keys.copy()
    sw[0::2], sw[1::2] = r.keys[1::2], r.keys[0::2]
    rid = ctx.load_reference(small["sid"], sw, r.coef, e0)
    try:
        swp = ctx.run(rid)["e2"]
    finally:
        ctx.unload(rid)
    assert abs(swp - base) <= 1e-12 * abs(base)


def _keys_of(dets):
    k = np.empty(2 * len(dets), dtype=np.uint64)
    k[0::2] = [d[0] for d in dets]
    k[1::2] = [d[1] for d in dets]
    return k


@pytest.mark.parametrize("n_orb,na,nb,n_ref,seed", [(4, 2, 2, 3, 1), (5, 2, 1, 4, 3), (6, 3, 3, 5, 5),
                                                    (6, 3, 2, 1, 6)])
def test_tiny_systems_match_brute_force(ctx, n_orb, na, nb, n_ref, seed):
    from test_oracle_pins import strong_integrals

    h, eri = strong_integrals(n_orb, seed)
    dets = brute.basis(n_orb, na, nb)
    H = brute.hamiltonian(h, eri, dets)
    rng = np.random.default_rng(100 + seed)
    idx = sorted(rng.choice(len(dets), size=n_ref, replace=False).tolist())
    coef = rng.normal(0, 1, n_ref)
    e0 = float(min(H[i, i] for i in idx) - 0.37)
    bf = brute.pt2(h, eri, dets, H, idx, coef, e0)
    sid = ctx.load_system(h, eri)
    rid = ctx.load_reference(sid, _keys_of([dets[i] for i in idx]), coef, e0)
    try:
        got = ctx.run(rid)
        k, num, haa = ctx.dump_external(rid, len(dets))
    finally:
        ctx.unload(rid)
        ctx.unload(sid)
    k, num, haa = sort_keys(k, num, haa)
    assert np.array_equal(k, bf["keys"])
    np.testing.assert_allclose(num, bf["num"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(haa, bf["haa"], rtol=0, atol=1e-12)
    assert e2_close(got["e2"], bf["e2"])


def test_edge_cases(ctx):
    # no excitations at all: one orbital, one alpha electron, no beta electron
    h = np.array([[-1.0]])
    eri = np.array([[[[0.5]]]])
    sid = ctx.load_system(h, eri)
    rid = ctx.load_reference(sid, np.array([1, 0], dtype=np.uint64), np.array([1.0]), -2.0)
    got = ctx.run(rid)
    ctx.unload(rid)
    ctx.unload(sid)
    assert got["n_terms"] == 0 and got["n_external"] == 0 and got["e2"] == 0.0
    # a filled alpha shell (no alpha virtuals), single-determinant reference
    s = inputs.make_integrals(6, 5)
    keys = np.array([0b111111, 0b000011], dtype=np.uint64)
    e0 = float(oracle.diagonals(s.h, s.eri, keys)[0] - 0.2)
    ref = oracle.pt2(s.h, s.eri, keys, np.array([1.0]), e0)
    sid = ctx.load_system(s.h, s.eri)
    rid = ctx.load_reference(sid, keys, np.array([1.0]), e0)
    got = ctx.run(rid)
    ctx.unload(rid)
    ctx.unload(sid)
    assert_same_result(got, ref)


def test_64_orbitals_top_bit(ctx):
    # n_orb = 64 exercises bit 63 of both words
    s = inputs.make_integrals(64, 77)
    r = inputs.make_reference(64, 2, 6, 2, 78)
    # move one electron of each spin to orbital 63 in one determinant
    keys = r.keys.copy()
    keys[2] = np.uint64((1 << 63) | 1)
    keys[3] = np.uint64((1 << 63) | 2)
    e0 = oracle.e0_of(s.h, s.eri, keys)
    ref = oracle.pt2(s.h, s.eri, keys, r.coef, e0)
    sid = ctx.load_system(s.h, s.eri)
    rid = ctx.load_reference(sid, keys, r.coef, e0)
    got = ctx.run(rid)
    ctx.unload(rid)
    ctx.unload(sid)
    assert_same_result(got, ref)


def test_invalid_inputs_are_rejected(ctx, small):
    s, r = small["s"], small["r"]
    bad = r.keys.copy()
    bad[2], bad[3] = bad[0], bad[1]
    with pytest.raises(pt2.Pt2Error) as e:
        ctx.load_reference(small["sid"], bad, r.coef, -1.0)
    assert e.value.code == pt2.PT2_ERR_INVALID
    bad = r.keys.copy()
    bad[0] = np.uint64(bad[0]) | np.uint64(1 << 40)
    with pytest.raises(pt2.Pt2Error) as e:
        ctx.load_reference(small["sid"], bad, r.coef, -1.0)
    assert e.value.code == pt2.PT2_ERR_INVALID
    coef = r.coef.copy()
    coef[3] = np.nan
    with pytest.raises(pt2.Pt2Error) as e:
        ctx.load_reference(small["sid"], r.keys, coef, -1.0)
    assert e.value.code == pt2.PT2_ERR_INVALID
    hb = s.h.copy()
    hb[0, 1] += 1e-6
    with pytest.raises(pt2.Pt2Error) as e:
        ctx.load_system(hb, s.eri)
    assert e.value.code == pt2.PT2_ERR_INVALID
    # the integral check runs over rows in parallel and reports the first
    # element (in index order) that breaks the 8-fold symmetry
    eb = s.eri.copy()
    eb[7, 3, 9, 5] += 1e-6
    eb[2, 11, 4, 6] += 1e-6
    with pytest.raises(pt2.Pt2Error) as e:
        ctx.load_system(s.h, eb)
    assert e.value.code == pt2.PT2_ERR_INVALID
    assert "(2 11|4 6)" in str(e.value), str(e.value)
    with pytest.raises(pt2.Pt2Error) as e:
        ctx.load_system(np.eye(65), np.zeros((65,) * 4))
    assert e.value.code == pt2.PT2_ERR_UNSUPPORTED
    with pytest.raises(pt2.Pt2Error) as e:
        ctx.run(987654)
    assert e.value.code == pt2.PT2_ERR_NOT_FOUND
    with pytest.raises(pt2.Pt2Error) as e:
        ctx.run(small["rid"], constraint=(3, 5))
    assert e.value.code == pt2.PT2_ERR_INVALID
    with pytest.raises(pt2.Pt2Error) as e:
        ctx.unload(small["sid"])  # still used by a reference
    assert e.value.code == pt2.PT2_ERR_INVALID


def T(n, v):
    return 2 * n * v + 2 * math.comb(n, 2) * math.comb(v, 2) + (n * v) ** 2


def test_class_slices_partition_the_solve(ctx, small):
    # the alpha-class slices are non-overlapping, complete constraint classes
    # (Algorithm 2): their counts and set digests add up to the full run's
    # exactly and their energies to its energy
    full = ctx.run(small["rid"])
    for m in (7, 20):
        parts = [ctx.run(small["rid"], class_slice=(k, m)) for k in range(m)]
        for f in ("n_terms", "n_unique", "n_in_ref", "n_external", "n_pos_denom"):
            assert sum(p[f] for p in parts) == full[f], (m, f)
        assert sum(p["digest_sum"] for p in parts) % (1 << 64) == full["digest_sum"]
        x = 0
        for p in parts:
            x ^= p["digest_xor"]
        assert x == full["digest_xor"]
        assert abs(sum(p["e2"] for p in parts) - full["e2"]) <= 1e-14 * abs(full["e2"])
        assert sum(p["n_terms"] > 0 for p in parts) > m // 2
    assert_same_result(full, small["ref"])


def test_class_slices_with_duplicate_subtraction_and_constraint(ctx, small):
    # each slice subtracts the reference determinants of its own classes only
    full = ctx.run(small["rid"], subtract_ref=True, constraint=(3, 1))
    parts = [ctx.run(small["rid"], subtract_ref=True, constraint=(3, 1), class_slice=(k, 5)) for k in range(5)]
    assert sum(p["n_terms"] for p in parts) == full["n_terms"]
    assert abs(sum(p["e2"] for p in parts) - full["e2"]) <= 1e-14 * abs(full["e2"])


def test_class_slice_options_are_validated(ctx, small):
    for sl in ((5, 5), (0, 5000), (9, 3)):
        with pytest.raises(pt2.Pt2Error) as e:
            ctx.run(small["rid"], class_slice=sl)
        assert e.value.code == pt2.PT2_ERR_INVALID
