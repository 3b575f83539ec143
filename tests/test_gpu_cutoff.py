"""Numerator cutoff (the Results section and the subsection on the
matrix-element cutoff): a contribution c_i H_ai with |c_i H_ai| below the
cutoff is dropped before it gets a record, a denominator or a sort.

Against the oracle with the same cutoff: counts (kept contributions, unique
keys, reference hits, external set and its digest, positive denominators)
exact, E2 within 1e-10, the dump key for key (numerators within 1e-13,
diagonals within 1e-11).  The decision |c H| >= cutoff is taken in FP64 on
both sides; an element that rounds differently on the two sides right at
the cutoff would change a count, which the seeded inputs do not hit.
"""

import numpy as np
import pytest

import oracle
from paper_1808_02049_gb300 import inputs, pt2

pytestmark = pytest.mark.gpu

STATS = ("n_terms", "n_unique", "n_in_ref", "n_external", "digest_sum", "digest_xor", "n_pos_denom")
SAME = ("e2",) + STATS + ("min_abs_denom",)


def same(a, b):
    return all(a[k] == b[k] for k in SAME)


def e2_close(a, b, tol=1e-10):
    return abs(a - b) <= max(tol, tol * abs(b))


def assert_matches_oracle(got, ref):
    for k in STATS:
        assert got[k] == ref[k], (k, got[k], ref[k])
    assert e2_close(got["e2"], ref["e2"]), (got["e2"], ref["e2"])


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
    return dict(s=s, r=r, e0=e0, sid=sid, rid=rid, full=oracle.pt2(s.h, s.eri, r.keys, r.coef, e0))


# 1e-8 is the paper's value; the larger ones drop a growing share of the
# small workload's contributions (its coefficients are larger than those of
# a 1e5-determinant reference)
@pytest.mark.parametrize("cut", [1e-8, 1e-6, 1e-5, 1e-4])
def test_cutoff_matches_oracle(ctx, small, cut):
    s, r, e0 = small["s"], small["r"], small["e0"]
    ref = oracle.pt2(s.h, s.eri, r.keys, r.coef, e0, cutoff=cut)
    got = ctx.run(small["rid"], cutoff=cut)
    assert_matches_oracle(got, ref)
    if cut >= 1e-5:
        assert ref["n_terms"] < 0.8 * small["full"]["n_terms"]


def test_cutoff_dump_matches_oracle(ctx, small):
    s, r, e0 = small["s"], small["r"], small["e0"]
    cut = 1e-5
    ok, onum, ohaa, ref = oracle.dump_external(s.h, s.eri, r.keys, r.coef, e0, cutoff=cut)
    assert ref["n_external"] < small["full"]["n_external"]  # whole determinants leave the set
    k, num, haa = ctx.dump_external(small["rid"], ref["n_external"] + 10, cutoff=cut)
    order = np.lexsort((k[:, 1], k[:, 0]))
    k, num, haa = k[order], num[order], haa[order]
    assert np.array_equal(k, ok)
    np.testing.assert_allclose(num, onum, rtol=0, atol=1e-13)
    np.testing.assert_allclose(haa, ohaa, rtol=0, atol=1e-11)


def test_cutoff_zero_is_the_exact_path(ctx, small):
    assert same(ctx.run(small["rid"], cutoff=0.0), ctx.run(small["rid"]))


def test_cutoff_bit_identical_across_tilings_pass_plans_and_heavy_split(ctx, small):
    cut = 1e-5
    base = ctx.run(small["rid"], cutoff=cut)
    for kw in [dict(tile_target=16), dict(tile_target=1024), dict(pass_budget_bytes=12 << 20),
               dict(pass_budget_bytes=1 << 20)]:  # the last splits the Hartree-Fock alpha class by beta class
        got = ctx.run(small["rid"], cutoff=cut, **kw)
        assert same(got, base), kw
    assert got["n_passes"] > 30


def test_cutoff_passes_are_planned_from_kept_counts(ctx, small):
    # the work list of a cutoff run counts the contributions it keeps (the
    # same decisions as the emission: each pass's record count is then checked
    # for equality), so its tiles hold the target and its passes run full
    s, r, e0 = small["s"], small["r"], small["e0"]
    cut, tt = 1e-5, 64
    ref = oracle.pt2(s.h, s.eri, r.keys, r.coef, e0, cutoff=cut)
    for budget in (12 << 20, 3 << 20):
        got = ctx.run(small["rid"], cutoff=cut, tile_target=tt, pass_budget_bytes=budget)
        exact = ctx.run(small["rid"], tile_target=tt, pass_budget_bytes=budget)
        assert_matches_oracle(got, ref)
        kept = got["n_terms"]
        assert kept < 0.6 * exact["n_terms"]
        assert kept / tt <= got["n_tiles"] <= kept / tt + got["n_passes"]
        assert got["n_passes"] <= 0.7 * exact["n_passes"] + 1, (got["n_passes"], exact["n_passes"])


def test_cutoff_with_constraint_classes(ctx, small):
    s, r, e0 = small["s"], small["r"], small["e0"]
    cut = 1e-5
    tot = 0.0
    for k in range(3):
        got = ctx.run(small["rid"], cutoff=cut, constraint=(3, k))
        ref = oracle.pt2(s.h, s.eri, r.keys, r.coef, e0, cutoff=cut, constraint=(3, k))
        assert_matches_oracle(got, ref)
        tot += got["e2"]
    assert e2_close(tot, ctx.run(small["rid"], cutoff=cut)["e2"])


def test_cutoff_with_spin_symmetry(ctx):
    w = inputs.WORKLOADS["small"]
    seed = inputs.workload_seed(w["seed_index"])
    s = inputs.make_integrals(w["n_orb"], seed)
    r = inputs.make_symmetric_reference(w["n_orb"], w["n_elec_per_spin"], w["n_det"], w["max_level"], seed + 1)
    e0 = oracle.e0_of(s.h, s.eri, r.keys)
    sid = ctx.load_system(s.h, s.eri)
    rid = ctx.load_reference(sid, r.keys, r.coef, e0)
    try:
        cut = 1e-5
        k, num, haa, ref = oracle.dump_external(s.h, s.eri, r.keys, r.coef, e0, cutoff=cut)
        got = ctx.run(rid, cutoff=cut, spin_symmetric=True)
        full = ctx.run(rid, cutoff=cut)
        assert_matches_oracle(full, ref)
        kept = k[k[:, 0] >= k[:, 1]]
        assert got["n_external"] == len(kept)
        assert (got["digest_sum"], got["digest_xor"]) == oracle.digest(kept)
        assert e2_close(got["e2"], ref["e2"])
        assert e2_close(got["e2"], full["e2"], 1e-12)
    finally:
        ctx.unload(rid)
        ctx.unload(sid)


def test_grouped_counts_with_cutoff_symmetry_and_slices(ctx):
    # a cutoff run on a symmetric reference, one class slice, many passes:
    # the single run counts its tiles in groups of passes, a batch of the same
    # run counts them per step; both must give the same result bit for bit,
    # and the slices must add up to the whole run
    w = inputs.WORKLOADS["small"]
    seed = inputs.workload_seed(w["seed_index"])
    s = inputs.make_integrals(w["n_orb"], seed)
    r = inputs.make_symmetric_reference(w["n_orb"], w["n_elec_per_spin"], w["n_det"], w["max_level"], seed + 1)
    e0 = oracle.e0_of(s.h, s.eri, r.keys)
    sid = ctx.load_system(s.h, s.eri)
    rid = ctx.load_reference(sid, r.keys, r.coef, e0)
    try:
        kw = dict(cutoff=1e-5, spin_symmetric=True, pass_budget_bytes=1 << 19, tile_target=128)
        whole = ctx.run(rid, cutoff=1e-5, spin_symmetric=True)
        parts = []
        for k in range(3):
            got = ctx.run(rid, class_slice=(k, 3), **kw)
            bid = ctx.batch_create([rid], class_slice=(k, 3), **kw)
            try:
                (b,) = ctx.batch_run(bid, 1)
            finally:
                ctx.batch_destroy(bid)
            assert same(got, b), k
            assert got["n_passes"] > 5
            parts.append(got)
        assert sum(p["n_terms"] for p in parts) == whole["n_terms"]
        assert sum(p["n_external"] for p in parts) == whole["n_external"]
        assert e2_close(sum(p["e2"] for p in parts), whole["e2"], 1e-13)
    finally:
        ctx.unload(rid)
        ctx.unload(sid)


def test_invalid_cutoff_is_rejected(ctx, small):
    for bad in (-1e-8, float("nan"), float("inf")):
        with pytest.raises(pt2.Pt2Error) as e:
            ctx.run(small["rid"], cutoff=bad)
        assert e.value.code == pt2.PT2_ERR_INVALID


def test_cutoff_in_batches_and_served_mix(ctx, small):
    cut = 1e-5
    s2, r2 = inputs.make_instance(dict(inputs.batch_instance_params(0), n_det=700))
    sid2 = ctx.load_system(s2.h, s2.eri)
    rid2 = ctx.load_reference(sid2, r2.keys, r2.coef, float(ctx.diagonal(sid2, r2.keys).min() - 0.1))
    try:
        ids = [small["rid"], rid2]
        alone = {i: ctx.run(i, cutoff=cut) for i in ids}
        exact = {i: ctx.run(i) for i in ids}
        bid = ctx.batch_create(ids, cutoff=cut)
        try:
            res = ctx.batch_run(bid, 2)
        finally:
            ctx.batch_destroy(bid)
        assert all(same(x, alone[i]) for x, i in zip(res, ids))
        # requests with and without the cutoff share the server's steps
        tickets = [(ctx.submit(ids[i % 2], cutoff=cut if i % 3 else 0.0), ids[i % 2], i % 3 != 0) for i in range(6)]
        for t, i, cutting in tickets:
            assert same(ctx.wait(t, timeout_s=600), alone[i] if cutting else exact[i])
    finally:
        ctx.unload(rid2)
        ctx.unload(sid2)
