"""Spin-flip (Z2) symmetric runs (subsection on Z2 spin symmetry for S_z = 0)
through the C ABI: only excited determinants with alpha >= beta (as 64-bit
words) are generated, sorted and reduced, and those with alpha > beta count
twice.

Against the oracle's full sum: E2 within 1e-10 (the tolerance of the other
parity tests); the kept half of the oracle's external set (alpha >= beta)
equals the symmetric run's external set bit-exactly (count, digest, keys),
numerators within 1e-13 and diagonals within 1e-11.  Against the ordinary
GPU path: E2 within 1e-12 relative (mirrored numerators are sums of the same
products computed with the two spins' loops in swapped order, so they may
differ in the last bit).  Symmetric runs are bit-identical across tilings,
pass plans (including a heavy alpha class split by beta class), batches and
served mixes with ordinary requests.
"""

import numpy as np
import pytest

import oracle
from paper_1808_02049_gb300 import inputs, pt2

pytestmark = pytest.mark.gpu

SAME = ("e2", "n_terms", "n_unique", "n_in_ref", "n_external", "digest_sum", "digest_xor", "n_pos_denom",
        "min_abs_denom")


def same(a, b):
    return all(a[k] == b[k] for k in SAME)


def e2_close(a, b, tol=1e-10):
    return abs(a - b) <= max(tol, tol * abs(b))


def sort_keys(k, *vals):
    order = np.lexsort((k[:, 1], k[:, 0]))
    return (k[order],) + tuple(v[order] for v in vals)


@pytest.fixture(scope="module")
def ctx():
    from paper_1808_02049_gb300 import build

    build.build_library()
    c = pt2.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def sym_small(ctx):
    w = inputs.WORKLOADS["small"]
    seed = inputs.workload_seed(w["seed_index"])
    s = inputs.make_integrals(w["n_orb"], seed)
    r = inputs.make_symmetric_reference(w["n_orb"], w["n_elec_per_spin"], w["n_det"], w["max_level"], seed + 1)
    e0 = oracle.e0_of(s.h, s.eri, r.keys)
    sid = ctx.load_system(s.h, s.eri)
    rid = ctx.load_reference(sid, r.keys, r.coef, e0)
    k, num, haa, ref = oracle.dump_external(s.h, s.eri, r.keys, r.coef, e0)
    keep = k[:, 0] >= k[:, 1]
    return dict(s=s, r=r, e0=e0, sid=sid, rid=rid, ref=ref, k=k[keep], num=num[keep], haa=haa[keep],
                sym=ctx.run(rid, spin_symmetric=True))


def test_symmetric_run_matches_oracle(sym_small):
    got, ref = sym_small["sym"], sym_small["ref"]
    assert e2_close(got["e2"], ref["e2"]), (got["e2"], ref["e2"])
    assert got["n_external"] == len(sym_small["k"])
    assert (got["digest_sum"], got["digest_xor"]) == oracle.digest(sym_small["k"])
    # about half of the terms are generated
    assert 0.4 * ref["n_terms"] < got["n_terms"] < 0.6 * ref["n_terms"]


def test_symmetric_dump_is_the_kept_half_of_the_oracle_set(ctx, sym_small):
    k, num, haa = ctx.dump_external(sym_small["rid"], len(sym_small["k"]) + 10, spin_symmetric=True)
    assert np.all(k[:, 0] >= k[:, 1])
    k, num, haa = sort_keys(k, num, haa)
    ok, onum, ohaa = sort_keys(sym_small["k"], sym_small["num"], sym_small["haa"])
    assert np.array_equal(k, ok)
    np.testing.assert_allclose(num, onum, rtol=0, atol=1e-13)
    np.testing.assert_allclose(haa, ohaa, rtol=0, atol=1e-11)


def test_symmetric_run_matches_full_gpu_path(ctx, sym_small):
    full = ctx.run(sym_small["rid"])
    assert e2_close(sym_small["sym"]["e2"], full["e2"], 1e-12)
    assert full["n_external"] == sym_small["ref"]["n_external"]


def test_symmetric_run_is_bit_identical_for_any_tiling_and_pass_plan(ctx, sym_small):
    base = sym_small["sym"]
    for kw in [dict(tile_target=16), dict(tile_target=1024), dict(pass_budget_bytes=12 << 20),
               dict(pass_budget_bytes=40 << 20, tile_target=100)]:
        got = ctx.run(sym_small["rid"], spin_symmetric=True, **kw)
        assert same(got, base), kw


def test_symmetric_heavy_alpha_class_split_by_beta_class(ctx, sym_small):
    # 150 determinants share the alpha string T of the four highest orbitals,
    # the largest 4-electron word, so every term they give with alpha' = T is
    # kept (T >= any beta'): at least 150 * (4*12 + 6*66) = 66,600 terms in
    # T's alpha class, where a 256 KB pass budget holds about 8,000 records.
    # The class must be split by beta class with the symmetric beta-class
    # counts (the run fails otherwise).
    s, n_orb, n = sym_small["s"], 16, 4
    top = ((1 << n) - 1) << (n_orb - n)
    rng = np.random.default_rng(5)
    ys = set()
    while len(ys) < 150:
        y = sum(1 << int(q) for q in rng.choice(n_orb, n, replace=False))
        if y != top:
            ys.add(y)
    dets, coef = [(top, top)], [0.9]
    for y in sorted(ys):
        v = float(rng.normal())
        dets += [(top, y), (y, top)]
        coef += [v, v]
    coef = np.array(coef)
    coef[1:] *= np.sqrt(1 - 0.81) / np.linalg.norm(coef[1:])
    keys = np.array([w for d in dets for w in d], dtype=np.uint64)
    e0 = oracle.e0_of(s.h, s.eri, keys)
    rid = ctx.load_reference(sym_small["sid"], keys, coef, e0)
    try:
        base = ctx.run(rid, spin_symmetric=True)
        got = ctx.run(rid, spin_symmetric=True, pass_budget_bytes=256 << 10)
        full = ctx.run(rid)
    finally:
        ctx.unload(rid)
    ref = oracle.pt2(s.h, s.eri, keys, coef, e0)
    assert got["n_passes"] > 30
    assert same(got, base)
    assert e2_close(base["e2"], ref["e2"]), (base["e2"], ref["e2"])
    assert e2_close(base["e2"], full["e2"], 1e-12)


def test_asymmetric_reference_is_rejected(ctx, sym_small):
    r = sym_small["r"]
    coef = r.coef.copy()
    coef[1] += 1e-3  # breaks c(beta, alpha) = c(alpha, beta) for one pair
    rid = ctx.load_reference(sym_small["sid"], r.keys, coef, sym_small["e0"])
    try:
        with pytest.raises(pt2.Pt2Error) as e:
            ctx.run(rid, spin_symmetric=True)
        assert e.value.code == pt2.PT2_ERR_INVALID
        ctx.run(rid)  # the ordinary path still runs
    finally:
        ctx.unload(rid)
    # drop one member of a mirror pair (alpha != beta)
    i = int(np.flatnonzero(r.keys[0::2] != r.keys[1::2])[0])
    keep = np.arange(r.n_det) != i
    keys = np.stack([r.keys[0::2][keep], r.keys[1::2][keep]], axis=1).reshape(-1)
    rid = ctx.load_reference(sym_small["sid"], keys, r.coef[keep], sym_small["e0"])
    try:
        with pytest.raises(pt2.Pt2Error) as e:
            ctx.run(rid, spin_symmetric=True)
        assert e.value.code == pt2.PT2_ERR_INVALID
    finally:
        ctx.unload(rid)


def test_symmetric_batches_and_served_mix(ctx, sym_small):
    refs = [sym_small]
    for k in range(3):
        prm = inputs.batch_instance_params(k)
        s = inputs.make_integrals(prm["n_orb"], prm["seed"])
        r = inputs.make_symmetric_reference(prm["n_orb"], prm["n_elec_per_spin"], min(prm["n_det"], 801),
                                            prm["max_level"], prm["seed"] + 1)
        sid = ctx.load_system(s.h, s.eri)
        e0 = float(ctx.diagonal(sid, r.keys).min() - 0.1)
        rid = ctx.load_reference(sid, r.keys, r.coef, e0)
        refs.append(dict(sid=sid, rid=rid, sym=ctx.run(rid, spin_symmetric=True)))
    full = {x["rid"]: ctx.run(x["rid"]) for x in refs}
    try:
        ids = [x["rid"] for x in refs]
        bid = ctx.batch_create(ids, spin_symmetric=True)
        try:
            res = ctx.batch_run(bid, len(ids))
        finally:
            ctx.batch_destroy(bid)
        for x, got in zip(refs, res):
            assert same(got, x["sym"])
            assert e2_close(got["e2"], full[x["rid"]]["e2"], 1e-12)
        # symmetric and ordinary requests share the server's steps
        tickets = [(ctx.submit(x["rid"], spin_symmetric=(i % 2 == 0)), x, i % 2 == 0)
                   for i, x in enumerate(refs + refs)]
        for t, x, sym in tickets:
            got = ctx.wait(t, timeout_s=600)
            assert same(got, x["sym"] if sym else full[x["rid"]])
    finally:
        for x in refs[1:]:
            ctx.unload(x["rid"])
            ctx.unload(x["sid"])


def test_symmetric_large_system_matches_full_gpu_path(ctx):
    # the 20-electron, 40-orbital system with a symmetric reference of 100,000
    # determinants: full size, against the ordinary path
    w = inputs.WORKLOADS["large"]
    seed = inputs.workload_seed(w["seed_index"])
    s = inputs.make_integrals(w["n_orb"], seed)
    r = inputs.make_symmetric_reference(w["n_orb"], w["n_elec_per_spin"], w["n_det"], w["max_level"], seed + 1)
    sid = ctx.load_system(s.h, s.eri)
    e0 = float(ctx.diagonal(sid, r.keys).min() - 0.1)
    rid = ctx.load_reference(sid, r.keys, r.coef, e0)
    try:
        full = ctx.run(rid)
        sym = ctx.run(rid, spin_symmetric=True)
    finally:
        ctx.unload(rid)
        ctx.unload(sid)
    assert e2_close(sym["e2"], full["e2"], 1e-12), (sym["e2"], full["e2"])
    assert 0.45 * full["n_terms"] < sym["n_terms"] < 0.55 * full["n_terms"]
    # each kept external determinant with alpha > beta stands for two
    assert sym["n_external"] < full["n_external"] <= 2 * sym["n_external"]
