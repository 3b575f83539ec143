"""Triplet and quadruplet constraints (the "Triplet constraints" section and
Algorithm 3) through the C ABI, against the oracle.

A run with pt2_opts.top_alpha = T sums only the excited determinants whose
k = popcount(T) highest occupied alpha orbitals are T; its alpha-alpha
doubles are generated directly (Algorithm 3) instead of through the bucket
table of the hash classes.  Every such class must match the oracle (set
bit-exactly, E2 within 1e-10), and the classes of each k must add up to the
unconstrained run exactly.
"""

import itertools

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
    return dict(s=s, r=r, e0=e0, sid=sid, rid=rid)


def same(got, ref):
    for f in ("n_terms", "n_external", "n_in_ref", "n_unique", "digest_sum", "digest_xor", "n_pos_denom"):
        assert got[f] == ref[f], f
    assert e2_close(got["e2"], ref["e2"]), (got["e2"], ref["e2"])


def test_triplets_partition_the_run(ctx, small):
    full = ctx.run(small["rid"])
    tot = dict(n_terms=0, n_external=0, n_in_ref=0, digest_sum=0, digest_xor=0, e2=0.0)
    nonzero = []
    for orbs in itertools.combinations(range(16), 3):
        T = sum(1 << q for q in orbs)
        g = ctx.run(small["rid"], top_alpha=T)
        for f in ("n_terms", "n_external", "n_in_ref"):
            tot[f] += g[f]
        tot["digest_sum"] = (tot["digest_sum"] + g["digest_sum"]) % 2 ** 64
        tot["digest_xor"] ^= g["digest_xor"]
        tot["e2"] += g["e2"]
        if g["n_terms"]:
            nonzero.append((g["n_terms"], T))
    for f in ("n_terms", "n_external", "n_in_ref", "digest_sum", "digest_xor"):
        assert tot[f] == full[f], f
    assert abs(tot["e2"] - full["e2"]) <= 1e-13 * abs(full["e2"])
    small["heavy"] = [T for _, T in sorted(nonzero, reverse=True)]
    assert len(nonzero) > 100


def test_triplet_classes_match_oracle(ctx, small):
    s, r, e0 = small["s"], small["r"], small["e0"]
    heavy = small.get("heavy") or []
    rng = np.random.default_rng(7)
    picks = heavy[:6] + [heavy[i] for i in rng.choice(len(heavy), size=6, replace=False)] if heavy else []
    if not picks:
        picks = [0b111 << 1, 0b1011 << 2, (1 << 15) | (1 << 3) | (1 << 2)]
    for T in picks:
        got = ctx.run(small["rid"], top_alpha=T)
        ref = oracle.pt2(s.h, s.eri, r.keys, r.coef, e0, top_alpha=T)
        same(got, ref)


def test_quadruplet_classes_match_oracle_and_partition(ctx, small):
    s, r, e0 = small["s"], small["r"], small["e0"]
    full = ctx.run(small["rid"])
    tot_terms, tot_e2, checked = 0, 0.0, 0
    for orbs in itertools.combinations(range(16), 4):
        T = sum(1 << q for q in orbs)
        g = ctx.run(small["rid"], top_alpha=T)
        tot_terms += g["n_terms"]
        tot_e2 += g["e2"]
        if g["n_terms"] and checked < 8 and orbs[0] >= 2:
            same(g, oracle.pt2(s.h, s.eri, r.keys, r.coef, e0, top_alpha=T))
            checked += 1
    assert tot_terms == full["n_terms"]
    assert abs(tot_e2 - full["e2"]) <= 1e-13 * abs(full["e2"])
    assert checked == 8


def test_triplet_with_slices_and_subtraction(ctx, small):
    # the triplet constraint combines with the class slices and with
    # duplicate subtraction; per triplet the slices add up to the triplet run
    T = small.get("heavy", [0b1110])[0]
    whole = ctx.run(small["rid"], top_alpha=T, subtract_ref=True)
    parts = [ctx.run(small["rid"], top_alpha=T, subtract_ref=True, class_slice=(k, 3)) for k in range(3)]
    assert sum(p["n_terms"] for p in parts) == whole["n_terms"]
    assert abs(sum(p["e2"] for p in parts) - whole["e2"]) <= 1e-14 * max(1e-300, abs(whole["e2"]))


def test_triplet_on_a_brute_force_system(ctx):
    from test_oracle_pins import strong_integrals

    n_orb, na, nb, n_ref, seed = 6, 3, 3, 5, 5
    h, eri = strong_integrals(n_orb, seed)
    dets = brute.basis(n_orb, na, nb)
    H = brute.hamiltonian(h, eri, dets)
    rng = np.random.default_rng(100 + seed)
    idx = sorted(rng.choice(len(dets), size=n_ref, replace=False).tolist())
    coef = rng.normal(0, 1, n_ref)
    e0 = float(min(H[i, i] for i in idx) - 0.37)
    keys = np.empty(2 * n_ref, dtype=np.uint64)
    keys[0::2] = [dets[i][0] for i in idx]
    keys[1::2] = [dets[i][1] for i in idx]
    sid = ctx.load_system(h, eri)
    rid = ctx.load_reference(sid, keys, coef, e0)
    try:
        for orbs in itertools.combinations(range(n_orb), 3):
            T = sum(1 << q for q in orbs)
            got = ctx.run(rid, top_alpha=T)
            ref = oracle.pt2(h, eri, keys, coef, e0, top_alpha=T)
            same(got, ref)
    finally:
        ctx.unload(rid)
        ctx.unload(sid)
