"""Pins of the CPU oracle against things other than itself.

* brute force: full determinant space, H built by second-quantised operator
  application (tests/brute.py), E2 of Eq. 3 evaluated from the dense matrix;
* the closed-form term count T(n, v) = 2 n v + 2 C(n,2) C(v,2) + (n v)^2 per
  determinant (all singles and doubles, structural);
* the duplicate-removal identity of the paper (subtracting c_i^2 (E - H_ii)
  from the unfiltered sum gives the filtered one when c is an eigenvector of
  H in the reference space), for the whole sum and per constraint class;
* the numerator cutoff against brute force (contributions filtered column by
  column in the dense H), and its constraint classes partitioning the sum;
* invariants: c -> 2c scales E2 by exactly 4; swapping alpha and beta words of
  every determinant leaves E2 unchanged; reordering the reference leaves E2
  unchanged; the constraint classes alpha % m = r partition the sum
  (Algorithm 2: non-overlapping and complete constraints).
"""

import math

import numpy as np
import pytest

import brute
import oracle
from paper_1808_02049_gb300 import inputs


def strong_integrals(n, seed, scale=0.3):
    """Random real integrals with full 8-fold symmetry and O(0.1-1) entries,
    so that a wrong sign or index shows up far above rounding."""
    rng = np.random.default_rng(seed)
    h = rng.normal(0, scale, (n, n))
    h = h + h.T
    h[np.diag_indices(n)] = -2.0 + 0.4 * np.arange(n)
    a = rng.normal(0, scale, (n, n, n, n))
    perms = [(0, 1, 2, 3), (1, 0, 2, 3), (0, 1, 3, 2), (1, 0, 3, 2),
             (2, 3, 0, 1), (3, 2, 0, 1), (2, 3, 1, 0), (3, 2, 1, 0)]
    eri = sum(a.transpose(p) for p in perms) / 8.0
    for p in range(n):
        for q in range(n):
            eri[p, p, q, q] = eri[q, q, p, p] = 0.5 + 0.1 * abs(math.sin(p + 3 * q + seed))
    return np.ascontiguousarray(h), np.ascontiguousarray(eri)


def keys_of(dets):
    k = np.empty(2 * len(dets), dtype=np.uint64)
    k[0::2] = [d[0] for d in dets]
    k[1::2] = [d[1] for d in dets]
    return k


CASES = [
    # (n_orb, n_alpha, n_beta, n_ref, seed)
    (4, 2, 2, 3, 1),
    (5, 2, 2, 6, 2),
    (5, 2, 1, 4, 3),
    (6, 2, 2, 8, 4),
    (6, 3, 3, 5, 5),
    (6, 3, 2, 1, 6),
]


@pytest.fixture(scope="module")
def brute_cases():
    out = []
    for n_orb, na, nb, n_ref, seed in CASES:
        h, eri = strong_integrals(n_orb, seed)
        dets = brute.basis(n_orb, na, nb)
        H = brute.hamiltonian(h, eri, dets)
        rng = np.random.default_rng(100 + seed)
        ref_idx = sorted(rng.choice(len(dets), size=n_ref, replace=False).tolist())
        coef = rng.normal(0, 1, n_ref)
        ref = [dets[i] for i in ref_idx]
        e0 = float(min(H[i, i] for i in ref_idx) - 0.37)
        out.append(dict(h=h, eri=eri, dets=dets, H=H, ref_idx=ref_idx, coef=coef, ref=ref, e0=e0))
    return out


def test_brute_hamiltonian_is_symmetric(brute_cases):
    for c in brute_cases:
        assert np.abs(c["H"] - c["H"].T).max() < 1e-13


def test_brute_rank_above_two_has_no_coupling(brute_cases):
    # H only connects determinants at most two excitations apart
    for c in brute_cases:
        res = brute.pt2(c["h"], c["eri"], c["dets"], c["H"], c["ref_idx"], c["coef"], c["e0"])
        assert res["far_max"] < 1e-13


def test_oracle_matches_brute_force(brute_cases):
    for c in brute_cases:
        keys = keys_of(c["ref"])
        bf = brute.pt2(c["h"], c["eri"], c["dets"], c["H"], c["ref_idx"], c["coef"], c["e0"])
        k, num, haa, res = oracle.dump_external(c["h"], c["eri"], keys, c["coef"], c["e0"])
        # connected external set: bit-exact
        assert k.shape == bf["keys"].shape
        assert np.array_equal(k, bf["keys"])
        assert res["n_external"] == len(bf["keys"])
        # numerators <a|H|psi> and diagonals
        np.testing.assert_allclose(num, bf["num"], rtol=0, atol=1e-12)
        np.testing.assert_allclose(haa, bf["haa"], rtol=0, atol=1e-12)
        assert abs(res["e2"] - bf["e2"]) <= 1e-12 * max(1.0, abs(bf["e2"]))


def test_numerator_cutoff_matches_brute_force(brute_cases):
    # the cutoff of the Results section: contributions |c_i H_ai| below it are
    # ignored; with the cutoff at the median contribution about half go, and
    # whole determinants leave the set when all of theirs do
    for c in brute_cases:
        keys = keys_of(c["ref"])
        ref_idx = c["ref_idx"]
        contrib = np.abs(c["H"][:, ref_idx] * c["coef"][None, :])
        conn = np.array([[brute.rank(d, c["dets"][i]) in (1, 2) for i in ref_idx] for d in c["dets"]])
        cut = float(np.median(contrib[conn]))
        bf = brute.pt2(c["h"], c["eri"], c["dets"], c["H"], ref_idx, c["coef"], c["e0"], cutoff=cut)
        full = brute.pt2(c["h"], c["eri"], c["dets"], c["H"], ref_idx, c["coef"], c["e0"])
        k, num, haa, res = oracle.dump_external(c["h"], c["eri"], keys, c["coef"], c["e0"], cutoff=cut)
        assert np.array_equal(k, bf["keys"])
        np.testing.assert_allclose(num, bf["num"], rtol=0, atol=1e-12)
        np.testing.assert_allclose(haa, bf["haa"], rtol=0, atol=1e-12)
        assert abs(res["e2"] - bf["e2"]) <= 1e-12 * max(1.0, abs(bf["e2"]))
        assert len(bf["keys"]) <= len(full["keys"]) and bf["e2"] != full["e2"]
        # kept contributions: the connected pairs at or above the cutoff (terms
        # landing on reference determinants included)
        assert res["n_terms"] == int((contrib[conn] >= cut).sum())
        assert oracle.pt2(c["h"], c["eri"], keys, c["coef"], c["e0"], cutoff=0.0) == \
            oracle.pt2(c["h"], c["eri"], keys, c["coef"], c["e0"])


def test_oracle_diagonal_matches_brute_force(brute_cases):
    for c in brute_cases:
        keys = keys_of(c["dets"])
        d = oracle.diagonals(c["h"], c["eri"], keys)
        np.testing.assert_allclose(d, np.diag(c["H"]), rtol=0, atol=1e-12)


def test_det_terms_match_brute_force_columns(brute_cases):
    # every single/double of a determinant, with H_ai c_i equal to the
    # brute-force matrix element times c_i
    for c in brute_cases:
        dets = c["dets"]
        idx = {d: k for k, d in enumerate(dets)}
        i = c["ref_idx"][0]
        d = dets[i]
        k, v, haa = oracle.det_terms(c["h"], c["eri"], d[0], d[1], 0.75)
        expect = [k2 for k2, dd in enumerate(dets) if brute.rank(d, dd) in (1, 2)]
        assert sorted(idx[(int(a), int(b))] for a, b in k) == sorted(expect)
        for (a, b), val, hh in zip(k.tolist(), v, haa):
            j = idx[(a, b)]
            assert abs(val - 0.75 * c["H"][j, i]) < 1e-12
            assert abs(hh - c["H"][j, j]) < 1e-12


def T(n, v):
    return 2 * n * v + 2 * math.comb(n, 2) * math.comb(v, 2) + (n * v) ** 2


def test_term_count_closed_form_small_workload():
    s, r = inputs.make_workload("small")
    e0 = oracle.e0_of(s.h, s.eri, r.keys)
    res = oracle.pt2(s.h, s.eri, r.keys, r.coef, e0)
    n, v = 4, 12
    assert T(n, v) == 3192
    assert res["n_terms"] == T(n, v) * r.n_det
    assert res["n_unique"] == res["n_in_ref"] + res["n_external"]
    # every reference determinant except possibly isolated ones is reached
    assert res["n_in_ref"] <= r.n_det


def test_det_terms_count_and_uniqueness():
    s, r = inputs.make_workload("small")
    for i in (0, 17, 999):
        k, v, _ = oracle.det_terms(s.h, s.eri, r.keys[2 * i], r.keys[2 * i + 1], r.coef[i])
        assert k.shape[0] == T(4, 12)
        assert len({(a, b) for a, b in k.tolist()}) == k.shape[0]
        for a, b in k.tolist():
            rk = (bin(a ^ int(r.keys[2 * i])).count("1") + bin(b ^ int(r.keys[2 * i + 1])).count("1")) // 2
            assert rk in (1, 2)


def test_subtraction_identity_eigenvector_reference():
    # Sec. "Removal of duplicate PT2 contributions": with c the lowest
    # eigenvector of H in the reference space and E0 its eigenvalue, the
    # unfiltered sum minus sum_i c_i^2 (E0 - H_ii) equals the filtered E2.
    for seed, (n_orb, na, nb, n_ref) in enumerate([(5, 2, 2, 7), (6, 2, 2, 12), (6, 3, 3, 9)]):
        h, eri = strong_integrals(n_orb, 40 + seed)
        dets = brute.basis(n_orb, na, nb)
        rng = np.random.default_rng(7 + seed)
        ref = [dets[i] for i in sorted(rng.choice(len(dets), n_ref, replace=False))]
        keys = keys_of(ref)
        Hr = brute.hamiltonian(h, eri, dets)
        idx = {d: k for k, d in enumerate(dets)}
        ri = [idx[d] for d in ref]
        w, V = np.linalg.eigh(Hr[np.ix_(ri, ri)])
        c, e0 = V[:, 0], w[0]
        res = oracle.pt2(h, eri, keys, c, e0, include_ref=True)
        hii = oracle.diagonals(h, eri, keys)
        sub = float(np.sum(c ** 2 * (e0 - hii)))
        # reference keys the enumeration never reaches contribute c_i^2 (E0 - H_ii)
        # to the subtraction but nothing to the unfiltered sum
        reached = set()
        for d in ref:
            kk, _, _ = oracle.det_terms(h, eri, d[0], d[1], 1.0)
            reached |= {(a, b) for a, b in kk.tolist()}
        unreached = [i for i, d in enumerate(ref) if d not in reached]
        sub_reached = sub - float(np.sum(c[unreached] ** 2 * (e0 - hii[unreached])))
        unfiltered = res["e2"] + res["e2_ref_like"]
        assert abs((unfiltered - sub_reached) - res["e2"]) < 1e-11


def test_subtraction_identity_per_constraint_class():
    # the identity holds key by key, so it holds in every constraint class:
    # the class's unfiltered sum minus c_i^2 (E0 - H_ii) over the reference
    # determinants of the class equals the class's filtered E2
    for seed, (n_orb, n, n_ref) in enumerate([(6, 2, 14), (6, 3, 12)]):
        h, eri = strong_integrals(n_orb, 60 + seed)
        dets = brute.basis(n_orb, n, n)
        rng = np.random.default_rng(70 + seed)
        ref = [dets[i] for i in sorted(rng.choice(len(dets), n_ref, replace=False))]
        keys = keys_of(ref)
        H = brute.hamiltonian(h, eri, dets)
        idx = {d: k for k, d in enumerate(dets)}
        ri = [idx[d] for d in ref]
        w, V = np.linalg.eigh(H[np.ix_(ri, ri)])
        c, e0 = V[:, 0], w[0]
        hii = oracle.diagonals(h, eri, keys)
        reached = set()
        for d in ref:
            kk, _, _ = oracle.det_terms(h, eri, d[0], d[1], 1.0)
            reached |= {(a, b) for a, b in kk.tolist()}
        for m, r in [(3, 0), (3, 1), (3, 2)]:
            res = oracle.pt2(h, eri, keys, c, e0, constraint=(m, r), include_ref=True)
            sub = sum(c[i] ** 2 * (e0 - hii[i]) for i, d in enumerate(ref) if d[0] % m == r and d in reached)
            assert abs(res["e2"] + res["e2_ref_like"] - sub - res["e2"]) < 1e-11


def test_cutoff_constraint_classes_partition_the_sum():
    s = inputs.make_integrals(12, inputs.workload_seed(8))
    r = inputs.make_reference(12, 3, 200, 3, inputs.workload_seed(8) + 1)
    e0 = oracle.e0_of(s.h, s.eri, r.keys)
    cut = 1e-4
    full = oracle.pt2(s.h, s.eri, r.keys, r.coef, e0, cutoff=cut)
    exact = oracle.pt2(s.h, s.eri, r.keys, r.coef, e0)
    assert full["n_terms"] < exact["n_terms"]
    parts = [oracle.pt2(s.h, s.eri, r.keys, r.coef, e0, cutoff=cut, constraint=(4, k)) for k in range(4)]
    assert sum(p["n_terms"] for p in parts) == full["n_terms"]
    assert sum(p["n_external"] for p in parts) == full["n_external"]
    assert abs(sum(p["e2"] for p in parts) - full["e2"]) < 1e-12 * abs(full["e2"])


def test_scaling_swap_permutation_invariants():
    s, r = inputs.make_workload("small", n_det=200)
    e0 = oracle.e0_of(s.h, s.eri, r.keys)
    base = oracle.pt2(s.h, s.eri, r.keys, r.coef, e0)
    dbl = oracle.pt2(s.h, s.eri, r.keys, 2.0 * r.coef, e0)
    assert dbl["e2"] == 4.0 * base["e2"]  # power-of-two scaling is exact in FP64
    sw = r.keys.copy()
    sw[0::2], sw[1::2] = r.keys[1::2], r.keys[0::2]
    swp = oracle.pt2(s.h, s.eri, sw, r.coef, e0)
    assert abs(swp["e2"] - base["e2"]) <= 1e-12 * abs(base["e2"])
    assert swp["n_external"] == base["n_external"]
    perm = np.random.default_rng(3).permutation(r.n_det)
    pk = np.empty_like(r.keys)
    pk[0::2], pk[1::2] = r.keys[0::2][perm], r.keys[1::2][perm]
    pp = oracle.pt2(s.h, s.eri, pk, r.coef[perm], e0)
    assert abs(pp["e2"] - base["e2"]) <= 1e-12 * abs(base["e2"])
    assert (pp["digest_sum"], pp["digest_xor"]) == (base["digest_sum"], base["digest_xor"])


def test_constraint_classes_partition_the_sum():
    s, r = inputs.make_workload("small", n_det=150)
    e0 = oracle.e0_of(s.h, s.eri, r.keys)
    base = oracle.pt2(s.h, s.eri, r.keys, r.coef, e0)
    m = 7
    parts = [oracle.pt2(s.h, s.eri, r.keys, r.coef, e0, constraint=(m, k)) for k in range(m)]
    assert sum(p["n_terms"] for p in parts) == base["n_terms"]
    assert sum(p["n_external"] for p in parts) == base["n_external"]
    assert sum(p["digest_sum"] for p in parts) % 2 ** 64 == base["digest_sum"]
    x = 0
    for p in parts:
        x ^= p["digest_xor"]
    assert x == base["digest_xor"]
    assert abs(sum(p["e2"] for p in parts) - base["e2"]) <= 1e-13 * abs(base["e2"])


def test_single_alpha_string_classes_partition_the_sum():
    # With a modulus above every alpha word the constraint keeps one alpha
    # string, and the oracle skips reference determinants more than a double
    # excitation away from it.  Over all C(16, 4) = 1820 alpha strings the
    # classes are complete, so they must rebuild the unconstrained result;
    # a wrongly skipped determinant would lose its terms.
    import itertools

    s, r = inputs.make_workload("small", n_det=60)
    e0 = oracle.e0_of(s.h, s.eri, r.keys)
    base = oracle.pt2(s.h, s.eri, r.keys, r.coef, e0)
    mod = 1 << 40
    tot_terms = tot_ext = dsum = dxor = 0
    e2 = 0.0
    for occ in itertools.combinations(range(16), 4):
        a = sum(1 << q for q in occ)
        p = oracle.pt2(s.h, s.eri, r.keys, r.coef, e0, constraint=(mod, a))
        tot_terms += p["n_terms"]
        tot_ext += p["n_external"]
        dsum = (dsum + p["digest_sum"]) % 2 ** 64
        dxor ^= p["digest_xor"]
        e2 += p["e2"]
    assert tot_terms == base["n_terms"]
    assert tot_ext == base["n_external"]
    assert (dsum, dxor) == (base["digest_sum"], base["digest_xor"])
    assert abs(e2 - base["e2"]) <= 1e-13 * abs(base["e2"])


def test_oracle_rejects_invalid_reference():
    s, r = inputs.make_workload("small", n_det=10)
    bad = r.keys.copy()
    bad[2] = bad[0]
    bad[3] = bad[1]  # duplicate determinant
    with pytest.raises(ValueError):
        oracle.pt2(s.h, s.eri, bad, r.coef, -10.0)
    bad = r.keys.copy()
    bad[4] |= np.uint64(1 << 20)  # bit beyond n_orb = 16, wrong popcount
    with pytest.raises(ValueError):
        oracle.pt2(s.h, s.eri, bad, r.coef, -10.0)


def _top_orbitals(word, k):
    """The k highest set bits of word as a mask (a plain restatement of the
    triplet constraint's definition, independent of the oracle's C)."""
    bits = [p for p in range(64) if (int(word) >> p) & 1]
    return sum(1 << p for p in bits[-k:]) if len(bits) >= k else -1


def test_triplet_constraint_matches_brute_force(brute_cases):
    # per triplet T: the brute-force external set and energy restricted to
    # determinants whose three highest occupied alpha orbitals are T
    import itertools

    for c in brute_cases:
        n = c["h"].shape[0]
        na = bin(int(c["ref"][0][0])).count("1")
        if na < 3:
            continue
        keys = keys_of(c["ref"])
        bf = brute.pt2(c["h"], c["eri"], c["dets"], c["H"], c["ref_idx"], c["coef"], c["e0"])
        terms = bf["num"] ** 2 / (c["e0"] - bf["haa"])
        tops = np.array([_top_orbitals(k[0], 3) for k in bf["keys"]])
        seen = 0
        for trip in itertools.combinations(range(n), 3):
            T = sum(1 << p for p in trip)
            sel = tops == T
            res = oracle.pt2(c["h"], c["eri"], keys, c["coef"], c["e0"], top_alpha=T)
            assert res["n_external"] == int(sel.sum())
            assert abs(res["e2"] - terms[sel].sum()) <= 1e-12 * max(1.0, abs(bf["e2"]))
            seen += int(sel.sum())
        assert seen == len(bf["keys"])


@pytest.mark.parametrize("k", [3, 4])
def test_top_orbital_constraints_partition_the_sum(k):
    # the triplet (k = 3) and quadruplet (k = 4) constraints are
    # non-overlapping and complete: over every mask of k of the 16 orbitals
    # the classes rebuild the unconstrained result exactly
    import itertools

    s, r = inputs.make_workload("small", n_det=40 if k == 3 else 15)
    e0 = oracle.e0_of(s.h, s.eri, r.keys)
    base = oracle.pt2(s.h, s.eri, r.keys, r.coef, e0)
    tot = dict(n_terms=0, n_external=0, n_in_ref=0, digest_sum=0, digest_xor=0, e2=0.0)
    for orbs in itertools.combinations(range(16), k):
        p = oracle.pt2(s.h, s.eri, r.keys, r.coef, e0, top_alpha=sum(1 << q for q in orbs))
        for f in ("n_terms", "n_external", "n_in_ref"):
            tot[f] += p[f]
        tot["digest_sum"] = (tot["digest_sum"] + p["digest_sum"]) % 2 ** 64
        tot["digest_xor"] ^= p["digest_xor"]
        tot["e2"] += p["e2"]
    for f in ("n_terms", "n_external", "n_in_ref", "digest_sum", "digest_xor"):
        assert tot[f] == base[f], f
    assert abs(tot["e2"] - base["e2"]) <= 1e-12 * abs(base["e2"])
