"""Pins of the spin-flip (Z2) reading against the second-quantised Hamiltonian
and the oracle (subsection on Z2 spin symmetry for S_z = 0).

Exchanging the alpha and beta strings of every determinant changes each
determinant by the same sign (alpha creators are ordered before beta ones),
so H_(b,a),(b',a') = H_(a,b),(a',b').  For a reference closed under the
exchange with c(b, a) = c(a, b) the connected external set is closed under it
too, mirrored determinants have the same numerator and diagonal, and
E2 = sum over alpha == beta + 2 * sum over alpha > beta, which is what the
symmetric run computes from the kept half alpha >= beta.
"""

import numpy as np

import brute
import oracle
from paper_1808_02049_gb300 import inputs
from test_oracle_pins import keys_of, strong_integrals


def symmetric_ref(dets, n_ref, seed):
    """n_ref determinants (with their mirrors) of a brute-force basis and
    coefficients equal on mirror pairs."""
    rng = np.random.default_rng(seed)
    pos = {d: i for i, d in enumerate(dets)}
    chosen = []
    for i in rng.permutation(len(dets)).tolist():
        a, b = dets[i]
        if (a, b) in chosen:
            continue
        chosen.append((a, b))
        if a != b:
            chosen.append((b, a))
        if len(chosen) >= n_ref:
            break
    coef, seen = [], {}
    for a, b in chosen:
        key = (min(a, b), max(a, b))
        if key not in seen:
            seen[key] = float(rng.normal())
        coef.append(seen[key])
    return [pos[d] for d in chosen], chosen, np.array(coef)


def halves(keys2, num, haa, e0):
    term = num ** 2 / (e0 - haa)
    a, b = keys2[:, 0], keys2[:, 1]
    return term[a == b].sum() + 2.0 * term[a > b].sum()


def test_mirror_symmetry_brute_force():
    for n_orb, n, n_ref, seed in [(5, 2, 5, 1), (6, 2, 7, 2), (6, 3, 9, 3)]:
        h, eri = strong_integrals(n_orb, seed)
        dets = brute.basis(n_orb, n, n)
        H = brute.hamiltonian(h, eri, dets)
        pos = {d: i for i, d in enumerate(dets)}
        flip = np.array([pos[(b, a)] for a, b in dets])
        # the exchange is a symmetry of H in this phase convention
        assert np.abs(H[np.ix_(flip, flip)] - H).max() < 1e-13
        ref_idx, ref, coef = symmetric_ref(dets, n_ref, 10 + seed)
        e0 = float(min(H[i, i] for i in ref_idx) - 0.29)
        bf = brute.pt2(h, eri, dets, H, ref_idx, coef, e0)
        got = halves(bf["keys"], bf["num"], bf["haa"], e0)
        assert abs(got - bf["e2"]) <= 1e-12 * max(1.0, abs(bf["e2"]))
        # and the oracle's external set obeys the same identity
        k, num, haa, res = oracle.dump_external(h, eri, keys_of(ref), coef, e0)
        assert abs(halves(k, num, haa, e0) - res["e2"]) <= 1e-12 * max(1.0, abs(res["e2"]))


def mirror_check(k, num, haa):
    idx = {(a, b): i for i, (a, b) in enumerate(k.tolist())}
    worst = 0.0
    for i, (a, b) in enumerate(k.tolist()):
        j = idx.get((b, a))
        if j is None:
            return None
        worst = max(worst, abs(num[i] - num[j]), abs(haa[i] - haa[j]))
    return worst


def test_symmetric_reference_generator_and_oracle_mirrors():
    s = inputs.make_integrals(12, inputs.workload_seed(9))
    r = inputs.make_symmetric_reference(12, 3, 301, 3, inputs.workload_seed(9) + 1)
    a, b = r.keys[0::2], r.keys[1::2]
    pairs = {(x, y): c for x, y, c in zip(a.tolist(), b.tolist(), r.coef.tolist())}
    assert len(pairs) == r.n_det == 301
    assert all(pairs[(y, x)] == c for (x, y), c in pairs.items())
    assert abs(np.linalg.norm(r.coef) - 1.0) < 1e-12
    e0 = oracle.e0_of(s.h, s.eri, r.keys)
    k, num, haa, res = oracle.dump_external(s.h, s.eri, r.keys, r.coef, e0)
    worst = mirror_check(k, num, haa)
    assert worst is not None and worst < 1e-12
    assert abs(halves(k, num, haa, e0) - res["e2"]) <= 1e-12 * abs(res["e2"])
    # an ordinary reference is not closed under the exchange: the identity is not vacuous
    r2 = inputs.make_reference(12, 3, 301, 3, inputs.workload_seed(9) + 1)
    k2, num2, haa2, res2 = oracle.dump_external(s.h, s.eri, r2.keys, r2.coef, e0)
    w2 = mirror_check(k2, num2, haa2)
    assert w2 is None or w2 > 1e-6
    assert abs(halves(k2, num2, haa2, e0) - res2["e2"]) > 1e-9 * abs(res2["e2"])


def test_reference_generators_are_seeded_and_refuse_impossible_sizes():
    import pytest

    a = inputs.make_symmetric_reference(12, 3, 101, 3, 5)
    b = inputs.make_symmetric_reference(12, 3, 101, 3, 5)
    assert np.array_equal(a.keys, b.keys) and np.array_equal(a.coef, b.coef)
    # an even size needs one self-mirrored determinant besides Hartree-Fock
    c = inputs.make_symmetric_reference(12, 3, 100, 3, 5)
    assert int(np.sum(c.keys[0::2] == c.keys[1::2])) == 2
    with pytest.raises(ValueError):
        inputs.make_reference(6, 2, 10 ** 6, 2, 1)
    with pytest.raises(ValueError):
        inputs.make_symmetric_reference(6, 2, 10 ** 6, 2, 1)
    with pytest.raises(ValueError):
        inputs.make_symmetric_reference(12, 3, 100, 1, 1)
