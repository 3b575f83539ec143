"""The 24-electron / 60-orbital / 1,000,000-determinant workload (4.8e11
generated terms) at full size, in the launch configuration of a plain run.

Here the Hartree-Fock alpha string is shared by about 234,000 reference
determinants, so its alpha class holds about 1.8e10 terms, more than any pass;
the engine splits it by beta class.  The oracle cannot enumerate the full sum
in test time, so the full run is checked through properties that hold at any
size (closed-form term count, set bookkeeping, identical energy and set for a
different pass plan), and parity with the oracle on one alpha string: the
constraint with a modulus above every alpha word keeps exactly that string
(Algorithm 2 with a one-string constraint), which the oracle computes from
the few reference determinants within a double excitation of it.
"""

import math

import numpy as np
import pytest

import oracle
from paper_1808_02049_gb300 import inputs, pt2

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N_DET = 1_000_000
N_ORB, N_EL = 60, 12


@pytest.fixture(scope="module")
def million():
    from paper_1808_02049_gb300 import build

    build.build_library()
    s, r = inputs.make_workload("million")
    assert r.n_det == N_DET
    e0 = oracle.e0_of(s.h, s.eri, r.keys)
    c = pt2.Context(0)
    sid = c.load_system(s.h, s.eri)
    rid = c.load_reference(sid, r.keys, r.coef, e0)
    yield dict(c=c, s=s, r=r, e0=e0, rid=rid)
    c.close()


def test_full_size_with_heavy_alpha_class(million):
    c, rid = million["c"], million["rid"]
    alpha = million["r"].keys[0::2]
    assert np.unique(alpha, return_counts=True)[1].max() > 200_000
    a = c.run(rid)
    n, v = N_EL, N_ORB - N_EL
    T = 2 * n * v + 2 * math.comb(n, 2) * math.comb(v, 2) + (n * v) ** 2
    assert a["n_terms"] == T * N_DET == 481_824_000_000
    assert a["n_unique"] == a["n_in_ref"] + a["n_external"]
    assert a["n_in_ref"] <= N_DET
    assert a["n_passes"] >= a["n_terms"] * 32 // (96 << 30)  # passes of at most 96 GB
    assert math.isfinite(a["e2"]) and a["e2"] < 0
    # a smaller pass budget splits the classes differently: same energy and set
    b = c.run(rid, pass_budget_bytes=32 << 30)
    assert b["n_passes"] > a["n_passes"]
    assert b["e2"] == a["e2"]
    assert (b["digest_sum"], b["digest_xor"], b["n_external"]) == (a["digest_sum"], a["digest_xor"], a["n_external"])


@pytest.mark.parametrize("level", [3, 4])
def test_one_alpha_string_matches_oracle(million, level):
    # the smallest alpha string of the reference that is a triple (quadruple)
    # excitation of the Hartree-Fock one: a few thousand (hundred) reference
    # determinants lie within a double excitation of it
    c, s, r, e0, rid = million["c"], million["s"], million["r"], million["e0"], million["rid"]
    alpha = r.keys[0::2]
    hf = (1 << N_EL) - 1
    dist = np.array([bin(int(x) ^ hf).count("1") for x in alpha])
    a0 = int(alpha[dist == 2 * level].min())
    cls = (1 << 63, a0)
    got = c.run(rid, constraint=cls)
    ref = oracle.pt2(s.h, s.eri, r.keys, r.coef, e0, constraint=cls)
    assert ref["n_terms"] > 0
    assert got["n_terms"] == ref["n_terms"]
    assert got["n_external"] == ref["n_external"]
    assert got["n_in_ref"] == ref["n_in_ref"]
    assert (got["digest_sum"], got["digest_xor"]) == (ref["digest_sum"], ref["digest_xor"])
    assert got["n_pos_denom"] == ref["n_pos_denom"]
    assert abs(got["e2"] - ref["e2"]) <= max(1e-10, 1e-10 * abs(ref["e2"]))
    # the class energy is small, so check it relatively as well
    assert abs(got["e2"] - ref["e2"]) <= 1e-10 * abs(ref["e2"])


def test_slices_of_the_full_size_solve(million):
    # the benchmark's steps: 20 alpha-class slices, which together are one
    # complete solve of the 4.8e11 terms
    c, rid = million["c"], million["rid"]
    full = c.run(rid)
    parts = [c.run(rid, class_slice=(k, 20)) for k in range(20)]
    assert sum(p["n_terms"] for p in parts) == full["n_terms"] == 481_824_000_000
    assert sum(p["n_external"] for p in parts) == full["n_external"]
    assert sum(p["n_in_ref"] for p in parts) == full["n_in_ref"]
    assert sum(p["digest_sum"] for p in parts) % (1 << 64) == full["digest_sum"]
    assert abs(sum(p["e2"] for p in parts) - full["e2"]) <= 1e-14 * abs(full["e2"])
    # no slice is far from its share (the hash classes spread the terms)
    assert max(p["n_terms"] for p in parts) < 3 * full["n_terms"] / 20


def test_hashed_keys_on_a_slice_of_the_full_size_solve(million):
    c, rid = million["c"], million["rid"]
    a = c.run(rid, class_slice=(2, 20))
    b = c.run(rid, class_slice=(2, 20), hashed_keys=True)
    assert b["n_hash_collisions"] == 0
    assert a["e2"] == b["e2"]
    for f in ("n_terms", "n_unique", "n_in_ref", "n_external", "digest_sum", "digest_xor"):
        assert a[f] == b[f], f
