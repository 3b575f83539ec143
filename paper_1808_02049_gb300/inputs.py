"""Seeded synthetic PT2 inputs: integrals, reference determinants, coefficients.

This module only draws random numbers and lays them out.  It holds none of the
PT2 arithmetic (no matrix elements, no diagonals, no energies), so the CUDA
path and the CPU oracle can both consume its output without sharing any of the
method's code.  E0 is therefore not produced here: the recipe defines it as the
lowest reference diagonal minus 0.1 Ha, and each side computes that diagonal
with its own code.

Recipe (the paper's molecules and ASCI wavefunctions are not available, so
these stand in for them; Sec. "Results", Tables 1-6 use real FCIDUMPs):

* one-electron integrals h: symmetric, h_pp = -2.0 + 0.25 p, h_pq ~ N(0, 0.02);
* two-electron integrals (pq|rs), chemist notation, 8-fold symmetric:
  (pp|qq) ~ U(0.3, 0.7) for every orbital pair p <= q (p = q included), every
  other unique element ~ N(0, 0.01) * exp(-0.1 (|p-q| + |r-s|));
* reference: the Hartree-Fock determinant (lowest n orbitals of each spin) plus
  random excitations of it.  An excitation level l is drawn uniformly from
  1..max_level, split between alpha and beta uniformly over the feasible
  splits, and the removed/added orbitals are drawn uniformly without
  replacement; duplicates are rejected until n_det determinants exist;
* coefficients: c_HF = 0.95, the others N(0,1) * exp(-0.5 l), rescaled so that
  the non-HF part has norm sqrt(1 - 0.95^2) (the whole vector has unit norm
  and c_HF stays 0.95).

Keys are 64-bit occupation words, orbital p <-> bit p, stored as
keys[2 i] = alpha word, keys[2 i + 1] = beta word (alpha is the more
significant half of the 128-bit determinant key, Sec. "Triplet constraints").

Random numbers come from numpy's PCG64 generator seeded with the given seed.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "System",
    "Reference",
    "make_integrals",
    "make_reference",
    "make_symmetric_reference",
    "make_workload",
    "batch_instance_params",
    "WORKLOADS",
    "workload_seed",
]

SEED_BASE = 20181806


def workload_seed(index: int, instance: int = 0) -> int:
    """Seed of a workload with seed index `index`: base + 1000 * index + instance."""
    return SEED_BASE + 1000 * index + instance


@dataclasses.dataclass
class System:
    n_orb: int
    h: np.ndarray  # (n, n) float64, symmetric
    eri: np.ndarray  # (n, n, n, n) float64, chemist (pq|rs)


@dataclasses.dataclass
class Reference:
    n_alpha: int
    n_beta: int
    keys: np.ndarray  # (2 * n_det,) uint64: alpha, beta interleaved
    coef: np.ndarray  # (n_det,) float64
    level: np.ndarray  # (n_det,) int8, excitation level from HF

    @property
    def n_det(self) -> int:
        return int(self.coef.shape[0])


def make_integrals(n_orb: int, seed: int) -> System:
    """Integrals of the recipe above for n_orb spatial orbitals."""
    n = int(n_orb)
    rng = np.random.Generator(np.random.PCG64(seed))
    off = rng.normal(0.0, 0.02, size=(n, n))
    h = np.triu(off, 1)
    h = h + h.T
    h[np.diag_indices(n)] = -2.0 + 0.25 * np.arange(n)

    # unique orbital pairs P = (p >= q), indexed p (p + 1) / 2 + q
    p_of = np.concatenate([np.full(p + 1, p) for p in range(n)])
    q_of = np.concatenate([np.arange(p + 1) for p in range(n)])
    npair = p_of.shape[0]
    iu, ju = np.triu_indices(npair)  # P <= R, one draw per unique element
    unif = rng.uniform(0.3, 0.7, size=iu.shape[0])
    gaus = rng.normal(0.0, 1.0, size=iu.shape[0])
    p1, q1, p2, q2 = p_of[iu], q_of[iu], p_of[ju], q_of[ju]
    coulomb_like = (p1 == q1) & (p2 == q2)
    width = 0.01 * np.exp(-0.1 * (np.abs(p1 - q1) + np.abs(p2 - q2)))
    vals = np.where(coulomb_like, unif, gaus * width)
    v = np.zeros((npair, npair))
    v[iu, ju] = vals
    v[ju, iu] = vals
    pidx = np.empty((n, n), dtype=np.int64)
    for p in range(n):
        for q in range(p + 1):
            pidx[p, q] = pidx[q, p] = p * (p + 1) // 2 + q
    eri = v[pidx[:, :, None, None], pidx[None, None, :, :]]
    return System(n_orb=n, h=np.ascontiguousarray(h), eri=np.ascontiguousarray(eri))


def _bits(idx_lists: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """OR of 1 << idx over the entries of each row where mask is set."""
    sh = np.where(mask, idx_lists, 0).astype(np.uint64)
    w = np.left_shift(np.uint64(1), sh)
    w = np.where(mask, w, np.uint64(0))
    return np.bitwise_or.reduce(w, axis=1)


def _draw_excitations(rng, n_orb, n, levels, batch):
    """Random alpha/beta strings at the given excitation levels from HF."""
    v = n_orb - n
    lvl = levels
    # feasible alpha share la of a level l: max(0, l - m) <= la <= min(l, m)
    m = min(n, v)
    lo = np.maximum(0, lvl - m)
    hi = np.minimum(lvl, m)
    la = lo + np.floor(rng.random(batch) * (hi - lo + 1)).astype(np.int64)
    lb = lvl - la
    hf = np.uint64((1 << n) - 1) if n < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    out = []
    for share in (la, lb):
        occ_rank = np.argsort(np.argsort(rng.random((batch, n)), axis=1), axis=1)
        vir_rank = np.argsort(np.argsort(rng.random((batch, v)), axis=1), axis=1)
        occ_pick = occ_rank < share[:, None]
        vir_pick = vir_rank < share[:, None]
        occ_idx = np.broadcast_to(np.arange(n), (batch, n))
        vir_idx = np.broadcast_to(np.arange(n, n_orb), (batch, v))
        removed = _bits(occ_idx, occ_pick)
        added = _bits(vir_idx, vir_pick)
        out.append((hf ^ removed) | added)
    return out[0], out[1]


def make_reference(n_orb: int, n_elec_per_spin: int, n_det: int, max_level: int,
                   seed: int) -> Reference:
    """HF plus random excitations up to max_level, deduplicated, with coefficients."""
    n = int(n_elec_per_spin)
    if not (0 < n < n_orb <= 64):
        raise ValueError("need 0 < n_elec_per_spin < n_orb <= 64")
    if n_det > _count_within(n_orb, n, max_level):
        raise ValueError("n_det exceeds the determinants within max_level of HF")
    rng = np.random.Generator(np.random.PCG64(seed))
    hf = np.uint64((1 << n) - 1)
    alphas = [np.array([hf], dtype=np.uint64)]
    betas = [np.array([hf], dtype=np.uint64)]
    lvls = [np.array([0], dtype=np.int8)]
    seen = {(int(hf), int(hf))}
    have = 1
    while have < n_det:
        batch = max(1024, 2 * (n_det - have))
        lvl = 1 + np.floor(rng.random(batch) * max_level).astype(np.int64)
        a, b = _draw_excitations(rng, n_orb, n, lvl, batch)
        keep_a, keep_b, keep_l = [], [], []
        for x, y, l in zip(a.tolist(), b.tolist(), lvl.tolist()):
            if (x, y) in seen:
                continue
            seen.add((x, y))
            keep_a.append(x)
            keep_b.append(y)
            keep_l.append(l)
            have += 1
            if have == n_det:
                break
        alphas.append(np.array(keep_a, dtype=np.uint64))
        betas.append(np.array(keep_b, dtype=np.uint64))
        lvls.append(np.array(keep_l, dtype=np.int8))
    alpha = np.concatenate(alphas)[:n_det]
    beta = np.concatenate(betas)[:n_det]
    level = np.concatenate(lvls)[:n_det]
    keys = np.empty(2 * n_det, dtype=np.uint64)
    keys[0::2] = alpha
    keys[1::2] = beta

    coef = np.empty(n_det)
    coef[0] = 0.95
    if n_det > 1:
        z = rng.normal(0.0, 1.0, size=n_det - 1) * np.exp(-0.5 * level[1:].astype(np.float64))
        z *= math.sqrt(1.0 - 0.95 ** 2) / np.linalg.norm(z)
        coef[1:] = z
    return Reference(n_alpha=n, n_beta=n, keys=keys, coef=coef, level=level)


def make_symmetric_reference(n_orb: int, n_elec_per_spin: int, n_det: int, max_level: int,
                             seed: int) -> Reference:
    """A reference closed under exchange of the alpha and beta strings.

    Determinants are drawn as in make_reference (HF plus random excitations,
    deduplicated); each one with alpha != beta brings its mirror (beta, alpha)
    with the same coefficient, so c(beta, alpha) = c(alpha, beta) for every
    pair (the wavefunction is then an eigenvector of the spin flip).  n_det
    counts the mirrors; HF (alpha = beta) is its own mirror.
    """
    n = int(n_elec_per_spin)
    if not (0 < n < n_orb <= 64):
        raise ValueError("need 0 < n_elec_per_spin < n_orb <= 64")
    if n_det > _count_within(n_orb, n, max_level):
        raise ValueError("n_det exceeds the determinants within max_level of HF")
    if n_det % 2 == 0 and max_level < 2:
        raise ValueError("an even n_det needs a second self-mirrored determinant (max_level >= 2)")
    rng = np.random.Generator(np.random.PCG64(seed))
    hf = (1 << n) - 1
    pairs = [(hf, hf)]
    levels = [0]
    seen = {(hf, hf)}
    have = 1
    while have < n_det:
        batch = max(1024, n_det - have)
        lvl = 1 + np.floor(rng.random(batch) * max_level).astype(np.int64)
        a, b = _draw_excitations(rng, n_orb, n, lvl, batch)
        for x, y, l in zip(a.tolist(), b.tolist(), lvl.tolist()):
            if (x, y) in seen:
                continue
            need = 1 if x == y else 2
            if have + need > n_det:
                continue
            seen.add((x, y))
            seen.add((y, x))
            pairs.append((x, y))
            levels.append(l)
            have += need
            if have == n_det:
                break
    alpha, beta, level = [], [], []
    for (x, y), l in zip(pairs, levels):
        alpha.append(x)
        beta.append(y)
        level.append(l)
        if x != y:
            alpha.append(y)
            beta.append(x)
            level.append(l)
    keys = np.empty(2 * n_det, dtype=np.uint64)
    keys[0::2] = np.array(alpha, dtype=np.uint64)
    keys[1::2] = np.array(beta, dtype=np.uint64)
    level = np.array(level, dtype=np.int8)
    coef = np.empty(n_det)
    coef[0] = 0.95
    if n_det > 1:
        # one draw per mirror pair, shared by both members
        z = np.empty(n_det - 1)
        i = 1
        for (x, y), l in zip(pairs[1:], levels[1:]):
            v = rng.normal(0.0, 1.0) * math.exp(-0.5 * l)
            z[i - 1] = v
            i += 1
            if x != y:
                z[i - 1] = v
                i += 1
        z *= math.sqrt(1.0 - 0.95 ** 2) / np.linalg.norm(z)
        coef[1:] = z
    return Reference(n_alpha=n, n_beta=n, keys=keys, coef=coef, level=level)


def _count_within(n_orb: int, n: int, max_level: int) -> int:
    v = n_orb - n
    tot = 0
    for lvl in range(0, max_level + 1):
        for la in range(0, lvl + 1):
            lb = lvl - la
            tot += math.comb(n, la) * math.comb(v, la) * math.comb(n, lb) * math.comb(v, lb)
    return tot


# The named single-solve workloads: electrons per spin, spatial orbitals,
# N_det, maximum excitation level, and the index their seeds derive from.
WORKLOADS = {
    # 8 electrons in 16 orbitals, 1,000 determinants: about 3.2e6 terms
    "small": dict(n_elec_per_spin=4, n_orb=16, n_det=1000, max_level=3, seed_index=0),
    # 20 electrons in 40 orbitals, 100,000 determinants: 1.2975e10 terms
    "large": dict(n_elec_per_spin=10, n_orb=40, n_det=100_000, max_level=4, seed_index=1),
    # 24 electrons in 60 orbitals, 1,000,000 determinants: 4.8e11 terms
    "million": dict(n_elec_per_spin=12, n_orb=60, n_det=1_000_000, max_level=4, seed_index=2),
}
BATCH_SEED_INDEX = 3  # the 64-instance batched workload


def make_workload(name: str, n_det: int | None = None):
    """(System, Reference) of a named single-solve workload ("small", "large" or "million")."""
    c = WORKLOADS[name]
    seed = workload_seed(c["seed_index"])
    sys_ = make_integrals(c["n_orb"], seed)
    nd = c["n_det"] if n_det is None else n_det
    ref = make_reference(c["n_orb"], c["n_elec_per_spin"], nd, c["max_level"], seed + 1)
    return sys_, ref


def batch_instance_params(k: int):
    """Size of instance k of the batched workload (64 uneven instances).

    n_orb ~ U{16..40}, electrons per spin ~ U{4..10} (kept below n_orb),
    N_det log-uniform in [1e3, 5e4].  The maximum excitation level is 4 when
    N_det exceeds half the number of determinants within triples of HF, else 3.
    """
    rng = np.random.Generator(np.random.PCG64(workload_seed(BATCH_SEED_INDEX, k)))
    n_orb = int(rng.integers(16, 41))
    n = int(rng.integers(4, 11))
    n = min(n, n_orb - 1)
    n_det = int(round(math.exp(rng.uniform(math.log(1e3), math.log(5e4)))))
    max_level = 4 if n_det > _count_within(n_orb, n, 3) // 2 else 3
    return dict(n_orb=n_orb, n_elec_per_spin=n, n_det=n_det, max_level=max_level,
                seed=workload_seed(BATCH_SEED_INDEX, k) + 7)


def make_instance(params: dict):
    """(System, Reference) of one batched-workload instance."""
    sys_ = make_integrals(params["n_orb"], params["seed"])
    ref = make_reference(params["n_orb"], params["n_elec_per_spin"], params["n_det"],
                         params["max_level"], params["seed"] + 1)
    return sys_, ref
