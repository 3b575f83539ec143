"""Brute-force PT2 on tiny systems, by second-quantised operator application.

Independent of the oracle: it never uses Slater-Condon rules.  The full
determinant space is enumerated, the Hamiltonian

    H = sum_{pq,s} h_pq a+_{ps} a_{qs}
        + 1/2 sum_{pqrs,s,t} (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs}

is applied to every basis determinant operator by operator with explicit
anticommutation signs (Jordan-Wigner order: alpha spin-orbitals 0..n-1, then
beta spin-orbitals n..2n-1, i.e. the canonical alpha-then-beta ascending
order), and E2 of Eq. 3 is evaluated from the resulting dense matrix:

    E2 = sum_{a not in ref, rank(a) <= 2} (H c)_a^2 / (E0 - H_aa).
"""

from __future__ import annotations

import itertools

import numpy as np


def _sign_before(mask: int, so: int) -> int:
    return -1 if bin(mask & ((1 << so) - 1)).count("1") & 1 else 1


def _annihilate(mask, so):
    if not (mask >> so) & 1:
        return None, 0
    return mask & ~(1 << so), _sign_before(mask, so)


def _create(mask, so):
    if (mask >> so) & 1:
        return None, 0
    return mask | (1 << so), _sign_before(mask, so)


def basis(n_orb: int, n_alpha: int, n_beta: int):
    """All determinants as (alpha word, beta word)."""
    al = [sum(1 << p for p in c) for c in itertools.combinations(range(n_orb), n_alpha)]
    be = [sum(1 << p for p in c) for c in itertools.combinations(range(n_orb), n_beta)]
    return [(a, b) for a in al for b in be]


def hamiltonian(h: np.ndarray, eri: np.ndarray, dets):
    """Dense <D_i|H|D_j> over the given determinants."""
    n = h.shape[0]
    index = {(a | (b << n)): k for k, (a, b) in enumerate(dets)}
    m = len(dets)
    H = np.zeros((m, m))
    for j, (a, b) in enumerate(dets):
        ket = a | (b << n)
        occ = [so for so in range(2 * n) if (ket >> so) & 1]
        # one-body part
        for q in occ:
            m1, s1 = _annihilate(ket, q)
            spin = q // n
            for p in range(spin * n, spin * n + n):
                m2, s2 = _create(m1, p)
                if m2 is None:
                    continue
                H[index[m2], j] += s1 * s2 * h[p % n, q % n]
        # two-body part: a+_p a+_r a_s a_q, applied right to left
        for q in occ:
            m1, s1 = _annihilate(ket, q)
            sq = q // n
            for s in occ:
                if s == q:
                    continue
                m2, s2 = _annihilate(m1, s)
                st = s // n
                for r in range(st * n, st * n + n):
                    m3, s3 = _create(m2, r)
                    if m3 is None:
                        continue
                    for p in range(sq * n, sq * n + n):
                        m4, s4 = _create(m3, p)
                        if m4 is None:
                            continue
                        H[index[m4], j] += 0.5 * s1 * s2 * s3 * s4 * eri[p % n, q % n, r % n, s % n]
    return H


def rank(d1, d2) -> int:
    """Excitation rank between two determinants (alpha, beta)."""
    return (bin(d1[0] ^ d2[0]).count("1") + bin(d1[1] ^ d2[1]).count("1")) // 2


def pt2(h, eri, dets, H, ref_idx, coef, e0, cutoff=0.0):
    """E2, the connected external set (sorted keys) and its numerators and diagonals.

    With a cutoff, a contribution H_ai c_i of a connected reference
    determinant counts only if |H_ai c_i| >= cutoff, and a determinant
    belongs to the set only if one of its contributions counts."""
    ref_idx = list(ref_idx)
    refset = set(ref_idx)
    coef = np.asarray(coef)
    hc = H[:, ref_idx] @ coef
    contrib = H[:, ref_idx] * coef[None, :]
    ext = []
    for k, d in enumerate(dets):
        if k in refset:
            continue
        conn = [j for j, i in enumerate(ref_idx) if rank(d, dets[i]) in (1, 2)]
        if cutoff > 0:
            conn = [j for j in conn if abs(contrib[k, j]) >= cutoff]
            hc[k] = sum(contrib[k, j] for j in conn)
        if conn:
            ext.append(k)
    ext.sort(key=lambda k: (dets[k][0], dets[k][1]))
    e2 = sum(hc[k] ** 2 / (e0 - H[k, k]) for k in ext)
    keys = np.array([[dets[k][0], dets[k][1]] for k in ext], dtype=np.uint64).reshape(-1, 2)
    far = [k for k, d in enumerate(dets) if k not in refset
           and all(rank(d, dets[i]) > 2 for i in ref_idx)]
    return dict(e2=e2, keys=keys, num=hc[ext], haa=np.diag(H)[ext], far_max=
                float(np.abs(hc[far]).max()) if far else 0.0)
