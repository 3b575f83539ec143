/*
 * CPU oracle for the deterministic Epstein-Nesbet PT2 energy.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes (Eq. 3 and the single-pass loop of Algorithm 1, with the
 * square of the summed numerator as Eq. 3 prints it):
 *
 *   E2 = sum_{a in S} ( sum_{i : a in SD(D_i)} H_ai c_i )^2 / (E0 - H_aa)
 *
 * S is the connected external set: every determinant one single or double
 * excitation (spin conserved) away from some reference determinant D_i,
 * minus the reference determinants themselves (the explicit filter of the
 * section on duplicate removal; S is defined structurally, so keys whose
 * summed numerator is exactly zero still belong to S).
 *
 * Steps, in the paper's order, written plainly:
 *   1. for each reference determinant, enumerate alpha singles, beta singles,
 *      alpha-alpha doubles, beta-beta doubles and alpha-beta doubles, with
 *      the Slater-Condon matrix element and fermionic phase (Algorithm 1,
 *      "acting the Hamiltonian on each determinant");
 *   2. accumulate H_ai c_i per excited determinant in a hash map, in
 *      generation order (the paper contrasts hash maps with sorting; here the
 *      hash map is the plain definition, not a performance choice);
 *   3. drop the keys that are reference determinants;
 *   4. compute H_aa directly from the occupation lists (the textbook diagonal,
 *      not the incremental one of the appendix);
 *   5. sort the remaining keys (alpha word most significant) and sum
 *      num^2 / (E0 - H_aa) in that order with Neumaier compensation.
 *
 * Conventions.  Orbital p of spin alpha is bit p of the alpha word, of spin
 * beta bit p of the beta word.  A determinant is the product of alpha
 * creation operators in ascending orbital order followed by the beta ones in
 * ascending order, acting on the vacuum.  Integrals are chemist-notation
 * (pq|rs) = eri[((p*n + q)*n + r)*n + s].
 *
 * Optional constraint (Algorithm 2, one constraint class): when mod > 1 only
 * excited determinants whose alpha word satisfies alpha % mod == rem are kept;
 * when top != 0, only those whose k = popcount(top) highest occupied alpha
 * orbitals are exactly the orbitals of top (the triplet constraint of the
 * "Triplet constraints" section for k = 3, the quadruplet one for k = 4).
 * The classes r = 0..mod-1 are non-overlapping and complete, so their E2 sum
 * to the unconstrained E2.  When mod exceeds every alpha word (mod > 2^n_orb
 * - 1) the class is the single alpha string rem; a single or double
 * excitation changes at most two alpha orbitals, so a reference determinant
 * whose alpha word differs from rem in more than four bits contributes
 * nothing to it and is not enumerated.
 *
 * Optional numerator cutoff (the Results section and the subsection on the
 * matrix-element cutoff): a contribution c_i H_ai with |c_i H_ai| below the
 * cutoff is ignored before it reaches the map, so an excited determinant all
 * of whose contributions are below it is not in S.  Cutoff 0 keeps every
 * contribution.  n_terms then counts the kept contributions.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double e2;                 /* PT2 energy over the kept keys */
    double e2_ref_like;        /* PT2-like sum over reference keys (unfiltered part) */
    uint64_t n_terms;          /* generated (key, value) pairs kept by the constraint */
    uint64_t n_unique;         /* distinct keys generated */
    uint64_t n_in_ref;         /* distinct generated keys that are reference determinants */
    uint64_t n_external;       /* |S| */
    uint64_t digest_sum;       /* sum of mix1(key) over S, mod 2^64 */
    uint64_t digest_xor;       /* xor of mix2(key) over S */
    double min_abs_denom;      /* min |E0 - H_aa| over S */
    uint64_t n_pos_denom;      /* keys of S with E0 - H_aa > 0 */
} oracle_result;

/* ------------------------------------------------------------------ system */

typedef struct {
    int n;
    const double *h;
    const double *eri;
} sys_t;

static double ERI(const sys_t *s, int p, int q, int r, int t)
{
    int n = s->n;
    return s->eri[(((size_t)p * n + q) * n + r) * n + t];
}

static int popc64(uint64_t x) { return __builtin_popcountll(x); }

static int occ_list(uint64_t w, int n_orb, int *out)
{
    int k = 0;
    for (int p = 0; p < n_orb; ++p)
        if ((w >> p) & 1ull) out[k++] = p;
    return k;
}

/* (-1)^(number of occupied orbitals of w strictly between r and a) */
static double single_sign(uint64_t w, int r, int a)
{
    int lo = r < a ? r : a, hi = r < a ? a : r;
    int cnt = 0;
    for (int p = lo + 1; p < hi; ++p)
        if ((w >> p) & 1ull) ++cnt;
    return (cnt & 1) ? -1.0 : 1.0;
}

/* Direct diagonal <D|H|D> = sum_p h_pp + 1/2 sum_{p,q} [(pp|qq) - delta_spin (pq|qp)]. */
static double diag_direct(const sys_t *s, uint64_t wa, uint64_t wb)
{
    int oa[64], ob[64];
    int na = occ_list(wa, s->n, oa), nb = occ_list(wb, s->n, ob);
    double e = 0.0;
    for (int i = 0; i < na; ++i) e += s->h[oa[i] * s->n + oa[i]];
    for (int i = 0; i < nb; ++i) e += s->h[ob[i] * s->n + ob[i]];
    for (int i = 0; i < na; ++i)
        for (int j = i + 1; j < na; ++j)
            e += ERI(s, oa[i], oa[i], oa[j], oa[j]) - ERI(s, oa[i], oa[j], oa[j], oa[i]);
    for (int i = 0; i < nb; ++i)
        for (int j = i + 1; j < nb; ++j)
            e += ERI(s, ob[i], ob[i], ob[j], ob[j]) - ERI(s, ob[i], ob[j], ob[j], ob[i]);
    for (int i = 0; i < na; ++i)
        for (int j = 0; j < nb; ++j)
            e += ERI(s, oa[i], oa[i], ob[j], ob[j]);
    return e;
}

/* <D'|H|D> for D' = D with r -> a in the string `same` (spin sigma), `other`
 * the string of the opposite spin:
 *   sign * [ h_ar + sum_{j in same} ((ar|jj) - (aj|jr)) + sum_{j in other} (ar|jj) ].
 * The j = r term of the same-spin sum vanishes identically. */
static double single_element(const sys_t *s, uint64_t same, uint64_t other, int r, int a)
{
    int os[64], oo[64];
    int ns = occ_list(same, s->n, os), no = occ_list(other, s->n, oo);
    double v = s->h[a * s->n + r];
    for (int k = 0; k < ns; ++k) {
        int j = os[k];
        v += ERI(s, a, r, j, j) - ERI(s, a, j, j, r);
    }
    for (int k = 0; k < no; ++k) {
        int j = oo[k];
        v += ERI(s, a, r, j, j);
    }
    return single_sign(same, r, a) * v;
}

/* Same-spin double r1 < r2 -> a1 < a2 on string w:
 *   gamma * [ (a1 r1|a2 r2) - (a1 r2|a2 r1) ],
 * gamma = sign of r1 -> a1 on w times sign of r2 -> a2 on the result. */
static double same_double_element(const sys_t *s, uint64_t w, int r1, int r2, int a1, int a2)
{
    double g1 = single_sign(w, r1, a1);
    uint64_t w1 = (w & ~(1ull << r1)) | (1ull << a1);
    double g2 = single_sign(w1, r2, a2);
    return g1 * g2 * (ERI(s, a1, r1, a2, r2) - ERI(s, a1, r2, a2, r1));
}

/* Opposite-spin double: sign_alpha * sign_beta * (aA rA | aB rB). */
static double ab_double_element(const sys_t *s, uint64_t wa, uint64_t wb, int ra, int aa, int rb, int ab)
{
    return single_sign(wa, ra, aa) * single_sign(wb, rb, ab) * ERI(s, aa, ra, ab, rb);
}

/* --------------------------------------------------------------- hash map */

typedef struct {
    uint64_t *ka, *kb;
    double *val;
    uint8_t *used;
    size_t cap, size;
} map_t;

static uint64_t fmix(uint64_t z)
{
    /* SplitMix64 output function (Steele, Lea, Flood 2014; constants as
     * published by Vigna). */
    z ^= z >> 30;
    z *= 0xbf58476d1ce4e5b9ull;
    z ^= z >> 27;
    z *= 0x94d049bb133111ebull;
    z ^= z >> 31;
    return z;
}

static int map_init(map_t *m, size_t cap)
{
    size_t c = 1024;
    while (c < cap) c <<= 1;
    m->cap = c;
    m->size = 0;
    m->ka = malloc(c * sizeof(uint64_t));
    m->kb = malloc(c * sizeof(uint64_t));
    m->val = malloc(c * sizeof(double));
    m->used = calloc(c, 1);
    return (m->ka && m->kb && m->val && m->used) ? 0 : -1;
}

static void map_free(map_t *m)
{
    free(m->ka); free(m->kb); free(m->val); free(m->used);
    memset(m, 0, sizeof(*m));
}

static int map_add(map_t *m, uint64_t a, uint64_t b, double v);

static int map_grow(map_t *m)
{
    map_t n2;
    if (map_init(&n2, m->cap * 2)) return -1;
    for (size_t i = 0; i < m->cap; ++i)
        if (m->used[i]) map_add(&n2, m->ka[i], m->kb[i], m->val[i]);
    map_free(m);
    *m = n2;
    return 0;
}

static int map_add(map_t *m, uint64_t a, uint64_t b, double v)
{
    if (2 * (m->size + 1) > m->cap)
        if (map_grow(m)) return -1;
    size_t mask = m->cap - 1;
    size_t i = fmix(a ^ fmix(b)) & mask;
    while (m->used[i]) {
        if (m->ka[i] == a && m->kb[i] == b) {
            m->val[i] += v;
            return 0;
        }
        i = (i + 1) & mask;
    }
    m->used[i] = 1;
    m->ka[i] = a;
    m->kb[i] = b;
    m->val[i] = v;
    m->size++;
    return 0;
}

/* ----------------------------------------------------------- enumeration */

typedef void (*visit_fn)(void *ctx, uint64_t a, uint64_t b, double value);

typedef struct {
    uint64_t mod, rem;
    uint64_t top;
} constraint_t;

/* The k highest occupied orbitals of word a, as a mask (fewer if a has fewer). */
static uint64_t highest_occupied(uint64_t a, int k)
{
    uint64_t m = 0;
    for (int p = 63; p >= 0 && k > 0; --p)
        if ((a >> p) & 1ull) {
            m |= 1ull << p;
            --k;
        }
    return m;
}

static int keep_alpha(const constraint_t *c, uint64_t a)
{
    if (c->top && highest_occupied(a, __builtin_popcountll(c->top)) != c->top) return 0;
    return c->mod <= 1 || (a % c->mod) == c->rem;
}

/* All singles and doubles of (wa, wb), value H_ai * c_i, in the order:
 * alpha singles, beta singles, alpha-alpha doubles, beta-beta doubles,
 * alpha-beta doubles (alpha single outer, beta single inner).
 * Returns the number of visited terms. */
static uint64_t enumerate_det(const sys_t *s, uint64_t wa, uint64_t wb, double c,
                              const constraint_t *cons, visit_fn f, void *ctx)
{
    int n = s->n;
    int oa[64], ob[64], va[64], vb[64];
    int na = occ_list(wa, n, oa), nb = occ_list(wb, n, ob);
    int nva = 0, nvb = 0;
    for (int p = 0; p < n; ++p) {
        if (!((wa >> p) & 1ull)) va[nva++] = p;
        if (!((wb >> p) & 1ull)) vb[nvb++] = p;
    }
    uint64_t cnt = 0;

    /* alpha singles */
    for (int i = 0; i < na; ++i)
        for (int j = 0; j < nva; ++j) {
            int r = oa[i], a = va[j];
            uint64_t wa2 = (wa & ~(1ull << r)) | (1ull << a);
            if (!keep_alpha(cons, wa2)) continue;
            f(ctx, wa2, wb, c * single_element(s, wa, wb, r, a));
            ++cnt;
        }
    /* beta singles */
    if (keep_alpha(cons, wa))
        for (int i = 0; i < nb; ++i)
            for (int j = 0; j < nvb; ++j) {
                int r = ob[i], a = vb[j];
                uint64_t wb2 = (wb & ~(1ull << r)) | (1ull << a);
                f(ctx, wa, wb2, c * single_element(s, wb, wa, r, a));
                ++cnt;
            }
    /* alpha-alpha doubles */
    for (int i1 = 0; i1 < na; ++i1)
        for (int i2 = i1 + 1; i2 < na; ++i2)
            for (int j1 = 0; j1 < nva; ++j1)
                for (int j2 = j1 + 1; j2 < nva; ++j2) {
                    int r1 = oa[i1], r2 = oa[i2], a1 = va[j1], a2 = va[j2];
                    uint64_t wa2 = (wa & ~((1ull << r1) | (1ull << r2))) | (1ull << a1) | (1ull << a2);
                    if (!keep_alpha(cons, wa2)) continue;
                    f(ctx, wa2, wb, c * same_double_element(s, wa, r1, r2, a1, a2));
                    ++cnt;
                }
    /* beta-beta doubles */
    if (keep_alpha(cons, wa))
        for (int i1 = 0; i1 < nb; ++i1)
            for (int i2 = i1 + 1; i2 < nb; ++i2)
                for (int j1 = 0; j1 < nvb; ++j1)
                    for (int j2 = j1 + 1; j2 < nvb; ++j2) {
                        int r1 = ob[i1], r2 = ob[i2], a1 = vb[j1], a2 = vb[j2];
                        uint64_t wb2 = (wb & ~((1ull << r1) | (1ull << r2))) | (1ull << a1) | (1ull << a2);
                        f(ctx, wa, wb2, c * same_double_element(s, wb, r1, r2, a1, a2));
                        ++cnt;
                    }
    /* alpha-beta doubles */
    for (int i = 0; i < na; ++i)
        for (int j = 0; j < nva; ++j) {
            int ra = oa[i], aa = va[j];
            uint64_t wa2 = (wa & ~(1ull << ra)) | (1ull << aa);
            if (!keep_alpha(cons, wa2)) continue;
            for (int k = 0; k < nb; ++k)
                for (int l = 0; l < nvb; ++l) {
                    int rb = ob[k], ab = vb[l];
                    uint64_t wb2 = (wb & ~(1ull << rb)) | (1ull << ab);
                    f(ctx, wa2, wb2, c * ab_double_element(s, wa, wb, ra, aa, rb, ab));
                    ++cnt;
                }
        }
    return cnt;
}

static void visit_map(void *ctx, uint64_t a, uint64_t b, double v)
{
    map_t *m = (map_t *)ctx;
    if (map_add(m, a, b, v)) m->size = (size_t)-1; /* allocation failure marker */
}

typedef struct {
    map_t *m;
    double cutoff;
    uint64_t kept;
} cut_ctx;

/* The numerator cutoff in front of the map: contributions below it are dropped. */
static void visit_cut(void *ctx, uint64_t a, uint64_t b, double v)
{
    cut_ctx *k = (cut_ctx *)ctx;
    if (!(fabs(v) >= k->cutoff)) return;
    k->kept++;
    visit_map(k->m, a, b, v);
}

/* ------------------------------------------------------------ the energy */

typedef struct {
    uint64_t a, b;
} key_t;

static int key_cmp(const void *x, const void *y)
{
    const key_t *p = x, *q = y;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    if (p->b != q->b) return p->b < q->b ? -1 : 1;
    return 0;
}

typedef struct {
    uint64_t a, b;
    size_t slot;
} ent_t;

static int ent_cmp(const void *x, const void *y)
{
    const ent_t *p = x, *q = y;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    if (p->b != q->b) return p->b < q->b ? -1 : 1;
    return 0;
}

/* Neumaier's improvement of Kahan summation. */
typedef struct {
    double s, c;
} nsum_t;

static void nsum_add(nsum_t *t, double x)
{
    double s = t->s + x;
    if (fabs(t->s) >= fabs(x)) t->c += (t->s - s) + x;
    else t->c += (x - s) + t->s;
    t->s = s;
}

/* Set digest of the external set (a verification aid, not part of the
 * method): mix1 summed mod 2^64 and mix2 xor-ed over the keys.  Multiplying
 * by odd 64-bit constants and finishing with the SplitMix64 output function. */
uint64_t oracle_digest_mix1(uint64_t a, uint64_t b) { return fmix(a ^ (b * 0x9e3779b97f4a7c15ull)); }
uint64_t oracle_digest_mix2(uint64_t a, uint64_t b) { return fmix(b ^ (a * 0xc2b2ae3d27d4eb4full)); }

/* Validation shared by the entry points: returns 0 when the reference is a
 * set of distinct determinants with equal alpha and beta electron counts and
 * no bit at or above n_orb. */
static int check_ref(int n_orb, int64_t n_det, const uint64_t *keys)
{
    if (n_orb < 1 || n_orb > 64 || n_det < 0) return -1;
    uint64_t lim = n_orb == 64 ? ~0ull : ((1ull << n_orb) - 1);
    for (int64_t i = 0; i < n_det; ++i) {
        if ((keys[2 * i] & ~lim) || (keys[2 * i + 1] & ~lim)) return -1;
        if (popc64(keys[2 * i]) != popc64(keys[0]) || popc64(keys[2 * i + 1]) != popc64(keys[1])) return -1;
    }
    return 0;
}

/*
 * Full oracle run.  When include_ref is set the reference keys are kept as
 * well and their PT2-like contributions go to e2_ref_like (the quantity the
 * paper subtracts in its duplicate-removal section).  If dump_* are given
 * (cap entries), the external keys are written in sorted order with their
 * summed numerator and direct diagonal; the return value is then |S|.
 * Returns -1 on invalid input, -2 on allocation failure, else 0 (or |S|).
 */
int64_t oracle_pt2(int n_orb, const double *h, const double *eri, int64_t n_det,
                   const uint64_t *keys, const double *coef, double e0,
                   uint64_t cons_mod, uint64_t cons_rem, uint64_t top, int include_ref, double cutoff,
                   oracle_result *out, uint64_t *dump_keys, double *dump_num,
                   double *dump_haa, int64_t dump_cap)
{
    if (check_ref(n_orb, n_det, keys)) return -1;
    if (!(cutoff >= 0.0) || isinf(cutoff)) return -1;
    sys_t s = {n_orb, h, eri};
    constraint_t cons = {cons_mod, cons_rem, top};
    memset(out, 0, sizeof(*out));
    out->min_abs_denom = INFINITY;

    map_t m;
    if (map_init(&m, 1 << 16)) return -2;
    cut_ctx cc = {&m, cutoff, 0};
    const int exact_alpha = cons_mod > 1 && (n_orb >= 64 || cons_mod > (1ull << n_orb) - 1ull);
    for (int64_t i = 0; i < n_det; ++i) {
        if (exact_alpha && __builtin_popcountll(keys[2 * i] ^ cons_rem) > 4) continue;
        enumerate_det(&s, keys[2 * i], keys[2 * i + 1], coef[i], &cons, visit_cut, &cc);
        if (m.size == (size_t)-1) { map_free(&m); return -2; }
    }
    const uint64_t nterms = cc.kept;

    /* reference keys, sorted, for the explicit filter */
    key_t *rk = malloc((size_t)(n_det ? n_det : 1) * sizeof(key_t));
    ent_t *ent = malloc((m.size ? m.size : 1) * sizeof(ent_t));
    if (!rk || !ent) { free(rk); free(ent); map_free(&m); return -2; }
    for (int64_t i = 0; i < n_det; ++i) { rk[i].a = keys[2 * i]; rk[i].b = keys[2 * i + 1]; }
    qsort(rk, (size_t)n_det, sizeof(key_t), key_cmp);
    for (int64_t i = 1; i < n_det; ++i)
        if (rk[i].a == rk[i - 1].a && rk[i].b == rk[i - 1].b) { free(rk); free(ent); map_free(&m); return -1; }

    size_t ne = 0;
    for (size_t i = 0; i < m.cap; ++i)
        if (m.used[i]) { ent[ne].a = m.ka[i]; ent[ne].b = m.kb[i]; ent[ne].slot = i; ++ne; }
    qsort(ent, ne, sizeof(ent_t), ent_cmp);

    nsum_t e2 = {0, 0}, e2r = {0, 0};
    int64_t nd = 0;
    for (size_t k = 0; k < ne; ++k) {
        key_t q = {ent[k].a, ent[k].b};
        double num = m.val[ent[k].slot];
        int in_ref = bsearch(&q, rk, (size_t)n_det, sizeof(key_t), key_cmp) != NULL;
        if (in_ref) {
            out->n_in_ref++;
            if (include_ref) {
                double haa = diag_direct(&s, q.a, q.b);
                nsum_add(&e2r, num * num / (e0 - haa));
            }
            continue;
        }
        double haa = diag_direct(&s, q.a, q.b);
        double den = e0 - haa;
        nsum_add(&e2, num * num / den);
        out->n_external++;
        out->digest_sum += oracle_digest_mix1(q.a, q.b);
        out->digest_xor ^= oracle_digest_mix2(q.a, q.b);
        if (fabs(den) < out->min_abs_denom) out->min_abs_denom = fabs(den);
        if (den > 0) out->n_pos_denom++;
        if (dump_keys && nd < dump_cap) {
            dump_keys[2 * nd] = q.a;
            dump_keys[2 * nd + 1] = q.b;
            dump_num[nd] = num;
            dump_haa[nd] = haa;
        }
        ++nd;
    }
    out->e2 = e2.s + e2.c;
    out->e2_ref_like = e2r.s + e2r.c;
    out->n_terms = nterms;
    out->n_unique = ne;
    free(rk);
    free(ent);
    map_free(&m);
    return dump_keys ? nd : 0;
}

/* Direct diagonals H_kk of n determinants. */
void oracle_diagonals(int n_orb, const double *h, const double *eri, int64_t n,
                      const uint64_t *keys, double *out)
{
    sys_t s = {n_orb, h, eri};
    for (int64_t i = 0; i < n; ++i) out[i] = diag_direct(&s, keys[2 * i], keys[2 * i + 1]);
}

typedef struct {
    const sys_t *s;
    uint64_t *keys;
    double *val, *haa;
    int64_t cap, n;
} list_ctx;

static void visit_list(void *ctx, uint64_t a, uint64_t b, double v)
{
    list_ctx *l = (list_ctx *)ctx;
    if (l->n < l->cap) {
        l->keys[2 * l->n] = a;
        l->keys[2 * l->n + 1] = b;
        l->val[l->n] = v;
        l->haa[l->n] = diag_direct(l->s, a, b);
    }
    l->n++;
}

/* The terms one determinant generates, in enumeration order, with the direct
 * diagonal of each excited determinant.  Returns the number of terms (which
 * may exceed cap; only cap are written). */
int64_t oracle_det_terms(int n_orb, const double *h, const double *eri, uint64_t wa, uint64_t wb,
                         double c, uint64_t cons_mod, uint64_t cons_rem, uint64_t *keys,
                         double *val, double *haa, int64_t cap)
{
    sys_t s = {n_orb, h, eri};
    constraint_t cons = {cons_mod, cons_rem, 0};
    list_ctx l = {&s, keys, val, haa, cap, 0};
    enumerate_det(&s, wa, wb, c, &cons, visit_list, &l);
    return l.n;
}
