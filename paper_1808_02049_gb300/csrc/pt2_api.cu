// Host runtime of libpt2: contexts, resident systems and references, pass
// planning (the work list of the parallelisation-with-work-lists section),
// device memory under a budget, and the C ABI declared in include/pt2.h.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "pt2_runtime.h"

using namespace pt2;

namespace {
thread_local std::string g_create_error;
}  // namespace

namespace pt2 {

int fail(pt2_ctx *c, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_create_error = buf;
    return code;
}

int cuda_fail(pt2_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, PT2_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}


int dev_alloc(pt2_ctx *c, DevBuf &b, size_t bytes, const char *what)
{
    if (bytes == 0) bytes = 16;
    if (c->used + bytes > c->budget)
        return fail(c, PT2_ERR_OOM, "%s: %zu bytes would exceed the device budget (%llu of %llu used)", what, bytes,
                    (unsigned long long)c->used, (unsigned long long)c->budget);
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, PT2_ERR_OOM, "%s: cudaMalloc(%zu) failed: %s", what, bytes, cudaGetErrorString(e));
    }
    b.ptr = p;
    b.bytes = bytes;
    c->used += bytes;
    return PT2_OK;
}

void dev_free(pt2_ctx *c, DevBuf &b)
{
    if (b.ptr) {
        cudaFree(b.ptr);
        c->used -= b.bytes;
    }
    b.ptr = nullptr;
    b.bytes = 0;
}

// grow-only workspace buffer
int ensure(pt2_ctx *c, DevBuf &b, size_t bytes, const char *what)
{
    if (b.bytes >= bytes && b.ptr) return PT2_OK;
    dev_free(c, b);
    c->ws_gen++;
    return dev_alloc(c, b, bytes, what);
}

void free_system(pt2_ctx *c, SystemRes &s)
{
    DevBuf *b[] = {&s.h, &s.eri, &s.J, &s.WS, &s.Jx, &s.WSx, &s.hdx, &s.dpair};
    for (DevBuf *x : b) dev_free(c, *x);
}

void free_ref(pt2_ctx *c, RefRes &r)
{
    DevBuf *b[] = {&r.keys, &r.coef, &r.hii, &r.d0, &r.g};
    for (DevBuf *x : b) dev_free(c, *x);
}

uint64_t splitmix64(uint64_t &s)
{
    uint64_t z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

bool finite_all(const double *x, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(x[i])) return false;
    return true;
}

uint64_t comb2(uint64_t m) { return m * (m - 1) / 2; }

// f(lo, hi) over [0, n) in contiguous chunks, one per host thread (at most 16).
template <class F>
void parallel_chunks(size_t n, F &&f)
{
    const size_t hw = std::thread::hardware_concurrency();
    const size_t nt = std::max<size_t>(1, std::min<size_t>(n, std::min<size_t>(16, hw ? hw : 1)));
    std::vector<std::thread> th;
    for (size_t t = 1; t < nt; ++t) th.emplace_back([&f, n, nt, t] { f(n * t / nt, n * (t + 1) / nt); });
    f(0, n / nt);
    for (auto &x : th) x.join();
}

uint64_t terms_per_det(int n, int na, int nb)
{
    uint64_t va = n - na, vb = n - nb;
    uint64_t sa = (uint64_t)na * va, sb = (uint64_t)nb * vb;
    return sa + sb + comb2(na) * comb2(va) + comb2(nb) * comb2(vb) + sa * sb;
}

SysDev sys_dev(const SystemRes &s)
{
    SysDev d;
    d.n = s.n;
    d.h = (const double *)s.h.ptr;
    d.eri = (const double *)s.eri.ptr;
    d.J = (const double *)s.J.ptr;
    d.WS = (const double *)s.WS.ptr;
    d.Jx = (const int64_t *)s.Jx.ptr;
    d.WSx = (const int64_t *)s.WSx.ptr;
    d.hdx = (const int64_t *)s.hdx.ptr;
    d.dpair = (const double *)s.dpair.ptr;
    return d;
}

GenParams gen_params(pt2_ctx *c, const SystemRes &s, const RefRes &r)
{
    GenParams p;
    memset(&p, 0, sizeof p);
    p.sys = sys_dev(s);
    p.hash = (const HashTables *)c->hash.ptr;
    p.keys = (const uint64_t *)r.keys.ptr;
    p.coef = (const double *)r.coef.ptr;
    p.d0 = (const int64_t *)r.d0.ptr;
    p.g = (const int64_t *)r.g.ptr;
    p.e0 = r.e0;
    p.n_det = r.n_det;
    p.na = r.na;
    p.nb = r.nb;
    p.n_sa = r.na * (s.n - r.na);
    p.n_sb = r.nb * (s.n - r.nb);
    p.class_lo = 0;
    p.class_hi = kNumClasses;
    p.bclass_lo = 0;
    p.bclass_hi = kNumClasses;
    p.heavy_class = 0;
    p.sym = 0;
    p.cutoff = 0.0;
    p.subtract = 0;
    p.cons_mod = 1;
    p.top_mask = 0;
    p.top_hi = 0;
    p.err = (uint32_t *)c->err_word.ptr;
    return p;
}

int status_of_err(pt2_ctx *c, uint32_t err)
{
    if (!err) return PT2_OK;
    if (err & kErrWaitTimeout) return fail(c, PT2_ERR_TIMEOUT, "a bounded device wait timed out (err bits 0x%x)", err);
    if (err & kErrFixedRange)
        return fail(c, PT2_ERR_INVALID, "a numerator H_ai c_i exceeds 2^36 in magnitude (err bits 0x%x)", err);
    if (err & kErrScratch)
        return fail(c, PT2_ERR_OOM, "an oversize tile exceeds the chunked-path scratch (err bits 0x%x)", err);
    if (err & kErrNoProgress)
        return fail(c, PT2_ERR_OOM, "a tile has more distinct keys than the chunk capacity (err bits 0x%x)", err);
    if (err & kErrCount) return fail(c, PT2_ERR_CUDA, "emitted term count differs from the plan (err bits 0x%x)", err);
    return fail(c, PT2_ERR_CUDA, "device error bits 0x%x", err);
}

}  // namespace pt2

// ===================================================================== ABI

extern "C" {

int pt2_create(pt2_ctx **out, int device, uint64_t hbm_budget_bytes)
{
    if (!out) return fail(nullptr, PT2_ERR_INVALID, "out pointer is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0)
        return fail(nullptr, PT2_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
    if (device < 0 || device >= ndev) return fail(nullptr, PT2_ERR_INVALID, "device %d out of range", device);
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail(nullptr, PT2_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, device);
    if (prop.major < 10)
        return fail(nullptr, PT2_ERR_UNSUPPORTED, "device %d is sm_%d%d; this library is built for sm_103a", device,
                    prop.major, prop.minor);
    int tile_per_sm = 0, big_per_sm = 0;
    e = init_kernel_attributes(&tile_per_sm, &big_per_sm);
    if (e != cudaSuccess) return fail(nullptr, PT2_ERR_CUDA, "kernel attributes: %s", cudaGetErrorString(e));
    auto c = std::make_unique<pt2_ctx>();
    c->device = device;
    c->sm_count = prop.multiProcessorCount;
    c->tile_per_sm = tile_per_sm;
    c->big_per_sm = big_per_sm;
    size_t fr = 0, tot = 0;
    e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) return fail(nullptr, PT2_ERR_CUDA, "cudaMemGetInfo: %s", cudaGetErrorString(e));
    c->budget = hbm_budget_bytes ? hbm_budget_bytes : (uint64_t)(0.8 * (double)fr);
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail(nullptr, PT2_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
    for (auto &ev : c->ev) {
        e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return fail(nullptr, PT2_ERR_CUDA, "event: %s", cudaGetErrorString(e));
    }
    pt2_ctx *cp = c.get();
    int rc = dev_alloc(cp, c->hash, sizeof(HashTables), "hash tables");
    if (rc) {
        g_create_error = cp->err;
        return rc;
    }
    if ((rc = dev_alloc(cp, c->err_word, 16, "error word"))) {
        g_create_error = cp->err;
        return rc;
    }
    HashTables ht;
    uint64_t seed = 0x5eed1808020490ull;
    for (int i = 0; i < kMaxOrb; ++i) ht.zc[i] = splitmix64(seed);
    for (int i = 0; i < kMaxOrb; ++i) ht.zta[i] = splitmix64(seed);
    for (int i = 0; i < kMaxOrb; ++i) ht.ztb[i] = splitmix64(seed);
    for (int i = 0; i < kMaxOrb; ++i) ht.zcb[i] = splitmix64(seed);
    for (int j2 = 1, t = 0; j2 < kMaxOrb; ++j2)
        for (int j1 = 0; j1 < j2; ++j1, ++t) ht.pairs[t] = (uint16_t)(j1 | (j2 << 8));
    e = cudaMemcpy(c->hash.ptr, &ht, sizeof ht, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(nullptr, PT2_ERR_CUDA, "copy: %s", cudaGetErrorString(e));
    *out = c.release();
    return PT2_OK;
}

void pt2_destroy(pt2_ctx *c)
{
    if (!c) return;
    server_stop(c);
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    batches_release(c);
    for (auto &kv : c->refs) free_ref(c, *kv.second);
    for (auto &kv : c->systems) free_system(c, *kv.second);
    DevBuf *bufs[] = {&c->hash,     &c->class_counts, &c->tile_counts, &c->tile_off,   &c->cursor,
                      &c->scan_tmp, &c->recs,         &c->ref_tile,    &c->ref_count,  &c->ref_off,
                      &c->ref_cursor, &c->ref_keys,   &c->big_list,    &c->big_max,    &c->scratch,
                      &c->acc,      &c->err_word,     &c->steps,       &c->gen_tab,    &c->dump_keys,
                      &c->dump_num, &c->dump_haa,     &c->dump_count,  &c->grp_counts, &c->grp_tab};
    for (DevBuf *b : bufs) dev_free(c, *b);
    if (c->steps_pinned) cudaFreeHost(c->steps_pinned);
    for (auto &ev : c->ev)
        if (ev) cudaEventDestroy(ev);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char *pt2_last_error(const pt2_ctx *c) { return c ? c->err.c_str() : g_create_error.c_str(); }

int pt2_load_system(pt2_ctx *c, int n_orb, const double *h, const double *eri, uint32_t *system_id)
{
    if (!c) return PT2_ERR_INVALID;
    if (n_orb > kMaxOrb) return fail(c, PT2_ERR_UNSUPPORTED, "n_orb = %d above %d", n_orb, kMaxOrb);
    if (n_orb < 1 || !h || !eri || !system_id) return fail(c, PT2_ERR_INVALID, "bad arguments");
    const size_t n = (size_t)n_orb, n2 = n * n, n4 = n2 * n2;
    if (!finite_all(h, n2) || !finite_all(eri, n4)) return fail(c, PT2_ERR_INVALID, "non-finite integral");
    for (size_t p = 0; p < n; ++p)
        for (size_t q = 0; q < p; ++q)
            if (std::fabs(h[p * n + q] - h[q * n + p]) > 1e-12 * std::max(1.0, std::fabs(h[p * n + q])))
                return fail(c, PT2_ERR_INVALID, "h is not symmetric at (%zu, %zu)", p, q);
    auto E = [&](size_t p, size_t q, size_t r, size_t s) { return eri[((p * n + q) * n + r) * n + s]; };
    // the first element (in index order) that differs from a symmetry partner;
    // rows p are checked in parallel, each chunk keeps its first failure
    std::vector<size_t> first(n, n4);
    parallel_chunks(n, [&](size_t p0, size_t p1) {
        for (size_t p = p0; p < p1; ++p)
            for (size_t q = 0; q < n; ++q)
                for (size_t r = 0; r < n; ++r)
                    for (size_t s = 0; s < n; ++s) {
                        const double v = E(p, q, r, s), tol = 1e-12 * std::max(1.0, std::fabs(v));
                        if (std::fabs(v - E(q, p, r, s)) > tol || std::fabs(v - E(p, q, s, r)) > tol ||
                            std::fabs(v - E(r, s, p, q)) > tol) {
                            first[p0] = ((p * n + q) * n + r) * n + s;
                            return;
                        }
                    }
    });
    const size_t bad = *std::min_element(first.begin(), first.end());
    if (bad < n4)
        return fail(c, PT2_ERR_INVALID, "eri lacks 8-fold symmetry at (%zu %zu|%zu %zu)", bad / (n2 * n),
                    bad / n2 % n, bad / n % n, bad % n);
    // Canonical copies: every symmetry-equivalent element takes the value at one
    // canonical index, so the kernels may read whichever permutation gives them
    // contiguous addresses and still see bit-identical integrals.
    std::vector<double> hc(n2), ec(n4);
    for (size_t p = 0; p < n; ++p)
        for (size_t q = 0; q < n; ++q) hc[p * n + q] = p >= q ? h[p * n + q] : h[q * n + p];
    parallel_chunks(n, [&](size_t p0, size_t p1) {
        for (size_t p = p0; p < p1; ++p)
            for (size_t q = 0; q < n; ++q)
                for (size_t r = 0; r < n; ++r)
                    for (size_t t = 0; t < n; ++t) {
                        size_t a = p, b = q, x = r, y = t;
                        if (a < b) std::swap(a, b);
                        if (x < y) std::swap(x, y);
                        if (a * n + b < x * n + y) {
                            std::swap(a, x);
                            std::swap(b, y);
                        }
                        ec[((p * n + q) * n + r) * n + t] = E(a, b, x, y);
                    }
    });
    h = hc.data();
    eri = ec.data();
    cudaSetDevice(c->device);
    // Coulomb and same-spin pair energies, as doubles for the direct diagonal and
    // as exact 2^-48 Ha integers for the incremental diagonal of the generator
    std::vector<double> J(n2), WS(n2);
    std::vector<int64_t> Jx(n2), WSx(n2), hdx(n);
    double gbound = 0.0;
    for (size_t p = 0; p < n; ++p) {
        double row = std::fabs(h[p * n + p]);
        for (size_t q = 0; q < n; ++q) {
            J[p * n + q] = E(p, p, q, q);
            WS[p * n + q] = E(p, p, q, q) - E(p, q, q, p);
            row += std::max(std::fabs(J[p * n + q]), std::fabs(WS[p * n + q]));
            Jx[p * n + q] = std::llrint(J[p * n + q] * kDenScale);
            WSx[p * n + q] = std::llrint(WS[p * n + q] * kDenScale);
        }
        hdx[p] = std::llrint(h[p * n + p] * kDenScale);
        gbound = std::max(gbound, row);
    }
    if (gbound >= kDenRange)
        return fail(c, PT2_ERR_UNSUPPORTED,
                    "orbital energy bound %.1f Ha exceeds the %.0f Ha range of the fixed-point diagonal", gbound,
                    kDenRange);
    // same-spin double elements (a1 r1|a2 r2) - (a1 r2|a2 r1) by colex pairs
    // r1 < r2, a1 < a2, from the canonical integrals: the same two doubles and
    // the same subtraction as a direct evaluation, so the same value
    const size_t np = n * (n - 1) / 2;
    std::vector<double> dp(np * np);
    for (size_t r2 = 1, P = 0; r2 < n; ++r2)
        for (size_t r1 = 0; r1 < r2; ++r1, ++P)
            for (size_t a2 = 1, Q = 0; a2 < n; ++a2)
                for (size_t a1 = 0; a1 < a2; ++a1, ++Q)
                    dp[P * np + Q] = eri[((r2 * n + a2) * n + r1) * n + a1] - eri[((r1 * n + a2) * n + r2) * n + a1];
    auto s = std::make_unique<SystemRes>();
    s->n = n_orb;
    int rc;
    if ((rc = dev_alloc(c, s->h, n2 * 8, "h")) || (rc = dev_alloc(c, s->eri, n4 * 8, "eri")) ||
        (rc = dev_alloc(c, s->J, n2 * 8, "J")) || (rc = dev_alloc(c, s->WS, n2 * 8, "WS")) ||
        (rc = dev_alloc(c, s->Jx, n2 * 8, "Jx")) || (rc = dev_alloc(c, s->WSx, n2 * 8, "WSx")) ||
        (rc = dev_alloc(c, s->hdx, n * 8, "hdx")) || (rc = dev_alloc(c, s->dpair, np * np * 8, "pair integrals"))) {
        free_system(c, *s);
        return rc;
    }
    CK(cudaMemcpy(s->h.ptr, h, n2 * 8, cudaMemcpyHostToDevice), "copy h");
    CK(cudaMemcpy(s->eri.ptr, eri, n4 * 8, cudaMemcpyHostToDevice), "copy eri");
    CK(cudaMemcpy(s->J.ptr, J.data(), n2 * 8, cudaMemcpyHostToDevice), "copy J");
    CK(cudaMemcpy(s->WS.ptr, WS.data(), n2 * 8, cudaMemcpyHostToDevice), "copy WS");
    CK(cudaMemcpy(s->Jx.ptr, Jx.data(), n2 * 8, cudaMemcpyHostToDevice), "copy Jx");
    CK(cudaMemcpy(s->WSx.ptr, WSx.data(), n2 * 8, cudaMemcpyHostToDevice), "copy WSx");
    CK(cudaMemcpy(s->hdx.ptr, hdx.data(), n * 8, cudaMemcpyHostToDevice), "copy hdx");
    CK(cudaMemcpy(s->dpair.ptr, dp.data(), np * np * 8, cudaMemcpyHostToDevice), "copy pair integrals");
    uint32_t id = c->next_id++;
    c->systems[id] = std::move(s);
    *system_id = id;
    return PT2_OK;
}

int pt2_load_reference(pt2_ctx *c, uint32_t system_id, uint64_t n_det, const uint64_t *keys, const double *coef,
                       double e0, uint32_t *ref_id)
{
    if (!c) return PT2_ERR_INVALID;
    auto it = c->systems.find(system_id);
    if (it == c->systems.end()) return fail(c, PT2_ERR_NOT_FOUND, "unknown system id %u", system_id);
    if (n_det == 0 || !keys || !coef || !ref_id) return fail(c, PT2_ERR_INVALID, "bad arguments");
    if (n_det > (1ull << 31)) return fail(c, PT2_ERR_UNSUPPORTED, "n_det above 2^31");
    SystemRes &s = *it->second;
    const uint64_t lim = s.n == 64 ? ~0ull : ((1ull << s.n) - 1);
    const int na = __builtin_popcountll(keys[0]), nb = __builtin_popcountll(keys[1]);
    for (uint64_t i = 0; i < n_det; ++i) {
        if ((keys[2 * i] & ~lim) || (keys[2 * i + 1] & ~lim))
            return fail(c, PT2_ERR_INVALID, "determinant %llu has an orbital at or above n_orb", (unsigned long long)i);
        if (__builtin_popcountll(keys[2 * i]) != na || __builtin_popcountll(keys[2 * i + 1]) != nb)
            return fail(c, PT2_ERR_INVALID, "determinant %llu has a different electron count", (unsigned long long)i);
    }
    if (!finite_all(coef, n_det) || !std::isfinite(e0)) return fail(c, PT2_ERR_INVALID, "non-finite coefficient or E0");
    bool flip_symmetric = na == nb;
    {
        // sorted (alpha, beta, index): duplicates, and whether every determinant's
        // mirror (beta, alpha) is present with the same coefficient
        struct K {
            uint64_t a, b, i;
            bool operator<(const K &o) const { return a < o.a || (a == o.a && b < o.b); }
        };
        std::vector<K> k(n_det);
        for (uint64_t i = 0; i < n_det; ++i) k[i] = {keys[2 * i], keys[2 * i + 1], i};
        std::sort(k.begin(), k.end());
        for (uint64_t i = 1; i < n_det; ++i)
            if (k[i].a == k[i - 1].a && k[i].b == k[i - 1].b)
                return fail(c, PT2_ERR_INVALID, "duplicate determinant in the reference");
        for (uint64_t i = 0; flip_symmetric && i < n_det; ++i) {
            const K m{k[i].b, k[i].a, 0};
            auto it = std::lower_bound(k.begin(), k.end(), m);
            flip_symmetric = it != k.end() && it->a == m.a && it->b == m.b && coef[it->i] == coef[k[i].i];
        }
    }
    cudaSetDevice(c->device);
    auto r = std::make_unique<RefRes>();
    r->system = system_id;
    r->n_det = n_det;
    r->na = na;
    r->nb = nb;
    r->e0 = e0;
    r->flip_symmetric = flip_symmetric;
    int rc;
    if ((rc = dev_alloc(c, r->keys, n_det * 16, "reference keys")) ||
        (rc = dev_alloc(c, r->coef, n_det * 8, "coefficients")) ||
        (rc = dev_alloc(c, r->hii, n_det * 8, "diagonals")) || (rc = dev_alloc(c, r->d0, n_det * 8, "denominators")) ||
        (rc = dev_alloc(c, r->g, n_det * 2 * (size_t)s.n * 8, "orbital energies"))) {
        free_ref(c, *r);
        return rc;
    }
    CK(cudaMemcpyAsync(r->keys.ptr, keys, n_det * 16, cudaMemcpyHostToDevice, c->stream), "copy keys");
    CK(cudaMemcpyAsync(r->coef.ptr, coef, n_det * 8, cudaMemcpyHostToDevice, c->stream), "copy coef");
    CK(launch_diag(sys_dev(s), (const uint64_t *)r->keys.ptr, n_det, (double *)r->hii.ptr, c->stream),
       "diagonal kernel");
    CK(launch_ref_g(sys_dev(s), (const uint64_t *)r->keys.ptr, n_det, (int64_t *)r->g.ptr, c->stream),
       "orbital energy kernel");
    CK(launch_ref_d0(sys_dev(s), (const uint64_t *)r->keys.ptr, (const int64_t *)r->g.ptr, n_det, e0,
                     (int64_t *)r->d0.ptr, c->stream),
       "denominator kernel");
    {
        // E0 - H_ii must lie inside the fixed-point range of the diagonal
        std::vector<double> hii(n_det);
        CK(cudaMemcpyAsync(hii.data(), r->hii.ptr, n_det * 8, cudaMemcpyDeviceToHost, c->stream), "copy");
        CK(cudaStreamSynchronize(c->stream), "sync");
        for (uint64_t i = 0; i < n_det; ++i)
            if (!(std::fabs(e0 - hii[i]) < kDenRange)) {
                free_ref(c, *r);
                return fail(c, PT2_ERR_UNSUPPORTED, "|E0 - H_ii| = %g Ha for determinant %llu exceeds %.0f Ha",
                            std::fabs(e0 - hii[i]), (unsigned long long)i, kDenRange);
            }
    }
    s.refs++;
    uint32_t id = c->next_id++;
    c->refs[id] = std::move(r);
    *ref_id = id;
    return PT2_OK;
}

int pt2_unload(pt2_ctx *c, uint32_t id)
{
    if (!c) return PT2_ERR_INVALID;
    cudaSetDevice(c->device);
    {
        // a reference with unfinished requests in the serving engine is
        // refused at once: not after waiting for the engine's current step
        // (which holds the execution lock) or for the stream, by which time
        // they may have finished
        std::lock_guard<std::mutex> sl(c->served_mu);
        auto si = c->served.find(id);
        if (si != c->served.end() && si->second > 0)
            return fail(c, PT2_ERR_BUSY, "reference %u has requests in the serving engine", id);
    }
    cudaStreamSynchronize(c->stream);
    std::lock_guard<std::recursive_mutex> lock(c->exec);
    auto ri = c->refs.find(id);
    if (ri != c->refs.end()) {
        RefRes &r = *ri->second;
        if (r.busy) return fail(c, PT2_ERR_BUSY, "reference %u has requests in the serving engine", id);
        free_ref(c, r);
        c->systems.at(r.system)->refs--;
        c->refs.erase(ri);
        return PT2_OK;
    }
    auto si = c->systems.find(id);
    if (si != c->systems.end()) {
        if (si->second->refs > 0) return fail(c, PT2_ERR_INVALID, "system %u is still used by a reference", id);
        free_system(c, *si->second);
        c->systems.erase(si);
        return PT2_OK;
    }
    return fail(c, PT2_ERR_NOT_FOUND, "unknown id %u", id);
}

int pt2_diagonal(pt2_ctx *c, uint32_t system_id, uint64_t n, const uint64_t *keys, double *out)
{
    if (!c) return PT2_ERR_INVALID;
    auto it = c->systems.find(system_id);
    if (it == c->systems.end()) return fail(c, PT2_ERR_NOT_FOUND, "unknown system id %u", system_id);
    if (n == 0) return PT2_OK;
    if (!keys || !out) return fail(c, PT2_ERR_INVALID, "bad arguments");
    SystemRes &s = *it->second;
    const uint64_t lim = s.n == 64 ? ~0ull : ((1ull << s.n) - 1);
    for (uint64_t i = 0; i < 2 * n; ++i)
        if (keys[i] & ~lim) return fail(c, PT2_ERR_INVALID, "determinant %llu has an orbital at or above n_orb",
                                        (unsigned long long)(i / 2));
    cudaSetDevice(c->device);
    DevBuf k, d;
    int rc;
    if ((rc = dev_alloc(c, k, n * 16, "keys"))) return rc;
    if ((rc = dev_alloc(c, d, n * 8, "diagonals"))) {
        dev_free(c, k);
        return rc;
    }
    cudaError_t e = cudaMemcpyAsync(k.ptr, keys, n * 16, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_diag(sys_dev(s), (const uint64_t *)k.ptr, n, (double *)d.ptr, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d.ptr, n * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, k);
    dev_free(c, d);
    if (e != cudaSuccess) return cuda_fail(c, e, "diagonal");
    return PT2_OK;
}

int pt2_det_terms(pt2_ctx *c, uint32_t ref_id, uint64_t det_index, uint64_t *keys, double *val, double *haa,
                  uint64_t cap, uint64_t *n_out)
{
    if (!c) return PT2_ERR_INVALID;
    // the lock comes first: pt2_unload frees references and systems under it
    std::lock_guard<std::recursive_mutex> lock(c->exec);
    auto it = c->refs.find(ref_id);
    if (it == c->refs.end()) return fail(c, PT2_ERR_NOT_FOUND, "unknown reference id %u", ref_id);
    if (!n_out || (cap && (!keys || !val || !haa))) return fail(c, PT2_ERR_INVALID, "bad arguments");
    RefRes &r = *it->second;
    if (det_index >= r.n_det) return fail(c, PT2_ERR_INVALID, "determinant index out of range");
    SystemRes &s = *c->systems.at(r.system);
    cudaSetDevice(c->device);
    const uint64_t T = terms_per_det(s.n, r.na, r.nb);
    int rc;
    if ((rc = ensure(c, c->recs, std::max<uint64_t>(T, 1) * sizeof(Rec32), "term records"))) return rc;
    if ((rc = ensure(c, c->cursor, 8, "cursor"))) return rc;
    GenParams p = gen_params(c, s, r);
    p.n_tiles = 1;
    p.cursor = (unsigned int *)c->cursor.ptr;
    p.recs = (Rec32 *)c->recs.ptr;
    p.rec_cap = T;
    p.det_begin = det_index;
    gen_layout(p, kModeDetTerms);
    CK(cudaMemsetAsync(c->err_word.ptr, 0, 4, c->stream), "memset");
    CK(cudaMemsetAsync(c->cursor.ptr, 0, 4, c->stream), "memset");
    CK(launch_gen_single(kModeDetTerms, p, nullptr, nullptr, c->stream), "generator");
    unsigned int n32 = 0;
    uint32_t err = 0;
    CK(cudaMemcpyAsync(&n32, c->cursor.ptr, 4, cudaMemcpyDeviceToHost, c->stream), "copy");
    CK(cudaMemcpyAsync(&err, c->err_word.ptr, 4, cudaMemcpyDeviceToHost, c->stream), "copy");
    CK(cudaStreamSynchronize(c->stream), "sync");
    if ((rc = status_of_err(c, err))) return rc;
    const unsigned long long n = n32;
    *n_out = n;
    if (n > cap) return fail(c, PT2_ERR_OOM, "determinant has %llu terms, above cap %llu", n, (unsigned long long)cap);
    std::vector<Rec32> h(n);
    CK(cudaMemcpy(h.data(), c->recs.ptr, n * sizeof(Rec32), cudaMemcpyDeviceToHost), "copy");
    for (uint64_t i = 0; i < n; ++i) {
        keys[2 * i] = h[i].a;
        keys[2 * i + 1] = h[i].b;
        val[i] = h[i].num;
        double d;
        memcpy(&d, &h[i].den, 8);  // this mode stores H_aa itself
        haa[i] = d;
    }
    return PT2_OK;
}

int pt2_det_terms_noalloc(pt2_ctx *c, uint32_t ref_id, uint64_t det_index, uint64_t *keys, double *val,
                          double *haa, uint64_t cap, uint64_t *n_out)
{
    if (!c) return PT2_ERR_INVALID;
    // the lock comes first: pt2_unload frees references and systems under it
    std::lock_guard<std::recursive_mutex> lock(c->exec);
    auto it = c->refs.find(ref_id);
    if (it == c->refs.end()) return fail(c, PT2_ERR_NOT_FOUND, "unknown reference id %u", ref_id);
    if (!n_out || (cap && (!keys || !val || !haa))) return fail(c, PT2_ERR_INVALID, "bad arguments");
    RefRes &r = *it->second;
    if (det_index >= r.n_det) return fail(c, PT2_ERR_INVALID, "determinant index out of range");
    SystemRes &s = *c->systems.at(r.system);
    const uint64_t T = terms_per_det(s.n, r.na, r.nb);
    if (T > kNoAllocMaxTerms)
        return fail(c, PT2_ERR_OOM,
                    "a determinant of this system has %llu terms, above the %llu the fixed device scratch holds",
                    (unsigned long long)T, (unsigned long long)kNoAllocMaxTerms);
    cudaSetDevice(c->device);
    GenParams p = gen_params(c, s, r);
    p.det_begin = det_index;
    unsigned long long n = 0;
    // the error word is context memory allocated at creation; clear it so
    // that neither this call nor the next run sees a stale bit
    CK(cudaMemsetAsync(c->err_word.ptr, 0, 4, c->stream), "memset");
    CK(launch_det_terms_noalloc(c->device, p, cap, keys, val, haa, &n, c->stream), "allocation-free generation");
    uint32_t err = 0;
    CK(cudaMemcpyAsync(&err, c->err_word.ptr, 4, cudaMemcpyDeviceToHost, c->stream), "copy");
    CK(cudaStreamSynchronize(c->stream), "sync");
    int rc;
    if ((rc = status_of_err(c, err))) return rc;
    *n_out = n;
    if (n > cap) return fail(c, PT2_ERR_OOM, "determinant has %llu terms, above cap %llu", n, (unsigned long long)cap);
    return PT2_OK;
}

int pt2_eval_terms(pt2_ctx *c, uint64_t n, const double *num, const double *denom, double *term)
{
    if (!c) return PT2_ERR_INVALID;
    if (n == 0) return PT2_OK;
    if (!num || !denom || !term) return fail(c, PT2_ERR_INVALID, "bad arguments");
    for (uint64_t i = 0; i < n; ++i) {
        if (!std::isfinite(num[i]) || !std::isfinite(denom[i]) || !(std::fabs(denom[i]) < 32768.0) ||
            std::llrint(denom[i] * kDenScale) == 0)
            return fail(c, PT2_ERR_INVALID, "entry %llu: numerator or denominator out of range",
                        (unsigned long long)i);
    }
    std::lock_guard<std::recursive_mutex> lock(c->exec);
    cudaSetDevice(c->device);
    DevBuf dn, dd, dt;
    int rc;
    if ((rc = dev_alloc(c, dn, n * 8, "numerators"))) return rc;
    if ((rc = dev_alloc(c, dd, n * 8, "denominators")) || (rc = dev_alloc(c, dt, n * 8, "terms"))) {
        dev_free(c, dn);
        dev_free(c, dd);
        return rc;
    }
    cudaError_t e = cudaMemcpyAsync(dn.ptr, num, n * 8, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dd.ptr, denom, n * 8, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = launch_eval_terms((const double *)dn.ptr, (const double *)dd.ptr, n, (double *)dt.ptr, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(term, dt.ptr, n * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, dn);
    dev_free(c, dd);
    dev_free(c, dt);
    if (e != cudaSuccess) return cuda_fail(c, e, "term evaluation");
    return PT2_OK;
}

int pt2_phase_times(pt2_ctx *c, double *out, int n, uint64_t *launches)
{
    if (!c || (!out && n > 0)) return PT2_ERR_INVALID;
    for (int i = 0; i < n && i < kPhases; ++i) out[i] = c->phase_ms[i];
    if (launches) *launches = c->launches;
    return PT2_OK;
}

int pt2_memory_info(pt2_ctx *c, uint64_t *budget, uint64_t *used, uint64_t *device_free)
{
    if (!c) return PT2_ERR_INVALID;
    if (budget) *budget = c->budget;
    if (used) *used = c->used;
    if (device_free) {
        cudaSetDevice(c->device);
        size_t fr = 0, tot = 0;
        CK(cudaMemGetInfo(&fr, &tot), "cudaMemGetInfo");
        *device_free = fr;
    }
    return PT2_OK;
}

void *pt2_stream(pt2_ctx *c) { return c ? (void *)c->stream : nullptr; }

}  // extern "C"
