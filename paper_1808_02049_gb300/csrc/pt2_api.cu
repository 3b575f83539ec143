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
#include <vector>

#include "pt2.h"
#include "pt2_internal.cuh"

using namespace pt2;

namespace {

thread_local std::string g_create_error;

struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

struct SystemRes {
    int n = 0;
    DevBuf h, eri, J, WS, Jx, WSx, hdx;
    int refs = 0;  // references using this system
};

struct RefRes {
    uint32_t system = 0;
    uint64_t n_det = 0;
    int na = 0, nb = 0;
    double e0 = 0.0;
    DevBuf keys, coef, hii, d0;
};

constexpr int kPhases = 8;

}  // namespace

struct pt2_ctx {
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    uint64_t budget = 0, used = 0;
    std::string err;
    uint32_t next_id = 1;
    std::map<uint32_t, std::unique_ptr<SystemRes>> systems;
    std::map<uint32_t, std::unique_ptr<RefRes>> refs;
    DevBuf hash;
    // run workspace (grow-only)
    DevBuf class_counts, tile_counts, tile_off, cursor, scan_tmp, recs, ref_tile, ref_count, ref_off, ref_cursor,
        ref_keys, big_list, scratch, acc, err_word, dump_keys, dump_num, dump_haa, dump_count;
    cudaEvent_t ev[2 * kPhases + 2] = {};
    double phase_ms[kPhases] = {};
    uint64_t launches = 0;
};

namespace {

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

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

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
    return dev_alloc(c, b, bytes, what);
}

void free_system(pt2_ctx *c, SystemRes &s)
{
    DevBuf *b[] = {&s.h, &s.eri, &s.J, &s.WS, &s.Jx, &s.WSx, &s.hdx};
    for (DevBuf *x : b) dev_free(c, *x);
}

void free_ref(pt2_ctx *c, RefRes &r)
{
    DevBuf *b[] = {&r.keys, &r.coef, &r.hii, &r.d0};
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
    p.e0 = r.e0;
    p.n_det = r.n_det;
    p.na = r.na;
    p.nb = r.nb;
    p.n_sa = r.na * (s.n - r.na);
    p.n_sb = r.nb * (s.n - r.nb);
    p.class_lo = 0;
    p.class_hi = kNumClasses;
    p.cons_mod = 1;
    p.err = (uint32_t *)c->err_word.ptr;
    return p;
}

// Launch the generator over all determinants in slices (grid.x limit).
cudaError_t gen_all(pt2_ctx *c, GenMode mode, GenParams p, uint64_t n_det)
{
    gen_layout(p, mode);
    const uint64_t slice = 1ull << 30;
    for (uint64_t b = 0; b < n_det; b += slice) {
        p.det_begin = b;
        uint64_t m = std::min(slice, n_det - b);
        cudaError_t e = launch_gen(mode, p, m, c->stream);
        c->launches++;
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

struct Pass {
    uint32_t c_lo, c_hi;
    uint64_t records;
    uint64_t n_tiles;
};

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

struct DumpTarget {
    uint64_t *keys = nullptr;
    double *num = nullptr, *haa = nullptr;
    uint64_t cap = 0;
    uint64_t n_out = 0;
};

int run_impl(pt2_ctx *c, uint32_t ref_id, const pt2_opts *opts_in, pt2_result *out, DumpTarget *dump)
{
    auto it = c->refs.find(ref_id);
    if (it == c->refs.end()) return fail(c, PT2_ERR_NOT_FOUND, "unknown reference id %u", ref_id);
    if (!out) return fail(c, PT2_ERR_INVALID, "result pointer is NULL");
    RefRes &r = *it->second;
    SystemRes &s = *c->systems.at(r.system);
    pt2_opts o;
    memset(&o, 0, sizeof o);
    if (opts_in) o = *opts_in;
    if (o.constraint_mod > 1 && o.constraint_rem >= o.constraint_mod)
        return fail(c, PT2_ERR_INVALID, "constraint_rem must be below constraint_mod");
    uint64_t tile_target = o.tile_target ? o.tile_target : 576;
    if (tile_target > (uint64_t)kTileCap) return fail(c, PT2_ERR_INVALID, "tile_target above %d", kTileCap);
    const bool prof = (o.flags & PT2_FLAG_PROFILE) != 0;
    cudaStream_t st = c->stream;
    c->launches = 0;
    for (double &x : c->phase_ms) x = 0.0;
    int rc;

    // fixed workspace
    if ((rc = ensure(c, c->class_counts, kNumClasses * 8, "class counts"))) return rc;
    if ((rc = ensure(c, c->acc, sizeof(RunAcc), "accumulator"))) return rc;
    if ((rc = ensure(c, c->ref_tile, r.n_det * 4, "reference tiles"))) return rc;
    if ((rc = ensure(c, c->ref_keys, r.n_det * 16, "reference slices"))) return rc;
    if (dump) {
        if ((rc = ensure(c, c->dump_count, 16, "dump count"))) return rc;
        if ((rc = ensure(c, c->dump_keys, std::max<uint64_t>(dump->cap, 1) * 16, "dump keys"))) return rc;
        if ((rc = ensure(c, c->dump_num, std::max<uint64_t>(dump->cap, 1) * 8, "dump num"))) return rc;
        if ((rc = ensure(c, c->dump_haa, std::max<uint64_t>(dump->cap, 1) * 8, "dump haa"))) return rc;
        CK(cudaMemsetAsync(c->dump_count.ptr, 0, 8, st), "memset");
    }
    RunAcc *acc = (RunAcc *)c->acc.ptr;
    uint32_t *errw = (uint32_t *)c->err_word.ptr;

    CK(cudaEventRecord(c->ev[0], st), "event");
    CK(cudaMemsetAsync(errw, 0, 4, st), "memset");
    CK(launch_acc_init(acc, st), "acc init");
    c->launches++;

    // ---- work list: terms per alpha-hash class
    GenParams gp = gen_params(c, s, r);
    gp.cons_mod = o.constraint_mod > 1 ? o.constraint_mod : 1;
    gp.cons_rem = o.constraint_mod > 1 ? o.constraint_rem : 0;
    gp.class_counts = (unsigned long long *)c->class_counts.ptr;
    CK(cudaMemsetAsync(c->class_counts.ptr, 0, kNumClasses * 8, st), "memset");
    CK(gen_all(c, kModeClassCount, gp, r.n_det), "class count kernel");
    std::vector<unsigned long long> cls(kNumClasses);
    CK(cudaMemcpyAsync(cls.data(), c->class_counts.ptr, kNumClasses * 8, cudaMemcpyDeviceToHost, st), "copy");
    CK(cudaEventRecord(c->ev[1], st), "event");
    CK(cudaStreamSynchronize(st), "sync");
    if (prof) {
        float ms = 0;
        cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
        c->phase_ms[0] += ms;
    }

    // ---- plan passes under the memory budget
    uint64_t total = 0;
    for (auto x : cls) total += x;
    uint64_t pass_budget = o.pass_budget_bytes;
    if (!pass_budget) {
        // the pass workspace a previous run left allocated is reused, so it counts as available
        const DevBuf *ws[] = {&c->tile_counts, &c->tile_off, &c->cursor,   &c->scan_tmp, &c->ref_count,
                              &c->ref_off,     &c->ref_cursor, &c->big_list, &c->scratch,  &c->recs};
        uint64_t held = 0;
        for (const DevBuf *b : ws) held += b->bytes;
        const uint64_t fixed = c->used - held;
        const uint64_t reserve = (2ull << 30) + (64ull << 20);  // oversize scratch and slack
        pass_budget = c->budget > fixed + reserve ? c->budget - fixed - reserve : 0;
    }
    // per record: 32 bytes plus about 60 bytes of tile bookkeeping per tile
    const double per_rec = sizeof(Rec32) + 60.0 / (double)tile_target;
    uint64_t max_rec = (uint64_t)((double)pass_budget / per_rec);
    // Emission scatters every term to a random tile through an atomic cursor;
    // when the cursors of a pass no longer fit in L2 those atomics go to DRAM,
    // so a default pass holds at most kMaxTilesPerPass tiles.
    if (!o.pass_budget_bytes) max_rec = std::min<uint64_t>(max_rec, kMaxTilesPerPass * tile_target);
    // Random 32-byte writes spread over a larger footprint run slower (address
    // translation reach), so a default pass also stays below kMaxPassBytes.
    if (!o.pass_budget_bytes) max_rec = std::min<uint64_t>(max_rec, kMaxPassBytes / sizeof(Rec32));
    if (max_rec < 1024)
        return fail(c, PT2_ERR_OOM, "pass budget of %llu bytes is too small (context budget %llu, in use %llu)",
                    (unsigned long long)pass_budget, (unsigned long long)c->budget, (unsigned long long)c->used);
    std::vector<Pass> passes;
    {
        Pass cur{0, 0, 0, 0};
        for (int k = 0; k < kNumClasses; ++k) {
            if (cls[k] > max_rec)
                return fail(c, PT2_ERR_OOM,
                            "alpha class %d holds %llu terms, above the %llu a pass can hold; raise the budget", k,
                            (unsigned long long)cls[k], (unsigned long long)max_rec);
            if (cur.records + cls[k] > max_rec) {
                cur.c_hi = k;
                passes.push_back(cur);
                cur = Pass{(uint32_t)k, 0, 0, 0};
            }
            cur.records += cls[k];
        }
        cur.c_hi = kNumClasses;
        if (cur.records > 0 || passes.empty()) passes.push_back(cur);
    }
    uint64_t max_tiles = 1, max_records = 1;
    for (auto &p : passes) {
        p.n_tiles = std::max<uint64_t>(1, (p.records + tile_target - 1) / tile_target);
        max_tiles = std::max(max_tiles, p.n_tiles);
        max_records = std::max(max_records, p.records);
    }
    if (max_tiles >= 0xFFFFFFFFull) return fail(c, PT2_ERR_INVALID, "too many tiles in one pass");
    if ((rc = ensure(c, c->tile_counts, max_tiles * 4, "tile counts"))) return rc;
    if ((rc = ensure(c, c->tile_off, (max_tiles + 1) * 8, "tile offsets"))) return rc;
    if ((rc = ensure(c, c->cursor, max_tiles * 8, "tile cursors"))) return rc;
    if ((rc = ensure(c, c->scan_tmp, scan_tmp_elems(max_tiles) * 8 * 2, "scan scratch"))) return rc;
    if ((rc = ensure(c, c->ref_count, max_tiles * 4, "reference counts"))) return rc;
    if ((rc = ensure(c, c->ref_off, (max_tiles + 1) * 8, "reference offsets"))) return rc;
    if ((rc = ensure(c, c->ref_cursor, max_tiles * 8, "reference cursors"))) return rc;
    if ((rc = ensure(c, c->big_list, max_tiles * 4, "oversize list"))) return rc;
    if ((rc = ensure(c, c->recs, max_records * sizeof(Rec32), "term records"))) return rc;

    uint64_t n_tiles_total = 0;
    uint32_t n_big_total = 0;
    const int tile_ctas = 4 * c->sm_count;
    for (size_t pi = 0; pi < passes.size(); ++pi) {
        const Pass &P = passes[pi];
        n_tiles_total += P.n_tiles;
        cudaEvent_t *E = &c->ev[2];
        // tile counts
        if (prof) CK(cudaEventRecord(E[0], st), "event");
        GenParams g = gp;
        g.class_lo = P.c_lo;
        g.class_hi = P.c_hi;
        g.n_tiles = P.n_tiles;
        g.tile_counts = (uint32_t *)c->tile_counts.ptr;
        g.cursor = (unsigned long long *)c->cursor.ptr;
        g.recs = (Rec32 *)c->recs.ptr;
        g.rec_cap = P.records;
        CK(cudaMemsetAsync(g.tile_counts, 0, P.n_tiles * 4, st), "memset");
        CK(gen_all(c, kModeTileCount, g, r.n_det), "tile count kernel");
        if (prof) CK(cudaEventRecord(E[1], st), "event");
        CK(launch_scan_u32_to_u64(g.tile_counts, (unsigned long long *)c->tile_off.ptr, P.n_tiles,
                                  (unsigned long long *)c->scan_tmp.ptr, st),
           "scan");
        c->launches += 3;
        CK(cudaMemcpyAsync(c->cursor.ptr, c->tile_off.ptr, P.n_tiles * 8, cudaMemcpyDeviceToDevice, st), "copy");
        if (prof) CK(cudaEventRecord(E[2], st), "event");
        CK(gen_all(c, kModeEmit, g, r.n_det), "emit kernel");
        if (prof) CK(cudaEventRecord(E[3], st), "event");
        // reference slices of the pass
        RefPartParams rp;
        rp.keys = (const uint64_t *)r.keys.ptr;
        rp.n_det = r.n_det;
        rp.hash = (const HashTables *)c->hash.ptr;
        rp.class_lo = P.c_lo;
        rp.class_hi = P.c_hi;
        rp.cons_mod = gp.cons_mod;
        rp.cons_rem = gp.cons_rem;
        rp.n_tiles = P.n_tiles;
        rp.ref_tile = (uint32_t *)c->ref_tile.ptr;
        rp.ref_count = (uint32_t *)c->ref_count.ptr;
        rp.ref_cursor = (unsigned long long *)c->ref_cursor.ptr;
        rp.ref_keys_out = (uint64_t *)c->ref_keys.ptr;
        CK(cudaMemsetAsync(rp.ref_count, 0, P.n_tiles * 4, st), "memset");
        CK(launch_ref_partition(rp, 0, st), "reference tiles");
        CK(launch_scan_u32_to_u64(rp.ref_count, (unsigned long long *)c->ref_off.ptr, P.n_tiles,
                                  (unsigned long long *)c->scan_tmp.ptr + scan_tmp_elems(max_tiles), st),
           "scan");
        CK(cudaMemcpyAsync(rp.ref_cursor, c->ref_off.ptr, P.n_tiles * 8, cudaMemcpyDeviceToDevice, st), "copy");
        CK(launch_ref_partition(rp, 1, st), "reference scatter");
        CK(launch_sort_slices((const unsigned long long *)c->ref_off.ptr, (uint64_t *)c->ref_keys.ptr, P.n_tiles, st),
           "reference sort");
        c->launches += 6;
        if (prof) CK(cudaEventRecord(E[4], st), "event");
        // tiles
        TileParams tp;
        memset(&tp, 0, sizeof tp);
        tp.recs = (const Rec32 *)c->recs.ptr;
        tp.tile_off = (const unsigned long long *)c->tile_off.ptr;
        tp.ref_off = (const unsigned long long *)c->ref_off.ptr;
        tp.ref_keys = (const uint64_t *)c->ref_keys.ptr;
        tp.n_tiles = P.n_tiles;
        tp.e0 = r.e0;
        tp.acc = acc;
        tp.big_list = (uint32_t *)c->big_list.ptr;
        tp.err = errw;
        if (dump) {
            tp.dump_keys = (uint64_t *)c->dump_keys.ptr;
            tp.dump_num = (double *)c->dump_num.ptr;
            tp.dump_haa = (double *)c->dump_haa.ptr;
            tp.dump_count = (unsigned long long *)c->dump_count.ptr;
            tp.dump_cap = dump->cap;
        }
        CK(launch_tiles(tp, tile_ctas, st), "tile kernel");
        c->launches++;
        if (prof) CK(cudaEventRecord(E[5], st), "event");
        // oversize tiles: size the scratch from what the tile kernel found
        RunAcc bi;
        CK(cudaMemcpyAsync(&bi, acc, sizeof bi, cudaMemcpyDeviceToHost, st), "copy");
        CK(cudaStreamSynchronize(st), "sync");
        n_big_total += bi.n_big;
        if (bi.n_big) {
            uint64_t cap = bi.big_max;
            int ctas = (int)std::min<uint64_t>(bi.n_big, 4ull * (uint64_t)c->sm_count);
            // keep the scratch within 2 GB (or what a single tile needs)
            while (ctas > 1 && (uint64_t)ctas * 2 * cap * sizeof(Rec48) > (2ull << 30)) ctas /= 2;
            if ((rc = ensure(c, c->scratch, (size_t)ctas * 2 * cap * sizeof(Rec48), "oversize scratch"))) return rc;
            tp.scratch = (Rec48 *)c->scratch.ptr;
            tp.scratch_cap = cap;
            CK(launch_big_tiles(tp, ctas, st), "oversize tile kernel");
            c->launches++;
        }
        if (prof) CK(cudaEventRecord(E[6], st), "event");
        CK(launch_pass_finish(tp.tile_off, P.n_tiles, P.records, acc, errw, st), "pass finish");
        c->launches++;
        if (prof) {
            CK(cudaEventRecord(E[7], st), "event");
            CK(cudaEventSynchronize(E[7]), "sync");
            float ms;
            for (int k = 0; k < 7; ++k) {
                cudaEventElapsedTime(&ms, E[k], E[k + 1]);
                c->phase_ms[k + 1] += ms;
            }
        }
    }
    CK(launch_acc_finalize(acc, st), "finalize");
    c->launches++;
    RunAcc h;
    uint32_t err = 0;
    CK(cudaMemcpyAsync(&h, acc, sizeof h, cudaMemcpyDeviceToHost, st), "copy");
    CK(cudaMemcpyAsync(&err, errw, 4, cudaMemcpyDeviceToHost, st), "copy");
    CK(cudaEventRecord(c->ev[1], st), "event");
    CK(cudaStreamSynchronize(st), "sync");
    float ms = 0;
    cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
    err |= h.err;
    if ((rc = status_of_err(c, err))) return rc;
    memset(out, 0, sizeof *out);
    out->e2 = h.e2;
    out->n_terms = h.n_terms;
    out->n_unique = h.n_unique;
    out->n_in_ref = h.n_in_ref;
    out->n_external = h.n_ext;
    out->digest_sum = h.dsum;
    out->digest_xor = h.dxor;
    out->min_abs_denom = h.min_abs_den;
    out->n_pos_denom = h.n_pos;
    out->n_passes = (uint32_t)passes.size();
    out->n_tiles = (uint32_t)std::min<uint64_t>(n_tiles_total, 0xFFFFFFFFull);
    out->n_oversize = n_big_total;
    out->seconds = ms * 1e-3;
    if (h.n_terms != total)
        return fail(c, PT2_ERR_CUDA, "generated %llu terms, planned %llu", (unsigned long long)h.n_terms,
                    (unsigned long long)total);
    if (dump) {
        unsigned long long nd = 0;
        CK(cudaMemcpy(&nd, c->dump_count.ptr, 8, cudaMemcpyDeviceToHost), "copy");
        dump->n_out = nd;
        if (nd > dump->cap)
            return fail(c, PT2_ERR_OOM, "external set has %llu keys, above the dump capacity %llu", nd,
                        (unsigned long long)dump->cap);
        CK(cudaMemcpy(dump->keys, c->dump_keys.ptr, nd * 16, cudaMemcpyDeviceToHost), "copy");
        CK(cudaMemcpy(dump->num, c->dump_num.ptr, nd * 8, cudaMemcpyDeviceToHost), "copy");
        CK(cudaMemcpy(dump->haa, c->dump_haa.ptr, nd * 8, cudaMemcpyDeviceToHost), "copy");
    }
    return PT2_OK;
}

}  // namespace

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
    auto c = std::make_unique<pt2_ctx>();
    c->device = device;
    c->sm_count = prop.multiProcessorCount;
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
    e = cudaMemcpy(c->hash.ptr, &ht, sizeof ht, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(nullptr, PT2_ERR_CUDA, "copy: %s", cudaGetErrorString(e));
    *out = c.release();
    return PT2_OK;
}

void pt2_destroy(pt2_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (auto &kv : c->refs) free_ref(c, *kv.second);
    for (auto &kv : c->systems) free_system(c, *kv.second);
    DevBuf *bufs[] = {&c->hash,      &c->class_counts, &c->tile_counts, &c->tile_off, &c->cursor,
                      &c->scan_tmp,  &c->recs,         &c->ref_tile,    &c->ref_count, &c->ref_off,
                      &c->ref_cursor, &c->ref_keys,    &c->big_list,    &c->scratch,  &c->acc,
                      &c->err_word,  &c->dump_keys,    &c->dump_num,    &c->dump_haa, &c->dump_count};
    for (DevBuf *b : bufs) dev_free(c, *b);
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
    for (size_t p = 0; p < n; ++p)
        for (size_t q = 0; q < n; ++q)
            for (size_t r = 0; r < n; ++r)
                for (size_t s = 0; s < n; ++s) {
                    double v = E(p, q, r, s), tol = 1e-12 * std::max(1.0, std::fabs(v));
                    if (std::fabs(v - E(q, p, r, s)) > tol || std::fabs(v - E(p, q, s, r)) > tol ||
                        std::fabs(v - E(r, s, p, q)) > tol)
                        return fail(c, PT2_ERR_INVALID, "eri lacks 8-fold symmetry at (%zu %zu|%zu %zu)", p, q, r, s);
                }
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
    auto s = std::make_unique<SystemRes>();
    s->n = n_orb;
    int rc;
    if ((rc = dev_alloc(c, s->h, n2 * 8, "h")) || (rc = dev_alloc(c, s->eri, n4 * 8, "eri")) ||
        (rc = dev_alloc(c, s->J, n2 * 8, "J")) || (rc = dev_alloc(c, s->WS, n2 * 8, "WS")) ||
        (rc = dev_alloc(c, s->Jx, n2 * 8, "Jx")) || (rc = dev_alloc(c, s->WSx, n2 * 8, "WSx")) ||
        (rc = dev_alloc(c, s->hdx, n * 8, "hdx"))) {
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
    {
        std::vector<std::pair<uint64_t, uint64_t>> k(n_det);
        for (uint64_t i = 0; i < n_det; ++i) k[i] = {keys[2 * i], keys[2 * i + 1]};
        std::sort(k.begin(), k.end());
        for (uint64_t i = 1; i < n_det; ++i)
            if (k[i] == k[i - 1]) return fail(c, PT2_ERR_INVALID, "duplicate determinant in the reference");
    }
    cudaSetDevice(c->device);
    auto r = std::make_unique<RefRes>();
    r->system = system_id;
    r->n_det = n_det;
    r->na = na;
    r->nb = nb;
    r->e0 = e0;
    int rc;
    if ((rc = dev_alloc(c, r->keys, n_det * 16, "reference keys")) ||
        (rc = dev_alloc(c, r->coef, n_det * 8, "coefficients")) ||
        (rc = dev_alloc(c, r->hii, n_det * 8, "diagonals")) || (rc = dev_alloc(c, r->d0, n_det * 8, "denominators"))) {
        free_ref(c, *r);
        return rc;
    }
    CK(cudaMemcpyAsync(r->keys.ptr, keys, n_det * 16, cudaMemcpyHostToDevice, c->stream), "copy keys");
    CK(cudaMemcpyAsync(r->coef.ptr, coef, n_det * 8, cudaMemcpyHostToDevice, c->stream), "copy coef");
    CK(launch_diag(sys_dev(s), (const uint64_t *)r->keys.ptr, n_det, (double *)r->hii.ptr, c->stream),
       "diagonal kernel");
    CK(launch_ref_d0((const double *)r->hii.ptr, n_det, e0, (int64_t *)r->d0.ptr, c->stream), "denominator kernel");
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
    cudaStreamSynchronize(c->stream);
    auto ri = c->refs.find(id);
    if (ri != c->refs.end()) {
        RefRes &r = *ri->second;
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

int pt2_run(pt2_ctx *c, uint32_t ref_id, const pt2_opts *opts, pt2_result *out)
{
    if (!c) return PT2_ERR_INVALID;
    cudaSetDevice(c->device);
    return run_impl(c, ref_id, opts, out, nullptr);
}

int pt2_dump_external(pt2_ctx *c, uint32_t ref_id, const pt2_opts *opts, uint64_t *keys, double *num, double *haa,
                      uint64_t cap, uint64_t *n_out)
{
    if (!c) return PT2_ERR_INVALID;
    if ((cap && (!keys || !num || !haa)) || !n_out) return fail(c, PT2_ERR_INVALID, "bad arguments");
    cudaSetDevice(c->device);
    DumpTarget d;
    d.keys = keys;
    d.num = num;
    d.haa = haa;
    d.cap = cap;
    pt2_result res;
    int rc = run_impl(c, ref_id, opts, &res, &d);
    *n_out = d.n_out;
    return rc;
}

int pt2_det_terms(pt2_ctx *c, uint32_t ref_id, uint64_t det_index, uint64_t *keys, double *val, double *haa,
                  uint64_t cap, uint64_t *n_out)
{
    if (!c) return PT2_ERR_INVALID;
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
    p.cursor = (unsigned long long *)c->cursor.ptr;
    p.recs = (Rec32 *)c->recs.ptr;
    p.rec_cap = T;
    p.det_begin = det_index;
    gen_layout(p, kModeDetTerms);
    CK(cudaMemsetAsync(c->err_word.ptr, 0, 4, c->stream), "memset");
    CK(cudaMemsetAsync(c->cursor.ptr, 0, 8, c->stream), "memset");
    CK(launch_gen(kModeDetTerms, p, 1, c->stream), "generator");
    unsigned long long n = 0;
    CK(cudaMemcpyAsync(&n, c->cursor.ptr, 8, cudaMemcpyDeviceToHost, c->stream), "copy");
    CK(cudaStreamSynchronize(c->stream), "sync");
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
    CK(launch_det_terms_noalloc(c->device, p, cap, keys, val, haa, &n, c->stream), "allocation-free generation");
    *n_out = n;
    if (n > cap) return fail(c, PT2_ERR_OOM, "determinant has %llu terms, above cap %llu", n, (unsigned long long)cap);
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
