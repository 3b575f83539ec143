// Step engine of libpt2: planning (the work list of the section on
// parallelisation with work lists), packing of memory-bounded passes into
// steps, step execution, and on top of it single solves (pt2_run), batches
// captured as CUDA graphs (pt2_batch_*), the autotuner and the
// continuous-batching server (pt2_submit / pt2_poll / pt2_wait).
//
// A step runs one pass of each of a set of instances with one launch of
// every kernel: the instances' determinants and tiles are concatenated into
// one index space, and per-instance parameters and accumulators live in a
// device table of the step.  Steps issue no host synchronisation, so a
// batch's steps can be captured into a graph and replayed.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "pt2_runtime.h"

namespace pt2 {

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

constexpr uint64_t kDefaultTileTarget = 832;
constexpr uint32_t kTuneCandidates[] = {704, 768, 832, 896};

int size_class(uint64_t total)
{
    int k = 0;
    for (uint64_t t = total; t >= 10 && k < 7; t /= 10) ++k;
    return std::max(0, std::min(7, k - 5));  // <1e6, 1e6, 1e7, ..., >=1e11
}

// Records one step may hold: what the HBM budget leaves, and at most
// `passes` full-size passes (steps of batches and of the server hold two, so a
// full pass of a large solve and passes of smaller ones run side by side).
uint64_t records_budget(pt2_ctx *c, int passes = 1)
{
    // the step workspace a previous run left allocated is reused, so it counts as available
    const DevBuf *ws[] = {&c->tile_counts, &c->tile_off, &c->cursor, &c->scan_tmp, &c->ref_count,
                          &c->ref_off,     &c->ref_cursor, &c->big_list, &c->recs};
    uint64_t held = 0;
    for (const DevBuf *b : ws) held += b->bytes;
    const uint64_t fixed = c->used - held;
    const uint64_t scratch = (uint64_t)c->big_per_sm * c->sm_count * 2 * kBigScratch * sizeof(Rec48);
    const uint64_t reserve = scratch + (256ull << 20);
    const uint64_t avail = c->budget > fixed + reserve ? c->budget - fixed - reserve : 0;
    // per record: 32 bytes plus tile bookkeeping (about 60 bytes per tile of ~500 records)
    uint64_t rec = (uint64_t)((double)avail / (sizeof(Rec32) + 0.15));
    return std::min<uint64_t>(std::min<uint64_t>(rec, (uint64_t)passes * (kMaxPassBytes / sizeof(Rec32))),
                              kMaxStepRecords);
}

int init_job(pt2_ctx *c, Job &j, uint32_t ref_id, const pt2_opts *o)
{
    auto it = c->refs.find(ref_id);
    if (it == c->refs.end()) return fail(c, PT2_ERR_NOT_FOUND, "unknown reference id %u", ref_id);
    j.r = it->second.get();
    j.s = c->systems.at(j.r->system).get();
    j.ref_id = ref_id;
    memset(&j.o, 0, sizeof j.o);
    if (o) j.o = *o;
    if (j.o.constraint_mod > 1 && j.o.constraint_rem >= j.o.constraint_mod)
        return fail(c, PT2_ERR_INVALID, "constraint_rem must be below constraint_mod");
    if (j.o.tile_target > (uint32_t)kTileCap) return fail(c, PT2_ERR_INVALID, "tile_target above %d", kTileCap);
    if (j.o.class_slices > (uint32_t)kNumClasses || (j.o.class_slices > 1 && j.o.class_slice >= j.o.class_slices))
        return fail(c, PT2_ERR_INVALID, "class_slice must be below class_slices, and class_slices at most %d",
                    kNumClasses);
    if (j.o.reserved) return fail(c, PT2_ERR_INVALID, "pt2_opts.reserved must be 0");
    // alpha classes [cls_lo, cls_hi) of the slice
    if (j.o.class_slices > 1) {
        j.cls_lo = (uint32_t)((uint64_t)j.o.class_slice * kNumClasses / j.o.class_slices);
        j.cls_hi = (uint32_t)((uint64_t)(j.o.class_slice + 1) * kNumClasses / j.o.class_slices);
    } else {
        j.cls_lo = 0;
        j.cls_hi = kNumClasses;
    }
    j.gp = gen_params(c, *j.s, *j.r);
    j.gp.cons_mod = j.o.constraint_mod > 1 ? j.o.constraint_mod : 1;
    j.gp.cons_rem = j.o.constraint_mod > 1 ? j.o.constraint_rem : 0;
    // the highest occupied alpha orbitals of every summed excited determinant
    j.gp.top_mask = j.o.top_alpha;
    j.gp.top_hi = j.o.top_alpha ? ~((1ull << __builtin_ctzll(j.o.top_alpha)) - 1ull) : 0ull;
    if (j.o.flags & PT2_FLAG_SPIN_SYMMETRIC) {
        if (!j.r->flip_symmetric)
            return fail(c, PT2_ERR_INVALID,
                        "spin-flip symmetry needs a reference closed under alpha <-> beta exchange with equal coefficients");
        j.gp.sym = 1;
    }
    if (!(j.o.numerator_cutoff >= 0.0) || std::isinf(j.o.numerator_cutoff))
        return fail(c, PT2_ERR_INVALID, "numerator_cutoff must be finite and non-negative");
    j.gp.cutoff = j.o.numerator_cutoff;
    j.gp.subtract = (j.o.flags & PT2_FLAG_SUBTRACT_REF) ? 1u : 0u;
    return PT2_OK;
}

int ensure_pinned(pt2_ctx *c, size_t bytes)
{
    if (c->steps_pinned_bytes >= bytes) return PT2_OK;
    if (c->steps_pinned) cudaFreeHost(c->steps_pinned);
    c->steps_pinned = nullptr;
    c->steps_pinned_bytes = 0;
    cudaError_t e = cudaMallocHost(&c->steps_pinned, bytes);
    if (e != cudaSuccess) return cuda_fail(c, e, "pinned staging");
    c->steps_pinned_bytes = bytes;
    return PT2_OK;
}

// Launch the generator over n_ctas determinants of a batch (grid.x slices).
cudaError_t gen_launch(pt2_ctx *c, GenMode mode, GenBatch b, uint64_t n_ctas, int smem)
{
    const uint64_t slice = 1ull << 30;
    for (uint64_t o = 0; o < n_ctas; o += slice) {
        b.cta_offset = o;
        cudaError_t e = launch_gen(mode, b, std::min(slice, n_ctas - o), smem, c->stream);
        c->launches++;
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Duplicate subtraction of a job (none unless requested): after its
// accumulator is initialised, subtract its reference determinants' c_i^2 (E0 - H_ii).
cudaError_t job_subtract(pt2_ctx *c, const Job &j, RunAcc *acc, cudaStream_t st)
{
    if (!j.gp.subtract) return cudaSuccess;
    c->launches++;
    return launch_ref_subtract(reinterpret_cast<const uint64_t *>(j.r->keys.ptr),
                               reinterpret_cast<const double *>(j.r->coef.ptr),
                               reinterpret_cast<const double *>(j.r->hii.ptr), j.r->n_det, j.r->e0, j.gp.cons_mod,
                               j.gp.cons_rem, j.gp.top_hi, j.gp.top_mask,
                               reinterpret_cast<const HashTables *>(c->hash.ptr), j.cls_lo, j.cls_hi,
                               acc, reinterpret_cast<uint32_t *>(c->err_word.ptr), st);
}

// Whether a job generated the terms its plan counted: exactly, or for a run
// with a numerator cutoff at most the plan's count (its work list counts the
// kept terms, but the passes of a heavy alpha class are planned from bounds,
// so the check stays the bound those passes are held to).
bool terms_as_planned(const Job &j, uint64_t n_terms)
{
    return j.gp.cutoff > 0.0 ? n_terms <= j.total : n_terms == j.total;
}

// Checks a job's generator launches need (kFiltSym | kFiltCut).
int job_filt(const Job &j) { return (j.gp.sym ? kFiltSym : 0) | (j.gp.cutoff > 0.0 ? kFiltCut : 0); }

// Options of a job's instance in the tile kernels.
uint32_t job_iflags(const Job &j)
{
    return (j.gp.sym ? kInstSym : 0u) | ((j.o.debug_flags & PT2_DEBUG_NARROW_SORT_HASH) ? kInstNarrow : 0u) |
           ((j.o.debug_flags & PT2_DEBUG_SHORT_COPY_WAIT) ? kInstShortWait : 0u) |
           ((j.o.flags & PT2_FLAG_HASHED_KEYS) ? kInstHashed : 0u);
}

// Terms per beta class among the terms of alpha class k of a job (one
// beta-count launch over the job's determinants).
int beta_counts(pt2_ctx *c, const Job &j, uint32_t k, std::vector<unsigned long long> &out)
{
    GenParams g = j.gp;
    g.det_begin = 0;
    g.heavy_class = k;
    g.class_counts = reinterpret_cast<unsigned long long *>(c->class_counts.ptr);
    gen_layout(g, kModeBetaCount);
    cudaStream_t st = c->stream;
    CK(cudaMemsetAsync(c->class_counts.ptr, 0, kNumClasses * 8, st), "memset");
    GenBatch b{nullptr, nullptr, 1, 0, g, job_filt(j)};
    CK(gen_launch(c, kModeBetaCount, b, j.r->n_det, g.smem_bytes), "beta count kernel");
    out.assign(kNumClasses, 0);
    CK(cudaMemcpyAsync(out.data(), c->class_counts.ptr, kNumClasses * 8, cudaMemcpyDeviceToHost, st), "copy");
    CK(cudaStreamSynchronize(st), "sync");
    return PT2_OK;
}

// Work list: one class-count launch over all jobs (alpha-hash classes play
// the role of the paper's constraints), then each job's passes.  An alpha
// class with more terms than a pass holds (an alpha string shared by many
// reference determinants) is split further by the beta-hash classes of its
// terms, counted by a beta-count launch, as the paper splits a heavy
// constraint into finer ones.
int plan_jobs(pt2_ctx *c, const std::vector<Job *> &jobs, bool split_large, uint64_t step_cap)
{
    const size_t n = jobs.size();
    if (n == 0) return PT2_OK;
    if (n > (size_t)kMaxBatch) return fail(c, PT2_ERR_INVALID, "more than %d instances in one plan", kMaxBatch);
    int rc;
    if ((rc = ensure(c, c->class_counts, n * kNumClasses * 8, "class counts"))) return rc;
    const size_t tab = n * sizeof(GenParams) + (n + 1) * 8;
    if ((rc = ensure(c, c->gen_tab, tab, "generator table"))) return rc;
    if ((rc = ensure_pinned(c, std::max<size_t>(tab, sizeof(StepDev))))) return rc;
    GenParams *hp = reinterpret_cast<GenParams *>(c->steps_pinned);
    unsigned long long *hb = reinterpret_cast<unsigned long long *>(hp + n);
    uint64_t cta = 0;
    int smem = 0, filt = 0;
    for (size_t i = 0; i < n; ++i) {
        filt |= job_filt(*jobs[i]);
        GenParams g = jobs[i]->gp;
        g.class_lo = jobs[i]->cls_lo;  // the job's class slice only
        g.class_hi = jobs[i]->cls_hi;
        g.det_begin = 0;
        g.class_counts = reinterpret_cast<unsigned long long *>(c->class_counts.ptr) + i * kNumClasses;
        gen_layout(g, kModeClassCount);
        smem = std::max(smem, g.smem_bytes);
        hp[i] = g;
        hb[i] = cta;
        cta += jobs[i]->r->n_det;
    }
    hb[n] = cta;
    cudaStream_t st = c->stream;
    CK(cudaMemcpyAsync(c->gen_tab.ptr, c->steps_pinned, tab, cudaMemcpyHostToDevice, st), "copy");
    CK(cudaMemsetAsync(c->class_counts.ptr, 0, n * kNumClasses * 8, st), "memset");
    GenBatch b{reinterpret_cast<const GenParams *>(c->gen_tab.ptr),
               reinterpret_cast<const unsigned long long *>(static_cast<char *>(c->gen_tab.ptr) +
                                                            n * sizeof(GenParams)),
               (int)n, 0, hp[0], filt};
    CK(gen_launch(c, kModeClassCount, b, cta, smem), "class count kernel");
    std::vector<unsigned long long> cls(n * kNumClasses);
    CK(cudaMemcpyAsync(cls.data(), c->class_counts.ptr, n * kNumClasses * 8, cudaMemcpyDeviceToHost, st), "copy");
    CK(cudaStreamSynchronize(st), "sync");
    for (size_t i = 0; i < n; ++i) {
        Job &j = *jobs[i];
        const unsigned long long *cl = cls.data() + i * kNumClasses;
        j.total = 0;
        for (int k = (int)j.cls_lo; k < (int)j.cls_hi; ++k) j.total += cl[k];
        uint64_t tt = j.o.tile_target;
        if (!tt) tt = c->tuned_tile[size_class(j.total)];
        if (!tt) tt = kDefaultTileTarget;
        j.tile_target = tt;
        uint64_t cap = j.o.pass_budget_bytes ? (uint64_t)((double)j.o.pass_budget_bytes / (sizeof(Rec32) + 60.0 / tt))
                                             : step_cap;
        if (!j.o.pass_budget_bytes) {
            cap = std::min<uint64_t>(cap, kMaxTilesPerPass * tt);
            cap = std::min<uint64_t>(cap, std::max<uint64_t>(kLocalPassRecords, j.r->n_det * kTermsPerDetPass));
        }
        cap = std::min<uint64_t>(cap, (j.o.pass_budget_bytes ? kMaxPassBytesAsked : kMaxPassBytes) / sizeof(Rec32));
        if (split_large && !j.o.pass_budget_bytes) cap = std::min<uint64_t>(cap, std::max<uint64_t>(step_cap / 2, 1024));
        if (cap < 1024) return fail(c, PT2_ERR_OOM, "pass budget is too small (%llu records)", (unsigned long long)cap);
        j.pass_cap = cap;
        j.passes.clear();
        Pass cur;
        cur.c_lo = j.cls_lo;
        for (int k = (int)j.cls_lo; k < (int)j.cls_hi; ++k) {
            if (cl[k] > cap) {  // heavy alpha class: passes over its beta classes
                if (cur.records > 0) {
                    cur.c_hi = k;
                    j.passes.push_back(cur);
                }
                std::vector<unsigned long long> bh;
                if ((rc = beta_counts(c, j, (uint32_t)k, bh))) return rc;
                // the beta counts are of every term: in a run with a numerator
                // cutoff they bound what the beta-class passes keep
                const bool cutting = j.gp.cutoff > 0.0;
                unsigned long long sum = 0;
                Pass bp;
                bp.c_lo = k;
                bp.c_hi = k + 1;
                bp.b_lo = 0;
                bp.at_most = cutting;
                for (int b = 0; b < kNumClasses; ++b) {
                    sum += bh[b];
                    if (bh[b] > cap)
                        return fail(c, PT2_ERR_OOM,
                                    "alpha class %d, beta class %d holds %llu terms, above the %llu a pass can "
                                    "hold; raise the budget",
                                    k, b, (unsigned long long)bh[b], (unsigned long long)cap);
                    if (bp.records + bh[b] > cap) {
                        bp.b_hi = b;
                        j.passes.push_back(bp);
                        bp.b_lo = b;
                        bp.records = 0;
                        bp.at_most = cutting;
                    }
                    bp.records += bh[b];
                }
                bp.b_hi = kNumClasses;
                if (bp.records > 0) j.passes.push_back(bp);
                if (cutting ? sum < cl[k] : sum != cl[k])
                    return fail(c, PT2_ERR_CUDA, "beta counts of alpha class %d sum to %llu, not %llu", k, sum,
                                (unsigned long long)cl[k]);
                cur = Pass();
                cur.c_lo = k + 1;
                continue;
            }
            if (cur.records + cl[k] > cap) {
                cur.c_hi = k;
                j.passes.push_back(cur);
                cur = Pass();
                cur.c_lo = k;
            }
            cur.records += cl[k];
        }
        cur.c_hi = j.cls_hi;
        if (cur.records > 0 || j.passes.empty()) j.passes.push_back(cur);
        for (auto &p : j.passes) p.n_tiles = std::max<uint64_t>(1, (p.records + tt - 1) / tt);
        j.next = 0;
    }
    return PT2_OK;
}

// Greedy packing: a step takes the next pass of every job that still fits.
std::vector<StepPlan> pack_steps(const std::vector<Job *> &jobs, uint64_t step_cap)
{
    std::vector<size_t> next(jobs.size(), 0);
    std::vector<StepPlan> steps;
    for (;;) {
        StepPlan sp;
        for (size_t i = 0; i < jobs.size(); ++i) {
            if (next[i] >= jobs[i]->passes.size()) continue;
            if ((int)sp.items.size() >= kMaxBatch) break;
            const Pass &P = jobs[i]->passes[next[i]];
            if (!sp.items.empty() && sp.records + P.records > step_cap) continue;
            sp.items.push_back({jobs[i], next[i]});
            sp.records += P.records;
            sp.n_tiles += P.n_tiles;
            sp.n_ctas += jobs[i]->r->n_det;
            ++next[i];
        }
        if (sp.items.empty()) break;
        steps.push_back(sp);
    }
    return steps;
}

int ensure_step_workspace(pt2_ctx *c, const std::vector<StepPlan> &steps)
{
    uint64_t tiles = 1, recs = 1, refs = 1;
    for (const auto &sp : steps) {
        tiles = std::max(tiles, sp.n_tiles);
        recs = std::max(recs, sp.records);
        refs = std::max(refs, sp.n_ctas);
    }
    if (tiles >= 0xFFFFFFFFull) return fail(c, PT2_ERR_INVALID, "too many tiles in one step");
    int rc;
    if ((rc = ensure(c, c->tile_counts, tiles * 4, "tile counts"))) return rc;
    if ((rc = ensure(c, c->tile_off, (tiles + 1) * 8, "tile offsets"))) return rc;
    if ((rc = ensure(c, c->cursor, tiles * 4, "tile cursors"))) return rc;
    if ((rc = ensure(c, c->scan_tmp, scan_tmp_elems(tiles) * 8 * 2, "scan scratch"))) return rc;
    if ((rc = ensure(c, c->ref_count, tiles * 4, "reference counts"))) return rc;
    if ((rc = ensure(c, c->ref_off, (tiles + 1) * 8, "reference offsets"))) return rc;
    if ((rc = ensure(c, c->ref_cursor, tiles * 8, "reference cursors"))) return rc;
    if ((rc = ensure(c, c->big_list, tiles * 4, "oversize list"))) return rc;
    if ((rc = ensure(c, c->ref_tile, refs * 4, "reference tiles"))) return rc;
    if ((rc = ensure(c, c->ref_keys, refs * 16, "reference slices"))) return rc;
    if ((rc = ensure(c, c->big_max, 16, "oversize maximum"))) return rc;
    const uint64_t scratch = (uint64_t)c->big_per_sm * c->sm_count * 2 * kBigScratch * sizeof(Rec48);
    if ((rc = ensure(c, c->scratch, scratch, "oversize scratch"))) return rc;
    if ((rc = ensure(c, c->recs, recs * sizeof(Rec32), "term records"))) return rc;
    return PT2_OK;
}

int step_smem(const StepPlan &sp)
{
    int m = 0;
    for (const auto &it : sp.items) {
        GenParams g = it.job->gp;
        gen_layout(g, kModeEmit);
        m = std::max(m, g.smem_bytes);
    }
    return m;
}

// Generator parameters of item i of a step whose tiles start at tile_base.
GenParams step_item_params(pt2_ctx *c, const StepPlan &sp, size_t i, uint64_t tile_base)
{
    const Job &j = *sp.items[i].job;
    const Pass &P = j.passes[sp.items[i].pass];
    GenParams g = j.gp;
    g.class_lo = P.c_lo;
    g.class_hi = P.c_hi;
    g.bclass_lo = P.b_lo;
    g.bclass_hi = P.b_hi;
    g.n_tiles = P.n_tiles;
    g.tile_base = tile_base;
    g.det_begin = 0;
    g.class_counts = nullptr;
    g.tile_counts = reinterpret_cast<uint32_t *>(c->tile_counts.ptr);
    g.cursor = reinterpret_cast<unsigned int *>(c->cursor.ptr);
    g.recs = reinterpret_cast<Rec32 *>(c->recs.ptr);
    g.rec_cap = sp.records;
    gen_layout(g, kModeEmit);
    return g;
}

void fill_step(pt2_ctx *c, const StepPlan &sp, StepDev &h)
{
    uint64_t cta = 0, tb = 0;
    const size_t n = sp.items.size();
    for (size_t i = 0; i < n; ++i) {
        Job &j = *sp.items[i].job;
        const Pass &P = j.passes[sp.items[i].pass];
        h.params[i] = step_item_params(c, sp, i, tb);
        h.det_base[i] = cta;
        h.tile_base[i] = tb;
        h.e0[i] = j.r->e0;
        h.iflags[i] = job_iflags(j);
        h.expected[i] = P.records | (P.at_most ? kExpectAtMost : 0ull);
        h.acc[i] = j.acc;
        h.n_big[i] = 0;
        cta += j.r->n_det;
        tb += P.n_tiles;
    }
    h.det_base[n] = cta;
    h.tile_base[n] = tb;
}

struct DumpTarget {
    uint64_t *keys = nullptr;
    double *num = nullptr, *haa = nullptr;
    uint64_t cap = 0;
    uint64_t n_out = 0;
};

// Enqueue one step on the context stream (no host synchronisation unless
// profiling).  d is the step's device table.  pre: the step's tile counts,
// already counted by a grouped count (null: the step counts them itself).
int enqueue_step(pt2_ctx *c, const StepPlan &sp, StepDev *d, const DumpTarget *dump, bool prof,
                 const uint32_t *pre = nullptr)
{
    cudaStream_t st = c->stream;
    const int n = (int)sp.items.size();
    cudaEvent_t *E = &c->ev[2];
    if (prof) CK(cudaEventRecord(E[0], st), "event");
    GenBatch gb{d->params, d->det_base, n, 0, {}, 0};
    for (const StepItem &it : sp.items) gb.filt |= job_filt(*it.job);
    if (n == 1) gb.one = step_item_params(c, sp, 0, 0);
    const int smem = step_smem(sp);
    if (!pre) {
        CK(cudaMemsetAsync(c->tile_counts.ptr, 0, sp.n_tiles * 4, st), "memset");
        CK(gen_launch(c, kModeTileCount, gb, sp.n_ctas, smem), "tile count kernel");
    }
    if (prof) CK(cudaEventRecord(E[1], st), "event");
    unsigned long long *tile_off = reinterpret_cast<unsigned long long *>(c->tile_off.ptr);
    unsigned long long *tmp = reinterpret_cast<unsigned long long *>(c->scan_tmp.ptr);
    // tile offsets, and the same offsets as the 32-bit slot cursors of the emission
    CK(launch_scan_u32_to_u64(pre ? pre : reinterpret_cast<const uint32_t *>(c->tile_counts.ptr), tile_off,
                              reinterpret_cast<uint32_t *>(c->cursor.ptr), sp.n_tiles, tmp, st),
       "scan");
    c->launches += 3;
    if (prof) CK(cudaEventRecord(E[2], st), "event");
    CK(gen_launch(c, kModeEmit, gb, sp.n_ctas, smem), "emit kernel");
    if (prof) CK(cudaEventRecord(E[3], st), "event");
    RefPartParams rp;
    rp.params = d->params;
    rp.ref_base = d->det_base;
    rp.n_inst = n;
    rp.n_total = sp.n_ctas;
    rp.hash = reinterpret_cast<const HashTables *>(c->hash.ptr);
    rp.ref_tile = reinterpret_cast<uint32_t *>(c->ref_tile.ptr);
    rp.ref_count = reinterpret_cast<uint32_t *>(c->ref_count.ptr);
    rp.ref_cursor = reinterpret_cast<unsigned long long *>(c->ref_cursor.ptr);
    rp.ref_keys_out = reinterpret_cast<uint64_t *>(c->ref_keys.ptr);
    CK(cudaMemsetAsync(rp.ref_count, 0, sp.n_tiles * 4, st), "memset");
    CK(launch_ref_partition(rp, 0, st), "reference tiles");
    CK(launch_scan_u32_to_u64(rp.ref_count, reinterpret_cast<unsigned long long *>(c->ref_off.ptr), nullptr, sp.n_tiles,
                              tmp + scan_tmp_elems(c->tile_counts.bytes / 4), st),
       "scan");
    CK(cudaMemcpyAsync(rp.ref_cursor, c->ref_off.ptr, sp.n_tiles * 8, cudaMemcpyDeviceToDevice, st), "copy");
    CK(launch_ref_partition(rp, 1, st), "reference scatter");
    CK(launch_sort_slices(reinterpret_cast<const unsigned long long *>(c->ref_off.ptr),
                          reinterpret_cast<uint64_t *>(c->ref_keys.ptr), sp.n_tiles, st),
       "reference sort");
    c->launches += 6;
    if (prof) CK(cudaEventRecord(E[4], st), "event");
    TileParams tp;
    memset(&tp, 0, sizeof tp);
    tp.recs = reinterpret_cast<const Rec32 *>(c->recs.ptr);
    tp.tile_off = tile_off;
    tp.ref_off = reinterpret_cast<const unsigned long long *>(c->ref_off.ptr);
    tp.ref_keys = reinterpret_cast<const uint64_t *>(c->ref_keys.ptr);
    tp.n_tiles = sp.n_tiles;
    tp.tile_base = d->tile_base;
    tp.e0 = d->e0;
    tp.iflags = d->iflags;
    tp.sym_any = (gb.filt & kFiltSym) != 0;
    tp.acc = d->acc;
    tp.n_big = d->n_big;
    tp.big_max = reinterpret_cast<unsigned long long *>(c->big_max.ptr);
    tp.n_inst = n;
    tp.big_list = reinterpret_cast<uint32_t *>(c->big_list.ptr);
    tp.err = reinterpret_cast<uint32_t *>(c->err_word.ptr);
    tp.scratch = reinterpret_cast<Rec48 *>(c->scratch.ptr);
    tp.scratch_cap = kBigScratch;
    if (dump) {
        tp.dump_keys = reinterpret_cast<uint64_t *>(c->dump_keys.ptr);
        tp.dump_num = reinterpret_cast<double *>(c->dump_num.ptr);
        tp.dump_haa = reinterpret_cast<double *>(c->dump_haa.ptr);
        tp.dump_count = reinterpret_cast<unsigned long long *>(c->dump_count.ptr);
        tp.dump_cap = dump->cap;
    }
    CK(launch_tiles(tp, c->tile_per_sm * c->sm_count, st), "tile kernel");
    if (prof) CK(cudaEventRecord(E[5], st), "event");
    CK(launch_big_tiles(tp, c->big_per_sm * c->sm_count, st), "oversize tile kernel");
    if (prof) CK(cudaEventRecord(E[6], st), "event");
    CK(launch_pass_finish(tile_off, d->tile_base, n, d->expected, d->acc, d->n_big, tp.err, st), "pass finish");
    c->launches += 3;
    if (prof) {
        CK(cudaEventRecord(E[7], st), "event");
        CK(cudaEventSynchronize(E[7]), "sync");
        float ms;
        for (int k = 0; k < 7; ++k) {
            cudaEventElapsedTime(&ms, E[k], E[k + 1]);
            c->phase_ms[k + 1] += ms;
        }
    }
    return PT2_OK;
}

void result_of(const RunAcc &h, const Job &j, pt2_result *out)
{
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
    out->n_passes = (uint32_t)j.passes.size();
    uint64_t tiles = 0;
    for (const auto &p : j.passes) tiles += p.n_tiles;
    out->n_tiles = (uint32_t)std::min<uint64_t>(tiles, 0xFFFFFFFFull);
    out->n_oversize = h.n_big;
    out->n_hash_collisions = (uint32_t)std::min<unsigned long long>(h.n_coll, 0xFFFFFFFFull);
}

// Upload the device tables of a list of steps (one pinned staging copy).
// Consecutive passes of one run over whole alpha classes (every beta class)
// counted by one tile-count launch: each determinant's set-up (its singles,
// their classes, the bucket table) is then done once per group instead of
// once per pass.  A group's counts are kept until its passes have run.
constexpr uint64_t kGrpMaxTiles = 1ull << 28;  // 1 GiB of counts
struct CountGroup {
    size_t k0 = 0, n = 0;  // steps k0 .. k0 + n - 1, one pass each
    uint64_t tiles = 0;
    uint32_t tab[kGrpStride] = {};  // pass table, then the pass of each class (bytes)
};

std::vector<CountGroup> count_groups(const Job &j, const std::vector<StepPlan> &steps)
{
    std::vector<CountGroup> out;
    if (j.gp.top_mask) return out;  // triplet runs list their alpha-alpha doubles by Algorithm 3
    auto plain = [&](size_t k) {
        if (steps[k].items.size() != 1 || steps[k].items[0].job != &j) return false;
        const Pass &P = j.passes[steps[k].items[0].pass];
        return P.b_lo == 0 && P.b_hi >= (uint32_t)kNumClasses;
    };
    size_t k = 0;
    while (k < steps.size()) {
        if (!plain(k)) {
            ++k;
            continue;
        }
        CountGroup g;
        g.k0 = k;
        uint32_t hi = 0;
        while (k < steps.size() && plain(k) && g.n < (size_t)kMaxGrp) {
            const Pass &P = j.passes[steps[k].items[0].pass];
            if (g.n > 0 && (P.c_lo != hi || g.tiles + P.n_tiles > kGrpMaxTiles)) break;
            g.tab[g.n] = P.c_lo;
            g.tab[kMaxGrp + 1 + g.n] = (uint32_t)g.tiles;
            g.tab[2 * kMaxGrp + 1 + g.n] = (uint32_t)P.n_tiles;
            g.tiles += P.n_tiles;
            hi = P.c_hi;
            ++g.n;
            ++k;
        }
        g.tab[g.n] = hi;
        uint8_t *cls = reinterpret_cast<uint8_t *>(g.tab + kGrpClsOff);
        for (size_t q = 0; q < g.n; ++q)
            for (uint32_t c = g.tab[q]; c < g.tab[q + 1]; ++c) cls[c] = (uint8_t)q;
        if (g.n >= 2) out.push_back(g);
    }
    return out;
}

// One tile-count launch over the passes of group g (its table at dtab).
int enqueue_group_count(pt2_ctx *c, const Job &j, const CountGroup &g, const uint32_t *dtab, bool prof)
{
    cudaStream_t st = c->stream;
    cudaEvent_t *E = &c->ev[2];
    if (prof) CK(cudaEventRecord(E[0], st), "event");
    GenParams p = j.gp;
    p.class_lo = g.tab[0];
    p.class_hi = g.tab[g.n];
    p.bclass_lo = 0;
    p.bclass_hi = kNumClasses;
    p.n_tiles = g.tiles;
    p.tile_base = 0;
    p.det_begin = 0;
    p.class_counts = nullptr;
    p.tile_counts = reinterpret_cast<uint32_t *>(c->grp_counts.ptr);
    p.n_grp = (uint32_t)g.n;
    p.grp = dtab;
    gen_layout(p, kModeTileCount);
    CK(cudaMemsetAsync(c->grp_counts.ptr, 0, g.tiles * 4, st), "memset");
    GenBatch gb{nullptr, nullptr, 1, 0, p, job_filt(j)};
    CK(gen_launch(c, kModeTileCount, gb, j.r->n_det, p.smem_bytes), "grouped tile count kernel");
    if (prof) {
        CK(cudaEventRecord(E[1], st), "event");
        CK(cudaEventSynchronize(E[1]), "sync");
        float ms;
        cudaEventElapsedTime(&ms, E[0], E[1]);
        c->phase_ms[1] += ms;
    }
    return PT2_OK;
}

int upload_steps(pt2_ctx *c, const std::vector<StepPlan> &steps, DevBuf &dst)
{
    const size_t bytes = steps.size() * sizeof(StepDev);
    int rc;
    if ((rc = ensure(c, dst, std::max<size_t>(bytes, sizeof(StepDev)), "step tables"))) return rc;
    if ((rc = ensure_pinned(c, bytes))) return rc;
    StepDev *h = reinterpret_cast<StepDev *>(c->steps_pinned);
    for (size_t i = 0; i < steps.size(); ++i) fill_step(c, steps[i], h[i]);
    CK(cudaMemcpyAsync(dst.ptr, c->steps_pinned, bytes, cudaMemcpyHostToDevice, c->stream), "copy");
    CK(cudaStreamSynchronize(c->stream), "sync");  // the staging buffer is reused
    return PT2_OK;
}

int run_single(pt2_ctx *c, uint32_t ref_id, const pt2_opts *opts, pt2_result *out, DumpTarget *dump)
{
    if (!out) return fail(c, PT2_ERR_INVALID, "result pointer is NULL");
    std::lock_guard<std::recursive_mutex> lock(c->exec);
    cudaSetDevice(c->device);
    Job j;
    int rc;
    if ((rc = init_job(c, j, ref_id, opts))) return rc;
    const bool prof = (j.o.flags & PT2_FLAG_PROFILE) != 0;
    c->launches = 0;
    for (double &x : c->phase_ms) x = 0.0;
    if ((rc = ensure(c, c->acc, sizeof(RunAcc), "accumulator"))) return rc;
    j.acc = reinterpret_cast<RunAcc *>(c->acc.ptr);
    cudaStream_t st = c->stream;
    if (dump) {
        if ((rc = ensure(c, c->dump_count, 16, "dump count"))) return rc;
        if ((rc = ensure(c, c->dump_keys, std::max<uint64_t>(dump->cap, 1) * 16, "dump keys"))) return rc;
        if ((rc = ensure(c, c->dump_num, std::max<uint64_t>(dump->cap, 1) * 8, "dump num"))) return rc;
        if ((rc = ensure(c, c->dump_haa, std::max<uint64_t>(dump->cap, 1) * 8, "dump haa"))) return rc;
        CK(cudaMemsetAsync(c->dump_count.ptr, 0, 8, st), "memset");
    }
    CK(cudaEventRecord(c->ev[0], st), "event");
    std::vector<Job *> jobs{&j};
    if ((rc = plan_jobs(c, jobs, false, records_budget(c)))) return rc;
    CK(cudaEventRecord(c->ev[1], st), "event");
    if (prof) {
        CK(cudaEventSynchronize(c->ev[1]), "sync");
        float ms = 0;
        cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
        c->phase_ms[0] += ms;
    }
    std::vector<StepPlan> steps = pack_steps(jobs, ~0ull);
    if ((rc = ensure_step_workspace(c, steps))) return rc;
    if ((rc = upload_steps(c, steps, c->steps))) return rc;
    CK(cudaMemsetAsync(c->err_word.ptr, 0, 4, st), "memset");
    CK(launch_acc_init(j.acc, 1, st), "acc init");
    CK(job_subtract(c, j, j.acc, st), "duplicate subtraction");
    // passes whose tiles are counted in groups
    const std::vector<CountGroup> groups = count_groups(j, steps);
    if (!groups.empty()) {
        uint64_t mt = 0;
        std::vector<uint32_t> tabs;
        for (const CountGroup &g : groups) {
            mt = std::max(mt, g.tiles);
            tabs.insert(tabs.end(), g.tab, g.tab + kGrpStride);
        }
        if ((rc = ensure(c, c->grp_counts, mt * 4, "grouped tile counts"))) return rc;
        if ((rc = ensure(c, c->grp_tab, tabs.size() * 4, "pass tables"))) return rc;
        CK(cudaMemcpyAsync(c->grp_tab.ptr, tabs.data(), tabs.size() * 4, cudaMemcpyHostToDevice, st), "copy");
    }
    StepDev *d = reinterpret_cast<StepDev *>(c->steps.ptr);
    size_t gi = 0;
    for (size_t k = 0; k < steps.size(); ++k) {
        while (gi < groups.size() && k >= groups[gi].k0 + groups[gi].n) ++gi;
        const uint32_t *pre = nullptr;
        if (gi < groups.size() && k >= groups[gi].k0) {
            const CountGroup &g = groups[gi];
            if (k == g.k0 &&
                (rc = enqueue_group_count(c, j, g, reinterpret_cast<const uint32_t *>(c->grp_tab.ptr) + gi * kGrpStride,
                                          prof)))
                return rc;
            pre = reinterpret_cast<const uint32_t *>(c->grp_counts.ptr) + g.tab[kMaxGrp + 1 + (k - g.k0)];
        }
        if ((rc = enqueue_step(c, steps[k], d + k, dump, prof, pre))) return rc;
    }
    CK(launch_acc_finalize(j.acc, 1, st), "finalize");
    c->launches += 2;
    RunAcc h;
    uint32_t err = 0;
    CK(cudaMemcpyAsync(&h, j.acc, sizeof h, cudaMemcpyDeviceToHost, st), "copy");
    CK(cudaMemcpyAsync(&err, c->err_word.ptr, 4, cudaMemcpyDeviceToHost, st), "copy");
    CK(cudaEventRecord(c->ev[1], st), "event");
    CK(cudaStreamSynchronize(st), "sync");
    float ms = 0;
    cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
    if ((rc = status_of_err(c, err | h.err))) return rc;
    result_of(h, j, out);
    out->seconds = ms * 1e-3;
    if (!terms_as_planned(j, h.n_terms))
        return fail(c, PT2_ERR_CUDA, "generated %llu terms, planned %llu", (unsigned long long)h.n_terms,
                    (unsigned long long)j.total);
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

// ------------------------------------------------------------------ batches

struct Batch {
    std::vector<std::unique_ptr<Job>> jobs;
    std::vector<StepPlan> steps;
    DevBuf acc, tables;
    cudaGraphExec_t exec = nullptr;
    uint64_t ws_gen = 0;  // workspace generation the graph was captured with
    double capture_s = 0;
    bool profile = false;  // run the steps one by one with per-phase events instead of the graph
};

namespace {

int capture_batch(pt2_ctx *c, Batch &b)
{
    int rc;
    if ((rc = ensure_step_workspace(c, b.steps))) return rc;
    if ((rc = upload_steps(c, b.steps, b.tables))) return rc;
    if (b.exec) {
        cudaGraphExecDestroy(b.exec);
        b.exec = nullptr;
    }
    cudaStream_t st = c->stream;
    const double t0 = now_s();
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
    int n = (int)b.jobs.size();
    cudaError_t e = cudaMemsetAsync(c->err_word.ptr, 0, 4, st);
    if (e == cudaSuccess) e = launch_acc_init(reinterpret_cast<RunAcc *>(b.acc.ptr), n, st);
    for (int i = 0; e == cudaSuccess && i < n; ++i)
        e = job_subtract(c, *b.jobs[i], reinterpret_cast<RunAcc *>(b.acc.ptr) + i, st);
    StepDev *d = reinterpret_cast<StepDev *>(b.tables.ptr);
    for (size_t k = 0; e == cudaSuccess && k < b.steps.size(); ++k)
        if (enqueue_step(c, b.steps[k], d + k, nullptr, false) != PT2_OK) e = cudaErrorUnknown;
    if (e == cudaSuccess) e = launch_acc_finalize(reinterpret_cast<RunAcc *>(b.acc.ptr), n, st);
    cudaError_t e2 = cudaStreamEndCapture(st, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(c, PT2_ERR_CUDA, "capturing the batch failed: %s",
                    cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&b.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph instantiate");
    b.ws_gen = c->ws_gen;
    b.capture_s = now_s() - t0;
    return PT2_OK;
}

}  // namespace

void batches_release(pt2_ctx *c)
{
    for (auto &kv : c->batches) {
        Batch &b = *kv.second;
        if (b.exec) cudaGraphExecDestroy(b.exec);
        dev_free(c, b.acc);
        dev_free(c, b.tables);
    }
    c->batches.clear();
}

// ------------------------------------------------------------------ server

struct Server {
    std::thread th;
    std::mutex mu;
    std::condition_variable cv, done;
    bool stop = false;
    std::deque<Job *> pending;
    std::vector<Job *> active;
    std::map<uint64_t, std::unique_ptr<Job>> jobs;
    uint64_t next_ticket = 1;
    DevBuf acc_pool;
    std::vector<int> free_slots;
    uint64_t steps_run = 0;
    uint64_t inflight_bytes = 0;  // pass footprint of the admitted solves
};

namespace {

// A served request of reference ref_id is finished (done or failed).
void served_done(pt2_ctx *c, uint32_t ref_id)
{
    std::lock_guard<std::mutex> sl(c->served_mu);
    auto it = c->served.find(ref_id);
    if (it != c->served.end() && --it->second <= 0) c->served.erase(it);
}

void server_fail_jobs(pt2_ctx *c, std::vector<Job *> &js, int rc)
{
    Server &S = *c->server;
    for (Job *j : js) {
        j->status = rc;
        j->t_done = now_s();
        j->r->busy--;
        served_done(c, j->ref_id);
        S.inflight_bytes -= std::min(S.inflight_bytes, j->footprint);
        if (j->acc) S.free_slots.push_back((int)(j->acc - reinterpret_cast<RunAcc *>(S.acc_pool.ptr)));
    }
}

// One iteration of the serving loop: admit, run one step, retire.
void server_iteration(pt2_ctx *c)
{
    Server &S = *c->server;
    std::vector<Job *> admit;
    // Admission by HBM footprint: a solve's passes hold at most its terms or
    // one pass budget of 32-byte records; solves are admitted in arrival order
    // while the admitted footprint fits two steps of the context's record
    // budget (what stays free of the HBM budget after systems, references
    // and fixed workspace), and while slots are left.
    const uint64_t cap_now = [&] {
        std::lock_guard<std::recursive_mutex> lock(c->exec);
        return records_budget(c, 2);
    }();
    {
        std::lock_guard<std::mutex> lk(S.mu);
        while (!S.pending.empty() && S.active.size() + admit.size() < (size_t)kMaxBatch && !S.free_slots.empty()) {
            Job *j = S.pending.front();
            const uint64_t terms = terms_per_det(j->s->n, j->r->na, j->r->nb) * j->r->n_det;
            const uint64_t foot = std::min<uint64_t>(terms, std::max<uint64_t>(cap_now / 2, 1)) * sizeof(Rec32);
            const bool empty = S.active.empty() && admit.empty();
            if (!empty && S.inflight_bytes + foot > 2 * cap_now * sizeof(Rec32)) break;  // wait for room
            j->footprint = foot;
            S.inflight_bytes += foot;
            S.pending.pop_front();
            j->acc = reinterpret_cast<RunAcc *>(S.acc_pool.ptr) + S.free_slots.back();
            S.free_slots.pop_back();
            admit.push_back(j);
        }
    }
    std::lock_guard<std::recursive_mutex> lock(c->exec);
    cudaSetDevice(c->device);
    const uint64_t cap = records_budget(c, 2);
    if (!admit.empty()) {
        int rc = plan_jobs(c, admit, true, cap);
        for (Job *j : admit) j->t_admit = now_s();
        if (rc == PT2_OK)
            for (Job *j : admit)
                if (launch_acc_init(j->acc, 1, c->stream) != cudaSuccess ||
                    job_subtract(c, *j, j->acc, c->stream) != cudaSuccess)
                    rc = PT2_ERR_CUDA;
        std::lock_guard<std::mutex> lk(S.mu);
        if (rc != PT2_OK) {
            server_fail_jobs(c, admit, rc);
            S.done.notify_all();
        } else {
            for (Job *j : admit) S.active.push_back(j);
        }
    }
    // one step: the next pass of every active job that fits the step budget
    StepPlan sp;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        for (Job *j : S.active) {
            const Pass &P = j->passes[j->next];
            if (!sp.items.empty() && sp.records + P.records > cap) continue;
            sp.items.push_back({j, j->next});
            sp.records += P.records;
            sp.n_tiles += P.n_tiles;
            sp.n_ctas += j->r->n_det;
        }
    }
    if (sp.items.empty()) return;
    std::vector<StepPlan> one{sp};
    int rc = ensure_step_workspace(c, one);
    if (rc == PT2_OK) rc = upload_steps(c, one, c->steps);
    if (rc == PT2_OK) {
        if (cudaMemsetAsync(c->err_word.ptr, 0, 4, c->stream) != cudaSuccess) rc = PT2_ERR_CUDA;
    }
    if (rc == PT2_OK) rc = enqueue_step(c, sp, reinterpret_cast<StepDev *>(c->steps.ptr), nullptr, false);
    std::vector<Job *> finished;
    for (auto &it : sp.items) {
        it.job->next++;
        if (it.job->next == it.job->passes.size()) finished.push_back(it.job);
    }
    uint32_t err = 0;
    std::vector<RunAcc> h(finished.size());
    if (rc == PT2_OK) {
        for (size_t i = 0; i < finished.size(); ++i) {
            launch_acc_finalize(finished[i]->acc, 1, c->stream);
            cudaMemcpyAsync(&h[i], finished[i]->acc, sizeof(RunAcc), cudaMemcpyDeviceToHost, c->stream);
        }
        cudaMemcpyAsync(&err, c->err_word.ptr, 4, cudaMemcpyDeviceToHost, c->stream);
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) rc = PT2_ERR_CUDA;
    }
    if (rc == PT2_OK && err) rc = status_of_err(c, err);
    std::lock_guard<std::mutex> lk(S.mu);
    S.steps_run++;
    if (rc != PT2_OK) {  // the whole step failed: fail its jobs
        std::vector<Job *> js;
        for (auto &it : sp.items) js.push_back(it.job);
        server_fail_jobs(c, js, rc);
        S.active.erase(std::remove_if(S.active.begin(), S.active.end(),
                                      [&](Job *j) { return std::find(js.begin(), js.end(), j) != js.end(); }),
                       S.active.end());
        S.done.notify_all();
        return;
    }
    const double t = now_s();
    for (size_t i = 0; i < finished.size(); ++i) {
        Job *j = finished[i];
        result_of(h[i], *j, &j->result);
        j->t_done = t;
        j->result.seconds = t - j->t_submit;
        j->status = terms_as_planned(*j, h[i].n_terms) ? PT2_OK : PT2_ERR_CUDA;
        j->r->busy--;
        served_done(c, j->ref_id);
        S.inflight_bytes -= std::min(S.inflight_bytes, j->footprint);
        S.free_slots.push_back((int)(j->acc - reinterpret_cast<RunAcc *>(S.acc_pool.ptr)));
        S.active.erase(std::find(S.active.begin(), S.active.end(), j));
    }
    if (!finished.empty()) S.done.notify_all();
}

void server_loop(pt2_ctx *c)
{
    Server &S = *c->server;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(S.mu);
            S.cv.wait(lk, [&] { return S.stop || !S.pending.empty() || !S.active.empty(); });
            if (S.stop && S.pending.empty() && S.active.empty()) return;
        }
        server_iteration(c);
    }
}

int server_start(pt2_ctx *c)
{
    if (c->server) return PT2_OK;
    auto S = std::make_unique<Server>();
    int rc;
    if ((rc = dev_alloc(c, S->acc_pool, kMaxBatch * sizeof(RunAcc), "serving accumulators"))) return rc;
    for (int i = kMaxBatch - 1; i >= 0; --i) S->free_slots.push_back(i);
    c->server = std::move(S);
    c->server->th = std::thread(server_loop, c);
    return PT2_OK;
}

}  // namespace

void server_stop(pt2_ctx *c)
{
    if (!c->server) return;
    {
        std::lock_guard<std::mutex> lk(c->server->mu);
        c->server->stop = true;
    }
    c->server->cv.notify_all();
    if (c->server->th.joinable()) c->server->th.join();
    dev_free(c, c->server->acc_pool);
    c->server.reset();
}

}  // namespace pt2

pt2_ctx::pt2_ctx() = default;
pt2_ctx::~pt2_ctx() = default;

using namespace pt2;

// ===================================================================== ABI

extern "C" {

int pt2_run(pt2_ctx *c, uint32_t ref_id, const pt2_opts *opts, pt2_result *out)
{
    if (!c) return PT2_ERR_INVALID;
    return run_single(c, ref_id, opts, out, nullptr);
}

int pt2_dump_external(pt2_ctx *c, uint32_t ref_id, const pt2_opts *opts, uint64_t *keys, double *num, double *haa,
                      uint64_t cap, uint64_t *n_out)
{
    if (!c) return PT2_ERR_INVALID;
    if ((cap && (!keys || !num || !haa)) || !n_out) return fail(c, PT2_ERR_INVALID, "bad arguments");
    DumpTarget d;
    d.keys = keys;
    d.num = num;
    d.haa = haa;
    d.cap = cap;
    pt2_result res;
    int rc = run_single(c, ref_id, opts, &res, &d);
    *n_out = d.n_out;
    return rc;
}

int pt2_batch_create(pt2_ctx *c, uint32_t n, const uint32_t *ref_ids, const pt2_opts *opts, uint32_t *batch_id)
{
    if (!c) return PT2_ERR_INVALID;
    if (n == 0 || !ref_ids || !batch_id) return fail(c, PT2_ERR_INVALID, "bad arguments");
    if (n > (uint32_t)kMaxBatch) return fail(c, PT2_ERR_INVALID, "a batch holds at most %d instances", kMaxBatch);
    std::lock_guard<std::recursive_mutex> lock(c->exec);
    cudaSetDevice(c->device);
    auto b = std::make_unique<Batch>();
    std::vector<Job *> jobs;
    int rc;
    for (uint32_t i = 0; i < n; ++i) {
        b->jobs.push_back(std::make_unique<Job>());
        if ((rc = init_job(c, *b->jobs.back(), ref_ids[i], opts))) return rc;
        jobs.push_back(b->jobs.back().get());
    }
    if (opts && (opts->flags & PT2_FLAG_AUTOTUNE)) {
        uint32_t best;
        // tune each size class on its largest instance, before planning the batch
        std::vector<Job *> probe = jobs;
        if ((rc = plan_jobs(c, probe, true, records_budget(c, 2)))) return rc;
        std::map<int, Job *> largest;
        for (Job *j : jobs) {
            int k = size_class(j->total);
            if (!largest.count(k) || largest[k]->total < j->total) largest[k] = j;
        }
        for (auto &kv : largest)
            if ((rc = pt2_autotune(c, kv.second->ref_id, opts, &best))) return rc;
    }
    if ((rc = plan_jobs(c, jobs, true, records_budget(c, 2)))) return rc;
    if ((rc = dev_alloc(c, b->acc, n * sizeof(RunAcc), "batch accumulators"))) return rc;
    for (uint32_t i = 0; i < n; ++i) jobs[i]->acc = reinterpret_cast<RunAcc *>(b->acc.ptr) + i;
    b->steps = pack_steps(jobs, records_budget(c, 2));
    b->profile = opts && (opts->flags & PT2_FLAG_PROFILE);
    if ((rc = capture_batch(c, *b))) {
        dev_free(c, b->acc);
        dev_free(c, b->tables);
        return rc;
    }
    const uint32_t id = c->next_id++;
    c->batches[id] = std::move(b);
    *batch_id = id;
    return PT2_OK;
}

int pt2_batch_run(pt2_ctx *c, uint32_t batch_id, pt2_result *results)
{
    if (!c) return PT2_ERR_INVALID;
    std::lock_guard<std::recursive_mutex> lock(c->exec);
    auto it = c->batches.find(batch_id);
    if (it == c->batches.end()) return fail(c, PT2_ERR_NOT_FOUND, "unknown batch id %u", batch_id);
    if (!results) return fail(c, PT2_ERR_INVALID, "results pointer is NULL");
    Batch &b = *it->second;
    cudaSetDevice(c->device);
    int rc;
    // the shared workspace may have moved since capture (another run grew it)
    if (b.ws_gen != c->ws_gen)
        if ((rc = capture_batch(c, b))) return rc;
    cudaStream_t st = c->stream;
    const size_t n = b.jobs.size();
    std::vector<RunAcc> h(n);
    uint32_t err = 0;
    CK(cudaEventRecord(c->ev[0], st), "event");
    if (b.profile) {  // the captured work, launched step by step with per-phase events
        for (double &x : c->phase_ms) x = 0.0;
        c->launches = 0;
        CK(cudaMemsetAsync(c->err_word.ptr, 0, 4, st), "memset");
        CK(launch_acc_init(reinterpret_cast<RunAcc *>(b.acc.ptr), (int)n, st), "acc init");
        for (size_t i = 0; i < n; ++i)
            CK(job_subtract(c, *b.jobs[i], reinterpret_cast<RunAcc *>(b.acc.ptr) + i, st), "duplicate subtraction");
        StepDev *d = reinterpret_cast<StepDev *>(b.tables.ptr);
        for (size_t k = 0; k < b.steps.size(); ++k)
            if ((rc = enqueue_step(c, b.steps[k], d + k, nullptr, true))) return rc;
        CK(launch_acc_finalize(reinterpret_cast<RunAcc *>(b.acc.ptr), (int)n, st), "acc finalize");
    } else {
        CK(cudaGraphLaunch(b.exec, st), "graph launch");
    }
    CK(cudaEventRecord(c->ev[1], st), "event");
    CK(cudaMemcpyAsync(h.data(), b.acc.ptr, n * sizeof(RunAcc), cudaMemcpyDeviceToHost, st), "copy");
    CK(cudaMemcpyAsync(&err, c->err_word.ptr, 4, cudaMemcpyDeviceToHost, st), "copy");
    CK(cudaStreamSynchronize(st), "sync");
    float ms = 0;
    cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
    if ((rc = status_of_err(c, err))) return rc;
    for (size_t i = 0; i < n; ++i) {
        result_of(h[i], *b.jobs[i], &results[i]);
        results[i].seconds = ms * 1e-3;  // the whole batch
        if (!terms_as_planned(*b.jobs[i], h[i].n_terms))
            return fail(c, PT2_ERR_CUDA, "instance %zu generated %llu terms, planned %llu", i,
                        (unsigned long long)h[i].n_terms, (unsigned long long)b.jobs[i]->total);
    }
    return PT2_OK;
}

int pt2_batch_info(pt2_ctx *c, uint32_t batch_id, uint32_t *n_steps, uint64_t *n_terms, uint64_t *launches)
{
    if (!c) return PT2_ERR_INVALID;
    std::lock_guard<std::recursive_mutex> lock(c->exec);
    auto it = c->batches.find(batch_id);
    if (it == c->batches.end()) return fail(c, PT2_ERR_NOT_FOUND, "unknown batch id %u", batch_id);
    Batch &b = *it->second;
    if (n_steps) *n_steps = (uint32_t)b.steps.size();
    if (n_terms) {
        uint64_t t = 0;
        for (auto &j : b.jobs) t += j->total;
        *n_terms = t;
    }
    if (launches) {
        // per step: 2 generators + 3 scan + 7 reference/tile/oversize/finish, plus init/finalize
        *launches = 2 + 12 * (uint64_t)b.steps.size();
    }
    return PT2_OK;
}

int pt2_batch_destroy(pt2_ctx *c, uint32_t batch_id)
{
    if (!c) return PT2_ERR_INVALID;
    std::lock_guard<std::recursive_mutex> lock(c->exec);
    auto it = c->batches.find(batch_id);
    if (it == c->batches.end()) return fail(c, PT2_ERR_NOT_FOUND, "unknown batch id %u", batch_id);
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    Batch &b = *it->second;
    if (b.exec) cudaGraphExecDestroy(b.exec);
    dev_free(c, b.acc);
    dev_free(c, b.tables);
    c->batches.erase(it);
    return PT2_OK;
}

int pt2_autotune(pt2_ctx *c, uint32_t ref_id, const pt2_opts *opts, uint32_t *best_tile_target)
{
    if (!c) return PT2_ERR_INVALID;
    std::lock_guard<std::recursive_mutex> lock(c->exec);
    pt2_opts o;
    memset(&o, 0, sizeof o);
    if (opts) o = *opts;
    o.flags &= ~(uint32_t)PT2_FLAG_AUTOTUNE;
    double best_s = 1e300;
    uint32_t best = 0;
    uint64_t total = 0;
    for (uint32_t cand : kTuneCandidates) {
        o.tile_target = cand;
        pt2_result r;
        double s = 1e300;
        for (int rep = 0; rep < 2; ++rep) {  // the first run also warms the workspace
            int rc = run_single(c, ref_id, &o, &r, nullptr);
            if (rc) return rc;
            s = std::min(s, r.seconds);
        }
        total = r.n_terms;
        if (s < best_s) {
            best_s = s;
            best = cand;
        }
    }
    c->tuned_tile[size_class(total)] = best;
    if (best_tile_target) *best_tile_target = best;
    return PT2_OK;
}

int pt2_submit(pt2_ctx *c, uint32_t ref_id, const pt2_opts *opts, uint64_t *ticket)
{
    if (!c) return PT2_ERR_INVALID;
    if (!ticket) return fail(c, PT2_ERR_INVALID, "ticket pointer is NULL");
    auto j = std::make_unique<Job>();
    int rc;
    {
        std::lock_guard<std::recursive_mutex> lock(c->exec);
        if ((rc = init_job(c, *j, ref_id, opts))) return rc;
        if ((rc = server_start(c))) return rc;
        j->r->busy++;
        std::lock_guard<std::mutex> sl(c->served_mu);
        c->served[ref_id]++;
    }
    Server &S = *c->server;
    std::lock_guard<std::mutex> lk(S.mu);
    j->ticket = S.next_ticket++;
    j->t_submit = now_s();
    *ticket = j->ticket;
    S.pending.push_back(j.get());
    S.jobs[j->ticket] = std::move(j);
    S.cv.notify_all();
    return PT2_OK;
}

int pt2_poll(pt2_ctx *c, uint64_t ticket, pt2_result *out)
{
    if (!c) return PT2_ERR_INVALID;
    if (!c->server) return fail(c, PT2_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Server &S = *c->server;
    std::lock_guard<std::mutex> lk(S.mu);
    auto it = S.jobs.find(ticket);
    if (it == S.jobs.end()) return fail(c, PT2_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Job &j = *it->second;
    if (j.status == PT2_ERR_BUSY) return PT2_ERR_BUSY;
    const int st = j.status;
    if (out) *out = j.result;
    S.jobs.erase(it);  // a finished ticket is reported once
    return st == PT2_OK ? PT2_OK : fail(c, st, "request %llu failed", (unsigned long long)ticket);
}

int pt2_wait(pt2_ctx *c, uint64_t ticket, uint64_t timeout_ns, pt2_result *out)
{
    if (!c) return PT2_ERR_INVALID;
    if (!c->server) return fail(c, PT2_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Server &S = *c->server;
    {
        std::unique_lock<std::mutex> lk(S.mu);
        auto it = S.jobs.find(ticket);
        if (it == S.jobs.end()) return fail(c, PT2_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
        Job *j = it->second.get();
        const bool ok = S.done.wait_for(lk, std::chrono::nanoseconds(timeout_ns),
                                        [&] { return j->status != PT2_ERR_BUSY; });
        if (!ok) return fail(c, PT2_ERR_TIMEOUT, "request %llu still running", (unsigned long long)ticket);
    }
    return pt2_poll(c, ticket, out);
}

int pt2_server_stats(pt2_ctx *c, uint64_t *pending, uint64_t *active, uint64_t *steps)
{
    if (!c) return PT2_ERR_INVALID;
    if (!c->server) {
        if (pending) *pending = 0;
        if (active) *active = 0;
        if (steps) *steps = 0;
        return PT2_OK;
    }
    Server &S = *c->server;
    std::lock_guard<std::mutex> lk(S.mu);
    if (pending) *pending = S.pending.size();
    if (active) *active = S.active.size();
    if (steps) *steps = S.steps_run;
    return PT2_OK;
}

}  // extern "C"
