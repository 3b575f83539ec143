/*
 * libpt2 -- deterministic, sort-based Epstein-Nesbet PT2 on one GB300 (sm_103a).
 *
 * The library computes the second-order Epstein-Nesbet correction of a
 * selected-CI reference wavefunction psi = sum_i c_i |D_i> (Eq. 3 of Tubman
 * et al., arXiv:1808.02049, "Overview of ASCI"):
 *
 *     E2 = sum_{a not in psi} ( sum_i <D_a|H|D_i> c_i )^2 / (E0 - H_aa)
 *
 * where a runs over every determinant one single or double excitation away
 * from some reference determinant (Algorithm 1; the sum is split into
 * non-overlapping, complete constraint classes as in Algorithm 2).
 *
 * Conventions used by every entry point:
 *  - orbitals are numbered 0..n_orb-1, n_orb <= 64;
 *  - a determinant is a 128-bit key held as two 64-bit words, the alpha word
 *    (bit p set = alpha spin-orbital p occupied) and the beta word; the alpha
 *    word is the more significant half ("Triplet constraints" section);
 *  - key arrays interleave the words: keys[2 i] = alpha, keys[2 i + 1] = beta;
 *  - the determinant's sign convention is alpha creators in ascending order,
 *    then beta creators in ascending order, acting on the vacuum;
 *  - integrals are real, chemist notation: h[p*n + q] = h_pq (symmetric) and
 *    eri[((p*n + q)*n + r)*n + s] = (pq|rs) with 8-fold symmetry.
 *
 * Memory and ownership: every pointer argument is a HOST pointer.  Input arrays
 * are copied into device memory the library owns during the call and are
 * never retained; output arrays are written before the call returns.  The
 * context owns all device memory and one CUDA stream; nothing is allocated by
 * the caller on the device.
 *
 * Errors: every int-returning call returns PT2_OK (0) or a negative
 * pt2_status; pt2_last_error() then holds a message.  No call aborts or
 * exits.  A context is not thread-safe: one host thread at a time.
 */
#ifndef PT2_H
#define PT2_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pt2_ctx pt2_ctx;

typedef enum {
    PT2_OK = 0,
    PT2_ERR_INVALID = -1,     /* bad argument or inconsistent input data */
    PT2_ERR_OOM = -2,         /* device memory budget or capacity exceeded */
    PT2_ERR_CUDA = -3,        /* a CUDA runtime call failed */
    PT2_ERR_TIMEOUT = -4,     /* a bounded device-side wait ran out */
    PT2_ERR_BUSY = -5,        /* a submitted request has not finished */
    PT2_ERR_NOT_FOUND = -6,   /* unknown system, reference or ticket id */
    PT2_ERR_UNSUPPORTED = -7  /* e.g. n_orb > 64 */
} pt2_status;

/* Create a context on CUDA device `device`.  hbm_budget_bytes bounds the
 * device memory the context may hold (0 = 80% of the free memory at creation).
 * On success *out receives the context. */
int pt2_create(pt2_ctx **out, int device, uint64_t hbm_budget_bytes);

/* Release every device resource of the context.  NULL is ignored. */
void pt2_destroy(pt2_ctx *ctx);

/* Message of the last failed call on this context (or of the last failed
 * pt2_create when ctx is NULL).  Valid until the next call on the context. */
const char *pt2_last_error(const pt2_ctx *ctx);

/* Load the integrals of one system (the Hamiltonian of Eq. 3).
 * h: n_orb*n_orb doubles, symmetric to 1e-12; eri: n_orb^4 doubles with
 * (pq|rs) = (qp|rs) = (pq|sr) = (rs|pq) to 1e-12.  All values finite.
 * The library keeps one canonical element of each symmetry class (h_pq with
 * p >= q; (pq|rs) with p >= q, r >= s and pq >= rs as pair indices), so
 * inputs symmetric only to the tolerance give the same result whichever
 * equivalent element a kernel reads.
 * Errors: PT2_ERR_UNSUPPORTED for n_orb > 64, PT2_ERR_INVALID otherwise. */
int pt2_load_system(pt2_ctx *ctx, int n_orb, const double *h, const double *eri,
                    uint32_t *system_id);

/* Load a reference wavefunction {D_i, c_i} and its variational energy E0
 * (E_ASCI of Eq. 3) for a loaded system.  keys: 2*n_det words as described
 * above; coef: n_det finite doubles.  Every determinant must have the same
 * alpha and the same beta electron count, no bit at or above n_orb, and no
 * determinant may repeat (PT2_ERR_INVALID otherwise).  The reference is kept
 * resident on the device until pt2_unload. */
int pt2_load_reference(pt2_ctx *ctx, uint32_t system_id, uint64_t n_det, const uint64_t *keys,
                       const double *coef, double e0, uint32_t *ref_id);

/* Free a loaded system or reference (a system may only be unloaded once no
 * reference uses it; PT2_ERR_INVALID otherwise).  A reference with submitted
 * requests that have not finished is refused at once with PT2_ERR_BUSY, also
 * while the serving engine is running a step. */
int pt2_unload(pt2_ctx *ctx, uint32_t id);

/* Direct diagonal H_kk (Slater-Condon, the denominator term of Eq. 3) of n
 * determinants of a loaded system, computed on the device.  keys: 2*n words;
 * out: n doubles.  Used e.g. to set E0 = min_i H_ii - shift. */
int pt2_diagonal(pt2_ctx *ctx, uint32_t system_id, uint64_t n, const uint64_t *keys, double *out);

/* Run options.  Zero-initialise and set what you need. */
typedef struct {
    uint64_t constraint_mod;  /* 0 or 1: no constraint.  Otherwise only excited
                                 determinants with alpha % constraint_mod ==
                                 constraint_rem are summed: one class of a
                                 non-overlapping, complete partition
                                 (Algorithm 2). */
    uint64_t constraint_rem;
    uint64_t pass_budget_bytes; /* device bytes for one pass of generated
                                   terms (0 = chosen from the context budget
                                   and the reference size, at most 96 GB);
                                   smaller values mean more passes */
    uint32_t tile_target;       /* mean terms per hash tile, at most 1024
                                   (0 = default 832, or the tuned value) */
    uint32_t flags;             /* PT2_FLAG_* below */
    double numerator_cutoff;    /* 0 = exact.  Otherwise a contribution c_i H_ai
                                   with |c_i H_ai| < numerator_cutoff is
                                   ignored before it gets a record, a
                                   denominator or a sort (the Results section
                                   and the subsection on the matrix-element
                                   cutoff use 1e-8); a determinant all of
                                   whose contributions are ignored is not in
                                   the external set.  n_terms counts the kept
                                   contributions.  PT2_ERR_INVALID if negative
                                   or not finite. */
    uint32_t debug_flags;       /* PT2_DEBUG_* test aids below; 0 in normal use */
    uint32_t class_slices;      /* 0 or 1: every alpha class.  Otherwise only
                                   excited determinants whose alpha-hash class
                                   (a fixed 12-bit Zobrist hash of the alpha
                                   string, 4096 classes) lies in slice
                                   class_slice of class_slices contiguous
                                   slices are summed: another non-overlapping,
                                   complete partition of Algorithm 2, the one
                                   the memory-bounded passes are made of, so a
                                   slice costs about 1/class_slices of the
                                   solve (plus its own work-list launch).  At
                                   most 4096; combines with constraint_mod. */
    uint32_t class_slice;
    uint32_t reserved;          /* must be 0 */
    uint64_t top_alpha;         /* 0: none.  Otherwise a bit mask T of k alpha
                                   orbitals: only excited determinants whose k
                                   highest occupied alpha orbitals are exactly
                                   T are summed (the "Triplet constraints"
                                   section: k = 3 a triplet, k = 4 a
                                   quadruplet constraint; for each k the masks
                                   T form a non-overlapping, complete
                                   partition).  The alpha-alpha doubles of
                                   such a run are generated directly
                                   (Algorithm 3).  Combines with the other
                                   constraints. */
} pt2_opts;

#define PT2_FLAG_PROFILE 1u   /* record per-phase device times (pt2_phase_times); a batch created
                                 with it runs its steps one by one instead of replaying its graph */
#define PT2_FLAG_AUTOTUNE 2u  /* pt2_batch_create: tune the tile target per size class first */
/* Spin-flip symmetry (the subsection on Z2 spin symmetry for S_z = 0): for a reference closed under
 * exchange of the alpha and beta strings with c(beta, alpha) = c(alpha, beta),
 * the contributions of (alpha', beta') and (beta', alpha') to E2 are equal, so
 * only excited determinants with alpha' >= beta' (as 64-bit words) are
 * generated, sorted and reduced; those with alpha' > beta' count twice.  E2 is
 * that of the full sum; n_terms, n_unique, n_in_ref, n_external, the digest,
 * min_abs_denom and n_pos_denom then describe the kept half (alpha' >= beta').
 * PT2_ERR_INVALID if the reference is not symmetric. */
#define PT2_FLAG_SPIN_SYMMETRIC 4u
/* Duplicate subtraction (the section on removing duplicate contributions):
 * instead of filtering the reference determinants out of the external set,
 * keep them in the sum and subtract sum_i c_i^2 (E0 - H_ii) over the reference
 * determinants of the constraint class.  Equal to the filtered E2 when c is an
 * eigenvector of H in the reference space with eigenvalue E0 (the E0 given to
 * pt2_load_reference); otherwise it differs by the eigenvector residual.
 * n_in_ref is then 0 and n_external, the digest, min_abs_denom and
 * n_pos_denom cover every generated key, reference keys included. */
#define PT2_FLAG_SUBTRACT_REF 8u
/* Hashed keys (the section on compression with hash functions): inside each
 * hash tile the records are grouped by a 54-bit hash of the 128-bit key (a
 * 64-bit mix with the record's index in its low bits) instead of by the key
 * itself, so the grouping reads no keys.  Two different keys of one tile
 * with the same 54-bit hash would be merged; the run then still compares
 * every merged record with its group's first key and reports the number of
 * mismatches in pt2_result.n_hash_collisions (0: the hashed grouping was
 * exact, so E2, the counts and the external set equal an ordinary run's).
 * With about 450 keys per tile the expected number of such merges is about
 * 450^2 / 2^55 per tile, 3e-3 for a 4.8e11-term solve. */
#define PT2_FLAG_HASHED_KEYS 16u

/* Test aids (pt2_opts.debug_flags).  They exercise paths that ordinary inputs
 * reach only rarely; neither changes a result.
 * PT2_DEBUG_NARROW_SORT_HASH: the 32-bit hash that orders the records of a
 *   tile keeps only 4 bits, so most keys of a tile share their hash and their
 *   bucket: the grouping tells them apart by the full 128-bit comparison and
 *   hands long buckets to its warp path.  Slower; E2, counts and the external
 *   set are those of an ordinary run (pt2_result.n_hash_collisions counts the
 *   comparisons that met different keys with equal hashes).
 * PT2_DEBUG_SHORT_COPY_WAIT: the tile kernels give up waiting for a tile's
 *   bulk copy after 64 SM cycles instead of about a second.  The copy still
 *   lands (a second bounded wait), the CTA stops, and the run returns
 *   PT2_ERR_TIMEOUT; the context stays usable. */
#define PT2_DEBUG_NARROW_SORT_HASH 1u
#define PT2_DEBUG_SHORT_COPY_WAIT 2u

typedef struct {
    double e2;                /* the PT2 energy, Hartree */
    uint64_t n_terms;         /* generated (key, H_ai c_i) pairs */
    uint64_t n_unique;        /* distinct generated determinants */
    uint64_t n_in_ref;        /* distinct generated determinants that are in psi */
    uint64_t n_external;      /* |connected external set| */
    uint64_t digest_sum;      /* sum over the external set of mix1(key) mod 2^64 */
    uint64_t digest_xor;      /* xor over the external set of mix2(key) */
    double min_abs_denom;     /* min |E0 - H_aa| over the external set */
    uint64_t n_pos_denom;     /* external determinants with E0 - H_aa > 0 */
    uint32_t n_passes;        /* memory-bounded passes used */
    uint32_t n_tiles;         /* hash tiles over all passes */
    uint32_t n_oversize;      /* tiles handled by the chunked path */
    uint32_t n_hash_collisions; /* comparisons inside a tile that met two different keys with
                                   the same 32-bit sort hash; with PT2_FLAG_HASHED_KEYS, records
                                   merged into a group whose first key differs from theirs
                                   (saturates at 2^32 - 1) */
    double seconds;           /* device time of the run (CUDA events) */
} pt2_result;

/* Compute E2 for a loaded reference (blocking).  opts may be NULL.  The
 * result is bit-identical across runs for the same inputs and options. */
int pt2_run(pt2_ctx *ctx, uint32_t ref_id, const pt2_opts *opts, pt2_result *out);

/* Like pt2_run, and also write the connected external set: for each of its
 * determinants the key (2 words), the summed numerator sum_i H_ai c_i and the
 * diagonal H_aa.  Order is unspecified.  At most cap entries are written;
 * *n_out receives |S| (PT2_ERR_OOM if it exceeds cap).  Parity aid. */
int pt2_dump_external(pt2_ctx *ctx, uint32_t ref_id, const pt2_opts *opts, uint64_t *keys,
                      double *num, double *haa, uint64_t cap, uint64_t *n_out);

/* ------------------------------------------------------------------ batches
 *
 * Many independent solves of uneven size (different systems, orbital counts,
 * reference sizes) run together: their memory-bounded passes (Algorithm 2)
 * are packed into steps, and every step runs one pass of each of its
 * instances with a single launch of every kernel.  pt2_batch_create plans the
 * batch (one work-list launch over all instances), allocates its workspace
 * and captures all steps into one CUDA graph; pt2_batch_run replays it.
 * Results are bit-identical to pt2_run of each instance alone. */

/* Plan and capture a batch of n loaded references (n <= 256).  opts applies
 * to every instance (NULL: defaults); with PT2_FLAG_AUTOTUNE the tile target
 * of each size class present is tuned first (pt2_autotune). */
int pt2_batch_create(pt2_ctx *ctx, uint32_t n, const uint32_t *ref_ids, const pt2_opts *opts,
                     uint32_t *batch_id);

/* Run a created batch (blocking); results: n entries in creation order.
 * results[i].seconds is the device time of the whole batch. */
int pt2_batch_run(pt2_ctx *ctx, uint32_t batch_id, pt2_result *results);

/* Steps, total generated terms and kernel launches of one batch run (with a
 * numerator cutoff, n_terms is the work list's count of the kept terms). */
int pt2_batch_info(pt2_ctx *ctx, uint32_t batch_id, uint32_t *n_steps, uint64_t *n_terms, uint64_t *launches);

/* Release a batch and its device memory. */
int pt2_batch_destroy(pt2_ctx *ctx, uint32_t batch_id);

/* Autotuner: time every candidate tile target (the terms per hash tile, which
 * sets the bucket count of each pass and the in-shared-memory sort size) on
 * one reference and remember the fastest for the reference's size class
 * (decades of generated terms); later plans of that class use it.  The energy
 * does not depend on the choice. */
int pt2_autotune(pt2_ctx *ctx, uint32_t ref_id, const pt2_opts *opts, uint32_t *best_tile_target);

/* ------------------------------------------------------------------ serving
 *
 * Continuous batching: submitted solves queue and are admitted in arrival
 * order while fewer than 256 are in flight and their planned pass footprint
 * (terms, at most one pass of 32-byte records each) fits two steps of the
 * context's HBM record budget; admitted solves are planned (work-list launch)
 * and then advance one pass per engine step together with every other
 * admitted solve whose next pass fits the step's memory budget; finished
 * solves leave and waiting ones join between steps.  A background host thread of the context runs the engine;
 * systems and references stay resident, and a reference with requests in
 * flight cannot be unloaded (PT2_ERR_BUSY).  Each result is bit-identical to
 * pt2_run of the same reference alone. */

/* Queue a solve of a loaded reference; *ticket identifies it. */
int pt2_submit(pt2_ctx *ctx, uint32_t ref_id, const pt2_opts *opts, uint64_t *ticket);

/* PT2_ERR_BUSY while the request runs; otherwise its status, with the result
 * in *out (seconds = latency from submission to completion).  A finished
 * ticket is reported once and then forgotten (PT2_ERR_NOT_FOUND after). */
int pt2_poll(pt2_ctx *ctx, uint64_t ticket, pt2_result *out);

/* Like pt2_poll, but first wait up to timeout_ns for the request to finish;
 * PT2_ERR_TIMEOUT if it is still running then. */
int pt2_wait(pt2_ctx *ctx, uint64_t ticket, uint64_t timeout_ns, pt2_result *out);

/* Requests waiting for admission, in flight, and engine steps run so far. */
int pt2_server_stats(pt2_ctx *ctx, uint64_t *pending, uint64_t *active, uint64_t *steps);

/* Generate the terms of one reference determinant (index in the caller's
 * original order): every single and double excitation D_a with its numerator
 * <D_a|H|D_i> c_i and diagonal H_aa, as the generation kernel emits them
 * (Algorithm 1, first step).  Order is unspecified; *n_out receives the count
 * (PT2_ERR_OOM if it exceeds cap).  Parity aid. */
int pt2_det_terms(pt2_ctx *ctx, uint32_t ref_id, uint64_t det_index, uint64_t *keys,
                  double *val, double *haa, uint64_t cap, uint64_t *n_out);

/* Allocation-free variant of pt2_det_terms, for callers that cannot allocate
 * device memory at the moment they call: code that runs under a memory pool
 * or arena it must not bypass, a serving loop that forbids allocations on its
 * latency path, or a process whose device memory is already fully reserved.
 * The paper has no counterpart; this is a library convenience.
 *
 * keys (2*cap uint64), val and haa (cap doubles each) are DEVICE pointers the
 * caller owns; the terms of determinant det_index are written there (at most
 * cap of them) and *n_out (host) receives their number (PT2_ERR_OOM if it
 * exceeds cap).  Order is unspecified, as for pt2_det_terms.
 *
 * The call allocates nothing: it stages the terms in a fixed device array
 * built into the library (16 MiB, 524288 terms; every GPU that loads the
 * library holds it until the process exits).  A determinant with more terms
 * is rejected with PT2_ERR_OOM.  The first call on a device looks up the
 * array's device address; make that first call before any stream capture.
 * All calls share the array and clear its counter when they start, so calls
 * whose GPU work overlaps (several threads or contexts) race and must be
 * serialised by the caller.  The call writes keys, val and haa on the
 * context's stream (pt2_stream): work the caller has queued on its own
 * streams that reads or writes these buffers must be finished, or ordered
 * before the call (for example by synchronising), when the call is made.
 * A device error of the generation is reported like pt2_run's (the
 * context's error word is cleared first and read after).
 * Blocking: returns after the terms are written. */
int pt2_det_terms_noalloc(pt2_ctx *ctx, uint32_t ref_id, uint64_t det_index, uint64_t *keys, double *val,
                          double *haa, uint64_t cap, uint64_t *n_out);

/* The per-key term of Eq. 3, num^2 / (E0 - H_aa), evaluated with the device
 * arithmetic of the tile kernels: the denominator rounded to the library's
 * fixed point (multiples of 2^-48 Ha), its reciprocal taken from the
 * single-precision hardware estimate refined by one Newton-Raphson step in
 * FP64 (relative error below 2^-44), FP64 products.  num and denom (E0 - H_aa
 * in Hartree) are n host doubles each, term receives n doubles.  Every entry
 * must be finite with 0 < |denom| < 2^15 Ha after rounding (PT2_ERR_INVALID
 * otherwise).  Parity aid: tests bound this arithmetic against exact values. */
int pt2_eval_terms(pt2_ctx *ctx, uint64_t n, const double *num, const double *denom, double *term);

/* Per-phase device milliseconds of the last run made with PT2_FLAG_PROFILE:
 * out[0] class count, [1] tile count, [2] scan, [3] generate/emit,
 * [4] reference partition, [5] tile sort-reduce, [6] oversize tiles,
 * [7] pass reduction.  n = number of slots in out (at most 8 written).
 * launches (may be NULL) receives the number of kernel launches. */
int pt2_phase_times(pt2_ctx *ctx, double *out, int n, uint64_t *launches);

/* Device memory accounting of the context: *budget is the byte budget fixed
 * at creation, *used what the context holds now (systems, references and the
 * grow-only run workspace), *device_free what the device reports free.  Any
 * pointer may be NULL. */
int pt2_memory_info(pt2_ctx *ctx, uint64_t *budget, uint64_t *used, uint64_t *device_free);

/* The context's CUDA stream (a cudaStream_t), for callers that want to
 * order or time their own work against the library's. */
void *pt2_stream(pt2_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* PT2_H */
