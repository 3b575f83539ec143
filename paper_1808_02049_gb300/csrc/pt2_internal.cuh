// Internal types shared by the host runtime (pt2_api.cu) and the kernels
// (pt2_kernels.cu).  Not part of the public C ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pt2 {

// ---------------------------------------------------------------- constants
constexpr int kMaxOrb = 64;
constexpr int kClassBits = 12;               // alpha-hash classes used to form passes
constexpr int kNumClasses = 1 << kClassBits;
constexpr int kGenThreads = 256;             // generator CTA
constexpr int kGenBatch = 8;                 // terms whose slots a lane requests before storing any
constexpr int kTileThreads = 256;            // tile sort-reduce CTA (four per SM)
constexpr int kTileCap = 1024;               // records a tile CTA sorts in shared memory
constexpr int kRefSliceSmem = 32;            // reference keys per tile kept in shared memory (larger slices are searched in global memory)
constexpr uint64_t kMaxTilesPerPass = 6400000;  // keeps the tile cursors (4 B each) resident in L2
constexpr uint64_t kMaxPassBytes = 64ull << 30;  // bound on one pass's term records unless the caller asks for more
constexpr uint64_t kMaxPassBytesAsked = ((1ull << 32) - 1) * 32;  // an explicit pass budget: up to the 32-bit slot limit
// Emission scatters records over the tiles of a pass; up to about 1.5e9
// records (1.8M tiles) per pass the partly written tile lines stay in L2.  A
// pass grows beyond that only when its determinants would otherwise emit
// fewer than kTermsPerDetPass terms each, where the per-determinant set-up
// of every pass costs more than the scatter.
constexpr uint64_t kLocalPassRecords = (48ull << 30) / 32;
constexpr uint64_t kTermsPerDetPass = 10000;
constexpr uint64_t kMaxStepRecords = (1ull << 32) - 1;  // record slots of a step are 32-bit
static_assert(kMaxPassBytes / 32 <= kMaxStepRecords, "record slots of a pass must fit 32-bit tile cursors");
constexpr int kBigThreads = 256;
constexpr int kBigChunk = 1024;             // records of an oversize tile grouped per chunk
constexpr int kBigCap = 640;                // partial records finished per grouping (oversize path)
constexpr uint64_t kBigScratch = 16384;      // partial records per buffer of one oversize CTA
constexpr int kBigBuckets = 256;             // most hash buckets the partials of one oversize tile split into
static_assert(kBigBuckets * kBigCap >= 2 * kBigScratch, "the hash split can always make buckets fit a chunk");
static_assert(kBigScratch <= 65535, "bucket starts of the hash split are 16-bit");
constexpr int kMaxBatch = 256;               // instances in one step
// Passes whose tiles one tile-count launch counts together (a group of
// consecutive passes of one run).  A group's table: kGrpTab u32 entries (class
// boundaries lo[0..kMaxGrp], tile bases base[kMaxGrp], tile counts nt[kMaxGrp]),
// then from u32 entry kGrpClsOff on the pass of every class, one byte per class
constexpr int kMaxGrp = 64;
constexpr int kGrpTab = 3 * kMaxGrp + 1;
constexpr int kGrpClsOff = 196;                           // 16-byte aligned
constexpr int kGrpStride = kGrpClsOff + kNumClasses / 4;  // u32 entries of one group's table
static_assert(kMaxGrp <= 64, "a pass index of a grouped count takes 6 bits");
static_assert(kGrpClsOff >= kGrpTab && kGrpClsOff % 4 == 0, "the class table follows the pass table, aligned");

// Fixed-point scales.  Diagonal quantities (E0 - H_aa and the pieces it is
// assembled from) are int64 multiples of 2^-48 Ha; numerator and energy sums
// are int128 multiples of 2^-90.  Integer sums are exact and associative, so
// results do not depend on the order in which terms meet.
constexpr int kDenShift = 48;
constexpr double kDenScale = 281474976710656.0;  // 2^48
constexpr double kDenRange = 2048.0;             // |component| bound validated at load (2^11 Ha)
constexpr int kFxShift = 90;

// Device error bits (OR-ed into the run's error word).
constexpr uint32_t kErrFixedRange = 1u;      // |numerator| or |term| beyond the fixed-point range
constexpr uint32_t kErrWaitTimeout = 2u;     // a bounded mbarrier wait ran out
constexpr uint32_t kErrScratch = 4u;         // oversize tile larger than its scratch
constexpr uint32_t kErrNoProgress = 8u;      // the partials of an oversize tile could not be split to fit a chunk
constexpr uint32_t kErrCount = 16u;          // emitted terms differ from the plan

// Per-instance run options the tile kernels read (TileParams::iflags).
constexpr uint32_t kInstSym = 1u;        // spin-flip symmetric run
constexpr uint32_t kInstNarrow = 2u;     // narrowed sort hash (test aid: most keys of a tile share hash and bucket)
constexpr uint32_t kInstShortWait = 4u;  // bulk-copy waits give up almost at once (test aid: exercises the timeout)
constexpr uint32_t kInstHashed = 8u;     // keys of a tile identified by a 54-bit hash (the hashing section)

// One generated term: the excited determinant, its numerator H_ai c_i and
// its denominator E0 - H_aa in units of 2^-48 Ha (from the parent's diagonal
// plus the exact incremental change, see the appendix on fast diagonals).
struct __align__(32) Rec32 {
    uint64_t a, b;
    double num;
    int64_t den;
};

// A partially reduced key (oversize path): exact fixed-point numerator sum.
struct __align__(16) Rec48 {
    uint64_t a, b;
    uint64_t fx_lo;
    int64_t fx_hi;
    int64_t den;
    uint64_t pad;
};

struct SysDev {
    int n;
    const double *h;     // n*n
    const double *eri;   // n^4
    const int64_t *Jx;   // n*n: (pp|qq) * 2^48
    const int64_t *WSx;  // n*n: ((pp|qq) - (pq|qp)) * 2^48, same-spin pair energy
    const int64_t *hdx;  // n: h_pp * 2^48
    const double *J;     // n*n (direct diagonal kernel)
    const double *WS;    // n*n
    // same-spin double elements by colex pair: dpair[P(r1, r2) * np + P(a1, a2)] =
    // (a1 r1|a2 r2) - (a1 r2|a2 r1) for r1 < r2, a1 < a2, P(i, j) = j (j - 1) / 2 + i,
    // np = n (n - 1) / 2 (one load per element instead of two)
    const double *dpair;
};

struct HashTables {
    uint64_t zc[kMaxOrb];   // alpha class hash (Zobrist)
    uint64_t zcb[kMaxOrb];  // beta class hash: splits the passes of a heavy alpha class
    uint64_t zta[kMaxOrb];  // tile hash, alpha part
    uint64_t ztb[kMaxOrb];  // tile hash, beta part
    uint16_t pairs[kMaxOrb * (kMaxOrb - 1) / 2];  // colex pair t -> (j1 | j2 << 8), j1 < j2
};

enum GenMode { kModeClassCount = 0, kModeTileCount = 1, kModeEmit = 2, kModeDetTerms = 3, kModeBetaCount = 4 };

struct GenParams {
    SysDev sys;
    const HashTables *hash;
    const uint64_t *keys;  // 2 * n_det
    const double *coef;
    const int64_t *d0;     // (E0 - H_ii) * 2^48 per determinant, exact from the integer tables
    const int64_t *g;      // per determinant, 2 n values: (h_xx + p(x)) * 2^48, alpha x then beta x
    double e0;
    uint64_t n_det;
    uint64_t det_begin;    // first determinant of this launch
    int na, nb;            // electrons per spin (same for all determinants)
    // pass selection
    uint32_t class_lo, class_hi;  // alpha classes [lo, hi) belong to the pass
    uint32_t bclass_lo, bclass_hi;  // and, within them, beta classes [lo, hi) (all: 0, kNumClasses)
    uint32_t heavy_class;         // beta-count mode: the alpha class whose beta classes are counted
    uint32_t sym;                 // spin-flip symmetric run: only terms with alpha' >= beta'
    double cutoff;                // numerator cutoff: contributions |c_i H_ai| below it are dropped (0: none)
    uint32_t subtract;            // duplicate subtraction: reference keys stay in the sum (no reference slices)
    uint64_t cons_mod, cons_rem;  // alpha % mod == rem (mod <= 1: none)
    uint64_t top_mask, top_hi;    // alpha & top_hi == top_mask: the highest occupied alpha orbitals are top_mask (0, 0: none)
    uint64_t n_tiles;                  // tiles of this instance in the pass
    uint64_t tile_base;                // first global tile index of this instance
    // tile-count mode over a group of n_grp > 0 passes (classes [class_lo,
    // class_hi) = the union of theirs): a term of class cl belongs to pass
    // q = byte cl of the class table (the last q with grp[q] <= cl) and counts
    // in tile grp[kMaxGrp + 1 + q] + tile_of(zt, grp[2 kMaxGrp + 1 + q]);
    // 0: one pass, n_tiles tiles
    uint32_t n_grp;
    const uint32_t *grp;               // kGrpStride entries (16-byte aligned)
    // outputs
    unsigned long long *class_counts;  // kNumClasses per instance; the class-count mode fills [class_lo, class_hi)
    uint32_t *tile_counts;             // n_tiles
    unsigned int *cursor;              // n_tiles: next free slot of each tile (a pass holds < 2^32 records)
    Rec32 *recs;
    unsigned long long rec_cap;        // records the launch may write (emit and det-terms modes)
    uint32_t *err;
    // dynamic shared memory layout (byte offsets)
    int smem_sa, smem_sb, smem_pairs, smem_vec, smem_hist, smem_vbk, smem_gcls, smem_bytes;
    int n_sa, n_sb;                    // singles per determinant: na*(n-na), nb*(n-nb)
};

// A launch of the generator over several instances: CTA g (global index
// cta_offset + blockIdx.x) belongs to the instance with
// det_base[i] <= g < det_base[i + 1] and handles its determinant
// params[i].det_begin + g - det_base[i].
// Checks a generator variant carries (template argument): the spin-flip
// drop rule and the numerator cutoff.
constexpr int kFiltSym = 1, kFiltCut = 2;
// Top bit of a pass's expected record count: the count is an upper bound (a
// beta-class pass of a heavy alpha class in a run with a numerator cutoff is
// planned from the counts of all terms).
constexpr unsigned long long kExpectAtMost = 1ull << 63;

struct GenBatch {
    const GenParams *params;
    const unsigned long long *det_base;  // n_inst + 1
    int n_inst;
    unsigned long long cta_offset;
    // n_inst == 1: the instance's parameters, read from the launch arguments
    // (constant bank) instead of the device table
    GenParams one;
    int filt;     // kFiltSym | kFiltCut: the checks some instance needs (selects the kernel variant)
};

// Run accumulator: every field is an exact integer reduction.
struct RunAcc {
    unsigned long long e2_lo;  // E2 * 2^90 as a 128-bit two's-complement integer
    long long e2_hi;
    unsigned long long n_terms, n_unique, n_in_ref, n_ext, n_pos, dsum, dxor;
    unsigned long long min_den;  // min |E0 - H_aa| * 2^48
    double e2;                   // filled by the finalize kernel
    double min_abs_den;
    unsigned int err;
    unsigned int n_big;          // oversize tiles over all passes
    unsigned long long n_coll;   // times two different keys of a tile shared their sort hash
};

// Tiles of a step cover several instances: tile t belongs to the instance
// with tile_base[i] <= t < tile_base[i + 1].
struct TileParams {
    const Rec32 *recs;
    const unsigned long long *tile_off;  // n_tiles + 1
    const unsigned long long *ref_off;   // n_tiles + 1
    const uint64_t *ref_keys;            // 2 * (refs in pass), grouped by tile, sorted per tile
    uint64_t n_tiles;                    // over all instances
    const unsigned long long *tile_base; // n_inst + 1
    const double *e0;                    // per instance
    const uint32_t *iflags;              // per instance: options of the tile kernels (kInst* bits: spin-flip
                                         // symmetric run, narrowed sort hash, short copy waits)
    RunAcc *const *acc;                  // per instance
    unsigned int *n_big;                 // per instance: oversize tiles of the pass
    unsigned long long *big_max;         // largest oversize tile (diagnostic)
    int n_inst;
    uint32_t *big_list;                  // oversize tiles of instance i start at tile_base[i]
    uint32_t *err;
    // dump of the external set (optional)
    uint64_t *dump_keys;
    double *dump_num, *dump_haa;
    unsigned long long *dump_count;
    unsigned long long dump_cap;
    // oversize path scratch: per CTA two buffers of scratch_cap Rec48
    Rec48 *scratch;
    unsigned long long scratch_cap;
    int sym_any;  // some instance is a spin-flip symmetric run: launch the variant that checks
};

// Reference determinants of a step: global index g belongs to the instance
// with ref_base[i] <= g < ref_base[i + 1] (keys, pass and tiles from params[i]).
struct RefPartParams {
    const GenParams *params;
    const unsigned long long *ref_base;  // n_inst + 1
    int n_inst;
    uint64_t n_total;
    const HashTables *hash;
    uint32_t *ref_tile;             // n_total: global tile or UINT32_MAX
    uint32_t *ref_count;            // n_tiles
    unsigned long long *ref_cursor; // n_tiles (initialised to offsets)
    uint64_t *ref_keys_out;         // 2 * refs in pass
};

// ---------------------------------------------------------------- launchers
// All launchers enqueue on `s` and return the launch error (cudaSuccess if ok).
void gen_layout(GenParams &p, GenMode mode);  // fills the smem_* fields from n_sa, n_sb
cudaError_t launch_gen(GenMode mode, const GenBatch &b, uint64_t n_ctas, int smem_bytes, cudaStream_t s);
cudaError_t launch_gen_single(GenMode mode, const GenParams &p, GenParams *d_params, unsigned long long *d_base,
                              cudaStream_t s);  // one determinant (parity aid); d_* are 1- and 2-entry scratch
cudaError_t launch_diag(const SysDev &sys, const uint64_t *keys, uint64_t n, double *out, cudaStream_t s);
// (E0 - H_ii) 2^48 exactly from the integer tables (needs the g tables of launch_ref_g)
cudaError_t launch_ref_d0(const SysDev &sys, const uint64_t *keys, const int64_t *g, uint64_t n, double e0,
                          int64_t *d0, cudaStream_t s);
cudaError_t launch_ref_g(const SysDev &sys, const uint64_t *keys, uint64_t n, int64_t *g, cudaStream_t s);
cudaError_t launch_scan_u32_to_u64(const uint32_t *in, unsigned long long *out, uint32_t *out32, uint64_t n,
                                   unsigned long long *tmp, cudaStream_t s);
size_t scan_tmp_elems(uint64_t n);
cudaError_t launch_ref_partition(const RefPartParams &p, int phase, cudaStream_t s);
cudaError_t launch_sort_slices(const unsigned long long *ref_off, uint64_t *ref_keys, uint64_t n_tiles,
                               cudaStream_t s);
cudaError_t launch_tiles(const TileParams &p, int n_ctas, cudaStream_t s);
cudaError_t launch_big_tiles(const TileParams &p, int n_ctas, cudaStream_t s);
cudaError_t launch_pass_finish(const unsigned long long *tile_off, const unsigned long long *tile_base, int n_inst,
                               const unsigned long long *expected, RunAcc *const *acc, unsigned int *n_big,
                               uint32_t *err, cudaStream_t s);
cudaError_t launch_acc_init(RunAcc *acc, int n, cudaStream_t s);
// acc.E2 -= sum over the reference determinants of the constraint class (alpha % cons_mod == cons_rem,
// the top-orbital constraint and alpha class in [cls_lo, cls_hi)) of c_i^2 (E0 - H_ii), exactly
cudaError_t launch_ref_subtract(const uint64_t *keys, const double *coef, const double *hii, uint64_t n, double e0,
                                uint64_t cons_mod, uint64_t cons_rem, uint64_t top_hi, uint64_t top_mask,
                                const HashTables *hash, uint32_t cls_lo, uint32_t cls_hi, RunAcc *acc, uint32_t *err,
                                cudaStream_t s);
cudaError_t launch_acc_finalize(RunAcc *acc, int n, cudaStream_t s);
// num^2 / den with the tile kernels' arithmetic (den in Hartree, rounded to 2^-48)
cudaError_t launch_eval_terms(const double *num, const double *den, uint64_t n, double *out, cudaStream_t s);
cudaError_t init_kernel_attributes(int *tile_per_sm, int *big_per_sm);  // once per process and device, before any capture
size_t tile_smem_bytes();
size_t big_smem_bytes();

// Allocation-free generation of one determinant's terms into caller-owned
// device arrays, staged in a fixed device array of kNoAllocMaxTerms records.
constexpr uint64_t kNoAllocMaxTerms = 1ull << 19;
constexpr int kMaxDevices = 64;
cudaError_t launch_det_terms_noalloc(int device, GenParams p, uint64_t cap, uint64_t *keys, double *val, double *haa,
                                     unsigned long long *n_host, cudaStream_t s);

}  // namespace pt2
