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
constexpr int kTileThreads = 512;            // tile sort-reduce CTA
constexpr int kTileCap = 2048;               // records a tile CTA groups in shared memory
constexpr int kRefSliceSmem = 64;            // reference keys per tile kept in shared memory
constexpr int kBigThreads = 512;
constexpr int kBigCap = 2048;                // Rec48 records grouped per chunk (oversize path)

// Device error bits (OR-ed into RunAcc::err).
constexpr uint32_t kErrFixedRange = 1u;      // |numerator| beyond the fixed-point range
constexpr uint32_t kErrWaitTimeout = 2u;     // a bounded mbarrier wait ran out
constexpr uint32_t kErrScratch = 4u;         // oversize tile larger than its scratch
constexpr uint32_t kErrNoProgress = 8u;      // chunked grouping could not shrink a tile
constexpr uint32_t kErrCount = 16u;          // emitted terms differ from the plan
constexpr uint32_t kErrDump = 32u;           // dump capacity exceeded

// One generated term: the excited determinant, its numerator H_ai c_i and
// its diagonal H_aa (computed incrementally from the parent determinant).
struct __align__(32) Rec32 {
    uint64_t a, b;
    double num, haa;
};

// A partially reduced key (oversize path): exact fixed-point numerator sum.
struct __align__(16) Rec48 {
    uint64_t a, b;
    uint64_t fx_lo;
    int64_t fx_hi;
    double haa;
    uint64_t pad;
};

struct SysDev {
    int n;
    const double *h;    // n*n
    const double *eri;  // n^4
    const double *J;    // n*n: (pp|qq)
    const double *WS;   // n*n: (pp|qq) - (pq|qp), same-spin pair energy
};

struct HashTables {
    uint64_t zc[kMaxOrb];   // alpha class hash (Zobrist)
    uint64_t zta[kMaxOrb];  // tile hash, alpha part
    uint64_t ztb[kMaxOrb];  // tile hash, beta part
};

enum GenMode { kModeClassCount = 0, kModeTileCount = 1, kModeEmit = 2, kModeDetTerms = 3 };

struct GenParams {
    SysDev sys;
    const HashTables *hash;
    const uint64_t *keys;  // 2 * n_det
    const double *coef;
    const double *hii;
    uint64_t n_det;
    uint64_t det_begin;    // first determinant of this launch
    int na, nb;            // electrons per spin (same for all determinants)
    // pass selection
    uint32_t class_lo, class_hi;  // classes [lo, hi) belong to the pass
    uint64_t cons_mod, cons_rem;  // alpha % mod == rem (mod <= 1: none)
    uint64_t n_tiles;
    // outputs
    unsigned long long *class_counts;  // kNumClasses
    uint32_t *tile_counts;             // n_tiles
    unsigned long long *cursor;        // n_tiles
    Rec32 *recs;
    unsigned long long rec_cap;        // records the launch may write (emit and det-terms modes)
    uint32_t *err;
    // dynamic shared memory layout (byte offsets)
    int smem_sa, smem_sb, smem_pairs, smem_vec, smem_hist, smem_bytes;
    int n_sa, n_sb;                    // singles per determinant: na*(n-na), nb*(n-nb)
};

struct TilePart {
    double e2;
    double min_den;
    uint64_t dsum, dxor;
    uint32_t n_unique, n_in_ref, n_ext, n_pos;
};

struct RunAcc {
    double e2_s, e2_c;  // Neumaier-compensated pass sums
    double min_den;
    unsigned long long n_terms, n_unique, n_in_ref, n_ext, dsum, dxor, n_pos;
    unsigned int err;
    unsigned int n_big;
};

struct TileParams {
    const Rec32 *recs;
    const unsigned long long *tile_off;  // n_tiles + 1
    const unsigned long long *ref_off;   // n_tiles + 1
    const uint64_t *ref_keys;            // 2 * (refs in pass), grouped by tile, sorted per tile
    uint64_t n_tiles;
    double e0;
    TilePart *parts;
    uint32_t *big_list;
    unsigned int *big_count;
    uint32_t *err;
    // dump of the external set (optional)
    uint64_t *dump_keys;
    double *dump_num, *dump_haa;
    unsigned long long *dump_count;
    unsigned long long dump_cap;
    // oversize path scratch: per CTA two buffers of scratch_cap Rec48
    Rec48 *scratch;
    unsigned long long scratch_cap;
};

struct RefPartParams {
    const uint64_t *keys;  // 2 * n_det (input order)
    uint64_t n_det;
    const HashTables *hash;
    uint32_t class_lo, class_hi;
    uint64_t cons_mod, cons_rem;
    uint64_t n_tiles;
    uint32_t *ref_tile;             // n_det: tile or UINT32_MAX
    uint32_t *ref_count;            // n_tiles
    unsigned long long *ref_cursor; // n_tiles (initialised to offsets)
    uint64_t *ref_keys_out;         // 2 * refs in pass
};

// ---------------------------------------------------------------- launchers
// All launchers enqueue on `s` and return the launch error (cudaSuccess if ok).
void gen_layout(GenParams &p, GenMode mode);  // fills the smem_* fields from n_sa, n_sb
cudaError_t launch_gen(GenMode mode, const GenParams &p, uint64_t n_dets, cudaStream_t s);
cudaError_t launch_diag(const SysDev &sys, const uint64_t *keys, uint64_t n, double *out, cudaStream_t s);
cudaError_t launch_scan_u32_to_u64(const uint32_t *in, unsigned long long *out, uint64_t n,
                                   unsigned long long *tmp, cudaStream_t s);
size_t scan_tmp_elems(uint64_t n);
cudaError_t launch_ref_partition(const RefPartParams &p, int phase, cudaStream_t s);
cudaError_t launch_sort_slices(const unsigned long long *ref_off, uint64_t *ref_keys, uint64_t n_tiles,
                               cudaStream_t s);
cudaError_t launch_tiles(const TileParams &p, cudaStream_t s);
cudaError_t launch_big_tiles(const TileParams &p, int n_ctas, cudaStream_t s);
cudaError_t launch_pass_reduce(const TilePart *parts, uint64_t n_tiles, TilePart *chunk_tmp,
                               const unsigned long long *tile_off, unsigned long long expected_terms,
                               RunAcc *acc, cudaStream_t s);
cudaError_t launch_acc_init(RunAcc *acc, cudaStream_t s);
int big_grid();
size_t tile_smem_bytes();
size_t big_smem_bytes();

}  // namespace pt2
