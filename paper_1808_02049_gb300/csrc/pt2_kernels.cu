// sm_103a kernels of the sort-based Epstein-Nesbet PT2 path.
//
// Path (Algorithm 2 with hash-defined constraint classes):
//   at load          H_ii, E0 - H_ii and the orbital energies g(x) of every
//                    reference determinant
//   gen<ClassCount>  work list: terms per alpha-hash class (sizes the passes);
//   gen<BetaCount>   for an alpha class too heavy for one pass, its terms per
//                    beta-hash class (splits it into several passes)
//   per pass:
//     gen<TileCount>  terms per hash tile of the pass
//     scan            tile offsets (and the 32-bit slot cursors)
//     gen<Emit>       every single/double of every reference determinant whose
//                     key falls in the pass: key, H_ai c_i (Slater-Condon,
//                     fermionic phase) and E0 - H_aa (exact incremental diagonal),
//                     written into its tile
//     ref partition   reference keys of the pass, grouped by tile and sorted
//     tile            per tile, in shared memory: stable LSD radix sort of the
//                     keys' 24-bit hashes (equal keys adjacent, collisions
//                     checked on the full key), reduce by key, explicit filter
//                     of reference keys by binary search, num^2 / (E0 - H_aa)
//                     accumulated exactly
//     big tile        tiles larger than shared memory, in chunks reduced to
//                     exact partials
//
// Run options, as template variants launched only where a step needs them
// (ordinary runs keep their registers): a spin-flip symmetric run keeps only
// terms with alpha' >= beta' and counts alpha' > beta' twice (the Z2
// subsection); the numerator cutoff drops contributions |c_i H_ai| below it in
// the tile count and the emission (the matrix-element cutoff subsection);
// duplicate subtraction leaves the reference keys in the sum and subtracts
// c_i^2 (E0 - H_ii) per reference determinant (ref_subtract_kernel).
//
// FP64 is the scarce unit on this GPU, so every quantity with a natural exact
// integer form is kept as one: the diagonal difference (int64, 2^-48 Ha), the
// per-key numerator sum and the energy sum (int128, 2^-90).  FP64 is used for
// the Slater-Condon products, the square and the reciprocal of the
// denominator.  Integer sums are associative, so the energy is bit-identical
// for any tiling, pass plan, reference order or atomic interleaving.
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "pt2_internal.cuh"

namespace pt2 {

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ uint32_t class_of(uint64_t zc) { return (uint32_t)(zc >> (64 - kClassBits)); }

__device__ __forceinline__ bool cons_ok(uint64_t mod, uint64_t rem, uint64_t alpha)
{
    return mod <= 1 || (alpha % mod) == rem;
}

// bits strictly between orbitals x and y
__device__ __forceinline__ uint64_t between_mask(int x, int y)
{
    int lo = x < y ? x : y, hi = x < y ? y : x;
    return ((1ull << hi) - 1ull) & ~((2ull << lo) - 1ull);
}

__device__ __forceinline__ double flip_sign(double v, uint32_t s)
{
    return __longlong_as_double(__double_as_longlong(v) ^ ((unsigned long long)(s & 1u) << 63));
}

// SplitMix64 output function (Steele, Lea, Flood 2014).
__device__ __forceinline__ uint64_t fmix64(uint64_t z)
{
    z ^= z >> 30;
    z *= 0xbf58476d1ce4e5b9ull;
    z ^= z >> 27;
    z *= 0x94d049bb133111ebull;
    z ^= z >> 31;
    return z;
}

// Order-independent digest of the external set.
__device__ __forceinline__ uint64_t digest1(uint64_t a, uint64_t b) { return fmix64(a ^ (b * 0x9e3779b97f4a7c15ull)); }
__device__ __forceinline__ uint64_t digest2(uint64_t a, uint64_t b) { return fmix64(b ^ (a * 0xc2b2ae3d27d4eb4full)); }

// Hash of a key that spreads it over the buckets of its tile.
__device__ __forceinline__ uint32_t bucket_hash(uint64_t a, uint64_t b)
{
    uint64_t h = (a * 0x9E3779B97F4A7C15ull) ^ b;
    h ^= h >> 29;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 32;
    return (uint32_t)h;
}

__device__ __forceinline__ bool key_less(uint64_t a0, uint64_t b0, uint64_t a1, uint64_t b1)
{
    return a0 < a1 || (a0 == a1 && b0 < b1);
}

// ---------------------------------------------------- exact fixed point

// Add value * 2^90 (rounded half away from zero) to the 128-bit integer
// (lo, hi).  |value| must stay below 2^36, else the range bit is set.
__device__ __forceinline__ void fx_add_double(uint64_t &lo, int64_t &hi, double v, uint32_t &err)
{
    uint64_t bits = (uint64_t)__double_as_longlong(v);
    int e = (int)((bits >> 52) & 0x7FF);
    if (e == 0) return;  // zero / subnormal: below the resolution
    if (e >= 1023 + 36) {
        err |= kErrFixedRange;
        return;
    }
    uint64_t m = (bits & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
    int sh = e - 1075 + kFxShift;  // value = m * 2^(e - 1075)
    uint64_t ml, mh;
    if (sh >= 0) {
        if (sh == 0) {
            ml = m;
            mh = 0;
        } else if (sh < 64) {
            ml = m << sh;
            mh = m >> (64 - sh);
        } else {
            ml = 0;
            mh = m << (sh - 64);
        }
    } else {
        int r = -sh;
        if (r > 63) return;
        ml = (m + (1ull << (r - 1))) >> r;
        mh = 0;
    }
    if (bits >> 63) {
        uint64_t nlo = lo - ml;
        uint64_t borrow = lo < ml;
        hi = hi - (int64_t)mh - (int64_t)borrow;
        lo = nlo;
    } else {
        uint64_t nlo = lo + ml;
        uint64_t carry = nlo < lo;
        hi = hi + (int64_t)mh + (int64_t)carry;
        lo = nlo;
    }
}

__device__ __forceinline__ void fx_add_fx(uint64_t &lo, int64_t &hi, uint64_t blo, int64_t bhi)
{
    uint64_t nlo = lo + blo;
    uint64_t carry = nlo < lo;
    hi = hi + bhi + (int64_t)carry;
    lo = nlo;
}

// Round a 128-bit magnitude times 2^-scale to the nearest double (ties to
// even), by assembling the IEEE bits with integer operations.
__device__ __forceinline__ double u128_to_double(uint64_t ulo, uint64_t uhi, int scale, bool neg)
{
    if ((ulo | uhi) == 0) return neg ? -0.0 : 0.0;
    int msb = uhi ? 127 - __clzll((long long)uhi) : 63 - __clzll((long long)ulo);
    uint64_t mant;
    int ex = msb - scale;
    if (msb <= 52) {
        mant = ulo << (52 - msb);
    } else {
        int sh = msb - 52;  // 1..75
        uint64_t lo2 = sh < 64 ? (ulo >> sh) | (uhi << (64 - sh)) : (uhi >> (sh - 64));
        int rb = sh - 1;
        uint64_t round = rb < 64 ? (ulo >> rb) & 1ull : (uhi >> (rb - 64)) & 1ull;
        bool sticky;
        if (rb == 0) sticky = false;
        else if (rb < 64) sticky = (ulo & ((1ull << rb) - 1ull)) != 0;
        else if (rb == 64) sticky = ulo != 0;
        else sticky = ulo != 0 || (uhi & ((1ull << (rb - 64)) - 1ull)) != 0;
        mant = lo2;
        if (round && (sticky || (mant & 1ull))) {
            ++mant;
            if (mant >> 53) {
                mant >>= 1;
                ++ex;
            }
        }
    }
    uint64_t bits = ((uint64_t)neg << 63) | ((uint64_t)(ex + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull);
    return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ double fx_to_double(uint64_t lo, int64_t hi)
{
    bool neg = hi < 0;
    uint64_t ulo = lo, uhi = (uint64_t)hi;
    if (neg) {
        ulo = ~ulo + 1ull;
        uhi = ~uhi + (ulo == 0 ? 1ull : 0ull);
    }
    return u128_to_double(ulo, uhi, kFxShift, neg);
}

// E0 - H_aa as a double: the int64 is rounded to nearest (ties to even) by the
// conversion instruction and the power-of-two scale is exact.
__device__ __forceinline__ double den_to_double(int64_t d) { return __ll2double_rn((long long)d) * 0x1p-48; }
static_assert(kDenShift == 48, "den_to_double scales by 2^-48");

// Reciprocal of d: a single-precision hardware estimate refined by one
// Newton-Raphson step, x1 = x0 (2 - d x0) (relative error about 2^-46).
__device__ __forceinline__ double recip(double d, int64_t dfx)
{
    float f = __ll2float_rn((long long)dfx) * 0x1p-48f;
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(f));
    uint32_t fb = __float_as_uint(rf);
    uint32_t fe = (fb >> 23) & 0xFF;
    uint64_t db;
    if (fe == 0) db = (uint64_t)(fb >> 31) << 63;
    else if (fe == 0xFF) db = ((uint64_t)(fb >> 31) << 63) | (0x7FFull << 52) | ((uint64_t)(fb & 0x7FFFFF) << 29);
    else db = ((uint64_t)(fb >> 31) << 63) | ((uint64_t)(fe + 896) << 52) | ((uint64_t)(fb & 0x7FFFFF) << 29);
    double x = __longlong_as_double((long long)db);
    double e = __fma_rn(-d, x, 1.0);
    return __fma_rn(x, e, x);
}

// ------------------------------------------------- mbarrier + TMA bulk copy

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One elected thread: expect `bytes` and start a global -> shared bulk copy.
// dst, src 16-byte aligned, bytes a multiple of 16 and below 2^20.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity, giving up after ~2^31 SM cycles
// (about a second).  On a timeout the error bit is set and a second bounded
// wait gives the copy in flight the chance to land before the CTA moves on.
__device__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t *err)
{
    long long t0 = clock64();
    while (!mbar_test(bar, parity)) {
        if (clock64() - t0 > (1ll << 31)) {
            atomicOr(err, kErrWaitTimeout);
            long long t1 = clock64();
            while (!mbar_test(bar, parity) && clock64() - t1 < (1ll << 31)) {
            }
            return false;
        }
    }
    return true;
}

// ----------------------------------------------------------- block scans

// Exclusive scan of n <= 4 * blockDim.x uint32 in shared memory (in place).
// `warp_tot` needs blockDim.x / 32 entries.
__device__ void block_scan_excl_u32(uint32_t *a, int n, uint32_t *warp_tot)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    uint32_t v[4];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int i = 4 * tid + k;
        v[k] = i < n ? a[i] : 0u;
        s += v[k];
    }
    uint32_t incl = s;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? warp_tot[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, wi, off);
            if (lane >= off) wi += t;
        }
        if (lane < nw) warp_tot[lane] = wi - w;
    }
    __syncthreads();
    uint32_t run = warp_tot[warp] + incl - s;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int i = 4 * tid + k;
        if (i < n) a[i] = run;
        run += v[k];
    }
    __syncthreads();
}

// ======================================================= generation kernel

// Alpha-alpha doubles are found through a table of the determinant's virtual
// alpha pairs bucketed by the top kVbkBits bits of the pair's class hash.  The
// class of a double is (hash of the occupied part) xor (hash of the virtual
// pair), so the classes of a pass, as groups of 2^(kClassBits - kVbkBits)
// classes, split into at most 2 kVbkBits aligned blocks; xor with the
// occupied part's top bits maps each block onto one contiguous range of
// buckets, and only those pairs are visited (then checked class by class).
constexpr int kVbkBits = 10;
constexpr int kVbkBitsMax = kVbkBits;
constexpr int kVbkBuckets = 1 << kVbkBits;
constexpr int kMaxVirPairs = kMaxOrb * (kMaxOrb - 1) / 2;
static_assert(kVbkBuckets == 4 * kGenThreads, "the bucket scan takes four buckets per thread");
static_assert(2 * kVbkBits <= 32, "one lane per block of buckets");
__device__ __forceinline__ uint32_t vb_bucket(uint64_t z) { return (uint32_t)(z >> (64 - kVbkBits)); }

// Shared memory of the bucket table (in the histogram area, unused by the
// emitting modes): counts then cursors, starts, pair list, per-warp lookups.
constexpr size_t kVbkBytes = kVbkBuckets * 4 + (kVbkBuckets + 1) * 2 + kMaxVirPairs * 2 + (kGenThreads / 32) * 64 * 2 + 16;

struct GenFixed {
    uint64_t zc[kMaxOrb], zcb[kMaxOrb], zta[kMaxOrb], ztb[kMaxOrb];
    int64_t gA[kMaxOrb], gB[kMaxOrb];  // (h_xx + p(x)) * 2^48 for alpha / beta spin-orbital x
    int occA[kMaxOrb], virA[kMaxOrb], occB[kMaxOrb], virB[kMaxOrb];
    uint64_t A, B, ZcA, ZcbB, ZtaA, ZtbB;
    double c;
    int64_t d0;
    int n_sa_pass, a_in_pass, n_sb_pass, b_in_pass;
    uint32_t wsum[kGenThreads / 32];
    // the pass's alpha classes as aligned blocks of bucket groups (see above)
    uint16_t blk_g[2 * kVbkBitsMax];
    uint8_t blk_k[2 * kVbkBitsMax];
    int n_blk;
};

// beta class of a beta-string hash (splits the heavy alpha classes)
__device__ __forceinline__ uint32_t bclass_of(uint64_t zcb) { return (uint32_t)(zcb >> (64 - kClassBits)); }

// Matrix elements without sign and coefficient, shared by the tile-count and
// emit launches so that the numerator cutoff takes the same decision in both
// (the same operations in the same order).
// Single r -> a of a string with occupied list occ_s (n_s), the other spin's
// string having occupied list occ_o (n_o): h_ar + sum_j ((ar|jj) - (aj|jr))
// over the same spin + sum_j (ar|jj) over the other spin.
__device__ __forceinline__ double single_value(const double *__restrict__ ht, const double *__restrict__ eri, int N,
                                               const int *occ_s, int n_s, const int *occ_o, int n_o, int r, int a)
{
    double v = ht[a * N + r];
    for (int q = 0; q < n_s; ++q) {
        const int j = occ_s[q];
        v += eri[(((size_t)a * N + r) * N + j) * N + j] - eri[(((size_t)a * N + j) * N + j) * N + r];
    }
    for (int q = 0; q < n_o; ++q) {
        const int j = occ_o[q];
        v += eri[(((size_t)a * N + r) * N + j) * N + j];
    }
    return v;
}

// Same-spin double r1 r2 -> a1 a2: (a1 r1|a2 r2) - (a1 r2|a2 r1), read as
// (r2 a2|r1 a1) - (r1 a2|r2 a1) so that a1 varies fastest in memory.
__device__ __forceinline__ double same_double_value(const double *__restrict__ eri, int N, int r1, int r2, int a1,
                                                    int a2)
{
    return __ldg(eri + (((size_t)r2 * N + a2) * N + r1) * N + a1) - __ldg(eri + (((size_t)r1 * N + a2) * N + r2) * N + a1);
}

// Kept by the numerator cutoff: |c v| >= cut (the sign of the element does not matter).
__device__ __forceinline__ bool above_cut(double c, double v, double cut) { return fabs(c * v) >= cut; }

// The string W after the single excitation packed in `info` (r in bits 0-7, a in 8-15).
__device__ __forceinline__ uint64_t single_word(uint64_t W, uint32_t info)
{
    return W ^ (1ull << (info & 0xFFu)) ^ (1ull << ((info >> 8) & 0xFFu));
}


// Counter updates on global memory.  The counters may be reached through
// pointers read from a device table, so the global state space is named
// explicitly: the compiler would otherwise emit generic (returning) atomics.
__device__ __forceinline__ void red_add_global(uint32_t *p, uint32_t v)
{
    asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "r"(v));
}
__device__ __forceinline__ uint32_t atom_add_global(unsigned int *p, uint32_t v)
{
    uint32_t old;
    asm volatile("atom.relaxed.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(__cvta_generic_to_global(p)), "r"(v));
    return old;
}

// One 32-byte record written with a single 256-bit store (one L2 sector).
__device__ __forceinline__ void store_rec32(Rec32 *dst, uint64_t a, uint64_t b, double num, int64_t den)
{
    // no memory clobber: nothing in the generator reads records back
    asm volatile("st.global.v4.u64 [%0], {%1, %2, %3, %4};" ::"l"(dst), "l"(a), "l"(b),
                 "l"((uint64_t)__double_as_longlong(num)), "l"((uint64_t)den));
}

// One batch of up to kGenBatch terms of a lane, items i0, i0 + step, ...:
// first every term's tile is hashed and its slot requested (the atomics of
// the batch are then in flight together), then the values are computed and
// stored, so the arithmetic overlaps the atomic round trips.
//   key(i, zt, el) -> false if item i is outside the pass, else sets the tile
//                     hash (and el, the matrix element, if it computed it)
//   val(i, a, b, num, den, el) -> the record of item i
// Where one determinant's terms go, copied out of the instance parameters once
// (the counters and cursors already offset to the instance's first tile), so
// the hot loops hold them in registers whether the parameters live in the
// constant bank or in global memory.
struct EmitOut {
    uint32_t *counts;      // TileCount: terms per tile
    unsigned int *cursor;  // Emit / DetTerms: next slot per tile
    Rec32 *recs;
    uint64_t n_tiles;
    unsigned long long rec_cap;
    uint32_t *err;
    double e0;
};

template <int MODE, class KeyFn, class ValFn>
__device__ __forceinline__ void emit_batch(const EmitOut &p, int i0, int step, int n, KeyFn key, ValFn val)
{
    uint32_t slot[kGenBatch];
    bool ok[kGenBatch];
    double el[kGenBatch];
#pragma unroll
    for (int u = 0; u < kGenBatch; ++u) {
        const int i = i0 + u * step;
        uint64_t zt = 0;
        el[u] = 0.0;
        ok[u] = i < n && key(i, zt, el[u]);
        slot[u] = 0;
        if (ok[u]) {
            if constexpr (MODE == kModeTileCount) {
                red_add_global(&p.counts[__umul64hi(zt, p.n_tiles)], 1u);
            } else if constexpr (MODE == kModeEmit) {
                slot[u] = atom_add_global(&p.cursor[__umul64hi(zt, p.n_tiles)], 1u);
            } else {
                slot[u] = atom_add_global(&p.cursor[0], 1u);
            }
        }
    }
    if constexpr (MODE == kModeEmit || MODE == kModeDetTerms) {
#pragma unroll
        for (int u = 0; u < kGenBatch; ++u) {
            if (!ok[u]) continue;
            if (slot[u] >= p.rec_cap) {  // emission disagrees with the counts
                if constexpr (MODE == kModeEmit) atomicOr(p.err, kErrCount);
                continue;
            }
            uint64_t a, b;
            double num;
            int64_t den;
            val(i0 + u * step, a, b, num, den, el[u]);
            if constexpr (MODE == kModeDetTerms)  // this mode reports H_aa itself (as double bits)
                den = __double_as_longlong(p.e0 - den_to_double(den));
            store_rec32(p.recs + slot[u], a, b, num, den);
        }
    }
}

// All singles and doubles of determinant `det` of one instance (the body of
// both generator kernels).  FILT (kFiltSym | kFiltCut): the instance may be a
// spin-flip symmetric run, or have a numerator cutoff (the checks cost
// registers, so the emission of ordinary runs leaves them out).
template <int MODE, int FILT>
__device__ __forceinline__ void gen_body(const GenParams &p, const uint64_t det)
{
    extern __shared__ __align__(128) unsigned char smem[];
    GenFixed &F = *reinterpret_cast<GenFixed *>(smem);
    int64_t *sa_delta = reinterpret_cast<int64_t *>(smem + p.smem_sa);
    uint64_t *sa_zt = reinterpret_cast<uint64_t *>(sa_delta + p.n_sa);
    uint32_t *sa_info = reinterpret_cast<uint32_t *>(sa_zt + p.n_sa);
    uint16_t *sa_pass = reinterpret_cast<uint16_t *>(sa_info + p.n_sa);
    int64_t *sb_delta = reinterpret_cast<int64_t *>(smem + p.smem_sb);
    uint64_t *sb_zt = reinterpret_cast<uint64_t *>(sb_delta + p.n_sb);
    uint32_t *sb_info = reinterpret_cast<uint32_t *>(sb_zt + p.n_sb);
    uint16_t *sb_pass = reinterpret_cast<uint16_t *>(sb_info + p.n_sb);
    uint16_t *pairs = reinterpret_cast<uint16_t *>(smem + p.smem_pairs);
    int64_t *vec_all = reinterpret_cast<int64_t *>(smem + p.smem_vec);
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem + p.smem_hist);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nw = kGenThreads / 32;
    constexpr bool kVal = MODE == kModeEmit || MODE == kModeDetTerms;
    constexpr bool kCount = MODE == kModeClassCount || MODE == kModeBetaCount;
    // pass membership of a term: alpha class in [class_lo, class_hi) and beta
    // class in [bclass_lo, bclass_hi); most passes take every beta class
    const bool bfull = p.bclass_lo == 0 && p.bclass_hi >= (uint32_t)kNumClasses;
    const uint32_t blo = p.bclass_lo, bhi = p.bclass_hi;
    // spin-flip symmetric run: a term is kept only if its alpha string, as a
    // 64-bit word, is not below its beta string (every mode applies the same rule)
    const bool sym = (FILT & kFiltSym) && p.sym != 0;
    // numerator cutoff (Results section; subsection on the matrix-element
    // cutoff): a contribution c_i H_ai with |c_i H_ai| below it is dropped
    // before its slot is taken, so it gets no record, denominator or sort
    constexpr bool kCut = (FILT & kFiltCut) != 0;
    const double cut = kCut ? p.cutoff : 0.0;
    const bool cutting = kCut && cut > 0.0;
    const int N = p.sys.n;
    const int na = p.na, nb = p.nb, nva = N - na, nvb = N - nb;
    const double *__restrict__ eri = p.sys.eri;
    const int64_t *__restrict__ Jx = p.sys.Jx;
    const int64_t *__restrict__ WSx = p.sys.WSx;
    const double *__restrict__ ht = p.sys.h;
    int64_t *vec = vec_all + warp * kMaxOrb;

    for (int i = tid; i < kMaxOrb; i += kGenThreads) {
        F.zc[i] = p.hash->zc[i];
        F.zcb[i] = p.hash->zcb[i];
        F.zta[i] = p.hash->zta[i];
        F.ztb[i] = p.hash->ztb[i];
    }
    for (int t = tid; t < N * (N - 1) / 2; t += kGenThreads) pairs[t] = p.hash->pairs[t];
    if constexpr (kCount)
        for (int i = tid; i < kNumClasses; i += kGenThreads) hist[i] = 0;
    {
        // occupied and virtual lists, one orbital per thread: its rank among
        // the occupied (virtual) orbitals below it is a population count
        const uint64_t A = p.keys[2 * det], B = p.keys[2 * det + 1];
        if (tid < N) {
            const int q = tid;
            const uint64_t below = (1ull << q) - 1ull;
            const int ra = __popcll(A & below), rb = __popcll(B & below);
            if ((A >> q) & 1ull) F.occA[ra] = q;
            else F.virA[q - ra] = q;
            if ((B >> q) & 1ull) F.occB[rb] = q;
            else F.virB[q - rb] = q;
        }
        if constexpr (kVal)  // g(x) = h_xx + p(x), exact in 2^-48 units, from the reference tables
            for (int i = tid; i < 2 * N; i += kGenThreads) (i < N ? F.gA : F.gB)[i < N ? i : i - N] = p.g[det * 2 * N + i];
        if (tid == 0) {
            F.A = A;
            F.B = B;
            F.c = p.coef[det];
            F.d0 = p.d0[det];
        }
    }
    __syncthreads();
    if (warp == 0) {
        uint64_t zc = 0, za = 0, zb = 0, zcb = 0;
        for (int i = lane; i < na; i += 32) {
            zc ^= F.zc[F.occA[i]];
            za ^= F.zta[F.occA[i]];
        }
        for (int i = lane; i < nb; i += 32) {
            zb ^= F.ztb[F.occB[i]];
            zcb ^= F.zcb[F.occB[i]];
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            zc ^= __shfl_xor_sync(0xffffffffu, zc, off);
            za ^= __shfl_xor_sync(0xffffffffu, za, off);
            zb ^= __shfl_xor_sync(0xffffffffu, zb, off);
            zcb ^= __shfl_xor_sync(0xffffffffu, zcb, off);
        }
        if (lane == 0) {
            F.ZcA = zc;
            F.ZcbB = zcb;
            F.ZtaA = za;
            F.ZtbB = zb;
        }
    }
    __syncthreads();
    const uint64_t A = F.A, B = F.B;
    const double c = F.c;
    const int64_t d0 = F.d0;

    // singles lists; delta = H_aa - H_ii of the single, exact
    for (int s = tid; s < p.n_sa; s += kGenThreads) {
        int i = s / nva, j = s - (s / nva) * nva;
        int r = F.occA[i], a = F.virA[j];
        uint32_t sg = __popcll(A & between_mask(r, a)) & 1;
        uint64_t a2 = A ^ (1ull << r) ^ (1ull << a);
        uint64_t zc = F.ZcA ^ F.zc[r] ^ F.zc[a];
        uint32_t inp;
        if constexpr (MODE == kModeClassCount) {
            inp = cons_ok(p.cons_mod, p.cons_rem, a2);
        } else if constexpr (MODE == kModeBetaCount) {
            inp = class_of(zc) == p.heavy_class && cons_ok(p.cons_mod, p.cons_rem, a2);
        } else {
            uint32_t cl = class_of(zc);
            inp = cl >= p.class_lo && cl < p.class_hi && cons_ok(p.cons_mod, p.cons_rem, a2);
        }
        if constexpr (kVal) sa_delta[s] = F.gA[a] - F.gA[r] - WSx[r * N + a];
        sa_zt[s] = kCount ? zc : (F.ZtaA ^ F.zta[r] ^ F.zta[a]);
        sa_info[s] = (uint32_t)r | ((uint32_t)a << 8) | (sg << 16) | (inp << 17);
    }
    for (int s = tid; s < p.n_sb; s += kGenThreads) {
        int i = s / nvb, j = s - (s / nvb) * nvb;
        int r = F.occB[i], a = F.virB[j];
        uint32_t sg = __popcll(B & between_mask(r, a)) & 1;
        if constexpr (kVal) sb_delta[s] = F.gB[a] - F.gB[r] - WSx[r * N + a];
        const uint64_t zcb = F.ZcbB ^ F.zcb[r] ^ F.zcb[a];  // beta class hash of the excited beta string
        // the beta-count mode histograms beta classes, so it keeps that hash here
        sb_zt[s] = MODE == kModeBetaCount ? zcb : (F.ZtbB ^ F.ztb[r] ^ F.ztb[a]);
        const uint32_t bc = bclass_of(zcb);
        const uint32_t binp = bfull || (bc >= blo && bc < bhi);
        sb_info[s] = (uint32_t)r | ((uint32_t)a << 8) | (sg << 16) | (binp << 17);
    }
    if (tid == 0) {
        bool ok = cons_ok(p.cons_mod, p.cons_rem, A);
        if constexpr (MODE == kModeBetaCount) {
            ok = ok && class_of(F.ZcA) == p.heavy_class;
        } else if constexpr (MODE != kModeClassCount) {
            uint32_t cl = class_of(F.ZcA);
            ok = ok && cl >= p.class_lo && cl < p.class_hi;
        }
        F.a_in_pass = ok;
        const uint32_t bc = bclass_of(F.ZcbB);
        F.b_in_pass = bfull || (bc >= blo && bc < bhi);
    }
    __syncthreads();
    // compact the alpha singles of the pass (warp 0, ballot + popc)
    if (warp == 0) {
        int base = 0;
        for (int s0 = 0; s0 < p.n_sa; s0 += 32) {
            int s = s0 + lane;
            bool f = s < p.n_sa && ((sa_info[s] >> 17) & 1u);
            uint32_t m = __ballot_sync(0xffffffffu, f);
            if (f) sa_pass[base + __popc(m & ((1u << lane) - 1u))] = (uint16_t)s;
            base += __popc(m);
        }
        if (lane == 0) F.n_sa_pass = base;
    } else if (warp == 1 && !bfull) {
        // and the beta singles whose beta class belongs to the pass
        int base = 0;
        for (int s0 = 0; s0 < p.n_sb; s0 += 32) {
            int s = s0 + lane;
            bool f = s < p.n_sb && ((sb_info[s] >> 17) & 1u);
            uint32_t m = __ballot_sync(0xffffffffu, f);
            if (f) sb_pass[base + __popc(m & ((1u << lane) - 1u))] = (uint16_t)s;
            base += __popc(m);
        }
        if (lane == 0) F.n_sb_pass = base;
    }
    __syncthreads();
    const int n_sa_pass = F.n_sa_pass;
    const bool a_in = F.a_in_pass != 0;
    const bool b_in = F.b_in_pass != 0;

    const int n_occ_pairs_a = na * (na - 1) / 2, n_vir_pairs_a = nva * (nva - 1) / 2;
    const int n_occ_pairs_b = nb * (nb - 1) / 2, n_vir_pairs_b = nvb * (nvb - 1) / 2;

    if constexpr (MODE == kModeClassCount) {
        // work list (the paper's first pass over the wavefunction): terms per
        // class.  A run with a numerator cutoff plans from these counts of all
        // terms, an upper bound of what it keeps (the counting modes never
        // evaluate matrix elements)
        if (!sym) {
            if (tid == 0 && a_in)
                atomicAdd(&hist[class_of(F.ZcA)], (uint32_t)(p.n_sb + n_occ_pairs_b * n_vir_pairs_b));
            for (int k = tid; k < n_sa_pass; k += kGenThreads) {
                int s = sa_pass[k];
                atomicAdd(&hist[class_of(sa_zt[s])], (uint32_t)(1 + p.n_sb));
            }
        } else {
            // kept terms only (the drop rule of a symmetric run): an alpha
            // single itself (beta string B) and its alpha-beta doubles, one
            // alpha single per warp
            for (int k = warp; k < n_sa_pass; k += nw) {
                const int s = sa_pass[k];
                const uint64_t a2 = single_word(A, sa_info[s]);
                uint32_t cnt = 0;
                for (int sb = lane; sb < p.n_sb; sb += 32) cnt += single_word(B, sb_info[sb]) <= a2;
                cnt = __reduce_add_sync(0xffffffffu, cnt);
                if (lane == 0) atomicAdd(&hist[class_of(sa_zt[s])], cnt + (a2 >= B ? 1u : 0u));
            }
            if (a_in) {  // beta singles and beta-beta doubles keep alpha string A
                uint32_t cnt = 0;
                for (int sb = tid; sb < p.n_sb; sb += kGenThreads) cnt += single_word(B, sb_info[sb]) <= A;
                for (int pi = warp; pi < n_occ_pairs_b; pi += nw) {
                    const int pr = pairs[pi];
                    const uint64_t b12 = B ^ (1ull << F.occB[pr & 0xFF]) ^ (1ull << F.occB[pr >> 8]);
                    for (int t = lane; t < n_vir_pairs_b; t += 32) {
                        const int pv = pairs[t];
                        cnt += (b12 ^ (1ull << F.virB[pv & 0xFF]) ^ (1ull << F.virB[pv >> 8])) <= A;
                    }
                }
                cnt = __reduce_add_sync(0xffffffffu, cnt);
                if (lane == 0 && cnt) atomicAdd(&hist[class_of(F.ZcA)], cnt);
            }
        }
        for (int pi = warp; pi < n_occ_pairs_a; pi += nw) {
            int pr = pairs[pi];
            int r1 = F.occA[pr & 0xFF], r2 = F.occA[pr >> 8];
            uint64_t z12 = F.ZcA ^ F.zc[r1] ^ F.zc[r2];
            uint64_t a12 = A ^ (1ull << r1) ^ (1ull << r2);
            for (int t = lane; t < n_vir_pairs_a; t += 32) {
                int pv = pairs[t];
                int a1 = F.virA[pv & 0xFF], a2 = F.virA[pv >> 8];
                uint64_t al = a12 ^ (1ull << a1) ^ (1ull << a2);
                if (!cons_ok(p.cons_mod, p.cons_rem, al)) continue;
                if (sym && al < B) continue;
                atomicAdd(&hist[class_of(z12 ^ F.zc[a1] ^ F.zc[a2])], 1u);
            }
        }
        __syncthreads();
        for (int i = tid; i < kNumClasses; i += kGenThreads)
            if (hist[i]) atomicAdd(&p.class_counts[i], (unsigned long long)hist[i]);
        return;
    } else if constexpr (MODE == kModeBetaCount) {
        // beta classes of the terms whose alpha class is the heavy class K:
        // alpha singles and alpha-alpha doubles keep beta = B; beta singles
        // (alpha = A) and alpha-beta doubles (alpha single in K) take the
        // beta string of a beta single; beta-beta doubles one of their own
        const uint32_t K = p.heavy_class;
        const uint32_t per_sb = (uint32_t)n_sa_pass + (a_in ? 1u : 0u);
        if (!sym) {
            if (per_sb)
                for (int sb = tid; sb < p.n_sb; sb += kGenThreads) atomicAdd(&hist[bclass_of(sb_zt[sb])], per_sb);
        } else if (per_sb) {
            // a beta single's string B' is kept under A (if A is in K) and
            // under each alpha single of K that is not below it
            for (int sb = tid; sb < p.n_sb; sb += kGenThreads) {
                const uint64_t b2 = single_word(B, sb_info[sb]);
                uint32_t cnt = a_in && A >= b2;
                for (int k = 0; k < n_sa_pass; ++k) cnt += single_word(A, sa_info[sa_pass[k]]) >= b2;
                if (cnt) atomicAdd(&hist[bclass_of(sb_zt[sb])], cnt);
            }
        }
        uint32_t keepB = 0;  // terms of class K whose beta string is B
        if (tid == 0) {
            if (!sym) {
                keepB = (uint32_t)n_sa_pass;
            } else {
                for (int k = 0; k < n_sa_pass; ++k) keepB += single_word(A, sa_info[sa_pass[k]]) >= B;
            }
        }
        for (int pi = warp; pi < n_occ_pairs_a; pi += nw) {
            int pr = pairs[pi];
            int r1 = F.occA[pr & 0xFF], r2 = F.occA[pr >> 8];
            uint64_t z12 = F.ZcA ^ F.zc[r1] ^ F.zc[r2];
            uint64_t a12 = A ^ (1ull << r1) ^ (1ull << r2);
            for (int t = lane; t < n_vir_pairs_a; t += 32) {
                int pv = pairs[t];
                int a1 = F.virA[pv & 0xFF], a2 = F.virA[pv >> 8];
                if (class_of(z12 ^ F.zc[a1] ^ F.zc[a2]) != K) continue;
                const uint64_t al = a12 ^ (1ull << a1) ^ (1ull << a2);
                if (!cons_ok(p.cons_mod, p.cons_rem, al)) continue;
                if (sym && al < B) continue;
                ++keepB;
            }
        }
        if (keepB) atomicAdd(&hist[bclass_of(F.ZcbB)], keepB);
        if (a_in)
            for (int pi = warp; pi < n_occ_pairs_b; pi += nw) {
                int pr = pairs[pi];
                int r1 = F.occB[pr & 0xFF], r2 = F.occB[pr >> 8];
                uint64_t z12 = F.ZcbB ^ F.zcb[r1] ^ F.zcb[r2];
                const uint64_t b12 = B ^ (1ull << r1) ^ (1ull << r2);
                for (int t = lane; t < n_vir_pairs_b; t += 32) {
                    int pv = pairs[t];
                    const int v1 = F.virB[pv & 0xFF], v2 = F.virB[pv >> 8];
                    if (sym && (b12 ^ (1ull << v1) ^ (1ull << v2)) > A) continue;
                    atomicAdd(&hist[bclass_of(z12 ^ F.zcb[v1] ^ F.zcb[v2])], 1u);
                }
            }
        __syncthreads();
        for (int i = tid; i < kNumClasses; i += kGenThreads)
            if (hist[i]) atomicAdd(&p.class_counts[i], (unsigned long long)hist[i]);
        return;
    } else {
        const uint64_t ZtaA = F.ZtaA, ZtbB = F.ZtbB;
        EmitOut out;
        out.counts = MODE == kModeTileCount ? p.tile_counts + p.tile_base : nullptr;
        out.cursor = MODE == kModeEmit ? p.cursor + p.tile_base : p.cursor;
        out.recs = p.recs;
        out.n_tiles = p.n_tiles;
        out.rec_cap = p.rec_cap;
        out.err = p.err;
        out.e0 = p.e0;
        const uint32_t class_lo = p.class_lo, class_hi = p.class_hi;
        const uint64_t cons_mod = p.cons_mod, cons_rem = p.cons_rem;
        // beta singles of the pass: all of them, or the compacted list
        const int n_sb = bfull ? p.n_sb : F.n_sb_pass;
        auto sb_at = [&](int k) { return bfull ? k : (int)sb_pass[k]; };

        // bucket table of the virtual alpha pairs, and the pass's classes as
        // aligned blocks of bucket groups
        uint32_t *vb_cnt = reinterpret_cast<uint32_t *>(smem + p.smem_hist);
        uint16_t *vb_off = reinterpret_cast<uint16_t *>(vb_cnt + kVbkBuckets);
        uint16_t *vb_list = vb_off + kVbkBuckets + 1;
        uint16_t *vb_warp = vb_list + kMaxVirPairs;
        if (b_in) {  // uniform across the CTA
            if (tid == 0) {
                constexpr int gs = kClassBits - kVbkBits;
                uint32_t g = class_lo >> gs;
                const uint32_t g1 = ((class_hi - 1) >> gs) + 1;
                int nb = 0;
                while (g < g1) {
                    int k = kVbkBits;
                    while (k > 0 && ((g & ((1u << k) - 1u)) != 0 || g + (1u << k) > g1)) --k;
                    F.blk_g[nb] = (uint16_t)g;
                    F.blk_k[nb] = (uint8_t)k;
                    ++nb;
                    g += 1u << k;
                }
                F.n_blk = nb;
            }
            for (int b = tid; b < kVbkBuckets; b += kGenThreads) vb_cnt[b] = 0;
            __syncthreads();
            for (int t = tid; t < n_vir_pairs_a; t += kGenThreads) {
                const int pv = pairs[t];
                atomicAdd(&vb_cnt[vb_bucket(F.zc[F.virA[pv & 0xFF]] ^ F.zc[F.virA[pv >> 8]])], 1u);
            }
            __syncthreads();
            {
                const uint4 c4 = reinterpret_cast<const uint4 *>(vb_cnt)[tid];
                const uint32_t sum = c4.x + c4.y + c4.z + c4.w;
                uint32_t incl = sum;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
                    if (lane >= off) incl += v;
                }
                if (lane == 31) F.wsum[warp] = incl;
                __syncthreads();
                uint32_t run = incl - sum;
#pragma unroll
                for (int k = 0; k < nw; ++k) run += k < warp ? F.wsum[k] : 0u;
                const uint32_t c[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    vb_off[4 * tid + k] = (uint16_t)run;
                    vb_cnt[4 * tid + k] = run;  // scatter cursor
                    run += c[k];
                }
                if (tid == kGenThreads - 1) vb_off[kVbkBuckets] = (uint16_t)run;
            }
            __syncthreads();
            for (int t = tid; t < n_vir_pairs_a; t += kGenThreads) {
                const int pv = pairs[t];
                const uint32_t b = vb_bucket(F.zc[F.virA[pv & 0xFF]] ^ F.zc[F.virA[pv >> 8]]);
                vb_list[atomicAdd(&vb_cnt[b], 1u)] = (uint16_t)t;
            }
            __syncthreads();
        }

        // ---- alpha singles (few per determinant: O(n) element each); beta string B
        if (b_in)
        for (int k0 = tid; k0 < n_sa_pass; k0 += kGenThreads * kGenBatch)
            emit_batch<MODE>(
                out, k0, kGenThreads, n_sa_pass,
                [&](int k, uint64_t &zt, double &el) {
                    const int s = sa_pass[k];
                    if (sym && single_word(A, sa_info[s]) < B) return false;
                    if (cutting) {
                        const uint32_t info = sa_info[s];
                        el = single_value(ht, eri, N, F.occA, na, F.occB, nb, info & 0xFF, (info >> 8) & 0xFF);
                        if (!above_cut(c, el, cut)) return false;
                    }
                    zt = sa_zt[s] ^ ZtbB;
                    return true;
                },
                [&](int k, uint64_t &ka, uint64_t &kb, double &num, int64_t &den, double el) {
                    const int s = sa_pass[k];
                    const uint32_t info = sa_info[s];
                    const int r = info & 0xFF, a = (info >> 8) & 0xFF;
                    const double v = cutting ? el : single_value(ht, eri, N, F.occA, na, F.occB, nb, r, a);
                    ka = A ^ (1ull << r) ^ (1ull << a);
                    kb = B;
                    num = flip_sign(c * v, info >> 16);
                    den = d0 - sa_delta[s];
                });
        // ---- beta singles
        if (a_in)
            for (int s0 = tid; s0 < n_sb; s0 += kGenThreads * kGenBatch)
                emit_batch<MODE>(
                    out, s0, kGenThreads, n_sb,
                    [&](int k, uint64_t &zt, double &el) {
                        const int s = sb_at(k);
                        if (sym && single_word(B, sb_info[s]) > A) return false;
                        if (cutting) {
                            const uint32_t info = sb_info[s];
                            el = single_value(ht, eri, N, F.occB, nb, F.occA, na, info & 0xFF, (info >> 8) & 0xFF);
                            if (!above_cut(c, el, cut)) return false;
                        }
                        zt = ZtaA ^ sb_zt[s];
                        return true;
                    },
                    [&](int k, uint64_t &ka, uint64_t &kb, double &num, int64_t &den, double el) {
                        const int s = sb_at(k);
                        const uint32_t info = sb_info[s];
                        const int r = info & 0xFF, a = (info >> 8) & 0xFF;
                        const double v = cutting ? el : single_value(ht, eri, N, F.occB, nb, F.occA, na, r, a);
                        ka = A;
                        kb = B ^ (1ull << r) ^ (1ull << a);
                        num = flip_sign(c * v, info >> 16);
                        den = d0 - sb_delta[s];
                    });
        // ---- alpha-beta doubles: one alpha single per warp, beta singles over lanes
        for (int k = warp; k < n_sa_pass; k += nw) {
            const int s = sa_pass[k];
            const uint32_t info = sa_info[s];
            const int rA = info & 0xFF, aA = (info >> 8) & 0xFF;
            const uint64_t a2 = A ^ (1ull << rA) ^ (1ull << aA);
            const uint64_t ztA = sa_zt[s];
            int64_t baseD = 0;
            double cA = 0.0;
            // (aA rA|aB rB) = (rA aA|rB aB): lanes take consecutive beta
            // singles (same rB, ascending aB), so this layout is contiguous
            const double *slice = eri + ((size_t)rA * N + aA) * N * N;
            if constexpr (kVal) {
                // u[q] = J(aA, q) - J(rA, q): the alpha-beta cross terms of H_aa
                for (int q = lane; q < N; q += 32) vec[q] = Jx[aA * N + q] - Jx[rA * N + q];
                __syncwarp();
                baseD = d0 - sa_delta[s];
                cA = flip_sign(c, info >> 16);
            }
            for (int sb0 = lane; sb0 < n_sb; sb0 += 32 * kGenBatch)
                emit_batch<MODE>(
                    out, sb0, 32, n_sb,
                    [&](int k, uint64_t &zt, double &el) {
                        const int sb = sb_at(k);
                        if (sym && single_word(B, sb_info[sb]) > a2) return false;
                        if (cutting) {
                            const uint32_t bi = sb_info[sb];
                            el = __ldg(slice + (bi & 0xFF) * N + ((bi >> 8) & 0xFF));
                            if (!above_cut(c, el, cut)) return false;
                        }
                        zt = ztA ^ sb_zt[sb];
                        return true;
                    },
                    [&](int k, uint64_t &ka, uint64_t &kb, double &num, int64_t &den, double el) {
                        const int sb = sb_at(k);
                        const uint32_t bi = sb_info[sb];
                        const int rB = bi & 0xFF, aB = (bi >> 8) & 0xFF;
                        ka = a2;
                        kb = B ^ (1ull << rB) ^ (1ull << aB);
                        num = flip_sign(cA * (cutting ? el : __ldg(slice + rB * N + aB)), bi >> 16);
                        den = baseD - sb_delta[sb] - (vec[aB] - vec[rB]);
                    });
            __syncwarp();
        }
        // ---- same-spin doubles: one occupied pair per warp, virtual pairs over lanes
        for (int spin = 0; spin < 2; ++spin) {
            if (spin == 0 && !b_in) continue;  // alpha-alpha doubles keep beta string B
            if (spin == 1 && !a_in) break;
            const int npo = spin ? n_occ_pairs_b : n_occ_pairs_a;
            const int npv = spin ? n_vir_pairs_b : n_vir_pairs_a;
            const int *occ = spin ? F.occB : F.occA;
            const int *vir = spin ? F.virB : F.virA;
            const int nv = spin ? nvb : nva;
            const int64_t *g = spin ? F.gB : F.gA;
            const uint64_t W = spin ? B : A;
            for (int pi = warp; pi < npo; pi += nw) {
                const int pr = pairs[pi];
                const int r1 = occ[pr & 0xFF], r2 = occ[pr >> 8];
                const uint64_t w12 = W ^ (1ull << r1) ^ (1ull << r2);
                const uint64_t zc12 = F.ZcA ^ F.zc[r1] ^ F.zc[r2];
                const uint64_t zcb12 = F.ZcbB ^ F.zcb[r1] ^ F.zcb[r2];
                const uint64_t zt12 =
                    spin ? (ZtaA ^ ZtbB ^ F.ztb[r1] ^ F.ztb[r2]) : (ZtaA ^ ZtbB ^ F.zta[r1] ^ F.zta[r2]);
                // items: every virtual beta pair, or the alpha pairs of the bucket
                // ranges the pass's blocks map to (block xor top bits of zc12)
                const bool nar = spin == 0;
                int nitems = npv, nq = 0;
                uint16_t *ws = vb_warp + warp * 64;  // [0, 32): slice starts, [32, 64): item offsets
                if (nar) {
                    const uint32_t u = vb_bucket(zc12);
                    nq = F.n_blk;
                    uint32_t start = 0, sz = 0;
                    if (lane < nq) {
                        const uint32_t k = F.blk_k[lane];
                        const uint32_t b = (F.blk_g[lane] ^ u) & ~((1u << k) - 1u);
                        start = vb_off[b];
                        sz = (uint32_t)vb_off[b + (1u << k)] - start;
                    }
                    uint32_t incl = sz;
#pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
                        if (lane >= off) incl += v;
                    }
                    if (lane < nq) {
                        ws[lane] = (uint16_t)start;
                        ws[32 + lane] = (uint16_t)(incl - sz);
                    }
                    nitems = (int)__shfl_sync(0xffffffffu, incl, 31);
                    __syncwarp();
                }
                if (nitems == 0) continue;  // uniform across the warp
                int64_t base = 0;
                if constexpr (kVal) {
                    // H_aa - H_ii = -g(r1) - g(r2) + W(r1,r2) + v(a1) + v(a2) + W(a1,a2),
                    // v(x) = g(x) - W(r1,x) - W(r2,x)
                    for (int j = lane; j < nv; j += 32) {
                        int x = vir[j];
                        vec[j] = g[x] - WSx[r1 * N + x] - WSx[r2 * N + x];
                    }
                    __syncwarp();
                    base = d0 + g[r1] + g[r2] - WSx[r1 * N + r2];
                }
                // the same emission over items mapped to virtual pairs by `pair_at`
                // (instantiated separately for the direct and the bucketed case)
                auto emit_pairs = [&](int n_items, auto pair_at) {
                    for (int t0 = lane; t0 < n_items; t0 += 32 * kGenBatch)
                        emit_batch<MODE>(
                            out, t0, 32, n_items,
                            [&](int i, uint64_t &zt, double &el) {
                                const int t = pair_at(i);
                                const int pv = pairs[t];
                                const int a1 = vir[pv & 0xFF], a2 = vir[pv >> 8];
                                if (spin == 0) {
                                    uint32_t cl = class_of(zc12 ^ F.zc[a1] ^ F.zc[a2]);
                                    if (cl < class_lo || cl >= class_hi) return false;
                                    const uint64_t w2 = w12 ^ (1ull << a1) ^ (1ull << a2);
                                    if (!cons_ok(cons_mod, cons_rem, w2)) return false;
                                    if (sym && w2 < B) return false;
                                    if (cutting) {
                                        el = same_double_value(eri, N, r1, r2, a1, a2);
                                        if (!above_cut(c, el, cut)) return false;
                                    }
                                    zt = zt12 ^ F.zta[a1] ^ F.zta[a2];
                                } else {
                                    if (!bfull) {
                                        const uint32_t bc = bclass_of(zcb12 ^ F.zcb[a1] ^ F.zcb[a2]);
                                        if (bc < blo || bc >= bhi) return false;
                                    }
                                    if (sym && (w12 ^ (1ull << a1) ^ (1ull << a2)) > A) return false;
                                    if (cutting) {
                                        el = same_double_value(eri, N, r1, r2, a1, a2);
                                        if (!above_cut(c, el, cut)) return false;
                                    }
                                    zt = zt12 ^ F.ztb[a1] ^ F.ztb[a2];
                                }
                                return true;
                            },
                            [&](int i, uint64_t &ka, uint64_t &kb, double &num, int64_t &den, double el) {
                                const int t = pair_at(i);
                                const int pv = pairs[t];
                                const int j1 = pv & 0xFF, j2 = pv >> 8;
                                const int a1 = vir[j1], a2 = vir[j2];
                                const uint64_t w2 = w12 ^ (1ull << a1) ^ (1ull << a2);
                                ka = spin ? A : w2;
                                kb = spin ? w2 : B;
                                const uint64_t w1 = W ^ (1ull << r1) ^ (1ull << a1);
                                const uint32_t par =
                                    __popcll(W & between_mask(r1, a1)) + __popcll(w1 & between_mask(r2, a2));
                                // a1 is the fastest-varying index across lanes
                                const double e = cutting ? el : same_double_value(eri, N, r1, r2, a1, a2);
                                num = flip_sign(c * e, par);
                                den = base - vec[j1] - vec[j2] - __ldg(WSx + a1 * N + a2);
                            });
                };
                if (nar)
                    emit_pairs(nitems, [&](int i) -> int {
                        int lo = 0, hi = nq;  // last slice whose offset is at most i
                        while (hi - lo > 1) {
                            const int mid = (lo + hi) >> 1;
                            if ((int)ws[32 + mid] <= i) lo = mid;
                            else hi = mid;
                        }
                        return vb_list[ws[lo] + (i - (int)ws[32 + lo])];
                    });
                else
                    emit_pairs(npv, [](int i) -> int { return i; });
                __syncwarp();
            }
        }
    }
}

// Generator over the determinants of several instances (one CTA each).
// Four CTAs per SM (64 registers): more warps hide the L2 round trips of the
// slot atomics.  The emission with the cutoff, which carries each term's
// matrix element from the key phase to the store phase, gets three (80 registers).
template <int MODE, int FILT>
__global__ void __launch_bounds__(kGenThreads, (MODE == kModeEmit && (FILT & kFiltCut)) ? 3 : 4)
    gen_kernel(const GenBatch b)
{
    if (b.n_inst == 1) {
        gen_body<MODE, FILT>(b.one, b.one.det_begin + b.cta_offset + blockIdx.x);
        return;
    }
    // instance of this CTA (thread 0 searches, the others read the result);
    // its parameters are read in place through the read-only data path
    __shared__ int sinst;
    __shared__ unsigned long long sdet;
    if (threadIdx.x == 0) {
        const unsigned long long g = b.cta_offset + blockIdx.x;
        int lo = 0, hi = b.n_inst;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (b.det_base[mid] <= g) lo = mid;
            else hi = mid;
        }
        sinst = lo;
        sdet = b.params[lo].det_begin + (g - b.det_base[lo]);
    }
    __syncthreads();
    const GenParams *__restrict__ gp = b.params + sinst;
    gen_body<MODE, FILT>(*gp, sdet);
}

// Generator for one determinant with its parameters passed by value.
template <int MODE>
__global__ void __launch_bounds__(kGenThreads, 3) gen_kernel_one(const GenParams p)
{
    gen_body<MODE, 0>(p, p.det_begin);
}

// ============================================================= diagonal

__global__ void diag_kernel(const SysDev sys, const uint64_t *__restrict__ keys, uint64_t n,
                            double *__restrict__ out)
{
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int N = sys.n;
    uint64_t A = keys[2 * i], B = keys[2 * i + 1];
    double e = 0.0;
    for (uint64_t x = A; x; x &= x - 1) {
        int p = __ffsll((long long)x) - 1;
        e += sys.h[p * N + p];
        for (uint64_t y = x & (x - 1); y; y &= y - 1) e += sys.WS[p * N + (__ffsll((long long)y) - 1)];
        for (uint64_t y = B; y; y &= y - 1) e += sys.J[p * N + (__ffsll((long long)y) - 1)];
    }
    for (uint64_t x = B; x; x &= x - 1) {
        int p = __ffsll((long long)x) - 1;
        e += sys.h[p * N + p];
        for (uint64_t y = x & (x - 1); y; y &= y - 1) e += sys.WS[p * N + (__ffsll((long long)y) - 1)];
    }
    out[i] = e;
}

__global__ void ref_d0_kernel(const double *__restrict__ hii, uint64_t n, double e0, int64_t *__restrict__ d0)
{
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    d0[i] = __double2ll_rn((e0 - hii[i]) * kDenScale);
}

// g(x) = h_xx + p(x) of every reference determinant, p(x) = sum over its
// occupied spin-orbitals j of <xj||xj> (the appendix on fast diagonals), exact
// in 2^-48 Ha: alpha x takes same-spin pair energies with the alpha electrons
// and Coulomb energies with the beta ones, and conversely.  One CTA of kMaxOrb
// threads per determinant; computed once per reference, read by every pass.
__global__ void ref_g_kernel(const SysDev sys, const uint64_t *__restrict__ keys, uint64_t n,
                             int64_t *__restrict__ g)
{
    const uint64_t det = blockIdx.x;
    const int N = sys.n, x = threadIdx.x;
    if (det >= n || x >= N) return;
    const uint64_t A = keys[2 * det], B = keys[2 * det + 1];
    int64_t ga = sys.hdx[x], gb = sys.hdx[x];
    for (uint64_t m = A; m; m &= m - 1) {
        const int k = __ffsll((long long)m) - 1;
        ga += sys.WSx[x * N + k];
        gb += sys.Jx[x * N + k];
    }
    for (uint64_t m = B; m; m &= m - 1) {
        const int k = __ffsll((long long)m) - 1;
        ga += sys.Jx[x * N + k];
        gb += sys.WSx[x * N + k];
    }
    g[det * 2 * N + x] = ga;
    g[det * 2 * N + N + x] = gb;
}

cudaError_t launch_ref_g(const SysDev &sys, const uint64_t *keys, uint64_t n, int64_t *g, cudaStream_t s)
{
    for (uint64_t o = 0; o < n; o += (1ull << 30)) {
        const uint64_t m = n - o < (1ull << 30) ? n - o : (1ull << 30);
        ref_g_kernel<<<(unsigned)m, kMaxOrb, 0, s>>>(sys, keys + 2 * o, m, g + o * 2 * sys.n);
    }
    return cudaGetLastError();
}

cudaError_t launch_ref_d0(const double *hii, uint64_t n, double e0, int64_t *d0, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    ref_d0_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(hii, n, e0, d0);
    return cudaGetLastError();
}

// ================================================================ scans

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

size_t scan_tmp_elems(uint64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

__device__ void block_scan_excl_u64(unsigned long long local_sum, unsigned long long &prefix,
                                    unsigned long long *warp_tot, unsigned long long &total)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    unsigned long long incl = local_sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        unsigned long long t = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = lane < nw ? warp_tot[lane] : 0ull;
        unsigned long long wi = w;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            unsigned long long t = __shfl_up_sync(0xffffffffu, wi, off);
            if (lane >= off) wi += t;
        }
        if (lane < nw) warp_tot[lane] = wi - w;
        if (lane == nw - 1) warp_tot[32] = wi;
    }
    __syncthreads();
    prefix = warp_tot[warp] + incl - local_sum;
    total = warp_tot[32];
    __syncthreads();
}

__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(const uint32_t *__restrict__ in, uint64_t n,
                                                                 unsigned long long *__restrict__ part)
{
    __shared__ unsigned long long wt[33];
    uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += in[base + k];
    unsigned long long pre, tot;
    block_scan_excl_u64(s, pre, wt, tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) scan_parts_kernel(unsigned long long *part, uint64_t nparts)
{
    __shared__ unsigned long long wt[33];
    unsigned long long carry = 0;
    for (uint64_t b0 = 0; b0 < nparts; b0 += kScanThreads) {
        uint64_t i = b0 + threadIdx.x;
        unsigned long long v = i < nparts ? part[i] : 0ull;
        unsigned long long pre, tot;
        block_scan_excl_u64(v, pre, wt, tot);
        if (i < nparts) part[i] = carry + pre;
        carry += tot;
    }
    if (threadIdx.x == 0) part[nparts] = carry;
}

__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const uint32_t *__restrict__ in, uint64_t n,
                                                                  const unsigned long long *__restrict__ part,
                                                                  uint64_t nparts,
                                                                  unsigned long long *__restrict__ out,
                                                                  uint32_t *__restrict__ out32)
{
    __shared__ unsigned long long wt[33];
    uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
    unsigned long long v[kScanItems];
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? in[base + k] : 0ull;
        s += v[k];
    }
    unsigned long long pre, tot;
    block_scan_excl_u64(s, pre, wt, tot);
    unsigned long long run = part[blockIdx.x] + pre;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) {
            out[base + k] = run;
            if (out32) out32[base + k] = (uint32_t)run;
        }
        run += v[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = part[nparts];
}

cudaError_t launch_scan_u32_to_u64(const uint32_t *in, unsigned long long *out, uint32_t *out32, uint64_t n,
                                   unsigned long long *tmp, cudaStream_t s)
{
    uint64_t nparts = (n + kScanTile - 1) / kScanTile;
    if (nparts == 0) return cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
    scan_sums_kernel<<<(unsigned)nparts, kScanThreads, 0, s>>>(in, n, tmp);
    scan_parts_kernel<<<1, kScanThreads, 0, s>>>(tmp, nparts);
    scan_apply_kernel<<<(unsigned)nparts, kScanThreads, 0, s>>>(in, n, tmp, nparts, out, out32);
    return cudaGetLastError();
}

// ===================================================== reference partition

__device__ __forceinline__ int ref_instance(const RefPartParams &p, uint64_t g)
{
    int lo = 0, hi = p.n_inst;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (p.ref_base[mid] <= g) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void ref_tile_kernel(const RefPartParams p)
{
    const uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (g >= p.n_total) return;
    const int inst = ref_instance(p, g);
    const GenParams &q = p.params[inst];
    const uint64_t i = g - p.ref_base[inst];
    const uint64_t A = q.keys[2 * i], B = q.keys[2 * i + 1];
    uint64_t zc = 0, zt = 0;
    for (uint64_t x = A; x; x &= x - 1) {
        int k = __ffsll((long long)x) - 1;
        zc ^= p.hash->zc[k];
        zt ^= p.hash->zta[k];
    }
    uint64_t zcb = 0;
    for (uint64_t x = B; x; x &= x - 1) {
        int k = __ffsll((long long)x) - 1;
        zt ^= p.hash->ztb[k];
        zcb ^= p.hash->zcb[k];
    }
    const uint32_t cl = class_of(zc), bc = bclass_of(zcb);
    uint32_t t = 0xFFFFFFFFu;
    // a run with duplicate subtraction keeps the reference keys in the sum
    if (!q.subtract && cl >= q.class_lo && cl < q.class_hi && bc >= q.bclass_lo && bc < q.bclass_hi &&
        cons_ok(q.cons_mod, q.cons_rem, A)) {
        t = (uint32_t)(q.tile_base + __umul64hi(zt, q.n_tiles));
        atomicAdd(&p.ref_count[t], 1u);
    }
    p.ref_tile[g] = t;
}

__global__ void ref_scatter_kernel(const RefPartParams p)
{
    const uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (g >= p.n_total) return;
    const uint32_t t = p.ref_tile[g];
    if (t == 0xFFFFFFFFu) return;
    const int inst = ref_instance(p, g);
    const GenParams &q = p.params[inst];
    const uint64_t i = g - p.ref_base[inst];
    const unsigned long long slot = atomicAdd(&p.ref_cursor[t], 1ull);
    p.ref_keys_out[2 * slot] = q.keys[2 * i];
    p.ref_keys_out[2 * slot + 1] = q.keys[2 * i + 1];
}

cudaError_t launch_ref_partition(const RefPartParams &p, int phase, cudaStream_t s)
{
    const unsigned g = (unsigned)((p.n_total + 255) / 256);
    if (g == 0) return cudaSuccess;
    if (phase == 0) ref_tile_kernel<<<g, 256, 0, s>>>(p);
    else ref_scatter_kernel<<<g, 256, 0, s>>>(p);
    return cudaGetLastError();
}

// Sort each tile's reference slice by key (slices are short: insertion sort).
__global__ void sort_slices_kernel(const unsigned long long *__restrict__ off, uint64_t *keys, uint64_t n_tiles)
{
    uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    unsigned long long s = off[t], e = off[t + 1];
    for (unsigned long long i = s + 1; i < e; ++i) {
        uint64_t a = keys[2 * i], b = keys[2 * i + 1];
        unsigned long long j = i;
        while (j > s && key_less(a, b, keys[2 * (j - 1)], keys[2 * (j - 1) + 1])) {
            keys[2 * j] = keys[2 * (j - 1)];
            keys[2 * j + 1] = keys[2 * (j - 1) + 1];
            --j;
        }
        keys[2 * j] = a;
        keys[2 * j + 1] = b;
    }
}

cudaError_t launch_sort_slices(const unsigned long long *ref_off, uint64_t *ref_keys, uint64_t n_tiles,
                               cudaStream_t s)
{
    unsigned g = (unsigned)((n_tiles + 255) / 256);
    if (g == 0) return cudaSuccess;
    sort_slices_kernel<<<g, 256, 0, s>>>(ref_off, ref_keys, n_tiles);
    return cudaGetLastError();
}

// ============================================================ tile kernels

// Per-thread statistics, all exact integers.
struct KeyStats {
    uint64_t e2_lo;
    int64_t e2_hi;
    uint64_t dsum, dxor, min_den;
    uint32_t n_unique, n_in_ref, n_ext, n_pos;
    uint32_t err;
    __device__ void clear()
    {
        e2_lo = 0;
        e2_hi = 0;
        dsum = dxor = 0;
        min_den = ~0ull;
        n_unique = n_in_ref = n_ext = n_pos = 0;
        err = 0;
    }
};

// Group `cnt` keys held in shared memory so that equal keys are adjacent:
// counting sort by a key hash into B buckets (B a power of two, about cnt/2),
// then within each bucket equal keys are gathered: small buckets by an
// insertion sort on the 128-bit key (alpha word most significant), large ones
// (a key with many duplicates) by repeated warp-wide partitions.  On return
// perm[0..cnt) lists record indices bucket by bucket with equal keys
// contiguous.  hist must be zero on entry and is left zero.
template <class KeyAt>
__device__ void group_keys(int cnt, int max_buckets, KeyAt key, uint16_t *perm, uint16_t *rnk, uint16_t *bkt,
                           uint32_t *hist, uint32_t *warp_tot, unsigned int *nbig)
{
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    int B = 32;
    while (2 * B < cnt && B < max_buckets) B <<= 1;
    if (tid == 0) *nbig = 0;
    for (int i = tid; i < cnt; i += nt) {
        uint64_t a, b;
        key(i, a, b);
        const uint32_t bb = bucket_hash(a, b) & (uint32_t)(B - 1);
        bkt[i] = (uint16_t)bb;
        rnk[i] = (uint16_t)atomicAdd(&hist[bb], 1u);
    }
    __syncthreads();
    block_scan_excl_u32(hist, B, warp_tot);
    for (int i = tid; i < cnt; i += nt) perm[hist[bkt[i]] + rnk[i]] = (uint16_t)i;
    __syncthreads();
    // small buckets: one thread each; large ones are queued for a warp (bkt is free now)
    for (int bb = tid; bb < B; bb += nt) {
        const int s = (int)hist[bb];
        const int e = bb + 1 < B ? (int)hist[bb + 1] : cnt;
        if (e - s <= 1) continue;
        if (e - s > 24) {
            bkt[atomicAdd(nbig, 1u)] = (uint16_t)bb;
            continue;
        }
        uint64_t la, lb;  // last key of the sorted prefix
        key(perm[s], la, lb);
        for (int i = s + 1; i < e; ++i) {
            const uint16_t x = perm[i];
            uint64_t a, b;
            key(x, a, b);
            if (!key_less(a, b, la, lb)) {
                la = a;
                lb = b;
                continue;
            }
            int j = i;
            while (j > s) {
                uint64_t pa, pb;
                key(perm[j - 1], pa, pb);
                if (!key_less(a, b, pa, pb)) break;
                perm[j] = perm[j - 1];
                --j;
            }
            perm[j] = x;
        }
    }
    __syncthreads();
    const int nb = (int)*nbig;
    for (int q = warp; q < nb; q += nw) {
        const int bb = bkt[q];
        const int s = (int)hist[bb];
        const int e = bb + 1 < B ? (int)hist[bb + 1] : cnt;
        int pos = s;
        while (pos < e) {
            uint64_t ka, kb;
            key(perm[pos], ka, kb);
            int n_eq = 0, n_ne = 0;
            for (int base = pos; base < e; base += 32) {
                const int j = base + lane;
                uint16_t x = 0;
                bool eq = false;
                if (j < e) {
                    x = perm[j];
                    uint64_t a, b;
                    key(x, a, b);
                    eq = a == ka && b == kb;
                }
                const unsigned m_eq = __ballot_sync(0xffffffffu, j < e && eq);
                const unsigned m_ne = __ballot_sync(0xffffffffu, j < e && !eq);
                const unsigned lt = (1u << lane) - 1u;
                if (j < e) {
                    if (eq) rnk[pos + n_eq + __popc(m_eq & lt)] = x;
                    else rnk[e - 1 - (n_ne + __popc(m_ne & lt))] = x;
                }
                n_eq += __popc(m_eq);
                n_ne += __popc(m_ne);
            }
            __syncwarp();
            for (int j = pos + lane; j < e; j += 32) perm[j] = rnk[j];
            __syncwarp();
            pos += n_eq;
        }
    }
    __syncthreads();
    for (int i = tid; i < B; i += nt) hist[i] = 0;  // ready for the next call
}

__device__ __forceinline__ bool in_slice(const uint64_t *rk, unsigned long long n, uint64_t a, uint64_t b)
{
    unsigned long long lo = 0, hi = n;
    while (lo < hi) {
        unsigned long long mid = (lo + hi) >> 1;
        uint64_t ma = rk[2 * mid], mb = rk[2 * mid + 1];
        if (ma == a && mb == b) return true;
        if (key_less(ma, mb, a, b)) lo = mid + 1;
        else hi = mid;
    }
    return false;
}

// One unique key: explicit filter against the reference slice, then the
// Epstein-Nesbet term num^2 / (E0 - H_aa) of Eq. 3, added exactly.
// In a spin-flip symmetric run (sym) a key with a > b stands for itself and
// its mirror (b, a), whose term is the same, so it counts twice.
__device__ __forceinline__ void finish_key(const TileParams &p, double e0, bool sym, const uint64_t *rk,
                                           unsigned long long nrk, uint64_t a, uint64_t b, double num, int64_t den,
                                           KeyStats &st)
{
    st.n_unique++;
    if (in_slice(rk, nrk, a, b)) {
        st.n_in_ref++;
        return;
    }
    double d = den_to_double(den);
    double term = (num * num) * recip(d, den);
    if (sym && a != b) term += term;
    fx_add_double(st.e2_lo, st.e2_hi, term, st.err);
    st.n_ext++;
    uint64_t ad = den < 0 ? (uint64_t)(-den) : (uint64_t)den;
    st.min_den = ad < st.min_den ? ad : st.min_den;
    st.n_pos += den > 0;
    st.dsum += digest1(a, b);
    st.dxor ^= digest2(a, b);
    if (p.dump_keys) {
        unsigned long long slot = atomicAdd(p.dump_count, 1ull);
        if (slot < p.dump_cap) {
            p.dump_keys[2 * slot] = a;
            p.dump_keys[2 * slot + 1] = b;
            p.dump_num[slot] = num;
            p.dump_haa[slot] = e0 - d;
        }
    }
}

// Sum the per-thread statistics of the CTA and add them to an instance's total.
__device__ void flush_stats(const TileParams &p, RunAcc *acc, KeyStats st, unsigned long long (*red)[32])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        uint64_t olo = __shfl_down_sync(0xffffffffu, st.e2_lo, off);
        int64_t ohi = __shfl_down_sync(0xffffffffu, st.e2_hi, off);
        fx_add_fx(st.e2_lo, st.e2_hi, olo, ohi);
        st.dsum += __shfl_down_sync(0xffffffffu, st.dsum, off);
        st.dxor ^= __shfl_down_sync(0xffffffffu, st.dxor, off);
        uint64_t om = __shfl_down_sync(0xffffffffu, st.min_den, off);
        st.min_den = om < st.min_den ? om : st.min_den;
        st.n_unique += __shfl_down_sync(0xffffffffu, st.n_unique, off);
        st.n_in_ref += __shfl_down_sync(0xffffffffu, st.n_in_ref, off);
        st.n_ext += __shfl_down_sync(0xffffffffu, st.n_ext, off);
        st.n_pos += __shfl_down_sync(0xffffffffu, st.n_pos, off);
        st.err |= __shfl_down_sync(0xffffffffu, st.err, off);
    }
    if (lane == 0) {
        red[0][warp] = st.e2_lo;
        red[1][warp] = (unsigned long long)st.e2_hi;
        red[2][warp] = st.dsum;
        red[3][warp] = st.dxor;
        red[4][warp] = st.min_den;
        red[5][warp] = st.n_unique;
        red[6][warp] = st.n_in_ref;
        red[7][warp] = st.n_ext;
        red[8][warp] = st.n_pos;
        red[9][warp] = st.err;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t lo = 0, dsum = 0, dxor = 0, mind = ~0ull, nu = 0, nr = 0, ne = 0, np = 0, er = 0;
        int64_t hi = 0;
        for (int w = 0; w < nw; ++w) {
            fx_add_fx(lo, hi, red[0][w], (int64_t)red[1][w]);
            dsum += red[2][w];
            dxor ^= red[3][w];
            mind = red[4][w] < mind ? red[4][w] : mind;
            nu += red[5][w];
            nr += red[6][w];
            ne += red[7][w];
            np += red[8][w];
            er |= red[9][w];
        }
        unsigned long long old = atomicAdd(&acc->e2_lo, (unsigned long long)lo);
        unsigned long long carry = (old + lo) < old ? 1ull : 0ull;
        atomicAdd((unsigned long long *)&acc->e2_hi, (unsigned long long)hi + carry);
        atomicAdd(&acc->dsum, dsum);
        atomicXor(&acc->dxor, dxor);
        atomicMin(&acc->min_den, mind);
        atomicAdd(&acc->n_unique, nu);
        atomicAdd(&acc->n_in_ref, nr);
        atomicAdd(&acc->n_ext, ne);
        atomicAdd(&acc->n_pos, np);
        if (er) atomicOr(p.err, (unsigned)er);
    }
}

// Load the tile's reference slice; returns a pointer usable for binary search.
__device__ const uint64_t *load_ref_slice(const TileParams &p, uint64_t t, uint64_t *rk_smem, unsigned long long &n)
{
    unsigned long long s = p.ref_off[t], e = p.ref_off[t + 1];
    n = e - s;
    if (n <= (unsigned long long)kRefSliceSmem) {
        for (unsigned long long i = threadIdx.x; i < 2 * n; i += blockDim.x) rk_smem[i] = p.ref_keys[2 * s + i];
        return rk_smem;
    }
    return p.ref_keys + 2 * s;
}

// ------------------------------------------- in-tile LSD radix sort + reduce
//
// A tile (or a chunk of an oversize tile) of at most kSortCap records sits in
// shared memory.  Each key is compressed to a 32-bit hash (the paper's
// compression of keys by hash functions) carried in a 64-bit word with the
// record's index, and the words are sorted with a stable LSD radix sort staged
// through shared memory: three 8-bit digit passes over the low 24 hash bits
// (a fourth over the top 8 bits only when two different keys share those 24),
// each ranking items within a warp with __match_any_sync, scanning the
// per-(digit, warp, item) counts into offsets and scattering.  Equal keys then
// form contiguous runs; every run is verified against the full 128-bit key (a
// remaining hash collision sends the chunk to an exact path) and reduced by
// key.

constexpr int kSortThreads = kTileThreads;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = kSortCap / kSortThreads;  // items per thread
constexpr int kWarpSpan = kSortCap / kSortWarps;     // positions a warp ranks in a digit pass
constexpr int kSortCtasPerSm = 1024 / kSortThreads;  // sorting CTAs per SM the registers are sized for
constexpr int kLongRun = 8;                          // longer runs are summed by a warp
static_assert(kSortItems * kSortThreads == kSortCap, "the sort holds whole items per thread");
static_assert(kWarpSpan == 32 * kSortItems, "a warp ranks whole rows of 32 positions");
static_assert(kSortThreads % 256 == 0, "the first 256 threads take one digit each in the offset scan");
static_assert(kBigThreads == kSortThreads, "every sorting CTA has the sort's width");
static_assert(kBigChunk <= kSortCap && kBigCap <= kSortCap && kTileCap <= kSortCap, "chunks fit one sort");

struct SortSmem {
    uint64_t words[2][kSortCap];  // (hash << 16) | record index
    union {
        uint16_t cnt[kSortWarps][256];  // digit pass: per-warp digit counts, then offsets
        struct {
            uint16_t heads[kSortCap], longq[kSortCap];  // after the passes: run heads, long runs
        } h;
        unsigned long long red[10][32];  // final statistics reduction
    } u;
    uint16_t dbase[256];
    uint32_t warp_tot[33];
    unsigned int nheads, nlong, collision;
};

__device__ __forceinline__ uint32_t key_hash32(uint64_t a, uint64_t b)
{
    uint64_t h = (a ^ 0x2545F4914F6CDD1Dull) * 0x9E3779B97F4A7C15ull;
    h ^= b;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 31;
    h *= 0x94D049BB133111EBull;
    return (uint32_t)(h >> 32);
}

// One stable counting-sort pass on the 8-bit digit at `shift` of the hash.
// Warp w ranks positions [w * kWarpSpan, (w + 1) * kWarpSpan) row by row (32
// positions per row, in order): __match_any_sync gives each item its rank
// among equal digits of the row, added to the warp's running count of that
// digit, which the row's lowest such lane then advances.  The counts live in
// a per-warp table, so it is cleared with a warp barrier only.  Thread d then
// turns digit d's per-warp counts into offsets and a block scan gives the
// digit bases; every item lands at base + warp offset + rank.
__device__ __forceinline__ void lsd_pass(const uint64_t *src, uint64_t *dst, int cnt, int shift, SortSmem &S)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint16_t *wc = S.u.cnt[warp];
    reinterpret_cast<uint4 *>(wc)[lane] = make_uint4(0, 0, 0, 0);  // 32 lanes x 16 B = 256 counts
    __syncwarp();
    uint64_t w[kSortItems];
    uint32_t dig[kSortItems], rank[kSortItems];
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const int pos = warp * kWarpSpan + it * 32 + lane;
        const bool valid = pos < cnt;
        w[it] = valid ? src[pos] : 0ull;
        const uint32_t d = (uint32_t)(w[it] >> (16 + shift)) & 0xFFu;
        // past-the-end lanes get a value no real digit has, so they match nobody
        const uint32_t peers = __match_any_sync(0xffffffffu, valid ? d : 256u + lane);
        dig[it] = d;
        const uint32_t before = valid ? wc[d] : 0u;
        rank[it] = before + __popc(peers & lt);
        __syncwarp();
        if (valid && (peers & lt) == 0) wc[d] = (uint16_t)(before + __popc(peers));
        __syncwarp();
    }
    __syncthreads();
    // thread d < 256: offsets of digit d within each warp's share, and its total
    uint32_t total_d = 0;
    if (tid < 256) {
        const int d = tid;
#pragma unroll
        for (int k = 0; k < kSortWarps; ++k) {
            const uint32_t c = S.u.cnt[k][d];
            S.u.cnt[k][d] = (uint16_t)total_d;
            total_d += c;
        }
    }
    // exclusive scan of the digit totals over warps 0..7: the digit bases
    {
        uint32_t incl = total_d;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += t;
        }
        if (lane == 31 && warp < 8) S.warp_tot[warp] = incl;
        __syncthreads();
        if (tid < 256) {
            uint32_t base = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) base += k < warp ? S.warp_tot[k] : 0u;
            S.dbase[tid] = (uint16_t)(base + incl - total_d);
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const int pos = warp * kWarpSpan + it * 32 + lane;
        if (pos < cnt) dst[S.dbase[dig[it]] + S.u.cnt[warp][dig[it]] + rank[it]] = w[it];
    }
    __syncthreads();
}

// Value of one unique key handed to a consumer: the numerator either as the
// FP64 value of a single record or as an exact fixed-point sum.
struct KeyVal {
    uint64_t a, b;
    bool fixed;
    double num;
    uint64_t fl;
    int64_t fh;
    int64_t den;
};

template <class Rec>
__device__ __forceinline__ void rec_value(const Rec &r, bool &fixed, double &num, uint64_t &fl, int64_t &fh);
template <>
__device__ __forceinline__ void rec_value<Rec32>(const Rec32 &r, bool &fixed, double &num, uint64_t &fl, int64_t &fh)
{
    fixed = false;
    num = r.num;
    fl = 0;
    fh = 0;
}
template <>
__device__ __forceinline__ void rec_value<Rec48>(const Rec48 &r, bool &fixed, double &num, uint64_t &fl, int64_t &fh)
{
    fixed = true;
    num = 0.0;
    fl = r.fx_lo;
    fh = r.fx_hi;
}
__device__ __forceinline__ void rec_add(const Rec32 &r, uint64_t &fl, int64_t &fh, uint32_t &err)
{
    fx_add_double(fl, fh, r.num, err);
}
__device__ __forceinline__ void rec_add(const Rec48 &r, uint64_t &fl, int64_t &fh, uint32_t &)
{
    fx_add_fx(fl, fh, r.fx_lo, r.fx_hi);
}

// Sort the chunk and hand every unique key to `emit` (any order; every thread
// may call it).  Returns false, for all threads, if two different keys share
// a hash; then nothing was emitted and the caller must use the exact path.
template <class Rec, class Emit>
__device__ bool sort_reduce_chunk(const Rec *recs, int cnt, SortSmem &S, uint32_t &err, Emit &&emit)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint64_t *A = S.words[0], *B = S.words[1];
    if (tid == 0) {
        S.nheads = 0;
        S.nlong = 0;
        S.collision = 0;
    }
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const int pos = it * kSortThreads + tid;
        if (pos < cnt) A[pos] = ((uint64_t)key_hash32(recs[pos].a, recs[pos].b) << 16) | (uint64_t)pos;
    }
    __syncthreads();
    // three digit passes order the words by the low 24 hash bits; a fourth
    // (the top 8 bits) runs only if two different keys share those 24 bits
    lsd_pass(A, B, cnt, 0, S);
    lsd_pass(B, A, cnt, 8, S);
    lsd_pass(A, B, cnt, 16, S);
    uint64_t hmask = 0xFFFFFFull << 16;
    A = S.words[1];
    for (int round = 0; round < 2; ++round) {
        // heads of equal-hash runs; a run must also hold a single 128-bit key
#pragma unroll
        for (int it = 0; it < kSortItems; ++it) {
            const int pos = it * kSortThreads + tid;
            bool head = false;
            if (pos < cnt) {
                const uint64_t wv = A[pos];
                head = pos == 0 || (A[pos - 1] & hmask) != (wv & hmask);
                if (!head) {
                    const Rec &r0 = recs[wv & 0xFFFF], &rp = recs[A[pos - 1] & 0xFFFF];
                    if (r0.a != rp.a || r0.b != rp.b) S.collision = 1;
                }
            }
            const uint32_t m = __ballot_sync(0xffffffffu, head);
            uint32_t base = 0;
            if (lane == 0 && m) base = atomicAdd(&S.nheads, (unsigned)__popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (head) S.u.h.heads[base + __popc(m & ((1u << lane) - 1u))] = (uint16_t)pos;
        }
        __syncthreads();
        if (!S.collision) break;
        if (round == 1) return false;
        __syncthreads();
        if (tid == 0) {
            S.nheads = 0;
            S.collision = 0;
        }
        lsd_pass(S.words[1], S.words[0], cnt, 24, S);
        A = S.words[0];
        hmask = 0xFFFFFFFFull << 16;
    }
    const int nh = (int)S.nheads;
    for (int h = tid; h < nh; h += kSortThreads) {
        const int j = S.u.h.heads[h];
        const uint64_t hj = A[j] & hmask;
        const Rec &r0 = recs[A[j] & 0xFFFF];
        KeyVal v;
        v.a = r0.a;
        v.b = r0.b;
        v.den = r0.den;
        rec_value(r0, v.fixed, v.num, v.fl, v.fh);
        if (j + 1 < cnt && (A[j + 1] & hmask) == hj) {
            if (j + kLongRun < cnt && (A[j + kLongRun] & hmask) == hj) {
                S.u.h.longq[atomicAdd(&S.nlong, 1u)] = (uint16_t)j;
                continue;
            }
            uint64_t fl = 0;
            int64_t fh = 0;
            rec_add(r0, fl, fh, err);
            for (int k = j + 1; k < cnt && (A[k] & hmask) == hj; ++k) {
                const Rec &r2 = recs[A[k] & 0xFFFF];
                rec_add(r2, fl, fh, err);
                v.den = r2.den < v.den ? r2.den : v.den;
            }
            v.fixed = true;
            v.fl = fl;
            v.fh = fh;
        }
        emit(v);
    }
    __syncthreads();
    const int nl = (int)S.nlong;
    for (int q = warp; q < nl; q += kSortThreads / 32) {
        const int j = S.u.h.longq[q];
        const uint64_t hj = A[j] & hmask;
        uint64_t fl = 0;
        int64_t fh = 0;
        int64_t den = recs[A[j] & 0xFFFF].den;
        for (int base = j; base < cnt; base += 32) {
            const int k = base + lane;
            const bool same = k < cnt && (A[k] & hmask) == hj;
            if (same) {
                const Rec &r = recs[A[k] & 0xFFFF];
                rec_add(r, fl, fh, err);
                den = r.den < den ? r.den : den;
            }
            if (__ballot_sync(0xffffffffu, same) != 0xffffffffu) break;
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            const uint64_t olo = __shfl_down_sync(0xffffffffu, fl, off);
            const int64_t ohi = __shfl_down_sync(0xffffffffu, fh, off);
            const int64_t od = __shfl_down_sync(0xffffffffu, den, off);
            fx_add_fx(fl, fh, olo, ohi);
            den = od < den ? od : den;
        }
        if (lane == 0) {
            const Rec &r0 = recs[A[j] & 0xFFFF];
            KeyVal v;
            v.a = r0.a;
            v.b = r0.b;
            v.fixed = true;
            v.num = 0.0;
            v.fl = fl;
            v.fh = fh;
            v.den = den;
            emit(v);
        }
    }
    __syncthreads();
    return true;
}

// Exact fallback for a chunk whose hash compression collided: bucket the keys
// by a second hash and insertion-sort each bucket by the full key (slow, and
// only reached with probability ~cnt^2 / 2^33 per chunk).
template <class Rec, class Emit>
__device__ void exact_reduce_chunk(const Rec *recs, int cnt, SortSmem &S, uint32_t &err, Emit &&emit)
{
    uint16_t *perm = reinterpret_cast<uint16_t *>(S.words[0]);
    uint16_t *rnk = reinterpret_cast<uint16_t *>(S.words[0]) + kSortCap;
    uint16_t *bkt = reinterpret_cast<uint16_t *>(S.words[0]) + 2 * kSortCap;
    uint32_t *hist = reinterpret_cast<uint32_t *>(S.words[1]);
    for (int i = threadIdx.x; i < kSortCap; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    auto key = [&](int i, uint64_t &a, uint64_t &b) {
        a = recs[i].a;
        b = recs[i].b;
    };
    group_keys(cnt, kSortCap, key, perm, rnk, bkt, hist, S.warp_tot, &S.nlong);
    const int nt = blockDim.x;
    const int chunk = (cnt + nt - 1) / nt;
    const int s = threadIdx.x * chunk, e = min(cnt, s + chunk);
    for (int j = s; j < e; ++j) {
        const Rec &r0 = recs[perm[j]];
        if (j > 0) {
            const Rec &rp = recs[perm[j - 1]];
            if (rp.a == r0.a && rp.b == r0.b) continue;
        }
        KeyVal v;
        v.a = r0.a;
        v.b = r0.b;
        v.fixed = true;
        v.num = 0.0;
        v.fl = 0;
        v.fh = 0;
        v.den = r0.den;
        for (int k = j; k < cnt; ++k) {
            const Rec &r2 = recs[perm[k]];
            if (k > j && (r2.a != r0.a || r2.b != r0.b)) break;
            rec_add(r2, v.fl, v.fh, err);
            v.den = r2.den < v.den ? r2.den : v.den;
        }
        emit(v);
    }
    __syncthreads();
}

// One unique key into the statistics (filter + Eq. 3 term).
__device__ __forceinline__ void finish_keyval(const TileParams &p, double e0, bool sym, const uint64_t *rk,
                                              unsigned long long nrk, const KeyVal &v, KeyStats &st)
{
    finish_key(p, e0, sym, rk, nrk, v.a, v.b, v.fixed ? fx_to_double(v.fl, v.fh) : v.num, v.den, st);
}

// Shared memory of the main tile kernel (several CTAs share an SM, so one CTA's
// tile load and barriers overlap the others' work).
struct MainSmem {
    Rec32 recs[kTileCap];
    SortSmem S;
    uint64_t rk[2 * kRefSliceSmem];
    unsigned long long meta[4];  // current tile: offset, count, reference offset, reference count
    uint64_t bar[2];
};

size_t tile_smem_bytes() { return sizeof(MainSmem); }

struct TileMeta {
    unsigned long long off, cnt, roff, rcnt;
};

__device__ __forceinline__ TileMeta tile_meta(const TileParams &p, uint64_t t)
{
    TileMeta m{0, 0, 0, 0};
    if (t < p.n_tiles) {
        m.off = p.tile_off[t];
        m.cnt = p.tile_off[t + 1] - m.off;
        m.roff = p.ref_off[t];
        m.rcnt = p.ref_off[t + 1] - m.roff;
    }
    return m;
}

__device__ __forceinline__ void issue_tile(const TileParams &p, MainSmem &M, const TileMeta &m)
{
    if (m.cnt == 0 || m.cnt > (unsigned long long)kTileCap) return;
    fence_proxy_async_smem();
    bulk_load(M.recs, p.recs + m.off, (uint32_t)(m.cnt * sizeof(Rec32)), &M.bar[0]);
}

__device__ __forceinline__ void push_oversize(const TileParams &p, int inst, uint64_t t, unsigned long long cnt)
{
    const unsigned idx = atomicAdd(&p.n_big[inst], 1u);
    p.big_list[p.tile_base[inst] + idx] = (uint32_t)t;
    atomicMax(p.big_max, cnt);
}

// Instance of global tile t.
__device__ __forceinline__ int tile_instance(const unsigned long long *__restrict__ tb, int n_inst, uint64_t t)
{
    int lo = 0, hi = n_inst;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (tb[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Persistent: CTA g handles tiles g, g + G, g + 2G, ...  Thread 0 keeps the
// tile metadata one tile ahead, so each tile's TMA load starts at once.
// Tiles of one instance are consecutive, so a CTA's statistics are flushed
// to an instance's accumulator when its tiles move on to the next instance.
template <bool SYM>
__global__ void __launch_bounds__(kTileThreads, kSortCtasPerSm) tile_kernel(const TileParams p)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MainSmem &M = *reinterpret_cast<MainSmem *>(smem_raw);
    const uint64_t G = gridDim.x;
    KeyStats st;
    st.clear();
    TileMeta nx{0, 0, 0, 0};
    if (threadIdx.x == 0) {
        mbar_init(&M.bar[0], 1);
        nx = tile_meta(p, blockIdx.x);
    }
    __syncthreads();
    // current instance, the first tile past it and its E0, kept in registers
    // (a CTA's tiles increase, so they only change at instance boundaries)
    int cur = tile_instance(p.tile_base, p.n_inst, blockIdx.x);
    unsigned long long cur_end = p.tile_base[cur + 1];
    double e0 = p.e0[cur];
    bool sym = SYM && p.sym[cur] != 0;
    bool dirty = false;
    uint32_t phase = 0;
    for (uint64_t t = blockIdx.x; t < p.n_tiles; t += G) {
        if (t >= cur_end) {  // uniform across the CTA
            if (dirty) flush_stats(p, p.acc[cur], st, M.S.u.red);
            st.clear();
            dirty = false;
            cur = tile_instance(p.tile_base, p.n_inst, t);
            cur_end = p.tile_base[cur + 1];
            e0 = p.e0[cur];
            sym = SYM && p.sym[cur] != 0;
        }
        const int inst = cur;
        if (threadIdx.x == 0) {
            issue_tile(p, M, nx);
            M.meta[0] = nx.off;
            M.meta[1] = nx.cnt;
            M.meta[2] = nx.roff;
            M.meta[3] = nx.rcnt;
            nx = tile_meta(p, t + G);  // consumed next iteration
        }
        __syncthreads();
        const unsigned long long cntl = M.meta[1];
        const unsigned long long roff = M.meta[2], rcnt = M.meta[3];
        if (cntl > (unsigned long long)kTileCap) {
            if (threadIdx.x == 0) push_oversize(p, inst, t, cntl);
        } else if (cntl > 0) {
            const int cnt = (int)cntl;
            const uint64_t *rk = M.rk;
            if (rcnt <= (unsigned long long)kRefSliceSmem) {
                for (unsigned long long i = threadIdx.x; i < 2 * rcnt; i += blockDim.x)
                    M.rk[i] = p.ref_keys[2 * roff + i];
            } else {
                rk = p.ref_keys + 2 * roff;
            }
            mbar_wait_bounded(&M.bar[0], phase, p.err);
            phase ^= 1u;
            const bool ok = sort_reduce_chunk(M.recs, cnt, M.S, st.err,
                                              [&](const KeyVal &v) { finish_keyval(p, e0, sym, rk, rcnt, v, st); });
            if (!ok && threadIdx.x == 0) push_oversize(p, inst, t, cntl);  // exact path for a hash collision
            dirty = true;
        }
        __syncthreads();  // records, slice and metadata free for the next tile
    }
    if (dirty) flush_stats(p, p.acc[cur], st, M.S.u.red);
    __syncthreads();
    if (threadIdx.x == 0) mbar_inval(&M.bar[0]);
}

cudaError_t launch_tiles(const TileParams &p, int n_ctas, cudaStream_t s)
{
    if (p.n_tiles == 0) return cudaSuccess;
    size_t sm = tile_smem_bytes();
    unsigned g = (unsigned)(p.n_tiles < (uint64_t)n_ctas ? p.n_tiles : (uint64_t)n_ctas);
    if (p.sym_any) tile_kernel<true><<<g, kTileThreads, sm, s>>>(p);
    else tile_kernel<false><<<g, kTileThreads, sm, s>>>(p);
    return cudaGetLastError();
}

// ------------------------------------------------------ oversize tiles

// Tiles above shared-memory capacity (keys with many duplicates, or a tile
// whose hash compression collided): each chunk is sorted and reduced to
// (key, exact fixed-point numerator, min denominator) records; the reduced
// list is processed again until it fits one chunk, then finished like a
// normal tile.  Exact sums make the result independent of the chunking.
struct BigSmem {
    union {
        Rec32 r32[kBigChunk];
        Rec48 r48[kBigCap];
    } u;
    SortSmem S;
    uint64_t rk[2 * kRefSliceSmem];
    uint64_t bar;
    unsigned int out_count;
    unsigned int big_pre[kMaxBatch + 1];  // oversize tiles before instance i
    unsigned int bk_cnt[kBigBuckets];     // hash split of partials: bucket sizes (fill cursors while scattering)
    unsigned short bk_off[kBigBuckets];   // bucket starts (< kBigScratch)
};

size_t big_smem_bytes() { return sizeof(BigSmem); }

template <class Rec>
__device__ void chunk_to_partials(const Rec *recs, int m, BigSmem &M, Rec48 *dst, uint32_t &err)
{
    auto put = [&](const KeyVal &v) {
        Rec48 o;
        o.a = v.a;
        o.b = v.b;
        if (v.fixed) {
            o.fx_lo = v.fl;
            o.fx_hi = v.fh;
        } else {
            uint64_t fl = 0;
            int64_t fh = 0;
            fx_add_double(fl, fh, v.num, err);
            o.fx_lo = fl;
            o.fx_hi = fh;
        }
        o.den = v.den;
        o.pad = 0;
        dst[atomicAdd(&M.out_count, 1u)] = o;
    };
    if (!sort_reduce_chunk(recs, m, M.S, err, put)) exact_reduce_chunk(recs, m, M.S, err, put);
}

// Persistent over the oversize tiles of all instances, numbered in one index
// space (instance i owns [big_pre[i], big_pre[i+1])) and dealt round-robin to
// the CTAs, so a step's oversize work spreads over the whole grid whatever
// its instance mix; a CTA flushes its statistics when its tiles move on to
// the next instance.  The partial lists live in a fixed per-CTA scratch of
// two buffers of scratch_cap records; a tile whose partials outgrow it sets
// kErrScratch.
template <bool SYM>
__global__ void __launch_bounds__(kBigThreads, kSortCtasPerSm) big_tile_kernel(const TileParams p)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    BigSmem &M = *reinterpret_cast<BigSmem *>(smem_raw);
    Rec48 *bufA = p.scratch + (size_t)blockIdx.x * 2 * p.scratch_cap;
    Rec48 *bufB = bufA + p.scratch_cap;
    uint32_t phase = 0;
    if (threadIdx.x == 0) mbar_init(&M.bar, 1);
    __syncthreads();
    const int nt = blockDim.x;
    if (threadIdx.x == 0) {
        unsigned int run = 0;
        for (int i = 0; i < p.n_inst; ++i) {
            M.big_pre[i] = run;
            run += p.n_big[i];
        }
        M.big_pre[p.n_inst] = run;
    }
    __syncthreads();
    const unsigned int total = M.big_pre[p.n_inst];
    int inst = -1;
    double e0 = 0.0;
    bool sym = false;
    KeyStats st;
    st.clear();
    {
        for (unsigned int idx = blockIdx.x; idx < total; idx += gridDim.x) {
            if (inst < 0 || idx >= M.big_pre[inst + 1]) {  // uniform across the CTA
                if (inst >= 0) {
                    flush_stats(p, p.acc[inst], st, M.S.u.red);
                    __syncthreads();
                }
                st.clear();
                int lo = 0, hi = p.n_inst;  // last instance whose range starts at or before idx
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (M.big_pre[mid] <= idx) lo = mid;
                    else hi = mid;
                }
                inst = lo;
                e0 = p.e0[inst];
                sym = SYM && p.sym[inst] != 0;
            }
            const uint64_t t = p.big_list[p.tile_base[inst] + (idx - M.big_pre[inst])];
            const unsigned long long off = p.tile_off[t];
            const unsigned long long cnt = p.tile_off[t + 1] - off;
            bool bad = false;
            // chunks of records -> exact partials (Rec48) in bufA
            unsigned long long u = 0;
            for (unsigned long long cs = 0; !bad && cs < cnt; cs += kBigChunk) {
                const int m = (int)min((unsigned long long)kBigChunk, cnt - cs);
                if (u + (unsigned long long)m > p.scratch_cap) {  // uniform
                    if (threadIdx.x == 0) atomicOr(p.err, kErrScratch);
                    bad = true;
                    break;
                }
                if (threadIdx.x == 0) {
                    fence_proxy_async_smem();
                    bulk_load(M.u.r32, p.recs + off + cs, (uint32_t)(m * sizeof(Rec32)), &M.bar);
                    M.out_count = 0;
                }
                mbar_wait_bounded(&M.bar, phase, p.err);
                phase ^= 1;
                __syncthreads();
                chunk_to_partials(M.u.r32, m, M, bufA + u, st.err);
                u += M.out_count;
                __syncthreads();
            }
            // Partials of different chunks may share a key.  If they fit one
            // chunk they are sorted and reduced together; otherwise they are
            // first split by a hash of the key into buckets that each fit a
            // chunk (equal keys share a bucket) and every bucket is finished
            // on its own.  Exact sums make the result independent of the split.
            unsigned long long nrk;
            const uint64_t *rk = load_ref_slice(p, t, M.rk, nrk);
            auto fin = [&](const KeyVal &v) { finish_keyval(p, e0, sym, rk, nrk, v, st); };
            auto finish_list = [&](const Rec48 *src, int m) {
                for (int i = threadIdx.x; i < m; i += nt) M.u.r48[i] = src[i];
                __syncthreads();
                if (!sort_reduce_chunk(M.u.r48, m, M.S, st.err, fin)) exact_reduce_chunk(M.u.r48, m, M.S, st.err, fin);
                __syncthreads();
            };
            if (!bad && u <= (unsigned long long)kBigCap) {
                finish_list(bufA, (int)u);
            } else if (!bad) {
                int nbk = 2;
                while ((unsigned long long)nbk * (kBigCap / 2) < u && nbk < kBigBuckets) nbk *= 2;
                for (;;) {  // uniform: every thread sees the same counts
                    for (int i = threadIdx.x; i < nbk; i += nt) M.bk_cnt[i] = 0;
                    __syncthreads();
                    for (unsigned long long i = threadIdx.x; i < u; i += nt)
                        atomicAdd(&M.bk_cnt[bucket_hash(bufA[i].a, bufA[i].b) & (nbk - 1)], 1u);
                    __syncthreads();
                    unsigned int mx = 0;
                    for (int i = 0; i < nbk; ++i) mx = max(mx, M.bk_cnt[i]);
                    if (mx <= (unsigned)kBigCap || nbk >= kBigBuckets) {
                        if (mx > (unsigned)kBigCap) {
                            if (threadIdx.x == 0) atomicOr(p.err, kErrNoProgress);
                            bad = true;
                        }
                        break;
                    }
                    nbk *= 2;
                    __syncthreads();
                }
                if (!bad) {
                    if (threadIdx.x == 0) {
                        unsigned int run = 0;
                        for (int i = 0; i < nbk; ++i) {
                            M.bk_off[i] = (unsigned short)run;
                            run += M.bk_cnt[i];
                            M.bk_cnt[i] = 0;  // refilled by the scatter below
                        }
                    }
                    __syncthreads();
                    for (unsigned long long i = threadIdx.x; i < u; i += nt) {
                        const Rec48 r = bufA[i];
                        const int k = bucket_hash(r.a, r.b) & (nbk - 1);
                        bufB[M.bk_off[k] + atomicAdd(&M.bk_cnt[k], 1u)] = r;
                    }
                    __syncthreads();
                    for (int k = 0; k < nbk; ++k)
                        if (M.bk_cnt[k]) finish_list(bufB + M.bk_off[k], (int)M.bk_cnt[k]);
                }
            }
            __syncthreads();
        }
        if (inst >= 0) flush_stats(p, p.acc[inst], st, M.S.u.red);
        __syncthreads();
    }
    if (threadIdx.x == 0) mbar_inval(&M.bar);
}

cudaError_t launch_big_tiles(const TileParams &p, int n_ctas, cudaStream_t s)
{
    if (n_ctas <= 0) return cudaSuccess;
    if (p.sym_any) big_tile_kernel<true><<<n_ctas, kBigThreads, big_smem_bytes(), s>>>(p);
    else big_tile_kernel<false><<<n_ctas, kBigThreads, big_smem_bytes(), s>>>(p);
    return cudaGetLastError();
}

// ========================================================= pass bookkeeping

// Per instance: count the pass's records, compare them with the plan and
// reset the oversize counter for the next pass.
__global__ void pass_finish_kernel(const unsigned long long *__restrict__ tile_off,
                                   const unsigned long long *__restrict__ tile_base, int n_inst,
                                   const unsigned long long *__restrict__ expected, RunAcc *const *acc,
                                   unsigned int *n_big, uint32_t *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_inst) return;
    const unsigned long long got = tile_off[tile_base[i + 1]] - tile_off[tile_base[i]];
    acc[i]->n_terms += got;
    acc[i]->n_big += n_big[i];
    // exact count, or (flag kExpectAtMost, a run with a numerator cutoff) an upper bound
    const unsigned long long e = expected[i] & ~kExpectAtMost;
    if ((expected[i] & kExpectAtMost) ? got > e : got != e) atomicOr(err, kErrCount);
    n_big[i] = 0;
}

cudaError_t launch_pass_finish(const unsigned long long *tile_off, const unsigned long long *tile_base, int n_inst,
                               const unsigned long long *expected, RunAcc *const *acc, unsigned int *n_big,
                               uint32_t *err, cudaStream_t s)
{
    pass_finish_kernel<<<(n_inst + 127) / 128, 128, 0, s>>>(tile_off, tile_base, n_inst, expected, acc, n_big, err);
    return cudaGetLastError();
}

__global__ void acc_init_kernel(RunAcc *acc, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    RunAcc a;
    a.e2_lo = 0;
    a.e2_hi = 0;
    a.n_terms = a.n_unique = a.n_in_ref = a.n_ext = a.n_pos = a.dsum = a.dxor = 0;
    a.min_den = ~0ull;
    a.e2 = 0.0;
    a.min_abs_den = 0.0;
    a.err = 0;
    a.n_big = 0;
    a.big_max = 0;
    acc[i] = a;
}

cudaError_t launch_acc_init(RunAcc *acc, int n, cudaStream_t s)
{
    acc_init_kernel<<<(n + 127) / 128, 128, 0, s>>>(acc, n);
    return cudaGetLastError();
}

// Duplicate subtraction (the section on removing duplicate contributions):
// when the reference keys are left in the sum, a reference determinant i of
// the constraint class receives the numerator (H c)_i - H_ii c_i, which is
// c_i (E0 - H_ii) if c is an eigenvector of H in the reference space with
// eigenvalue E0, so its PT2-like term is c_i^2 (E0 - H_ii).  That amount is
// subtracted here in the same exact fixed point as the sum.
__global__ void __launch_bounds__(256) ref_subtract_kernel(const uint64_t *__restrict__ keys,
                                                           const double *__restrict__ coef,
                                                           const double *__restrict__ hii, uint64_t n, double e0,
                                                           uint64_t cons_mod, uint64_t cons_rem, RunAcc *acc,
                                                           uint32_t *err)
{
    uint64_t lo = 0;
    int64_t hi = 0;
    uint32_t er = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        if (!cons_ok(cons_mod, cons_rem, keys[2 * i])) continue;
        const double c = coef[i];
        fx_add_double(lo, hi, -((c * c) * (e0 - hii[i])), er);
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        const uint64_t olo = __shfl_down_sync(0xffffffffu, lo, off);
        const int64_t ohi = __shfl_down_sync(0xffffffffu, hi, off);
        fx_add_fx(lo, hi, olo, ohi);
        er |= __shfl_down_sync(0xffffffffu, er, off);
    }
    __shared__ unsigned long long red[2][8];
    __shared__ uint32_t rer[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][warp] = lo;
        red[1][warp] = (unsigned long long)hi;
        rer[warp] = er;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t blo = 0;
        int64_t bhi = 0;
        uint32_t ber = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            fx_add_fx(blo, bhi, red[0][w], (int64_t)red[1][w]);
            ber |= rer[w];
        }
        const unsigned long long old = atomicAdd(&acc->e2_lo, (unsigned long long)blo);
        const unsigned long long carry = (old + blo) < old ? 1ull : 0ull;
        atomicAdd((unsigned long long *)&acc->e2_hi, (unsigned long long)bhi + carry);
        if (ber) atomicOr(err, ber);
    }
}

cudaError_t launch_ref_subtract(const uint64_t *keys, const double *coef, const double *hii, uint64_t n, double e0,
                                uint64_t cons_mod, uint64_t cons_rem, RunAcc *acc, uint32_t *err, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const uint64_t blocks = (n + 255) / 256 < 1216 ? (n + 255) / 256 : 1216;
    ref_subtract_kernel<<<(unsigned)blocks, 256, 0, s>>>(keys, coef, hii, n, e0, cons_mod, cons_rem, acc, err);
    return cudaGetLastError();
}

__global__ void acc_finalize_kernel(RunAcc *acc, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    acc[i].e2 = fx_to_double(acc[i].e2_lo, acc[i].e2_hi);
    acc[i].min_abs_den =
        acc[i].min_den == ~0ull ? INFINITY : u128_to_double(acc[i].min_den, 0, kDenShift, false);
}

cudaError_t launch_acc_finalize(RunAcc *acc, int n, cudaStream_t s)
{
    acc_finalize_kernel<<<(n + 127) / 128, 128, 0, s>>>(acc, n);
    return cudaGetLastError();
}

// ============================================================ launchers

void gen_layout(GenParams &p, GenMode mode)
{
    auto al = [](size_t x) { return (x + 127) & ~(size_t)127; };
    size_t off = al(sizeof(GenFixed));
    p.smem_sa = (int)off;
    off = al(off + (size_t)p.n_sa * (8 + 8 + 4 + 2));
    p.smem_sb = (int)off;
    off = al(off + (size_t)p.n_sb * (8 + 8 + 4 + 2));
    p.smem_pairs = (int)off;
    off = al(off + (size_t)(kMaxOrb * (kMaxOrb - 1) / 2) * 2);
    p.smem_vec = (int)off;
    off = al(off + (size_t)(kGenThreads / 32) * kMaxOrb * 8);
    p.smem_hist = (int)off;
    if (mode == kModeClassCount || mode == kModeBetaCount) off = al(off + (size_t)kNumClasses * 4);
    else off = al(off + kVbkBytes);
    p.smem_bytes = (int)off;
}

cudaError_t launch_gen(GenMode mode, const GenBatch &b, uint64_t n_ctas, int smem_bytes, cudaStream_t s)
{
    if (n_ctas == 0) return cudaSuccess;
    // the counting modes always carry the symmetry check (they have registers
    // to spare) and never the cutoff (they count every term)
    const unsigned g = (unsigned)n_ctas;
    constexpr int S = kFiltSym, C = kFiltCut;
    switch (mode) {
    case kModeClassCount: gen_kernel<kModeClassCount, S><<<g, kGenThreads, smem_bytes, s>>>(b); break;
    case kModeBetaCount: gen_kernel<kModeBetaCount, S><<<g, kGenThreads, smem_bytes, s>>>(b); break;
    case kModeTileCount:
        switch (b.filt & (S | C)) {
        case 0: gen_kernel<kModeTileCount, 0><<<g, kGenThreads, smem_bytes, s>>>(b); break;
        case S: gen_kernel<kModeTileCount, S><<<g, kGenThreads, smem_bytes, s>>>(b); break;
        case C: gen_kernel<kModeTileCount, C><<<g, kGenThreads, smem_bytes, s>>>(b); break;
        default: gen_kernel<kModeTileCount, S | C><<<g, kGenThreads, smem_bytes, s>>>(b); break;
        }
        break;
    case kModeEmit:
        switch (b.filt & (S | C)) {
        case 0: gen_kernel<kModeEmit, 0><<<g, kGenThreads, smem_bytes, s>>>(b); break;
        case S: gen_kernel<kModeEmit, S><<<g, kGenThreads, smem_bytes, s>>>(b); break;
        case C: gen_kernel<kModeEmit, C><<<g, kGenThreads, smem_bytes, s>>>(b); break;
        default: gen_kernel<kModeEmit, S | C><<<g, kGenThreads, smem_bytes, s>>>(b); break;
        }
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_gen_single(GenMode mode, const GenParams &p, GenParams *, unsigned long long *, cudaStream_t s)
{
    if (mode != kModeDetTerms) return cudaErrorInvalidValue;
    gen_kernel_one<kModeDetTerms><<<1, kGenThreads, p.smem_bytes, s>>>(p);
    return cudaGetLastError();
}

// Largest dynamic shared memory any generator layout needs (n_orb = 64).
static int gen_smem_max()
{
    GenParams p;
    p.n_sa = 32 * 32;
    p.n_sb = 32 * 32;
    gen_layout(p, kModeClassCount);
    return p.smem_bytes;
}

cudaError_t init_kernel_attributes(int *tile_per_sm, int *big_per_sm)
{
    const int g = gen_smem_max();
    cudaError_t e;
    constexpr int S = kFiltSym, C = kFiltCut;
    const void *gens[] = {(const void *)gen_kernel<kModeClassCount, S>, (const void *)gen_kernel<kModeBetaCount, S>,
                          (const void *)gen_kernel<kModeTileCount, 0>,  (const void *)gen_kernel<kModeTileCount, S>,
                          (const void *)gen_kernel<kModeTileCount, C>,  (const void *)gen_kernel<kModeTileCount, S | C>,
                          (const void *)gen_kernel<kModeEmit, 0>,       (const void *)gen_kernel<kModeEmit, S>,
                          (const void *)gen_kernel<kModeEmit, C>,       (const void *)gen_kernel<kModeEmit, S | C>,
                          (const void *)gen_kernel_one<kModeDetTerms>};
    for (const void *f : gens)
        if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, g))) return e;
    for (const void *f : {(const void *)tile_kernel<false>, (const void *)tile_kernel<true>})
        if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem_bytes())))
            return e;
    for (const void *f : {(const void *)big_tile_kernel<false>, (const void *)big_tile_kernel<true>})
        if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)big_smem_bytes())))
            return e;
    // the persistent kernels launch exactly the CTAs that fit at once (both
    // variants have the same launch bounds and shared memory)
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(tile_per_sm, tile_kernel<false>, kTileThreads,
                                                           tile_smem_bytes())))
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(big_per_sm, big_tile_kernel<false>, kBigThreads,
                                                           big_smem_bytes())))
        return e;
    if (*tile_per_sm < 1 || *big_per_sm < 1) return cudaErrorInvalidConfiguration;
    return cudaSuccess;
}

cudaError_t launch_diag(const SysDev &sys, const uint64_t *keys, uint64_t n, double *out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    diag_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sys, keys, n, out);
    return cudaGetLastError();
}

// ------------------------------------------------ allocation-free variant
//
// Scratch of the allocation-free term generation: a counter followed by a
// staging area of kNoAllocMaxTerms records, in a file-scope device array.
// Every GPU that loads the library holds this array (16 MiB + 256 bytes)
// until the process exits.  All calls share it: the counter is cleared at the
// start of every call, and calls that overlap on the GPU race on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[256 + kNoAllocMaxTerms * sizeof(Rec32)];

// The array's device address per device.  Host code may not use the symbol
// itself (it is a host-side stand-in), so the address is looked up with
// cudaGetSymbolAddress once per device, with that device current.
static void *g_noalloc_addr[kMaxDevices];
static std::mutex g_noalloc_mu;

static cudaError_t noalloc_scratch(int device, void **out)
{
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[device] = ptr;
    }
    *out = g_noalloc_addr[device];
    return cudaSuccess;
}

// Split staged records into the caller's key / numerator / diagonal arrays
// (at most cap of them).
__global__ void split_terms_kernel(const Rec32 *__restrict__ recs, const unsigned int *__restrict__ count,
                                   uint64_t cap, uint64_t *__restrict__ keys, double *__restrict__ val,
                                   double *__restrict__ haa)
{
    const uint64_t n = (uint64_t)*count < cap ? (uint64_t)*count : cap;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const Rec32 r = recs[i];
        keys[2 * i] = r.a;
        keys[2 * i + 1] = r.b;
        val[i] = r.num;
        haa[i] = __longlong_as_double((long long)r.den);  // this generation mode stores H_aa itself
    }
}

cudaError_t launch_det_terms_noalloc(int device, GenParams p, uint64_t cap, uint64_t *keys, double *val, double *haa,
                                     unsigned long long *n_host, cudaStream_t s)
{
    void *base = nullptr;
    cudaError_t e = noalloc_scratch(device, &base);
    if (e != cudaSuccess) return e;
    unsigned int *count = reinterpret_cast<unsigned int *>(base);
    Rec32 *recs = reinterpret_cast<Rec32 *>(static_cast<unsigned char *>(base) + 256);
    p.cursor = count;
    p.recs = recs;
    p.rec_cap = kNoAllocMaxTerms;
    p.n_tiles = 1;
    gen_layout(p, kModeDetTerms);
    if ((e = cudaMemsetAsync(count, 0, sizeof(unsigned int), s)) != cudaSuccess) return e;
    if ((e = launch_gen_single(kModeDetTerms, p, nullptr, nullptr, s)) != cudaSuccess) return e;
    split_terms_kernel<<<64, 256, 0, s>>>(recs, count, cap, keys, val, haa);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    unsigned int n32 = 0;
    if ((e = cudaMemcpyAsync(&n32, count, sizeof(unsigned int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    e = cudaStreamSynchronize(s);
    *n_host = n32;
    return e;
}

}  // namespace pt2
