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

// Constraint classes of Algorithm 2 on an excited alpha string: alpha % mod ==
// rem (mod <= 1: none), and the triplet constraint of the "Triplet
// constraints" section generalised to k orbitals: the k highest occupied
// alpha orbitals are exactly T (tmask = T, thi = every bit at or above T's
// lowest; both 0: none).
__device__ __forceinline__ bool cons_ok(uint64_t mod, uint64_t rem, uint64_t thi, uint64_t tmask, uint64_t alpha)
{
    return (alpha & thi) == tmask && (mod <= 1 || (alpha % mod) == rem);
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

// Add value * 2^shift (rounded half away from zero) to the 128-bit integer
// (lo, hi).  |value| * 2^shift must stay below 2^126, else the range bit is
// set.  Numerators use shift 90 (|value| < 2^36); energy terms, whose
// denominator is a 2^-48 fixed-point integer, fold that power of two in.
__device__ __forceinline__ void fx_add_double(uint64_t &lo, int64_t &hi, double v, uint32_t &err, int shift = kFxShift)
{
    uint64_t bits = (uint64_t)__double_as_longlong(v);
    int e = (int)((bits >> 52) & 0x7FF);
    if (e == 0) return;  // zero / subnormal: below the resolution
    if (e >= 1023 + 126 - shift) {
        err |= kErrFixedRange;
        return;
    }
    uint64_t m = (bits & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
    int sh = e - 1075 + shift;  // value * 2^shift = m * 2^sh
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

// 1 / dfx for a nonzero fixed-point denominator dfx (E0 - H_aa = dfx 2^-48):
// the single-precision hardware estimate x0 of rcp.approx.ftz.f32 (at most
// 1 ulp) of dfx rounded to float (half an ulp), together within 2^-22.4
// relative, refined by one Newton-Raphson step x1 = x0 + x0 (1 - dfx x0) in
// FP64, whose relative error is the square of x0's plus FP64 rounding:
// below 2^-44.  Every nonzero int64 has a reciprocal that is a normal
// float (between 2^-63 and 1), so x0's bits map onto a double directly
// (sign, exponent rebiased by 1023 - 127, mantissa widened).  dfx = 0 maps to
// a huge finite value (the float's infinity rebiased), so a term with a
// nonzero numerator overflows the fixed-point range and is reported.
__device__ __forceinline__ double recip_fx(int64_t dfx)
{
    const double d = __ll2double_rn((long long)dfx);
    const float f = __ll2float_rn((long long)dfx);
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(f));
    const uint32_t fb = __float_as_uint(rf);
    const uint64_t db = ((uint64_t)(fb >> 31) << 63) | ((uint64_t)(((fb >> 23) & 0xFFu) + 896u) << 52) |
                        ((uint64_t)(fb & 0x7FFFFFu) << 29);
    const double x = __longlong_as_double((long long)db);
    const double e = __fma_rn(-d, x, 1.0);
    return __fma_rn(x, e, x);
}

// The Epstein-Nesbet term num^2 / (E0 - H_aa) of Eq. 3 in units of 2^-48 Ha
// (the fixed-point addition of the energy applies the factor 2^48).
__device__ __forceinline__ double term_fx48(double num, int64_t dfx) { return (num * num) * recip_fx(dfx); }

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

// Non-blocking probe of the phase (try_wait may suspend the thread for a
// hardware time window before it answers; test_wait answers at once).
__device__ __forceinline__ bool mbar_probe(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity, giving up after `limit` SM
// cycles (2^31, about a second, in normal runs; a limit below 2^12 cycles
// polls with the non-blocking probe so that it can expire before a copy
// lands).  On a timeout the error bit is set and a second bounded wait (2^31
// cycles) gives the copy in flight the chance to land before the CTA stops.
__device__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t *err, long long limit)
{
    const bool quick = limit < (1ll << 12);
    long long t0 = clock64();
    while (!(quick ? mbar_probe(bar, parity) : mbar_test(bar, parity))) {
        if (clock64() - t0 > limit) {
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
    uint32_t chunk_a[32], chunk_b[32];  // pass flags of singles 32c .. 32c + 31 (n_sa, n_sb <= 1024)
    uint32_t grp[kGrpTab];              // pass table of a grouped tile count (GenParams::grp)
    uint32_t q_a;                       // its pass of the alpha string A
    uint32_t wsum[kGenThreads / 32];
    // the pass's alpha classes as aligned blocks of bucket groups (see above)
    uint16_t blk_g[2 * kVbkBitsMax];
    uint8_t blk_k[2 * kVbkBitsMax];
    int n_blk;
    unsigned int n_list;  // listed alpha-alpha doubles of the current round
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

// Same-spin double r1 r2 -> a1 a2 (r1 < r2, a1 < a2): (a1 r1|a2 r2) - (a1 r2|a2 r1),
// one load from the table of these elements by colex pair (SysDev::dpair).
__device__ __forceinline__ double same_double_value(const double *__restrict__ dpair, int np, int r1, int r2, int a1,
                                                    int a2)
{
    return __ldg(dpair + (size_t)(r2 * (r2 - 1) / 2 + r1) * np + (a2 * (a2 - 1) / 2 + a1));
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
    unsigned int *ctr;      // TileCount: terms per tile; Emit / DetTerms: next slot per tile
    Rec32 *recs;
    uint32_t n_tiles;       // tiles of the instance in the pass (< 2^32)
    uint32_t rec_cap;       // record slots of the step (< 2^32)
    uint32_t *err;
    double e0;              // DetTerms only
    // TileCount over a group of passes: tile bases then tile counts of the
    // passes (shared memory); the pass of a term rides in the low 6 bits of
    // its tile hash, which tile_of does not read.  Null: one pass.
    const uint32_t *gtab;
};

// Tile of a term from the high word of its tile hash: floor(zt_hi n_tiles / 2^32)
// (the reference partition uses the same map).
__device__ __forceinline__ uint32_t tile_of(uint64_t zt, uint32_t n_tiles)
{
    return __umulhi((uint32_t)(zt >> 32), n_tiles);
}

template <int MODE, int NB = kGenBatch, class KeyFn, class ValFn>
__device__ __forceinline__ void emit_batch(const EmitOut &p, int i0, int step, int n, KeyFn key, ValFn val)
{
    // The lanes of a warp hold consecutive items (i0 - lane is the warp's
    // first), so the steps in which some lane has an item are known to the
    // whole warp and the others are skipped.
    const int wbase = i0 - (int)(threadIdx.x & 31);
    const int nst = wbase >= n ? 0 : min(NB, (n - wbase + step - 1) / step);
    uint32_t slot[NB];
    uint32_t ok = 0;  // bit u: item of step u is a term of the pass
    double el[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        slot[u] = 0;
        el[u] = 0.0;
        if (u < nst) {
            const int i = i0 + u * step;
            uint64_t zt = 0;
            if (i < n && key(i, zt, el[u])) {
                ok |= 1u << u;
                if constexpr (MODE == kModeTileCount) {
                    uint32_t t;
                    if (p.gtab) {
                        const uint32_t q = (uint32_t)zt & 63u;
                        t = p.gtab[q] + tile_of(zt, p.gtab[kMaxGrp + q]);
                    } else {
                        t = tile_of(zt, p.n_tiles);
                    }
                    red_add_global(&p.ctr[t], 1u);
                } else if constexpr (MODE == kModeEmit) {
                    slot[u] = atom_add_global(&p.ctr[tile_of(zt, p.n_tiles)], 1u);
                } else {
                    slot[u] = atom_add_global(&p.ctr[0], 1u);
                }
            }
        }
    }
    if constexpr (MODE == kModeEmit || MODE == kModeDetTerms) {
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            if (u >= nst) break;
            if (!((ok >> u) & 1u)) continue;
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

// Bucket table of a determinant's virtual alpha pairs (entries vb_off[b] ..
// vb_off[b + 1] of vb_list are the indices, in the pair list, of the pairs
// whose class hash has top bits b), and the class range [class_lo, class_hi)
// as aligned blocks of bucket groups (F.blk_g, F.blk_k, F.n_blk).  Called by
// the whole CTA.
__device__ __forceinline__ void build_vbk(GenFixed &F, const uint16_t *pairs, int n_vir_pairs_a, uint32_t class_lo,
                                          uint32_t class_hi, uint32_t *vb_cnt, uint16_t *vb_off, uint16_t *vb_list)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nw = kGenThreads / 32;
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
    const double *__restrict__ dpair = p.sys.dpair;
    const int NP = N * (N - 1) / 2;
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
    // a tile count over a group of passes: its pass table, and the pass of
    // each class (one byte per class, copied 16 bytes per thread)
    const bool grouped = MODE == kModeTileCount && p.n_grp != 0;
    uint8_t *gcls = smem + p.smem_gcls;
    if (grouped) {
        for (int i = tid; i < kGrpTab; i += kGenThreads) F.grp[i] = p.grp[i];
        const uint4 *src = reinterpret_cast<const uint4 *>(p.grp + kGrpClsOff);
        for (int i = tid; i < kNumClasses / 16; i += kGenThreads) reinterpret_cast<uint4 *>(gcls)[i] = src[i];
    }
    auto grp_of = [&](uint32_t cl) { return (uint32_t)gcls[cl]; };
    // the tile hash of a term with its pass in the low 6 bits (grouped count)
    auto with_pass = [&](uint64_t zt, uint32_t q) { return grouped ? ((zt & ~63ull) | q) : zt; };
    // the class-count mode histograms the classes [class_lo, class_hi) only
    const uint32_t n_hist = MODE == kModeClassCount ? p.class_hi - p.class_lo : (uint32_t)kNumClasses;
    if constexpr (kCount)
        for (int i = tid; i < (int)n_hist; i += kGenThreads) hist[i] = 0;
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

    // singles lists; delta = H_aa - H_ii of the single, exact.  Single s is
    // lane s % 32 of its warp, so the warp's ballot of the pass flags is the
    // flag word of the 32 singles from 32 (s / 32) (compacted below)
    const uint32_t mva = nva ? (uint32_t)((0x100000000ull + nva - 1) / nva) : 0u;  // s / nva = umulhi(s, mva)
    const uint32_t mvb = nvb ? (uint32_t)((0x100000000ull + nvb - 1) / nvb) : 0u;  // exact while s * nv < 2^32
    for (int s0 = 0; s0 < p.n_sa; s0 += kGenThreads) {
        const int s = s0 + tid;
        uint32_t inp = 0, qs = 0;
        if (s < p.n_sa) {
            const int i = (int)__umulhi((uint32_t)s, mva), j = s - i * nva;
            const int r = F.occA[i], a = F.virA[j];
            const uint32_t sg = __popcll(A & between_mask(r, a)) & 1;
            const uint64_t a2 = A ^ (1ull << r) ^ (1ull << a);
            const uint64_t zc = F.ZcA ^ F.zc[r] ^ F.zc[a];
            if constexpr (MODE == kModeBetaCount) {
                inp = class_of(zc) == p.heavy_class && cons_ok(p.cons_mod, p.cons_rem, p.top_hi, p.top_mask, a2);
            } else {
                const uint32_t cl = class_of(zc);
                inp = cl >= p.class_lo && cl < p.class_hi && cons_ok(p.cons_mod, p.cons_rem, p.top_hi, p.top_mask, a2);
                if (grouped && inp) qs = grp_of(cl);
            }
            if constexpr (kVal) sa_delta[s] = F.gA[a] - F.gA[r] - WSx[r * N + a];
            sa_zt[s] = kCount ? zc : (F.ZtaA ^ F.zta[r] ^ F.zta[a]);
            // bits 0-7 r, 8-15 a, 16 sign, 17 in the pass, 18-23 pass of a grouped count
            sa_info[s] = (uint32_t)r | ((uint32_t)a << 8) | (sg << 16) | (inp << 17) | (qs << 18);
        }
        const uint32_t m = __ballot_sync(0xffffffffu, inp != 0);
        if (lane == 0) F.chunk_a[(s0 >> 5) + warp] = m;
    }
    for (int s0 = 0; s0 < p.n_sb; s0 += kGenThreads) {
        const int s = s0 + tid;
        uint32_t binp = 0;
        if (s < p.n_sb) {
            const int i = (int)__umulhi((uint32_t)s, mvb), j = s - i * nvb;
            const int r = F.occB[i], a = F.virB[j];
            const uint32_t sg = __popcll(B & between_mask(r, a)) & 1;
            if constexpr (kVal) sb_delta[s] = F.gB[a] - F.gB[r] - WSx[r * N + a];
            const uint64_t zcb = F.ZcbB ^ F.zcb[r] ^ F.zcb[a];  // beta class hash of the excited beta string
            // the beta-count mode histograms beta classes, so it keeps that hash here
            sb_zt[s] = MODE == kModeBetaCount ? zcb : (F.ZtbB ^ F.ztb[r] ^ F.ztb[a]);
            const uint32_t bc = bclass_of(zcb);
            binp = bfull || (bc >= blo && bc < bhi);
            sb_info[s] = (uint32_t)r | ((uint32_t)a << 8) | (sg << 16) | (binp << 17);
        }
        const uint32_t m = __ballot_sync(0xffffffffu, binp != 0);
        if (lane == 0) F.chunk_b[(s0 >> 5) + warp] = m;
    }
    if (tid == 0) {
        bool ok = cons_ok(p.cons_mod, p.cons_rem, p.top_hi, p.top_mask, A);
        if constexpr (MODE == kModeBetaCount) {
            ok = ok && class_of(F.ZcA) == p.heavy_class;
        } else {
            uint32_t cl = class_of(F.ZcA);
            ok = ok && cl >= p.class_lo && cl < p.class_hi;
            F.q_a = grouped && ok ? grp_of(cl) : 0u;
        }
        F.a_in_pass = ok;
        const uint32_t bc = bclass_of(F.ZcbB);
        F.b_in_pass = bfull || (bc >= blo && bc < bhi);
    }
    __syncthreads();
    // compact the alpha singles of the pass, and the beta singles whose beta
    // class belongs to it, in ascending order: every warp scans the chunk
    // counts (one chunk per lane) and writes the singles of its own chunks
    {
        const int nca = (p.n_sa + 31) >> 5, ncb = bfull ? 0 : (p.n_sb + 31) >> 5;
        const uint32_t ma = lane < nca ? F.chunk_a[lane] : 0u, mb = lane < ncb ? F.chunk_b[lane] : 0u;
        uint32_t ia = __popc(ma), ib = __popc(mb);  // inclusive prefix counts over the chunks
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t va = __shfl_up_sync(0xffffffffu, ia, off), vb = __shfl_up_sync(0xffffffffu, ib, off);
            if (lane >= off) {
                ia += va;
                ib += vb;
            }
        }
        const uint32_t lt = (1u << lane) - 1u;
        for (int ch = warp; ch < nca; ch += nw) {
            const uint32_t m = __shfl_sync(0xffffffffu, ma, ch), base = __shfl_sync(0xffffffffu, ia, ch) - __popc(m);
            if ((m >> lane) & 1u) sa_pass[base + __popc(m & lt)] = (uint16_t)(ch * 32 + lane);
        }
        for (int ch = warp; ch < ncb; ch += nw) {
            const uint32_t m = __shfl_sync(0xffffffffu, mb, ch), base = __shfl_sync(0xffffffffu, ib, ch) - __popc(m);
            if ((m >> lane) & 1u) sb_pass[base + __popc(m & lt)] = (uint16_t)(ch * 32 + lane);
        }
        const uint32_t ta = __shfl_sync(0xffffffffu, ia, 31), tb = __shfl_sync(0xffffffffu, ib, 31);
        if (tid == 0) {
            F.n_sa_pass = (int)ta;
            if (!bfull) F.n_sb_pass = (int)tb;
        }
    }
    __syncthreads();
    const int n_sa_pass = F.n_sa_pass;
    const bool a_in = F.a_in_pass != 0;
    const bool b_in = F.b_in_pass != 0;

    const int n_occ_pairs_a = na * (na - 1) / 2, n_vir_pairs_a = nva * (nva - 1) / 2;
    const int n_occ_pairs_b = nb * (nb - 1) / 2, n_vir_pairs_b = nvb * (nvb - 1) / 2;

    if constexpr (MODE == kModeClassCount) {
        // work list (the paper's first pass over the wavefunction): terms per
        // class of [class_lo, class_hi).  A run with a numerator cutoff counts
        // the contributions it keeps: it evaluates every matrix element with
        // the functions the emission uses, so both take the same decisions
        const uint32_t lo = p.class_lo;
        if (cutting) {
            // an alpha single (beta string B) and its alpha-beta doubles, one
            // alpha single per warp
            for (int k = warp; k < n_sa_pass; k += nw) {
                const int s = sa_pass[k];
                const uint32_t ia = sa_info[s];
                const uint64_t a2 = single_word(A, ia);
                const int rA = ia & 0xFF, aA = (ia >> 8) & 0xFF;
                uint32_t cnt = 0;
                for (int sb = lane; sb < p.n_sb; sb += 32) {
                    const uint32_t bi = sb_info[sb];
                    if (sym && single_word(B, bi) > a2) continue;
                    cnt += above_cut(c, __ldg(eri + (((size_t)rA * N + aA) * N + (bi & 0xFF)) * N + ((bi >> 8) & 0xFF)),
                                     cut);
                }
                cnt = __reduce_add_sync(0xffffffffu, cnt);
                if (lane == 0) {
                    if ((!sym || a2 >= B) && above_cut(c, single_value(ht, eri, N, F.occA, na, F.occB, nb, rA, aA), cut))
                        ++cnt;
                    if (cnt) atomicAdd(&hist[class_of(sa_zt[s]) - lo], cnt);
                }
            }
            if (a_in) {  // beta singles and beta-beta doubles keep alpha string A
                uint32_t cnt = 0;
                for (int sb = tid; sb < p.n_sb; sb += kGenThreads) {
                    const uint32_t bi = sb_info[sb];
                    if (sym && single_word(B, bi) > A) continue;
                    cnt += above_cut(c, single_value(ht, eri, N, F.occB, nb, F.occA, na, bi & 0xFF, (bi >> 8) & 0xFF),
                                     cut);
                }
                for (int pi = warp; pi < n_occ_pairs_b; pi += nw) {
                    const int pr = pairs[pi];
                    const int r1 = F.occB[pr & 0xFF], r2 = F.occB[pr >> 8];
                    const uint64_t b12 = B ^ (1ull << r1) ^ (1ull << r2);
                    for (int t = lane; t < n_vir_pairs_b; t += 32) {
                        const int pv = pairs[t];
                        const int a1 = F.virB[pv & 0xFF], a2 = F.virB[pv >> 8];
                        if (sym && (b12 ^ (1ull << a1) ^ (1ull << a2)) > A) continue;
                        cnt += above_cut(c, same_double_value(dpair, NP, r1, r2, a1, a2), cut);
                    }
                }
                cnt = __reduce_add_sync(0xffffffffu, cnt);
                if (lane == 0 && cnt) atomicAdd(&hist[class_of(F.ZcA) - lo], cnt);
            }
        } else if (!sym) {
            if (tid == 0 && a_in)
                atomicAdd(&hist[class_of(F.ZcA) - lo], (uint32_t)(p.n_sb + n_occ_pairs_b * n_vir_pairs_b));
            for (int k = tid; k < n_sa_pass; k += kGenThreads) {
                int s = sa_pass[k];
                atomicAdd(&hist[class_of(sa_zt[s]) - lo], (uint32_t)(1 + p.n_sb));
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
                if (lane == 0) atomicAdd(&hist[class_of(sa_zt[s]) - lo], cnt + (a2 >= B ? 1u : 0u));
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
                if (lane == 0 && cnt) atomicAdd(&hist[class_of(F.ZcA) - lo], cnt);
            }
        }
        // alpha-alpha doubles (beta string B): every candidate when all classes
        // are counted; for a narrower range only those of the bucket ranges
        // the range maps to (as the emission finds them), each checked class
        // by class
        auto count_aa = [&](uint64_t z12, uint64_t a12, int r1, int r2, int pv) {
            const int a1 = F.virA[pv & 0xFF], a2 = F.virA[pv >> 8];
            const uint32_t h = class_of(z12 ^ F.zc[a1] ^ F.zc[a2]) - lo;
            if (h >= n_hist) return;
            const uint64_t al = a12 ^ (1ull << a1) ^ (1ull << a2);
            if (!cons_ok(p.cons_mod, p.cons_rem, p.top_hi, p.top_mask, al)) return;
            if (sym && al < B) return;
            if (cutting && !above_cut(c, same_double_value(dpair, NP, r1, r2, a1, a2), cut)) return;
            atomicAdd(&hist[h], 1u);
        };
        if (n_hist == (uint32_t)kNumClasses) {
            for (int pi = warp; pi < n_occ_pairs_a; pi += nw) {
                const int pr = pairs[pi];
                const int r1 = F.occA[pr & 0xFF], r2 = F.occA[pr >> 8];
                const uint64_t z12 = F.ZcA ^ F.zc[r1] ^ F.zc[r2];
                const uint64_t a12 = A ^ (1ull << r1) ^ (1ull << r2);
                for (int t = lane; t < n_vir_pairs_a; t += 32) count_aa(z12, a12, r1, r2, pairs[t]);
            }
        } else {
            uint32_t *vb_cnt = reinterpret_cast<uint32_t *>(smem + p.smem_vbk);
            uint16_t *vb_off = reinterpret_cast<uint16_t *>(vb_cnt + kVbkBuckets);
            uint16_t *vb_list = vb_off + kVbkBuckets + 1;
            build_vbk(F, pairs, n_vir_pairs_a, p.class_lo, p.class_hi, vb_cnt, vb_off, vb_list);
            for (int pi = warp; pi < n_occ_pairs_a; pi += nw) {
                const int pr = pairs[pi];
                const int r1 = F.occA[pr & 0xFF], r2 = F.occA[pr >> 8];
                const uint64_t z12 = F.ZcA ^ F.zc[r1] ^ F.zc[r2];
                const uint64_t a12 = A ^ (1ull << r1) ^ (1ull << r2);
                const uint32_t u = vb_bucket(z12);
                for (int q = 0; q < F.n_blk; ++q) {
                    const uint32_t k = F.blk_k[q];
                    const uint32_t bb = (F.blk_g[q] ^ u) & ~((1u << k) - 1u);
                    const int st = vb_off[bb], en = vb_off[bb + (1u << k)];
                    for (int i = st + lane; i < en; i += 32) count_aa(z12, a12, r1, r2, pairs[vb_list[i]]);
                }
            }
        }
        __syncthreads();
        for (int i = tid; i < (int)n_hist; i += kGenThreads)
            if (hist[i]) atomicAdd(&p.class_counts[lo + i], (unsigned long long)hist[i]);
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
                if (!cons_ok(p.cons_mod, p.cons_rem, p.top_hi, p.top_mask, al)) continue;
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
        out.ctr = MODE == kModeTileCount ? p.tile_counts + p.tile_base
                  : MODE == kModeEmit    ? p.cursor + p.tile_base
                                         : p.cursor;
        out.recs = p.recs;
        out.n_tiles = (uint32_t)p.n_tiles;
        out.rec_cap = (uint32_t)min(p.rec_cap, (unsigned long long)0xFFFFFFFFull);
        out.err = p.err;
        out.e0 = p.e0;
        out.gtab = grouped ? F.grp + kMaxGrp + 1 : nullptr;
        const uint32_t q_a = F.q_a;  // pass of A (grouped count)
        const uint32_t class_lo = p.class_lo, class_hi = p.class_hi;
        // beta singles of the pass: all of them, or the compacted list
        const int n_sb = bfull ? p.n_sb : F.n_sb_pass;
        auto sb_at = [&](int k) { return bfull ? k : (int)sb_pass[k]; };

        // bucket table of the virtual alpha pairs, and the pass's classes as
        // aligned blocks of bucket groups
        uint32_t *vb_cnt = reinterpret_cast<uint32_t *>(smem + p.smem_vbk);
        uint16_t *vb_off = reinterpret_cast<uint16_t *>(vb_cnt + kVbkBuckets);
        uint16_t *vb_list = vb_off + kVbkBuckets + 1;
        if (b_in) build_vbk(F, pairs, n_vir_pairs_a, class_lo, class_hi, vb_cnt, vb_off, vb_list);  // uniform

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
                    zt = with_pass(sa_zt[s] ^ ZtbB, sa_info[s] >> 18);
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
                        zt = with_pass(ZtaA ^ sb_zt[s], q_a);
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
        // ---- alpha-beta doubles: every (alpha single of the pass, beta single)
        // item over the whole CTA, in groups of up to kAbGroup alpha singles (a
        // pass holding few classes has few alpha singles, and one per warp
        // would leave most warps idle).  Items of one alpha single are
        // consecutive, so lanes take consecutive beta singles (same rB,
        // ascending aB) and the integral (aA rA|aB rB) = (rA aA|rB aB) is read
        // contiguously.  Row j of vec holds u[q] = J(aA, q) - J(rA, q) for the
        // group's alpha single j: the alpha-beta cross terms of H_aa.
        {
            constexpr int kAbGroup = kGenThreads / 32;  // rows of vec
            const uint32_t nsb = (uint32_t)n_sb;
            // i / nsb = umulhi(i, ceil(2^32 / nsb)) exactly while i * nsb < 2^32
            const uint32_t magic = nsb ? (uint32_t)((0x100000000ull + nsb - 1) / nsb) : 0u;
            for (int g0 = 0; g0 < n_sa_pass; g0 += kAbGroup) {  // uniform across the CTA
                const int ng = min(kAbGroup, n_sa_pass - g0);
                __syncthreads();  // vec rows free
                if constexpr (kVal) {
                    for (int j = warp; j < ng; j += nw) {
                        const uint32_t ia = sa_info[sa_pass[g0 + j]];
                        const int rA = ia & 0xFF, aA = (ia >> 8) & 0xFF;
                        for (int q = lane; q < N; q += 32) vec_all[j * kMaxOrb + q] = Jx[aA * N + q] - Jx[rA * N + q];
                    }
                }
                __syncthreads();
                const int nitems = ng * n_sb;
                for (int i0 = tid; i0 < nitems; i0 += kGenThreads * kGenBatch)
                    emit_batch<MODE>(
                        out, i0, kGenThreads, nitems,
                        [&](int i, uint64_t &zt, double &el) {
                            const int j = (int)__umulhi((uint32_t)i, magic), k = i - j * n_sb;
                            const int s = sa_pass[g0 + j], sb = sb_at(k);
                            const uint32_t ia = sa_info[s];
                            if (sym && single_word(B, sb_info[sb]) > single_word(A, ia)) return false;
                            if (cutting) {
                                const uint32_t bi = sb_info[sb];
                                el = __ldg(eri + (((size_t)(ia & 0xFF) * N + ((ia >> 8) & 0xFF)) * N + (bi & 0xFF)) * N +
                                           ((bi >> 8) & 0xFF));
                                if (!above_cut(c, el, cut)) return false;
                            }
                            zt = with_pass(sa_zt[s] ^ sb_zt[sb], ia >> 18);
                            return true;
                        },
                        [&](int i, uint64_t &ka, uint64_t &kb, double &num, int64_t &den, double el) {
                            const int j = (int)__umulhi((uint32_t)i, magic), k = i - j * n_sb;
                            const int s = sa_pass[g0 + j], sb = sb_at(k);
                            const uint32_t ia = sa_info[s], bi = sb_info[sb];
                            const int rA = ia & 0xFF, aA = (ia >> 8) & 0xFF, rB = bi & 0xFF, aB = (bi >> 8) & 0xFF;
                            ka = A ^ (1ull << rA) ^ (1ull << aA);
                            kb = B ^ (1ull << rB) ^ (1ull << aB);
                            const double v =
                                cutting ? el : __ldg(eri + (((size_t)rA * N + aA) * N + rB) * N + aB);
                            num = flip_sign(c * v, (ia >> 16) ^ (bi >> 16));
                            const int64_t *u = vec_all + j * kMaxOrb;
                            den = d0 - sa_delta[s] - sb_delta[sb] - (u[aB] - u[rB]);
                        });
            }
        }
        // ---- alpha-alpha doubles (beta string B).  The candidates of an
        // occupied pair are the virtual pairs of the bucket ranges the pass's
        // class blocks map to (block xor the top bits of the occupied part's
        // class hash).  A pass holding few classes leaves each occupied pair
        // few candidates, so they are enumerated over the whole CTA: the
        // candidate count of every occupied pair, a block scan, one thread per
        // candidate checking its class and listing it, and the list emitted
        // with every lane busy, in rounds of at most kListCap candidates.
        if (b_in) {  // uniform across the CTA
            uint32_t *poff = vb_cnt;                                  // candidate offsets of the occupied pairs
            uint32_t *clist = reinterpret_cast<uint32_t *>(vec_all);  // (occupied pair << 16) | virtual pair
            constexpr int kPairGroup = kVbkBuckets - 1;
            constexpr uint32_t kListCap = (uint32_t)(kGenThreads / 32 * kMaxOrb * 8 / 4);
            constexpr int kAaBatch = 4;  // terms whose slots a lane requests together here (fewer live registers)
            const int npo = n_occ_pairs_a;
            const uint32_t lt = (1u << lane) - 1u;
            auto key_aa = [&](int k, uint64_t &zt, double &el) {
                const uint32_t e = clist[k];
                const int pr = pairs[(e >> 16) & 0x3FFu], pv = pairs[e & 0xFFFFu];
                const int r1 = F.occA[pr & 0xFF], r2 = F.occA[pr >> 8];
                const int a1 = F.virA[pv & 0xFF], a2 = F.virA[pv >> 8];
                if (cutting) {
                    el = same_double_value(dpair, NP, r1, r2, a1, a2);
                    if (!above_cut(c, el, cut)) return false;
                }
                zt = with_pass(ZtaA ^ ZtbB ^ F.zta[r1] ^ F.zta[r2] ^ F.zta[a1] ^ F.zta[a2], e >> 26);
                return true;
            };
            auto val_aa = [&](int k, uint64_t &ka, uint64_t &kb, double &num, int64_t &den, double el) {
                const uint32_t e = clist[k];
                const int pr = pairs[(e >> 16) & 0x3FFu], pv = pairs[e & 0xFFFFu];
                const int r1 = F.occA[pr & 0xFF], r2 = F.occA[pr >> 8];
                const int a1 = F.virA[pv & 0xFF], a2 = F.virA[pv >> 8];
                const uint64_t w1 = A ^ (1ull << r1) ^ (1ull << a1);
                ka = w1 ^ (1ull << r2) ^ (1ull << a2);
                kb = B;
                const uint32_t par = __popcll(A & between_mask(r1, a1)) + __popcll(w1 & between_mask(r2, a2));
                const double v = cutting ? el : same_double_value(dpair, NP, r1, r2, a1, a2);
                num = flip_sign(c * v, par);
                // H_aa - H_ii = -g(r1) - g(r2) + W(r1,r2) + v(a1) + v(a2) + W(a1,a2),
                // v(x) = g(x) - W(r1,x) - W(r2,x)
                den = d0 + F.gA[r1] + F.gA[r2] - __ldg(WSx + r1 * N + r2) -
                      (F.gA[a1] - __ldg(WSx + r1 * N + a1) - __ldg(WSx + r2 * N + a1)) -
                      (F.gA[a2] - __ldg(WSx + r1 * N + a2) - __ldg(WSx + r2 * N + a2)) - __ldg(WSx + a1 * N + a2);
            };
            __syncthreads();  // the alpha-beta warps are done with vec
            // list the candidates [c0, c1) that `cand` turns into items and emit
            // them, in rounds of at most kListCap
            auto list_and_emit = [&](uint32_t total, auto cand) {
                for (uint32_t c0 = 0; c0 < total; c0 += kListCap) {
                    if (tid == 0) F.n_list = 0;
                    __syncthreads();
                    const uint32_t c1 = min(total, c0 + kListCap);
                    for (uint32_t cb = c0; cb < c1; cb += kGenThreads) {
                        const uint32_t ci = cb + tid;
                        uint32_t item = 0;
                        const bool keep = ci < c1 && cand(ci, item);
                        const uint32_t m = __ballot_sync(0xffffffffu, keep);
                        if (m) {
                            const int leader = __ffs(m) - 1;
                            uint32_t base = 0;
                            if (lane == leader) base = atomicAdd(&F.n_list, (unsigned)__popc(m));
                            base = __shfl_sync(0xffffffffu, base, leader);
                            if (keep) clist[base + __popc(m & lt)] = item;
                        }
                    }
                    __syncthreads();
                    const int nl = (int)F.n_list;
                    for (int k0 = tid; k0 < nl; k0 += kGenThreads * kAaBatch)
                        emit_batch<MODE, kAaBatch>(out, k0, kGenThreads, nl, key_aa, val_aa);
                    __syncthreads();  // the list area is reused
                }
            };
            // an item of occupied pair pi and virtual pair vp (colex pair
            // indices into occA / virA) if its alpha class lies in the pass
            // and it meets the constraints
            auto aa_item = [&](int pi, int vp, uint32_t &item) {
                const int pr = pairs[pi], pv = pairs[vp];
                const int r1 = F.occA[pr & 0xFF], r2 = F.occA[pr >> 8];
                const int a1 = F.virA[pv & 0xFF], a2 = F.virA[pv >> 8];
                const uint32_t cl = class_of(F.ZcA ^ F.zc[r1] ^ F.zc[r2] ^ F.zc[a1] ^ F.zc[a2]);
                const uint64_t w2 = A ^ (1ull << r1) ^ (1ull << r2) ^ (1ull << a1) ^ (1ull << a2);
                const bool in = cl >= p.class_lo && cl < p.class_hi &&
                                cons_ok(p.cons_mod, p.cons_rem, p.top_hi, p.top_mask, w2) && !(sym && w2 < B);
                // bits 0-15 the virtual pair, 16-25 the occupied pair (< 1024
                // for 64 orbitals), 26-31 the pass of a grouped count
                item = ((grouped && in ? grp_of(cl) : 0u) << 26) | ((uint32_t)pi << 16) | (uint32_t)vp;
                return in;
            };
            if (p.top_mask) {
                // Algorithm 3 (fast generation for a triplet constraint T): the
                // double keeps T as the highest occupied orbitals iff it removes
                // every occupied orbital at or above T's lowest that is not in T
                // (R), adds the orbitals of T that are empty (Q), and takes its
                // other orbitals below T's lowest.  Those are the first L
                // occupied and the first Lv virtual orbitals, so the occupied
                // pairs (and likewise the virtual ones) are: R itself (|R| = 2),
                // R's orbital with each of the first L (|R| = 1), or every pair
                // of the first L (|R| = 0).
                const uint64_t T = p.top_mask;
                const uint64_t R = A & p.top_hi & ~T, Q = T & ~A;
                const int nr = __popcll(R), nq = __popcll(Q);
                const int tlo = __ffsll((long long)T) - 1;
                const int L = __popcll(A & ((1ull << tlo) - 1ull)), Lv = tlo - L;
                const bool fits = nr <= 2 && nq <= 2 && (N >= 64 || (T >> N) == 0);
                if (fits) {  // uniform across the CTA
                    auto colex = [](int i, int j) { return j * (j - 1) / 2 + i; };  // pair i < j
                    auto occ_pos = [&](uint64_t bits) { return __popcll(A & (bits - 1ull)); };
                    auto vir_pos = [&](uint64_t bits) { return (__ffsll((long long)bits) - 1) - occ_pos(bits); };
                    const uint64_t r1b = R & (~R + 1ull), q1b = Q & (~Q + 1ull);
                    const int ir1 = nr ? occ_pos(r1b) : 0, ir2 = nr == 2 ? occ_pos(R ^ r1b) : 0;
                    const int iq1 = nq ? vir_pos(q1b) : 0, iq2 = nq == 2 ? vir_pos(Q ^ q1b) : 0;
                    const uint32_t nO = nr == 2 ? 1u : nr == 1 ? (uint32_t)L : (uint32_t)(L * (L - 1) / 2);
                    const uint32_t nV = nq == 2 ? 1u : nq == 1 ? (uint32_t)Lv : (uint32_t)(Lv * (Lv - 1) / 2);
                    list_and_emit(nO * nV, [&](uint32_t ci, uint32_t &item) {
                        const int io = (int)(ci / nV), iv = (int)(ci - (uint32_t)io * nV);
                        const int pi = nr == 2 ? colex(ir1, ir2) : nr == 1 ? colex(io, ir1) : io;
                        const int vp = nq == 2 ? colex(iq1, iq2) : nq == 1 ? colex(iv, iq1) : iv;
                        return aa_item(pi, vp, item);
                    });
                }
            } else {
            for (int p0 = 0; p0 < npo; p0 += kPairGroup) {
                const int np = min(kPairGroup, npo - p0);
                for (int t = tid; t <= np; t += kGenThreads) {
                    uint32_t n = 0;
                    if (t < np) {
                        const int pr = pairs[p0 + t];
                        const uint32_t u = vb_bucket(F.ZcA ^ F.zc[F.occA[pr & 0xFF]] ^ F.zc[F.occA[pr >> 8]]);
                        for (int q = 0; q < F.n_blk; ++q) {
                            const uint32_t k = F.blk_k[q];
                            const uint32_t bb = (F.blk_g[q] ^ u) & ~((1u << k) - 1u);
                            n += (uint32_t)vb_off[bb + (1u << k)] - vb_off[bb];
                        }
                    }
                    poff[t] = n;
                }
                __syncthreads();
                block_scan_excl_u32(poff, np + 1, F.wsum);
                list_and_emit(poff[np], [&](uint32_t ci, uint32_t &item) {
                    int lo = 0, hi = np;  // the occupied pair: last t with poff[t] <= ci
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (poff[mid] <= ci) lo = mid;
                        else hi = mid;
                    }
                    const int pr = pairs[p0 + lo];
                    const uint32_t u = vb_bucket(F.ZcA ^ F.zc[F.occA[pr & 0xFF]] ^ F.zc[F.occA[pr >> 8]]);
                    uint32_t i = ci - poff[lo];
                    int vp = 0;
                    for (int q = 0; q < F.n_blk; ++q) {
                        const uint32_t k = F.blk_k[q];
                        const uint32_t bb = (F.blk_g[q] ^ u) & ~((1u << k) - 1u);
                        const uint32_t st = vb_off[bb], sz = (uint32_t)vb_off[bb + (1u << k)] - st;
                        if (i < sz) {
                            vp = vb_list[st + i];
                            break;
                        }
                        i -= sz;
                    }
                    return aa_item(p0 + lo, vp, item);
                });
            }
            }
        }
        // ---- beta-beta doubles (alpha string A): one occupied pair per warp,
        // virtual pairs over lanes.  In an ordinary pass every virtual pair
        // gives a term of the pass and the terms are emitted straight away.
        // Where an item needs a check (the beta class in a pass over part of
        // a heavy alpha class, the spin-flip rule) the warp first lists the
        // items that pass it, gathering several occupied pairs, and emits the
        // list with every lane busy.
        if (a_in) {  // uniform across the CTA
            uint32_t *wl = reinterpret_cast<uint32_t *>(vec);  // the warp's item list (its row of vec)
            constexpr int kWarpList = kMaxOrb * 8 / 4;
            const uint32_t lt = (1u << lane) - 1u;
            const int npo = n_occ_pairs_b, npv = n_vir_pairs_b;
            const bool listed = !bfull || sym;
            int nl = 0;
            // emit the listed items, each (occupied pair << 16) | virtual pair
            auto flush = [&]() {
                __syncwarp();
                for (int k0 = lane; k0 < nl; k0 += 32 * kGenBatch)
                    emit_batch<MODE>(
                        out, k0, 32, nl,
                        [&](int k, uint64_t &zt, double &el) {
                            const uint32_t e = wl[k];
                            const int pr = pairs[e >> 16], pv = pairs[e & 0xFFFFu];
                            const int r1 = F.occB[pr & 0xFF], r2 = F.occB[pr >> 8];
                            const int a1 = F.virB[pv & 0xFF], a2 = F.virB[pv >> 8];
                            if (cutting) {
                                el = same_double_value(dpair, NP, r1, r2, a1, a2);
                                if (!above_cut(c, el, cut)) return false;
                            }
                            zt = with_pass(ZtaA ^ ZtbB ^ F.ztb[r1] ^ F.ztb[r2] ^ F.ztb[a1] ^ F.ztb[a2], q_a);
                            return true;
                        },
                        [&](int k, uint64_t &ka, uint64_t &kb, double &num, int64_t &den, double el) {
                            const uint32_t e = wl[k];
                            const int pr = pairs[e >> 16], pv = pairs[e & 0xFFFFu];
                            const int r1 = F.occB[pr & 0xFF], r2 = F.occB[pr >> 8];
                            const int a1 = F.virB[pv & 0xFF], a2 = F.virB[pv >> 8];
                            const uint64_t w1 = B ^ (1ull << r1) ^ (1ull << a1);
                            ka = A;
                            kb = w1 ^ (1ull << r2) ^ (1ull << a2);
                            const uint32_t par =
                                __popcll(B & between_mask(r1, a1)) + __popcll(w1 & between_mask(r2, a2));
                            const double v = cutting ? el : same_double_value(dpair, NP, r1, r2, a1, a2);
                            num = flip_sign(c * v, par);
                            den = d0 + F.gB[r1] + F.gB[r2] - __ldg(WSx + r1 * N + r2) -
                                  (F.gB[a1] - __ldg(WSx + r1 * N + a1) - __ldg(WSx + r2 * N + a1)) -
                                  (F.gB[a2] - __ldg(WSx + r1 * N + a2) - __ldg(WSx + r2 * N + a2)) -
                                  __ldg(WSx + a1 * N + a2);
                        });
                __syncwarp();
                nl = 0;
            };
            for (int pi = warp; pi < npo; pi += nw) {
                const int pr = pairs[pi];
                const int r1 = F.occB[pr & 0xFF], r2 = F.occB[pr >> 8];
                const uint64_t w12 = B ^ (1ull << r1) ^ (1ull << r2);
                if (!listed) {
                    // every virtual pair is a term of the pass
                    int64_t base = 0;
                    if constexpr (kVal) {
                        for (int j = lane; j < nvb; j += 32) {
                            const int x = F.virB[j];
                            vec[j] = F.gB[x] - WSx[r1 * N + x] - WSx[r2 * N + x];
                        }
                        __syncwarp();
                        base = d0 + F.gB[r1] + F.gB[r2] - WSx[r1 * N + r2];
                    }
                    const uint64_t zt12 = ZtaA ^ ZtbB ^ F.ztb[r1] ^ F.ztb[r2];
                    for (int t0 = lane; t0 < npv; t0 += 32 * kGenBatch)
                        emit_batch<MODE>(
                            out, t0, 32, npv,
                            [&](int t, uint64_t &zt, double &el) {
                                const int pv = pairs[t];
                                const int a1 = F.virB[pv & 0xFF], a2 = F.virB[pv >> 8];
                                if (cutting) {
                                    el = same_double_value(dpair, NP, r1, r2, a1, a2);
                                    if (!above_cut(c, el, cut)) return false;
                                }
                                zt = with_pass(zt12 ^ F.ztb[a1] ^ F.ztb[a2], q_a);
                                return true;
                            },
                            [&](int t, uint64_t &ka, uint64_t &kb, double &num, int64_t &den, double el) {
                                const int pv = pairs[t];
                                const int j1 = pv & 0xFF, j2 = pv >> 8;
                                const int a1 = F.virB[j1], a2 = F.virB[j2];
                                const uint64_t w1 = B ^ (1ull << r1) ^ (1ull << a1);
                                ka = A;
                                kb = w12 ^ (1ull << a1) ^ (1ull << a2);
                                const uint32_t par =
                                    __popcll(B & between_mask(r1, a1)) + __popcll(w1 & between_mask(r2, a2));
                                // a1 is the fastest-varying index across lanes
                                const double v = cutting ? el : same_double_value(dpair, NP, r1, r2, a1, a2);
                                num = flip_sign(c * v, par);
                                den = base - vec[j1] - vec[j2] - __ldg(WSx + a1 * N + a2);
                            });
                    __syncwarp();
                    continue;
                }
                const uint64_t zcb12 = F.ZcbB ^ F.zcb[r1] ^ F.zcb[r2];
                for (int c0 = 0; c0 < npv; c0 += 32) {
                    const int t = c0 + lane;
                    bool keep = false;
                    if (t < npv) {
                        const int pv = pairs[t];
                        const int a1 = F.virB[pv & 0xFF], a2 = F.virB[pv >> 8];
                        const uint32_t bc = bclass_of(zcb12 ^ F.zcb[a1] ^ F.zcb[a2]);
                        keep = (bfull || (bc >= p.bclass_lo && bc < p.bclass_hi)) &&
                               !(sym && (w12 ^ (1ull << a1) ^ (1ull << a2)) > A);
                    }
                    const uint32_t m = __ballot_sync(0xffffffffu, keep);
                    if (nl + __popc(m) > kWarpList) flush();  // uniform across the warp
                    if (keep) wl[nl + __popc(m & lt)] = ((uint32_t)pi << 16) | (uint32_t)t;
                    nl += __popc(m);
                }
                if (nl > kWarpList - 32) flush();
            }
            flush();
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

// d0 = (E0 - H_ii) 2^48 of every reference determinant, exactly from the
// integer tables: sum over the occupied spin-orbitals x of (h_xx + g(x))
// counts each one-electron energy twice and each pair energy <xj||xj> twice,
// so it is 2 H_ii (2^-48 Ha).  A term's E0 - H_aa, assembled from its parent's
// d0 and integer increments, is then the same integer whichever reference
// determinant generated it.
__global__ void ref_d0_kernel(const SysDev sys, const uint64_t *__restrict__ keys, const int64_t *__restrict__ g,
                              uint64_t n, int64_t e0x, int64_t *__restrict__ d0)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int N = sys.n;
    const int64_t *gi = g + i * 2 * N;
    int64_t s = 0;
    for (uint64_t m = keys[2 * i]; m; m &= m - 1) {
        const int x = __ffsll((long long)m) - 1;
        s += sys.hdx[x] + gi[x];
    }
    for (uint64_t m = keys[2 * i + 1]; m; m &= m - 1) {
        const int x = __ffsll((long long)m) - 1;
        s += sys.hdx[x] + gi[N + x];
    }
    d0[i] = e0x - (s >> 1);
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

cudaError_t launch_ref_d0(const SysDev &sys, const uint64_t *keys, const int64_t *g, uint64_t n, double e0,
                          int64_t *d0, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    ref_d0_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sys, keys, g, n, (int64_t)std::llrint(e0 * kDenScale), d0);
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
        cons_ok(q.cons_mod, q.cons_rem, q.top_hi, q.top_mask, A)) {
        t = (uint32_t)(q.tile_base + tile_of(zt, (uint32_t)q.n_tiles));
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
    uint32_t n_in_ref, n_ext, n_pos, n_coll;  // distinct keys = n_in_ref + n_ext
    uint32_t err;
    __device__ void clear()
    {
        e2_lo = 0;
        e2_hi = 0;
        dsum = dxor = 0;
        min_den = ~0ull;
        n_in_ref = n_ext = n_pos = n_coll = 0;
        err = 0;
    }
};

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

// One distinct key: explicit filter against the reference slice, then the
// Epstein-Nesbet term num^2 / (E0 - H_aa) of Eq. 3, added exactly.
// In a spin-flip symmetric run (sym) a key with a > b stands for itself and
// its mirror (b, a), whose term is the same, so it counts twice (one more
// power of two in the fixed-point addition).
__device__ __forceinline__ void finish_key(const TileParams &p, double e0, bool sym, const uint64_t *rk,
                                           unsigned long long nrk, uint64_t a, uint64_t b, double num, int64_t den,
                                           KeyStats &st)
{
    if (nrk && in_slice(rk, nrk, a, b)) {
        st.n_in_ref++;
        return;
    }
    fx_add_double(st.e2_lo, st.e2_hi, term_fx48(num, den), st.err,
                  kFxShift + kDenShift + ((sym && a != b) ? 1 : 0));
    st.n_ext++;
    const uint64_t ad = den < 0 ? (uint64_t)(-den) : (uint64_t)den;
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
            p.dump_haa[slot] = e0 - den_to_double(den);
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
        st.n_in_ref += __shfl_down_sync(0xffffffffu, st.n_in_ref, off);
        st.n_ext += __shfl_down_sync(0xffffffffu, st.n_ext, off);
        st.n_pos += __shfl_down_sync(0xffffffffu, st.n_pos, off);
        st.n_coll += __shfl_down_sync(0xffffffffu, st.n_coll, off);
        st.err |= __shfl_down_sync(0xffffffffu, st.err, off);
    }
    if (lane == 0) {
        red[0][warp] = st.e2_lo;
        red[1][warp] = (unsigned long long)st.e2_hi;
        red[2][warp] = st.dsum;
        red[3][warp] = st.dxor;
        red[4][warp] = st.min_den;
        red[6][warp] = st.n_in_ref;
        red[7][warp] = st.n_ext;
        red[8][warp] = st.n_pos;
        red[9][warp] = st.err;
        red[10][warp] = st.n_coll;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t lo = 0, dsum = 0, dxor = 0, mind = ~0ull, nr = 0, ne = 0, np = 0, er = 0, nc = 0;
        int64_t hi = 0;
        for (int w = 0; w < nw; ++w) {
            fx_add_fx(lo, hi, red[0][w], (int64_t)red[1][w]);
            dsum += red[2][w];
            dxor ^= red[3][w];
            mind = red[4][w] < mind ? red[4][w] : mind;
            nr += red[6][w];
            ne += red[7][w];
            np += red[8][w];
            er |= red[9][w];
            nc += red[10][w];
        }
        unsigned long long old = atomicAdd(&acc->e2_lo, (unsigned long long)lo);
        unsigned long long carry = (old + lo) < old ? 1ull : 0ull;
        atomicAdd((unsigned long long *)&acc->e2_hi, (unsigned long long)hi + carry);
        atomicAdd(&acc->dsum, dsum);
        atomicXor(&acc->dxor, dxor);
        atomicMin(&acc->min_den, mind);
        atomicAdd(&acc->n_unique, nr + ne);
        atomicAdd(&acc->n_in_ref, nr);
        atomicAdd(&acc->n_ext, ne);
        atomicAdd(&acc->n_pos, np);
        if (nc) atomicAdd(&acc->n_coll, nc);
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

constexpr uint32_t kNarrowMask = 0x03C00000u;  // 4 hash bits, all inside the bucket digit
constexpr long long kWaitCycles = 1ll << 31;    // about a second
constexpr long long kShortWaitCycles = 64;      // shorter than any global-memory copy

// ------------------------------------------ in-tile bucket sort + reduce
//
// A tile (or a chunk of an oversize tile) of at most kGrpCap records sits in
// shared memory.  Its records are sorted so that equal keys share a bucket
// and every key is reduced once (the sort and the single pass of
// Algorithm 1):
//   1. one counting-sort pass on the top 10 bits of a 32-bit hash of the key
//      (1024 buckets): a record's rank inside its bucket from a
//      shared-memory atomic, bucket starts from a block scan, one scatter;
//   2. one lane per record: it heads its key if no earlier record of its
//      bucket has the same (hash, alpha word, beta word).  Keys that share
//      the 32-bit hash are told apart by the full 128-bit comparison, so the
//      grouping is exact whatever the hash does;
//   3. one lane per distinct key: the head adds up the records of its key
//      that follow it in the bucket and finishes the key; a head with a long
//      tail (a key with many duplicates) is summed by a warp.
// A key's numerator is the exact fixed-point sum of its contributions (a
// single contribution is rounded to the same 2^-90 grid), so the result does
// not depend on the order in which records meet, on the tiling or on which
// path summed the key.  E0 - H_aa is the same exact integer in every record of
// a key (it is assembled from integer tables), so the head record supplies it.

constexpr int kGrpThreads = kTileThreads;
constexpr int kGrpWarps = kGrpThreads / 32;
constexpr int kGrpCap = kTileCap;
constexpr int kGrpBuckets = 1024;
constexpr int kGrpItems = kGrpCap / kGrpThreads;  // records per thread
constexpr int kGrpBktShift = 22;                  // bucket = top 10 bits of the hash
constexpr int kLongTail = 16;                     // heads with more records after them are summed by a warp
constexpr int kTileCtasPerSm = 4;                 // resident tile CTAs the registers are sized for
static_assert(kGrpBuckets == 4 * kGrpThreads, "each thread clears four buckets");
static_assert(kGrpBuckets == (1 << (32 - kGrpBktShift)), "the bucket digit is the top bits of the hash");
static_assert(kGrpCap <= 1024 && kGrpItems * kGrpThreads == kGrpCap, "record indices take 10 bits");
static_assert(kBigThreads == kGrpThreads, "every grouping CTA has the grouping's width");
static_assert(kBigChunk <= kGrpCap && kBigCap <= kGrpCap, "chunks fit one grouping");
static_assert(kGrpCap / (kLongTail + 1) <= kGrpThreads, "long heads fit their list");

struct GrpSmem {
    uint64_t ent[kGrpCap];      // (hash << 32) | record index, bucket by bucket
    uint32_t cnt[kGrpBuckets];  // bucket sizes, then bucket starts; zero between groupings
    uint16_t uniq[kGrpCap];     // position (in ent) of the head of each distinct key
    uint16_t lng[kGrpThreads];  // heads with a long tail
    uint32_t warp_tot[kGrpWarps];
    unsigned int nuniq, nlong;
};

// 64-bit hash of a key for the hashed-key grouping (the hashing section):
// SplitMix64's finaliser on both words, combined by an odd multiplier.
__device__ __forceinline__ uint64_t key_hash64(uint64_t a, uint64_t b)
{
    return fmix64((a * 0x9E3779B97F4A7C15ull) ^ fmix64(b));
}

// Distinct keys listed by the last grouping (its heads, then its long heads).
__device__ __forceinline__ int group_keys(const GrpSmem &G) { return (int)(G.nuniq + G.nlong); }

// 32-bit hash that orders the records of a tile.  The keys of a tile share
// its tile hash (a Zobrist hash of the key), so this one mixes the two words
// with unrelated multipliers.
__device__ __forceinline__ uint32_t sort_hash(uint64_t a, uint64_t b)
{
    uint64_t h = (a * 0x9E3779B97F4A7C15ull) ^ b;
    h ^= h >> 32;
    h *= 0xD6E8FEB86659FD93ull;
    return (uint32_t)(h >> 32);
}

// A single contribution as the exact fixed-point sum gives it: values from
// 2^-38 up are on the 2^-90 grid already, smaller ones are rounded to it,
// values of 2^36 and more are out of range.
__device__ __forceinline__ double canon_num(double v, uint32_t &err)
{
    const int e = (int)((__double_as_longlong(v) >> 52) & 0x7FF);
    if (e >= 1023 - 38 && e < 1023 + 36) return v;
    uint64_t lo = 0;
    int64_t hi = 0;
    fx_add_double(lo, hi, v, err);
    return fx_to_double(lo, hi);
}

// Record access for the grouping: the key, and adding a record's numerator
// to an exact fixed-point sum.
struct R32 {
    using Rec = Rec32;
    static __device__ __forceinline__ void key(const Rec32 *r, int i, uint64_t &a, uint64_t &b)
    {
        const ulonglong2 k = *reinterpret_cast<const ulonglong2 *>(r + i);
        a = k.x;
        b = k.y;
    }
    static __device__ __forceinline__ void add(const Rec32 *r, int i, uint64_t &fl, int64_t &fh, uint32_t &err)
    {
        fx_add_double(fl, fh, r[i].num, err);
    }
};
struct R48 {
    using Rec = Rec48;
    static __device__ __forceinline__ void key(const Rec48 *r, int i, uint64_t &a, uint64_t &b)
    {
        const ulonglong2 k = *reinterpret_cast<const ulonglong2 *>(r + i);
        a = k.x;
        b = k.y;
    }
    static __device__ __forceinline__ void add(const Rec48 *r, int i, uint64_t &fl, int64_t &fh, uint32_t &)
    {
        fx_add_fx(fl, fh, r[i].fx_lo, r[i].fx_hi);
    }
};

// Group the cnt <= kGrpCap records of `recs` (shared memory) by key.  Every
// distinct key is handed to run(head, exact, fl, fh), once, by one thread:
// head is the index of one of its records; if exact, (fl, fh) is the exact
// numerator sum of all its records, otherwise head is its only record.  On
// return G.uniq[0, group_keys(G)) lists the head record of every distinct key
// (for a dense finish by the caller).  hmask narrows the hash (a test aid
// that makes most keys of a tile share their hash and bucket).  Returns how
// often this thread met two different keys with the same hash.  Every thread
// of the CTA must call it; it starts after and ends with a barrier.
template <class R, bool HK = false, class Run>
__device__ uint32_t group_records(const typename R::Rec *recs, int cnt, uint32_t hmask, GrpSmem &G, uint32_t &err,
                                  Run &&run)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    if (tid == 0) {
        G.nuniq = 0;
        G.nlong = 0;
    }
    // 1. hash and rank within the bucket.  An entry is (hash << 32) | index,
    // or with hashed keys (HK) the 64-bit key hash whose low 10 bits hold the
    // index; either way its top 10 bits are the bucket.
    uint64_t hh[kGrpItems];
    uint32_t rk[kGrpItems];
#pragma unroll
    for (int k = 0; k < kGrpItems; ++k) {
        const int i = tid + k * kGrpThreads;
        hh[k] = 0;
        rk[k] = 0;
        if (i < cnt) {
            uint64_t a, b;
            R::key(recs, i, a, b);
            if constexpr (HK) hh[k] = (key_hash64(a, b) & ~0x3FFull) | (uint64_t)i;
            else hh[k] = ((uint64_t)(sort_hash(a, b) & hmask) << 32) | (uint64_t)i;
            rk[k] = atomicAdd(&G.cnt[hh[k] >> 54], 1u);
        }
    }
    __syncthreads();
    // bucket starts (thread t scans buckets 4t .. 4t + 3)
    {
        const uint4 c4 = reinterpret_cast<const uint4 *>(G.cnt)[tid];
        const uint32_t sz = c4.x + c4.y + c4.z + c4.w;
        uint32_t incl = sz;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += t;
        }
        if (lane == 31) G.warp_tot[warp] = incl;
        __syncthreads();
        uint32_t lo = incl - sz;
#pragma unroll
        for (int w = 0; w < kGrpWarps; ++w) lo += w < warp ? G.warp_tot[w] : 0u;
        reinterpret_cast<uint4 *>(G.cnt)[tid] = make_uint4(lo, lo + c4.x, lo + c4.x + c4.y, lo + c4.x + c4.y + c4.z);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kGrpItems; ++k) {
        const int i = tid + k * kGrpThreads;
        if (i < cnt) G.ent[G.cnt[hh[k] >> 54] + rk[k]] = hh[k];
    }
    __syncthreads();
    // 2. one lane per record: does an earlier record of its bucket have its key?
    uint32_t coll = 0;
#pragma unroll
    for (int k = 0; k < kGrpItems; ++k) {
        const int pos = tid + k * kGrpThreads;
        bool head = false, longh = false;
        if (pos < cnt) {
            const uint64_t e = G.ent[pos];
            const uint32_t h = (uint32_t)(e >> 32);
            const uint32_t bk = h >> kGrpBktShift;
            const int bs = (int)G.cnt[bk];
            head = true;
            if (HK) {
                // with hashed keys an equal 54-bit hash stands for an equal key
                for (int j = bs; j < pos; ++j)
                    if (((G.ent[j] ^ e) >> 10) == 0) {
                        head = false;
                        break;
                    }
            } else if (bs < pos) {
                uint64_t a, b;
                R::key(recs, (int)(e & 0x3FFu), a, b);
                for (int j = bs; j < pos; ++j) {
                    const uint64_t ej = G.ent[j];
                    if ((uint32_t)(ej >> 32) != h) continue;
                    uint64_t a2, b2;
                    R::key(recs, (int)(ej & 0x3FFu), a2, b2);
                    if (a2 == a && b2 == b) {
                        head = false;
                        break;
                    }
                    ++coll;
                }
            }
            if (head) {
                const int be = bk + 1 < (uint32_t)kGrpBuckets ? (int)G.cnt[bk + 1] : cnt;
                longh = be - pos - 1 > kLongTail;
            }
        }
        const bool shorth = head && !longh;
        const uint32_t m = __ballot_sync(0xffffffffu, shorth);
        if (m) {
            const int leader = __ffs(m) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(&G.nuniq, (unsigned)__popc(m));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (shorth) G.uniq[base + __popc(m & lt)] = (uint16_t)pos;
        }
        if (longh) G.lng[atomicAdd(&G.nlong, 1u)] = (uint16_t)pos;
    }
    __syncthreads();
    // 3. one lane per distinct key: its records follow its head in the bucket
    const int nu = (int)G.nuniq;
    for (int u = tid; u < nu; u += kGrpThreads) {
        const int pos = G.uniq[u];
        const uint64_t e = G.ent[pos];
        const uint32_t h = (uint32_t)(e >> 32);
        const int idx = (int)(e & 0x3FFu);
        const uint32_t bk = h >> kGrpBktShift;
        const int be = bk + 1 < (uint32_t)kGrpBuckets ? (int)G.cnt[bk + 1] : cnt;
        bool multi = false;
        uint64_t fl = 0;
        int64_t fh = 0;
        if (pos + 1 < be) {
            uint64_t a, b;
            R::key(recs, idx, a, b);
            for (int q = pos + 1; q < be; ++q) {
                const uint64_t eq = G.ent[q];
                if (HK ? ((eq ^ e) >> 10) != 0 : (uint32_t)(eq >> 32) != h) continue;
                const int iq = (int)(eq & 0x3FFu);
                uint64_t a2, b2;
                R::key(recs, iq, a2, b2);
                if (a2 != a || b2 != b) {
                    // hashed keys: the records are merged all the same; the
                    // count reports that the hash identified different keys
                    if (!HK) continue;
                    ++coll;
                }
                if (!multi) R::add(recs, idx, fl, fh, err);
                multi = true;
                R::add(recs, iq, fl, fh, err);
            }
        }
        run(idx, multi, fl, fh);
        G.uniq[u] = (uint16_t)idx;
    }
    // heads with a long tail, a warp each
    const int nlg = (int)G.nlong;
    for (int q0 = warp; q0 < nlg; q0 += kGrpWarps) {
        const int pos = G.lng[q0];
        const uint64_t e = G.ent[pos];
        const uint32_t h = (uint32_t)(e >> 32);
        const int idx = (int)(e & 0x3FFu);
        const uint32_t bk = h >> kGrpBktShift;
        const int be = bk + 1 < (uint32_t)kGrpBuckets ? (int)G.cnt[bk + 1] : cnt;
        uint64_t a, b;
        R::key(recs, idx, a, b);
        uint64_t fl = 0;
        int64_t fh = 0;
        for (int base = pos; base < be; base += 32) {
            const int q = base + lane;
            if (q < be) {
                const uint64_t eq = G.ent[q];
                if (HK ? ((eq ^ e) >> 10) == 0 : (uint32_t)(eq >> 32) == h) {
                    const int iq = (int)(eq & 0x3FFu);
                    uint64_t a2, b2;
                    R::key(recs, iq, a2, b2);
                    if (a2 == a && b2 == b) R::add(recs, iq, fl, fh, err);
                    else if (HK) {
                        R::add(recs, iq, fl, fh, err);
                        ++coll;
                    }
                }
            }
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            const uint64_t ol = __shfl_down_sync(0xffffffffu, fl, off);
            const int64_t oh = __shfl_down_sync(0xffffffffu, fh, off);
            fx_add_fx(fl, fh, ol, oh);
        }
        if (lane == 0) {
            run(idx, true, fl, fh);
            G.uniq[nu + q0] = (uint16_t)idx;
        }
    }
    __syncthreads();  // every reader of the bucket starts is done
    reinterpret_cast<uint4 *>(G.cnt)[tid] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    return coll;
}

// Shared memory of the main tile kernel (several CTAs share an SM, so one CTA's
// tile load and barriers overlap the others' work).
struct MainSmem {
    Rec32 recs[kTileCap];
    GrpSmem G;
    uint64_t rk[2 * kRefSliceSmem];
    unsigned long long meta[4];  // current tile: offset, count, reference offset, reference count
    unsigned long long next[4];  // the same for the CTA's next tile (thread 0 reads it one tile ahead)
    uint64_t bar[2];
};
static_assert(sizeof(GrpSmem::ent) >= 11 * 32 * sizeof(unsigned long long), "statistics reduce in the entry area");  // rows 0-4, 6-10

size_t tile_smem_bytes() { return sizeof(MainSmem); }

__device__ __forceinline__ void tile_meta(const TileParams &p, uint64_t t, unsigned long long *m)
{
    m[0] = m[1] = m[2] = m[3] = 0;
    if (t < p.n_tiles) {
        m[0] = p.tile_off[t];
        m[1] = p.tile_off[t + 1] - m[0];
        m[2] = p.ref_off[t];
        m[3] = p.ref_off[t + 1] - m[2];
    }
}

// Thread 0: start the bulk copy of the tile described by m (if it fits).
__device__ __forceinline__ void issue_tile(const TileParams &p, MainSmem &M, const unsigned long long *m)
{
    if (m[1] == 0 || m[1] > (unsigned long long)kTileCap) return;
    fence_proxy_async_smem();
    bulk_load(M.recs, p.recs + m[0], (uint32_t)(m[1] * sizeof(Rec32)), &M.bar[0]);
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

// Statistics reduction area (the grouping's entries, free between tiles).
__device__ __forceinline__ unsigned long long (*red_area(GrpSmem &G))[32]
{
    return reinterpret_cast<unsigned long long (*)[32]>(G.ent);
}

// Persistent: CTA g handles tiles g, g + G, g + 2G, ...  Thread 0 keeps the
// tile metadata one tile ahead, so each tile's TMA load starts at once.
// Tiles of one instance are consecutive, so a CTA's statistics are flushed
// to an instance's accumulator when its tiles move on to the next instance.
// A bulk copy that does not complete within the wait limit stops the CTA
// (the run then reports the timeout).
template <bool SYM>
__global__ void __launch_bounds__(kTileThreads, kTileCtasPerSm) tile_kernel(const TileParams p)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MainSmem &M = *reinterpret_cast<MainSmem *>(smem_raw);
    const uint64_t G = gridDim.x;
    KeyStats st;
    st.clear();
    if (threadIdx.x == 0) {
        mbar_init(&M.bar[0], 1);
        tile_meta(p, blockIdx.x, M.next);
    }
    for (int i = threadIdx.x; i < kGrpBuckets; i += blockDim.x) M.G.cnt[i] = 0;
    __syncthreads();
    // current instance, the first tile past it and its options, kept in
    // registers (a CTA's tiles increase, so they only change at instance boundaries)
    int cur = tile_instance(p.tile_base, p.n_inst, blockIdx.x);
    unsigned long long cur_end = p.tile_base[cur + 1];
    double e0 = p.e0[cur];
    uint32_t fl = p.iflags[cur];
    bool dirty = false;
    uint32_t phase = 0;
    for (uint64_t t = blockIdx.x; t < p.n_tiles; t += G) {
        if (t >= cur_end) {  // uniform across the CTA
            if (dirty) flush_stats(p, p.acc[cur], st, red_area(M.G));
            st.clear();
            dirty = false;
            cur = tile_instance(p.tile_base, p.n_inst, t);
            cur_end = p.tile_base[cur + 1];
            e0 = p.e0[cur];
            fl = p.iflags[cur];
        }
        const bool sym = SYM && (fl & kInstSym);
        const uint32_t hmask = (fl & kInstNarrow) ? kNarrowMask : 0xFFFFFFFFu;
        const int inst = cur;
        if (threadIdx.x == 0) {
            issue_tile(p, M, M.next);
            for (int k = 0; k < 4; ++k) M.meta[k] = M.next[k];
            tile_meta(p, t + G, M.next);  // consumed next iteration
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
            const bool ok =
                mbar_wait_bounded(&M.bar[0], phase, p.err, (fl & kInstShortWait) ? kShortWaitCycles : kWaitCycles);
            phase ^= 1u;
            if (__syncthreads_or(!ok)) break;
            Rec32 *recs = M.recs;
            // the head record of each key takes the key's numerator ...
            auto run = [&](int head, bool exact, uint64_t sl, int64_t sh) {
                recs[head].num = exact ? fx_to_double(sl, sh) : canon_num(recs[head].num, st.err);
            };
            if (fl & kInstHashed) st.n_coll += group_records<R32, true>(recs, cnt, hmask, M.G, st.err, run);
            else st.n_coll += group_records<R32, false>(recs, cnt, hmask, M.G, st.err, run);
            // ... and every lane finishes one key at a time
            const int nk = group_keys(M.G);
            for (int u = threadIdx.x; u < nk; u += kTileThreads) {
                const Rec32 r = recs[M.G.uniq[u]];
                finish_key(p, e0, sym, rk, rcnt, r.a, r.b, r.num, r.den, st);
            }
            dirty = true;
        }
        __syncthreads();  // records, slice, entries and metadata free for the next tile
    }
    if (dirty) flush_stats(p, p.acc[cur], st, red_area(M.G));
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

// Tiles above shared-memory capacity (keys with many duplicates): each chunk
// is grouped and reduced to (key, exact fixed-point numerator, denominator)
// partials; the partial list is grouped again until it fits one chunk, then
// finished like a normal tile.  Exact sums make the result independent of
// the chunking.
struct BigSmem {
    union {
        Rec32 r32[kBigChunk];
        Rec48 r48[kBigCap];
    } u;
    GrpSmem G;
    uint64_t rk[2 * kRefSliceSmem];
    uint64_t bar;
    unsigned int out_count;
    unsigned int big_pre[kMaxBatch + 1];  // oversize tiles before instance i
    unsigned int bk_cnt[kBigBuckets];     // hash split of partials: bucket sizes (fill cursors while scattering)
    unsigned short bk_off[kBigBuckets];   // bucket starts (< kBigScratch)
};

size_t big_smem_bytes() { return sizeof(BigSmem); }

// One chunk of records -> exact partials appended to dst (out_count of them).
__device__ uint32_t chunk_to_partials(Rec32 *recs, int m, BigSmem &M, Rec48 *dst, uint32_t hmask, bool hashed,
                                      uint32_t &err)
{
    auto put = [&](int head, bool exact, uint64_t sl, int64_t sh) {
        const Rec32 &r = recs[head];
        Rec48 o;
        o.a = r.a;
        o.b = r.b;
        if (!exact) {
            sl = 0;
            sh = 0;
            fx_add_double(sl, sh, r.num, err);
        }
        o.fx_lo = sl;
        o.fx_hi = sh;
        o.den = r.den;
        o.pad = 0;
        dst[atomicAdd(&M.out_count, 1u)] = o;
    };
    return hashed ? group_records<R32, true>(recs, m, hmask, M.G, err, put)
                  : group_records<R32, false>(recs, m, hmask, M.G, err, put);
}

// Persistent over the oversize tiles of all instances, numbered in one index
// space (instance i owns [big_pre[i], big_pre[i+1])) and dealt round-robin to
// the CTAs, so a step's oversize work spreads over the whole grid whatever
// its instance mix; a CTA flushes its statistics when its tiles move on to
// the next instance.  The partial lists live in a fixed per-CTA scratch of
// two buffers of scratch_cap records; a tile whose partials outgrow it sets
// kErrScratch.
template <bool SYM>
__global__ void __launch_bounds__(kBigThreads, kTileCtasPerSm) big_tile_kernel(const TileParams p)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    BigSmem &M = *reinterpret_cast<BigSmem *>(smem_raw);
    Rec48 *bufA = p.scratch + (size_t)blockIdx.x * 2 * p.scratch_cap;
    Rec48 *bufB = bufA + p.scratch_cap;
    uint32_t phase = 0;
    if (threadIdx.x == 0) mbar_init(&M.bar, 1);
    for (int i = threadIdx.x; i < kGrpBuckets; i += blockDim.x) M.G.cnt[i] = 0;
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
    uint32_t fl = 0;
    KeyStats st;
    st.clear();
    bool stop = false;
    for (unsigned int idx = blockIdx.x; idx < total && !stop; idx += gridDim.x) {
        if (inst < 0 || idx >= M.big_pre[inst + 1]) {  // uniform across the CTA
            if (inst >= 0) {
                flush_stats(p, p.acc[inst], st, red_area(M.G));
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
            fl = p.iflags[inst];
        }
        const bool sym = SYM && (fl & kInstSym);
        const uint32_t hmask = (fl & kInstNarrow) ? kNarrowMask : 0xFFFFFFFFu;
        const long long wait = (fl & kInstShortWait) ? kShortWaitCycles : kWaitCycles;
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
            const bool ok = mbar_wait_bounded(&M.bar, phase, p.err, wait);
            phase ^= 1;
            if (__syncthreads_or(!ok)) {
                bad = true;
                stop = true;
                break;
            }
            st.n_coll += chunk_to_partials(M.u.r32, m, M, bufA + u, hmask, (fl & kInstHashed) != 0, st.err);
            u += M.out_count;
            __syncthreads();
        }
        // Partials of different chunks may share a key.  If they fit one
        // chunk they are grouped and reduced together; otherwise they are
        // first split by a hash of the key into buckets that each fit a
        // chunk (equal keys share a bucket) and every bucket is finished
        // on its own.  Exact sums make the result independent of the split.
        unsigned long long nrk;
        const uint64_t *rk = load_ref_slice(p, t, M.rk, nrk);
        auto finish_list = [&](const Rec48 *src, int m) {
            for (int i = threadIdx.x; i < m; i += nt) M.u.r48[i] = src[i];
            __syncthreads();
            Rec48 *r48 = M.u.r48;
            auto fin48 = [&](int head, bool exact, uint64_t sl, int64_t sh) {
                Rec48 &r = r48[head];
                if (!exact) {
                    sl = r.fx_lo;
                    sh = r.fx_hi;
                }
                r.pad = (uint64_t)__double_as_longlong(fx_to_double(sl, sh));
            };
            if (fl & kInstHashed) st.n_coll += group_records<R48, true>(r48, m, hmask, M.G, st.err, fin48);
            else st.n_coll += group_records<R48, false>(r48, m, hmask, M.G, st.err, fin48);
            const int nk = group_keys(M.G);
            for (int q = threadIdx.x; q < nk; q += nt) {
                const Rec48 &r = r48[M.G.uniq[q]];
                finish_key(p, e0, sym, rk, nrk, r.a, r.b, __longlong_as_double((long long)r.pad), r.den, st);
            }
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
    if (inst >= 0) flush_stats(p, p.acc[inst], st, red_area(M.G));
    __syncthreads();
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
    // exact count, or (flag kExpectAtMost: a beta-class pass of a heavy alpha
    // class in a run with a numerator cutoff) an upper bound
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
    a.n_coll = 0;
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
                                                           uint64_t cons_mod, uint64_t cons_rem, uint64_t top_hi,
                                                           uint64_t top_mask, const HashTables *__restrict__ hash,
                                                           uint32_t cls_lo,
                                                           uint32_t cls_hi, RunAcc *acc, uint32_t *err)
{
    uint64_t lo = 0;
    int64_t hi = 0;
    uint32_t er = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t A = keys[2 * i];
        if (!cons_ok(cons_mod, cons_rem, top_hi, top_mask, A)) continue;
        if (cls_lo > 0 || cls_hi < (uint32_t)kNumClasses) {  // a class slice: the alpha string's class
            uint64_t zc = 0;
            for (uint64_t x = A; x; x &= x - 1) zc ^= hash->zc[__ffsll((long long)x) - 1];
            const uint32_t cl = class_of(zc);
            if (cl < cls_lo || cl >= cls_hi) continue;
        }
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
                                uint64_t cons_mod, uint64_t cons_rem, uint64_t top_hi, uint64_t top_mask,
                                const HashTables *hash, uint32_t cls_lo, uint32_t cls_hi, RunAcc *acc, uint32_t *err,
                                cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const uint64_t blocks = (n + 255) / 256 < 1216 ? (n + 255) / 256 : 1216;
    ref_subtract_kernel<<<(unsigned)blocks, 256, 0, s>>>(keys, coef, hii, n, e0, cons_mod, cons_rem, top_hi, top_mask,
                                                         hash, cls_lo, cls_hi, acc, err);
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
    p.smem_vbk = (int)off;
    if (mode == kModeClassCount) {
        // a histogram of the counted class range; a range narrower than all
        // classes is counted through the bucket table of the virtual alpha pairs
        const uint32_t w = p.class_hi - p.class_lo;
        off = al(off + (size_t)w * 4);
        p.smem_vbk = (int)off;
        if (w < (uint32_t)kNumClasses) off = al(off + kVbkBytes);
    } else if (mode == kModeBetaCount) {
        off = al(off + (size_t)kNumClasses * 4);
    } else {
        off = al(off + kVbkBytes);
    }
    p.smem_gcls = (int)off;
    if (mode == kModeTileCount && p.n_grp) off = al(off + kNumClasses);  // pass of each class
    p.smem_bytes = (int)off;
}

cudaError_t launch_gen(GenMode mode, const GenBatch &b, uint64_t n_ctas, int smem_bytes, cudaStream_t s)
{
    if (n_ctas == 0) return cudaSuccess;
    // the counting modes always carry the symmetry check (they have registers
    // to spare); the class count carries the cutoff for runs that have one,
    // the beta count never (it counts every term of a heavy class)
    const unsigned g = (unsigned)n_ctas;
    constexpr int S = kFiltSym, C = kFiltCut;
    switch (mode) {
    case kModeClassCount:  // a run with a numerator cutoff counts what it keeps
        if (b.filt & C) gen_kernel<kModeClassCount, S | C><<<g, kGenThreads, smem_bytes, s>>>(b);
        else gen_kernel<kModeClassCount, S><<<g, kGenThreads, smem_bytes, s>>>(b);
        break;
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
    p.class_lo = 0;
    p.class_hi = kNumClasses - 1;  // the widest partial range: histogram and bucket table
    gen_layout(p, kModeClassCount);
    int m = p.smem_bytes;
    p.n_grp = 1;  // a grouped tile count: the emission's layout and a class table
    for (GenMode mode : {kModeBetaCount, kModeEmit, kModeTileCount}) {
        gen_layout(p, mode);
        m = m > p.smem_bytes ? m : p.smem_bytes;
    }
    return m;
}

cudaError_t init_kernel_attributes(int *tile_per_sm, int *big_per_sm)
{
    const int g = gen_smem_max();
    cudaError_t e;
    constexpr int S = kFiltSym, C = kFiltCut;
    const void *gens[] = {(const void *)gen_kernel<kModeClassCount, S>, (const void *)gen_kernel<kModeClassCount, S | C>,
                          (const void *)gen_kernel<kModeBetaCount, S>,
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

// The tile kernels' term arithmetic on given numerators and denominators
// (Hartree): the denominator rounded to the 2^-48 fixed point, then
// term_fx48, scaled back to Hartree.
__global__ void eval_terms_kernel(const double *__restrict__ num, const double *__restrict__ den, uint64_t n,
                                  double *__restrict__ out)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = term_fx48(num[i], __double2ll_rn(den[i] * kDenScale)) * kDenScale;
}

cudaError_t launch_eval_terms(const double *num, const double *den, uint64_t n, double *out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    eval_terms_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(num, den, n, out);
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
