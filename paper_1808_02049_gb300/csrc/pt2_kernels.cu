// sm_103a kernels of the sort-based Epstein-Nesbet PT2 path.
//
// Path (Algorithm 2 with hash-defined constraint classes):
//   gen<ClassCount>  work list: terms per alpha-hash class (sizes the passes)
//   per pass:
//     gen<TileCount>  terms per hash tile of the pass
//     scan            tile offsets
//     gen<Emit>       every single/double of every reference determinant whose
//                     alpha word falls in the pass: key, H_ai c_i (Slater-Condon,
//                     fermionic phase) and H_aa (incremental diagonal), written
//                     into its tile
//     ref partition   reference keys of the pass, grouped by tile and sorted
//     tile            per tile, in shared memory: bucket sort by key hash then
//                     insertion sort by the 128-bit key (equal keys adjacent),
//                     reduce_by_key, explicit filter of reference keys by binary
//                     search, num^2 / (E0 - H_aa), fixed-order block reduction
//     big tile        tiles larger than shared memory, grouped in chunks
//     pass reduce     fixed-order sum of tile partials into the run total
#include <cfloat>
#include <cmath>
#include <cstdint>

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
__device__ __forceinline__ uint64_t digest1(uint64_t a, uint64_t b) { return fmix64(fmix64(a) ^ b); }
__device__ __forceinline__ uint64_t digest2(uint64_t a, uint64_t b) { return fmix64(a ^ fmix64(b ^ 0x9e3779b97f4a7c15ull)); }

// Hash of a key that spreads it over the buckets of its tile.
__device__ __forceinline__ uint32_t bucket_hash(uint64_t a, uint64_t b)
{
    uint64_t h = (a * 0x9E3779B97F4A7C15ull) ^ b;
    h ^= h >> 29;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 32;
    return (uint32_t)h;
}

// Exact fixed-point accumulation of numerators: value * 2^90 as a 128-bit
// two's-complement integer.  Integer addition is associative, so the sum of
// the duplicates of a key does not depend on the order in which the tile
// received them; it is rounded to FP64 once.  |value| must stay below 2^36.
constexpr int kFxShift = 90;

__device__ __forceinline__ void fx_add_double(uint64_t &lo, int64_t &hi, double v, uint32_t &err)
{
    uint64_t bits = (uint64_t)__double_as_longlong(v);
    int e = (int)((bits >> 52) & 0x7FF);
    if (e == 0) return;                  // zero / subnormal: below the resolution
    if (e >= 1023 + 36) { err |= kErrFixedRange; return; }
    uint64_t m = (bits & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
    int sh = e - 1075 + kFxShift;        // value = m * 2^(e - 1075)
    uint64_t ml, mh;
    if (sh >= 0) {
        if (sh == 0) { ml = m; mh = 0; }
        else if (sh < 64) { ml = m << sh; mh = m >> (64 - sh); }
        else { ml = 0; mh = m << (sh - 64); }
    } else {
        int r = -sh;
        if (r > 63) return;
        ml = (m + (1ull << (r - 1))) >> r;  // round half away from zero on |value|
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

__device__ __forceinline__ double fx_to_double(uint64_t lo, int64_t hi)
{
    bool neg = hi < 0;
    uint64_t ulo = lo, uhi = (uint64_t)hi;
    if (neg) {
        ulo = ~ulo + 1ull;
        uhi = ~uhi + (ulo == 0 ? 1ull : 0ull);
    }
    double d = __fma_rn(__ull2double_rn(uhi), 0x1p64, __ull2double_rn(ulo));
    d *= 0x1p-90;
    return neg ? -d : d;
}

__device__ __forceinline__ bool key_less(uint64_t a0, uint64_t b0, uint64_t a1, uint64_t b1)
{
    return a0 < a1 || (a0 == a1 && b0 < b1);
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

struct GenFixed {
    uint64_t zc[kMaxOrb], zta[kMaxOrb], ztb[kMaxOrb];
    double gA[kMaxOrb], gB[kMaxOrb];
    int occA[kMaxOrb], virA[kMaxOrb], occB[kMaxOrb], virB[kMaxOrb];
    uint64_t A, B, ZcA, ZtaA, ZtbB;
    double c, hii;
    int n_sa_pass, a_in_pass;
};

// colex order of pairs: t = j2 (j2 - 1) / 2 + j1, j1 < j2
__device__ __forceinline__ void pair_of(int t, int &j1, int &j2)
{
    int k = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)t)) * 0.5f);
    while (k * (k - 1) / 2 > t) --k;
    while ((k + 1) * k / 2 <= t) ++k;
    j2 = k;
    j1 = t - k * (k - 1) / 2;
}

template <int MODE>
__device__ __forceinline__ void sink(const GenParams &p, uint64_t a, uint64_t b, uint64_t zt, double num,
                                     double haa)
{
    if constexpr (MODE == kModeTileCount) {
        uint64_t t = __umul64hi(zt, p.n_tiles);
        atomicAdd(&p.tile_counts[t], 1u);
    } else if constexpr (MODE == kModeEmit) {
        uint64_t t = __umul64hi(zt, p.n_tiles);
        unsigned long long slot = atomicAdd(&p.cursor[t], 1ull);
        if (slot >= p.rec_cap) {  // emission disagrees with the tile counts
            atomicOr(p.err, kErrCount);
            return;
        }
        double2 *dst = reinterpret_cast<double2 *>(p.recs + slot);
        dst[0] = make_double2(__longlong_as_double((long long)a), __longlong_as_double((long long)b));
        dst[1] = make_double2(num, haa);
    } else if constexpr (MODE == kModeDetTerms) {
        unsigned long long slot = atomicAdd(&p.cursor[0], 1ull);
        if (slot < p.rec_cap) {
            Rec32 r;
            r.a = a;
            r.b = b;
            r.num = num;
            r.haa = haa;
            p.recs[slot] = r;
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(kGenThreads) gen_kernel(const GenParams p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    GenFixed &F = *reinterpret_cast<GenFixed *>(smem);
    double *sa_delta = reinterpret_cast<double *>(smem + p.smem_sa);
    uint64_t *sa_zt = reinterpret_cast<uint64_t *>(sa_delta + p.n_sa);
    uint32_t *sa_info = reinterpret_cast<uint32_t *>(sa_zt + p.n_sa);
    uint16_t *sa_pass = reinterpret_cast<uint16_t *>(sa_info + p.n_sa);
    double *sb_delta = reinterpret_cast<double *>(smem + p.smem_sb);
    uint64_t *sb_zt = reinterpret_cast<uint64_t *>(sb_delta + p.n_sb);
    uint32_t *sb_info = reinterpret_cast<uint32_t *>(sb_zt + p.n_sb);
    uint16_t *pairs = reinterpret_cast<uint16_t *>(smem + p.smem_pairs);
    double *vec_all = reinterpret_cast<double *>(smem + p.smem_vec);
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem + p.smem_hist);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nw = kGenThreads / 32;
    const int N = p.sys.n;
    const int na = p.na, nb = p.nb, nva = N - na, nvb = N - nb;
    const uint64_t det = p.det_begin + blockIdx.x;
    const double *__restrict__ eri = p.sys.eri;
    const double *__restrict__ Jt = p.sys.J;
    const double *__restrict__ WSt = p.sys.WS;
    const double *__restrict__ ht = p.sys.h;
    double *vec = vec_all + warp * kMaxOrb;

    for (int i = tid; i < kMaxOrb; i += kGenThreads) {
        F.zc[i] = p.hash->zc[i];
        F.zta[i] = p.hash->zta[i];
        F.ztb[i] = p.hash->ztb[i];
    }
    const int max_m = N;  // pairs over at most N items
    for (int t = tid; t < max_m * (max_m - 1) / 2; t += kGenThreads) {
        int j1, j2;
        pair_of(t, j1, j2);
        pairs[t] = (uint16_t)(j1 | (j2 << 8));
    }
    if constexpr (MODE == kModeClassCount)
        for (int i = tid; i < kNumClasses; i += kGenThreads) hist[i] = 0;
    if (tid == 0) {
        uint64_t A = p.keys[2 * det], B = p.keys[2 * det + 1];
        F.A = A;
        F.B = B;
        F.c = p.coef[det];
        F.hii = p.hii[det];
        int ia = 0, iva = 0, ib = 0, ivb = 0;
        for (int q = 0; q < N; ++q) {
            if ((A >> q) & 1ull) F.occA[ia++] = q; else F.virA[iva++] = q;
            if ((B >> q) & 1ull) F.occB[ib++] = q; else F.virB[ivb++] = q;
        }
    }
    __syncthreads();
    if (warp == 0) {
        uint64_t zc = 0, za = 0, zb = 0;
        for (int i = lane; i < na; i += 32) { zc ^= F.zc[F.occA[i]]; za ^= F.zta[F.occA[i]]; }
        for (int i = lane; i < nb; i += 32) zb ^= F.ztb[F.occB[i]];
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            zc ^= __shfl_xor_sync(0xffffffffu, zc, off);
            za ^= __shfl_xor_sync(0xffffffffu, za, off);
            zb ^= __shfl_xor_sync(0xffffffffu, zb, off);
        }
        if (lane == 0) {
            F.ZcA = zc;
            F.ZtaA = za;
            F.ZtbB = zb;
        }
    } else if (warp == 1 || warp == 2) {
        // g(x) = h_xx + p(x), p(x) = sum over occupied j of <xj||xj>
        const int spin = warp - 1;  // 0: alpha x, 1: beta x
        const int *os = spin ? F.occB : F.occA;
        const int *oo = spin ? F.occA : F.occB;
        const int ns = spin ? nb : na, no = spin ? na : nb;
        for (int x = lane; x < N; x += 32) {
            double g = ht[x * N + x];
            for (int k = 0; k < ns; ++k) g += WSt[x * N + os[k]];
            for (int k = 0; k < no; ++k) g += Jt[x * N + oo[k]];
            (spin ? F.gB : F.gA)[x] = g;
        }
    }
    __syncthreads();
    const uint64_t A = F.A, B = F.B;
    const double c = F.c, hii = F.hii;

    // singles lists (alpha: with pass flag)
    for (int s = tid; s < p.n_sa; s += kGenThreads) {
        int i = s / nva, j = s - (s / nva) * nva;
        int r = F.occA[i], a = F.virA[j];
        uint32_t sg = __popcll(A & between_mask(r, a)) & 1;
        uint64_t a2 = A ^ (1ull << r) ^ (1ull << a);
        uint64_t zc = F.ZcA ^ F.zc[r] ^ F.zc[a];
        uint32_t inp;
        if constexpr (MODE == kModeClassCount) {
            inp = cons_ok(p.cons_mod, p.cons_rem, a2);
        } else {
            uint32_t cl = class_of(zc);
            inp = cl >= p.class_lo && cl < p.class_hi && cons_ok(p.cons_mod, p.cons_rem, a2);
        }
        sa_delta[s] = F.gA[a] - F.gA[r] - WSt[r * N + a];
        sa_zt[s] = (MODE == kModeClassCount) ? zc : (F.ZtaA ^ F.zta[r] ^ F.zta[a]);
        sa_info[s] = (uint32_t)r | ((uint32_t)a << 8) | (sg << 16) | (inp << 17);
    }
    for (int s = tid; s < p.n_sb; s += kGenThreads) {
        int i = s / nvb, j = s - (s / nvb) * nvb;
        int r = F.occB[i], a = F.virB[j];
        uint32_t sg = __popcll(B & between_mask(r, a)) & 1;
        sb_delta[s] = F.gB[a] - F.gB[r] - WSt[r * N + a];
        sb_zt[s] = F.ZtbB ^ F.ztb[r] ^ F.ztb[a];
        sb_info[s] = (uint32_t)r | ((uint32_t)a << 8) | (sg << 16);
    }
    if (tid == 0) {
        bool ok = cons_ok(p.cons_mod, p.cons_rem, A);
        if constexpr (MODE != kModeClassCount) {
            uint32_t cl = class_of(F.ZcA);
            ok = ok && cl >= p.class_lo && cl < p.class_hi;
        }
        F.a_in_pass = ok;
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
    }
    __syncthreads();
    const int n_sa_pass = F.n_sa_pass;
    const bool a_in = F.a_in_pass != 0;

    const int n_occ_pairs_a = na * (na - 1) / 2, n_vir_pairs_a = nva * (nva - 1) / 2;
    const int n_occ_pairs_b = nb * (nb - 1) / 2, n_vir_pairs_b = nvb * (nvb - 1) / 2;

    if constexpr (MODE == kModeClassCount) {
        // work list (the paper's first pass over the wavefunction): terms per class
        if (tid == 0 && a_in)
            atomicAdd(&hist[class_of(F.ZcA)],
                      (uint32_t)(p.n_sb + n_occ_pairs_b * n_vir_pairs_b));
        for (int k = tid; k < n_sa_pass; k += kGenThreads) {
            int s = sa_pass[k];
            atomicAdd(&hist[class_of(sa_zt[s])], (uint32_t)(1 + p.n_sb));
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
                atomicAdd(&hist[class_of(z12 ^ F.zc[a1] ^ F.zc[a2])], 1u);
            }
        }
        __syncthreads();
        for (int i = tid; i < kNumClasses; i += kGenThreads)
            if (hist[i]) atomicAdd(&p.class_counts[i], (unsigned long long)hist[i]);
        return;
    } else {
        constexpr bool kVal = MODE != kModeTileCount;
        const uint64_t ZtaA = F.ZtaA, ZtbB = F.ZtbB;

        // ---- alpha singles
        for (int k = tid; k < n_sa_pass; k += kGenThreads) {
            int s = sa_pass[k];
            uint32_t info = sa_info[s];
            int r = info & 0xFF, a = (info >> 8) & 0xFF;
            double num = 0.0, haa = 0.0;
            if constexpr (kVal) {
                double v = ht[a * N + r];
                for (int q = 0; q < na; ++q) {
                    int j = F.occA[q];
                    v += eri[(((size_t)a * N + r) * N + j) * N + j] - eri[(((size_t)a * N + j) * N + j) * N + r];
                }
                for (int q = 0; q < nb; ++q) {
                    int j = F.occB[q];
                    v += eri[(((size_t)a * N + r) * N + j) * N + j];
                }
                num = flip_sign(c * v, info >> 16);
                haa = hii + sa_delta[s];
            }
            sink<MODE>(p, A ^ (1ull << r) ^ (1ull << a), B, sa_zt[s] ^ ZtbB, num, haa);
        }
        // ---- beta singles
        if (a_in)
            for (int s = tid; s < p.n_sb; s += kGenThreads) {
                uint32_t info = sb_info[s];
                int r = info & 0xFF, a = (info >> 8) & 0xFF;
                double num = 0.0, haa = 0.0;
                if constexpr (kVal) {
                    double v = ht[a * N + r];
                    for (int q = 0; q < nb; ++q) {
                        int j = F.occB[q];
                        v += eri[(((size_t)a * N + r) * N + j) * N + j] -
                             eri[(((size_t)a * N + j) * N + j) * N + r];
                    }
                    for (int q = 0; q < na; ++q) {
                        int j = F.occA[q];
                        v += eri[(((size_t)a * N + r) * N + j) * N + j];
                    }
                    num = flip_sign(c * v, info >> 16);
                    haa = hii + sb_delta[s];
                }
                sink<MODE>(p, A, B ^ (1ull << r) ^ (1ull << a), ZtaA ^ sb_zt[s], num, haa);
            }
        // ---- alpha-beta doubles: one alpha single per warp, beta singles over lanes
        for (int k = warp; k < n_sa_pass; k += nw) {
            int s = sa_pass[k];
            uint32_t info = sa_info[s];
            int rA = info & 0xFF, aA = (info >> 8) & 0xFF;
            uint64_t a2 = A ^ (1ull << rA) ^ (1ull << aA);
            uint64_t ztA = sa_zt[s];
            double baseH = 0.0, cA = 0.0;
            const double *slice = nullptr;
            if constexpr (kVal) {
                // u[q] = J(aA, q) - J(rA, q): the alpha-beta cross terms of H_aa
                for (int q = lane; q < N; q += 32) vec[q] = Jt[aA * N + q] - Jt[rA * N + q];
                __syncwarp();
                baseH = hii + sa_delta[s];
                cA = flip_sign(c, info >> 16);
                slice = eri + ((size_t)aA * N + rA) * N * N;
            }
            for (int sb = lane; sb < p.n_sb; sb += 32) {
                uint32_t bi = sb_info[sb];
                int rB = bi & 0xFF, aB = (bi >> 8) & 0xFF;
                double num = 0.0, haa = 0.0;
                if constexpr (kVal) {
                    num = flip_sign(cA * slice[aB * N + rB], bi >> 16);
                    haa = baseH + sb_delta[sb] + (vec[aB] - vec[rB]);
                }
                sink<MODE>(p, a2, B ^ (1ull << rB) ^ (1ull << aB), ztA ^ sb_zt[sb], num, haa);
            }
            __syncwarp();
        }
        // ---- same-spin doubles: one occupied pair per warp, virtual pairs over lanes
        for (int spin = 0; spin < 2; ++spin) {
            if (spin == 1 && !a_in) break;
            const int npo = spin ? n_occ_pairs_b : n_occ_pairs_a;
            const int npv = spin ? n_vir_pairs_b : n_vir_pairs_a;
            const int *occ = spin ? F.occB : F.occA;
            const int *vir = spin ? F.virB : F.virA;
            const int nv = spin ? nvb : nva;
            const double *g = spin ? F.gB : F.gA;
            const uint64_t W = spin ? B : A;
            for (int pi = warp; pi < npo; pi += nw) {
                int pr = pairs[pi];
                int r1 = occ[pr & 0xFF], r2 = occ[pr >> 8];
                uint64_t w12 = W ^ (1ull << r1) ^ (1ull << r2);
                uint64_t zc12 = F.ZcA ^ F.zc[r1] ^ F.zc[r2];
                uint64_t zt12 = spin ? (ZtaA ^ ZtbB ^ F.ztb[r1] ^ F.ztb[r2]) : (ZtaA ^ ZtbB ^ F.zta[r1] ^ F.zta[r2]);
                double base = 0.0;
                if constexpr (kVal) {
                    for (int j = lane; j < nv; j += 32) {
                        int x = vir[j];
                        vec[j] = g[x] - WSt[r1 * N + x] - WSt[r2 * N + x];
                    }
                    __syncwarp();
                    base = hii - g[r1] - g[r2] + WSt[r1 * N + r2];
                }
                for (int t = lane; t < npv; t += 32) {
                    int pv = pairs[t];
                    int j1 = pv & 0xFF, j2 = pv >> 8;
                    int a1 = vir[j1], a2 = vir[j2];
                    uint64_t w2 = w12 ^ (1ull << a1) ^ (1ull << a2);
                    uint64_t zt;
                    if (spin == 0) {
                        uint32_t cl = class_of(zc12 ^ F.zc[a1] ^ F.zc[a2]);
                        if (cl < p.class_lo || cl >= p.class_hi) continue;
                        if (!cons_ok(p.cons_mod, p.cons_rem, w2)) continue;
                        zt = zt12 ^ F.zta[a1] ^ F.zta[a2];
                    } else {
                        zt = zt12 ^ F.ztb[a1] ^ F.ztb[a2];
                    }
                    double num = 0.0, haa = 0.0;
                    if constexpr (kVal) {
                        uint64_t w1 = W ^ (1ull << r1) ^ (1ull << a1);
                        uint32_t par = __popcll(W & between_mask(r1, a1)) + __popcll(w1 & between_mask(r2, a2));
                        double e = eri[(((size_t)a1 * N + r1) * N + a2) * N + r2] -
                                   eri[(((size_t)a1 * N + r2) * N + a2) * N + r1];
                        num = flip_sign(c * e, par);
                        haa = base + vec[j1] + vec[j2] + WSt[a1 * N + a2];
                    }
                    if (spin == 0) sink<MODE>(p, w2, B, zt, num, haa);
                    else sink<MODE>(p, A, w2, zt, num, haa);
                }
                __syncwarp();
            }
        }
    }
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

// ================================================================ scans

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

size_t scan_tmp_elems(uint64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

__device__ void block_scan_excl_u64(unsigned long long *v, int count_per_thread_dummy,
                                    unsigned long long local_sum, unsigned long long &prefix,
                                    unsigned long long *warp_tot, unsigned long long &total)
{
    (void)v;
    (void)count_per_thread_dummy;
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
    block_scan_excl_u64(nullptr, 0, s, pre, wt, tot);
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
        block_scan_excl_u64(nullptr, 0, v, pre, wt, tot);
        if (i < nparts) part[i] = carry + pre;
        carry += tot;
    }
    if (threadIdx.x == 0) part[nparts] = carry;
}

__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const uint32_t *__restrict__ in, uint64_t n,
                                                                  const unsigned long long *__restrict__ part,
                                                                  uint64_t nparts,
                                                                  unsigned long long *__restrict__ out)
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
    block_scan_excl_u64(nullptr, 0, s, pre, wt, tot);
    unsigned long long run = part[blockIdx.x] + pre;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = part[nparts];
}

cudaError_t launch_scan_u32_to_u64(const uint32_t *in, unsigned long long *out, uint64_t n,
                                   unsigned long long *tmp, cudaStream_t s)
{
    uint64_t nparts = (n + kScanTile - 1) / kScanTile;
    if (nparts == 0) {
        return cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
    }
    scan_sums_kernel<<<(unsigned)nparts, kScanThreads, 0, s>>>(in, n, tmp);
    scan_parts_kernel<<<1, kScanThreads, 0, s>>>(tmp, nparts);
    scan_apply_kernel<<<(unsigned)nparts, kScanThreads, 0, s>>>(in, n, tmp, nparts, out);
    return cudaGetLastError();
}

// ===================================================== reference partition

__global__ void ref_tile_kernel(const RefPartParams p)
{
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= p.n_det) return;
    uint64_t A = p.keys[2 * i], B = p.keys[2 * i + 1];
    uint64_t zc = 0, zt = 0;
    for (uint64_t x = A; x; x &= x - 1) {
        int q = __ffsll((long long)x) - 1;
        zc ^= p.hash->zc[q];
        zt ^= p.hash->zta[q];
    }
    for (uint64_t x = B; x; x &= x - 1) zt ^= p.hash->ztb[__ffsll((long long)x) - 1];
    uint32_t cl = class_of(zc);
    uint32_t t = 0xFFFFFFFFu;
    if (cl >= p.class_lo && cl < p.class_hi && cons_ok(p.cons_mod, p.cons_rem, A)) {
        t = (uint32_t)__umul64hi(zt, p.n_tiles);
        atomicAdd(&p.ref_count[t], 1u);
    }
    p.ref_tile[i] = t;
}

__global__ void ref_scatter_kernel(const RefPartParams p)
{
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= p.n_det) return;
    uint32_t t = p.ref_tile[i];
    if (t == 0xFFFFFFFFu) return;
    unsigned long long slot = atomicAdd(&p.ref_cursor[t], 1ull);
    p.ref_keys_out[2 * slot] = p.keys[2 * i];
    p.ref_keys_out[2 * slot + 1] = p.keys[2 * i + 1];
}

cudaError_t launch_ref_partition(const RefPartParams &p, int phase, cudaStream_t s)
{
    unsigned g = (unsigned)((p.n_det + 255) / 256);
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

struct TileSmem {
    uint64_t bar;
    uint32_t misc[4];
    uint32_t warp_tot[32];
    double red_d[2][32];
    unsigned long long red_u[3][32];
    uint32_t red_c[4][32];
    uint64_t rk[2 * kRefSliceSmem];
};

// Group `cnt` keys held in shared memory so that equal keys are adjacent:
// counting sort by a key hash into B >= cnt buckets, then insertion sort of
// each bucket by the 128-bit key (alpha word most significant).  On return
// perm[0..cnt) lists record indices in (bucket, key) order.
template <class KeyAt>
__device__ void group_keys(int cnt, KeyAt key, uint16_t *perm, uint16_t *bkt, uint16_t *rnk, uint32_t *hist,
                           uint32_t *warp_tot)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    int B = 32;
    while (B < cnt) B <<= 1;
    for (int i = tid; i < B; i += nt) hist[i] = 0;
    __syncthreads();
    for (int i = tid; i < cnt; i += nt) {
        uint64_t a, b;
        key(i, a, b);
        uint32_t bb = bucket_hash(a, b) & (uint32_t)(B - 1);
        bkt[i] = (uint16_t)bb;
        rnk[i] = (uint16_t)atomicAdd(&hist[bb], 1u);
    }
    __syncthreads();
    block_scan_excl_u32(hist, B, warp_tot);
    for (int i = tid; i < cnt; i += nt) perm[hist[bkt[i]] + rnk[i]] = (uint16_t)i;
    __syncthreads();
    for (int bb = tid; bb < B; bb += nt) {
        int s = (int)hist[bb];
        int e = bb + 1 < B ? (int)hist[bb + 1] : cnt;
        for (int i = s + 1; i < e; ++i) {
            uint16_t x = perm[i];
            uint64_t a, b;
            key(x, a, b);
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

struct KeyStats {
    double e2, min_den;
    unsigned long long dsum, dxor;
    uint32_t n_unique, n_in_ref, n_ext, n_pos;
    __device__ void clear()
    {
        e2 = 0.0;
        min_den = DBL_MAX;
        dsum = dxor = 0;
        n_unique = n_in_ref = n_ext = n_pos = 0;
    }
};

// One unique key: explicit filter against the reference slice, then the
// Epstein-Nesbet term num^2 / (E0 - H_aa) (Eq. 3).
__device__ __forceinline__ void finish_key(const TileParams &p, const uint64_t *rk, unsigned long long nrk,
                                           uint64_t a, uint64_t b, uint64_t fl, int64_t fh, double haa,
                                           KeyStats &st)
{
    st.n_unique++;
    if (in_slice(rk, nrk, a, b)) {
        st.n_in_ref++;
        return;
    }
    double num = fx_to_double(fl, fh);
    double den = p.e0 - haa;
    st.e2 += num * num / den;
    st.n_ext++;
    double ad = fabs(den);
    st.min_den = ad < st.min_den ? ad : st.min_den;
    st.n_pos += den > 0.0;
    st.dsum += digest1(a, b);
    st.dxor ^= digest2(a, b);
    if (p.dump_keys) {
        unsigned long long slot = atomicAdd(p.dump_count, 1ull);
        if (slot < p.dump_cap) {
            p.dump_keys[2 * slot] = a;
            p.dump_keys[2 * slot + 1] = b;
            p.dump_num[slot] = num;
            p.dump_haa[slot] = haa;
        }
    }
}

// Fixed-shape block reduction of the per-thread statistics; thread 0 returns them.
__device__ KeyStats block_reduce_stats(KeyStats st, TileSmem &S)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        st.e2 += __shfl_down_sync(0xffffffffu, st.e2, off);
        st.min_den = fmin(st.min_den, __shfl_down_sync(0xffffffffu, st.min_den, off));
        st.dsum += __shfl_down_sync(0xffffffffu, st.dsum, off);
        st.dxor ^= __shfl_down_sync(0xffffffffu, st.dxor, off);
        st.n_unique += __shfl_down_sync(0xffffffffu, st.n_unique, off);
        st.n_in_ref += __shfl_down_sync(0xffffffffu, st.n_in_ref, off);
        st.n_ext += __shfl_down_sync(0xffffffffu, st.n_ext, off);
        st.n_pos += __shfl_down_sync(0xffffffffu, st.n_pos, off);
    }
    if (lane == 0) {
        S.red_d[0][warp] = st.e2;
        S.red_d[1][warp] = st.min_den;
        S.red_u[0][warp] = st.dsum;
        S.red_u[1][warp] = st.dxor;
        S.red_c[0][warp] = st.n_unique;
        S.red_c[1][warp] = st.n_in_ref;
        S.red_c[2][warp] = st.n_ext;
        S.red_c[3][warp] = st.n_pos;
    }
    __syncthreads();
    KeyStats r;
    r.clear();
    if (threadIdx.x == 0)
        for (int w = 0; w < nw; ++w) {
            r.e2 += S.red_d[0][w];
            r.min_den = fmin(r.min_den, S.red_d[1][w]);
            r.dsum += S.red_u[0][w];
            r.dxor ^= S.red_u[1][w];
            r.n_unique += S.red_c[0][w];
            r.n_in_ref += S.red_c[1][w];
            r.n_ext += S.red_c[2][w];
            r.n_pos += S.red_c[3][w];
        }
    __syncthreads();
    return r;
}

__device__ void write_part(const TileParams &p, uint64_t t, const KeyStats &r)
{
    TilePart tp;
    tp.e2 = r.e2;
    tp.min_den = r.min_den;
    tp.dsum = r.dsum;
    tp.dxor = r.dxor;
    tp.n_unique = r.n_unique;
    tp.n_in_ref = r.n_in_ref;
    tp.n_ext = r.n_ext;
    tp.n_pos = r.n_pos;
    p.parts[t] = tp;
}

// Load the tile's reference slice; returns a pointer usable for binary search.
__device__ const uint64_t *load_ref_slice(const TileParams &p, uint64_t t, TileSmem &S, unsigned long long &n)
{
    unsigned long long s = p.ref_off[t], e = p.ref_off[t + 1];
    n = e - s;
    if (n <= (unsigned long long)kRefSliceSmem) {
        for (unsigned long long i = threadIdx.x; i < 2 * n; i += blockDim.x) S.rk[i] = p.ref_keys[2 * s + i];
        return S.rk;
    }
    return p.ref_keys + 2 * s;
}

// Shared memory of the main tile kernel.
struct MainSmem {
    Rec32 recs[kTileCap];
    uint16_t perm[kTileCap], bkt[kTileCap], rnk[kTileCap];
    uint32_t hist[kTileCap];
    TileSmem S;
};

size_t tile_smem_bytes() { return sizeof(MainSmem); }

__global__ void __launch_bounds__(kTileThreads, 2) tile_kernel(const TileParams p)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MainSmem &M = *reinterpret_cast<MainSmem *>(smem_raw);
    const uint64_t t = blockIdx.x;
    const unsigned long long off = p.tile_off[t];
    const int cnt64 = 0;
    (void)cnt64;
    const unsigned long long cntl = p.tile_off[t + 1] - off;
    if (cntl > (unsigned long long)kTileCap) {
        if (threadIdx.x == 0) {
            unsigned idx = atomicAdd(p.big_count, 1u);
            p.big_list[idx] = (uint32_t)t;
        }
        return;
    }
    const int cnt = (int)cntl;
    if (threadIdx.x == 0 && cnt > 0) {
        mbar_init(&M.S.bar, 1);
        bulk_load(M.recs, p.recs + off, (uint32_t)(cnt * sizeof(Rec32)), &M.S.bar);
    }
    unsigned long long nrk;
    const uint64_t *rk = load_ref_slice(p, t, M.S, nrk);
    __syncthreads();
    KeyStats st;
    st.clear();
    if (cnt > 0) {
        mbar_wait_bounded(&M.S.bar, 0, p.err);
        auto key = [&](int i, uint64_t &a, uint64_t &b) {
            a = M.recs[i].a;
            b = M.recs[i].b;
        };
        group_keys(cnt, key, M.perm, M.bkt, M.rnk, M.hist, M.S.warp_tot);
        uint32_t err = 0;
        const int nt = blockDim.x;
        const int chunk = (cnt + nt - 1) / nt;
        const int s = threadIdx.x * chunk, e = min(cnt, s + chunk);
        for (int j = s; j < e; ++j) {
            const Rec32 &r0 = M.recs[M.perm[j]];
            if (j > 0) {
                const Rec32 &rp = M.recs[M.perm[j - 1]];
                if (rp.a == r0.a && rp.b == r0.b) continue;
            }
            uint64_t fl = 0;
            int64_t fh = 0;
            double haa = r0.haa;
            fx_add_double(fl, fh, r0.num, err);
            for (int k = j + 1; k < cnt; ++k) {
                const Rec32 &rk2 = M.recs[M.perm[k]];
                if (rk2.a != r0.a || rk2.b != r0.b) break;
                fx_add_double(fl, fh, rk2.num, err);
                haa = fmin(haa, rk2.haa);
            }
            finish_key(p, rk, nrk, r0.a, r0.b, fl, fh, haa, st);
        }
        if (err) atomicOr(p.err, err);
        if (threadIdx.x == 0) mbar_inval(&M.S.bar);
    }
    KeyStats r = block_reduce_stats(st, M.S);
    if (threadIdx.x == 0) write_part(p, t, r);
}

cudaError_t launch_tiles(const TileParams &p, cudaStream_t s)
{
    if (p.n_tiles == 0) return cudaSuccess;
    size_t sm = tile_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    tile_kernel<<<(unsigned)p.n_tiles, kTileThreads, sm, s>>>(p);
    return cudaGetLastError();
}

// ------------------------------------------------------ oversize tiles

// Chunked grouping for tiles above shared-memory capacity: every chunk is
// grouped in shared memory and reduced to (key, exact fixed-point numerator,
// min H_aa) records; the reduced list is regrouped until it fits, then
// finished like a normal tile.  Fixed-point sums make the result independent
// of chunking.
struct BigSmem {
    union {
        Rec32 r32[kTileCap];
        Rec48 r48[kBigCap];
    } u;
    uint16_t perm[kBigCap > kTileCap ? kBigCap : kTileCap];
    uint16_t bkt[kBigCap > kTileCap ? kBigCap : kTileCap];
    uint16_t rnk[kBigCap > kTileCap ? kBigCap : kTileCap];
    uint32_t hist[kBigCap > kTileCap ? kBigCap : kTileCap];
    unsigned int out_count;
    TileSmem S;
};

size_t big_smem_bytes() { return sizeof(BigSmem); }
int big_grid() { return 64; }

__global__ void __launch_bounds__(kBigThreads, 1) big_tile_kernel(const TileParams p)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    BigSmem &M = *reinterpret_cast<BigSmem *>(smem_raw);
    Rec48 *bufA = p.scratch + (size_t)blockIdx.x * 2 * p.scratch_cap;
    Rec48 *bufB = bufA + p.scratch_cap;
    const unsigned int nbig = *p.big_count;
    uint32_t phase = 0;
    if (threadIdx.x == 0) mbar_init(&M.S.bar, 1);
    __syncthreads();
    const int nt = blockDim.x;
    for (unsigned int idx = blockIdx.x; idx < nbig; idx += gridDim.x) {
        const uint64_t t = p.big_list[idx];
        const unsigned long long off = p.tile_off[t];
        const unsigned long long cnt = p.tile_off[t + 1] - off;
        uint32_t err = 0;
        bool bad = false;
        if (cnt > p.scratch_cap) {
            if (threadIdx.x == 0) atomicOr(p.err, kErrScratch);
            bad = true;
        }
        // round 1: Rec32 chunks -> reduced Rec48 in bufA
        unsigned long long u = 0;
        for (unsigned long long cs = 0; !bad && cs < cnt; cs += kTileCap) {
            const int m = (int)min((unsigned long long)kTileCap, cnt - cs);
            if (threadIdx.x == 0) {
                fence_proxy_async_smem();
                bulk_load(M.u.r32, p.recs + off + cs, (uint32_t)(m * sizeof(Rec32)), &M.S.bar);
                M.out_count = 0;
            }
            mbar_wait_bounded(&M.S.bar, phase, p.err);
            phase ^= 1;
            __syncthreads();
            auto key = [&](int i, uint64_t &a, uint64_t &b) {
                a = M.u.r32[i].a;
                b = M.u.r32[i].b;
            };
            group_keys(m, key, M.perm, M.bkt, M.rnk, M.hist, M.S.warp_tot);
            const int chunk = (m + nt - 1) / nt;
            const int s = threadIdx.x * chunk, e = min(m, s + chunk);
            for (int j = s; j < e; ++j) {
                const Rec32 &r0 = M.u.r32[M.perm[j]];
                if (j > 0) {
                    const Rec32 &rp = M.u.r32[M.perm[j - 1]];
                    if (rp.a == r0.a && rp.b == r0.b) continue;
                }
                uint64_t fl = 0;
                int64_t fh = 0;
                double haa = r0.haa;
                fx_add_double(fl, fh, r0.num, err);
                for (int k = j + 1; k < m; ++k) {
                    const Rec32 &r2 = M.u.r32[M.perm[k]];
                    if (r2.a != r0.a || r2.b != r0.b) break;
                    fx_add_double(fl, fh, r2.num, err);
                    haa = fmin(haa, r2.haa);
                }
                unsigned int slot = atomicAdd(&M.out_count, 1u);
                Rec48 o;
                o.a = r0.a;
                o.b = r0.b;
                o.fx_lo = fl;
                o.fx_hi = fh;
                o.haa = haa;
                o.pad = 0;
                bufA[u + slot] = o;
            }
            __syncthreads();
            u += M.out_count;
            __syncthreads();
        }
        // further rounds until the reduced list fits one chunk
        Rec48 *src = bufA, *dst = bufB;
        while (!bad && u > (unsigned long long)kBigCap) {
            unsigned long long u2 = 0;
            for (unsigned long long cs = 0; cs < u; cs += kBigCap) {
                const int m = (int)min((unsigned long long)kBigCap, u - cs);
                __syncthreads();
                if (threadIdx.x == 0) M.out_count = 0;
                for (int i = threadIdx.x; i < m; i += nt) M.u.r48[i] = src[cs + i];
                __syncthreads();
                auto key = [&](int i, uint64_t &a, uint64_t &b) {
                    a = M.u.r48[i].a;
                    b = M.u.r48[i].b;
                };
                group_keys(m, key, M.perm, M.bkt, M.rnk, M.hist, M.S.warp_tot);
                const int chunk = (m + nt - 1) / nt;
                const int s = threadIdx.x * chunk, e = min(m, s + chunk);
                for (int j = s; j < e; ++j) {
                    const Rec48 &r0 = M.u.r48[M.perm[j]];
                    if (j > 0) {
                        const Rec48 &rp = M.u.r48[M.perm[j - 1]];
                        if (rp.a == r0.a && rp.b == r0.b) continue;
                    }
                    uint64_t fl = r0.fx_lo;
                    int64_t fh = r0.fx_hi;
                    double haa = r0.haa;
                    for (int k = j + 1; k < m; ++k) {
                        const Rec48 &r2 = M.u.r48[M.perm[k]];
                        if (r2.a != r0.a || r2.b != r0.b) break;
                        fx_add_fx(fl, fh, r2.fx_lo, r2.fx_hi);
                        haa = fmin(haa, r2.haa);
                    }
                    unsigned int slot = atomicAdd(&M.out_count, 1u);
                    Rec48 o = r0;
                    o.fx_lo = fl;
                    o.fx_hi = fh;
                    o.haa = haa;
                    dst[u2 + slot] = o;
                }
                __syncthreads();
                u2 += M.out_count;
            }
            __syncthreads();
            if (u2 >= u) {
                if (threadIdx.x == 0) atomicOr(p.err, kErrNoProgress);
                bad = true;
                break;
            }
            Rec48 *tmp = src;
            src = dst;
            dst = tmp;
            u = u2;
        }
        // final grouping and the energy
        unsigned long long nrk;
        __syncthreads();
        const uint64_t *rk = load_ref_slice(p, t, M.S, nrk);
        KeyStats st;
        st.clear();
        if (!bad) {
            const int m = (int)u;
            for (int i = threadIdx.x; i < m; i += nt) M.u.r48[i] = src[i];
            __syncthreads();
            auto key = [&](int i, uint64_t &a, uint64_t &b) {
                a = M.u.r48[i].a;
                b = M.u.r48[i].b;
            };
            group_keys(m, key, M.perm, M.bkt, M.rnk, M.hist, M.S.warp_tot);
            const int chunk = (m + nt - 1) / nt;
            const int s = threadIdx.x * chunk, e = min(m, s + chunk);
            for (int j = s; j < e; ++j) {
                const Rec48 &r0 = M.u.r48[M.perm[j]];
                if (j > 0) {
                    const Rec48 &rp = M.u.r48[M.perm[j - 1]];
                    if (rp.a == r0.a && rp.b == r0.b) continue;
                }
                uint64_t fl = r0.fx_lo;
                int64_t fh = r0.fx_hi;
                double haa = r0.haa;
                for (int k = j + 1; k < m; ++k) {
                    const Rec48 &r2 = M.u.r48[M.perm[k]];
                    if (r2.a != r0.a || r2.b != r0.b) break;
                    fx_add_fx(fl, fh, r2.fx_lo, r2.fx_hi);
                    haa = fmin(haa, r2.haa);
                }
                finish_key(p, rk, nrk, r0.a, r0.b, fl, fh, haa, st);
            }
        }
        if (err) atomicOr(p.err, err);
        KeyStats r = block_reduce_stats(st, M.S);
        if (threadIdx.x == 0) write_part(p, t, r);
        __syncthreads();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_inval(&M.S.bar);
}

cudaError_t launch_big_tiles(const TileParams &p, int n_ctas, cudaStream_t s)
{
    size_t sm = big_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(big_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    big_tile_kernel<<<n_ctas, kBigThreads, sm, s>>>(p);
    return cudaGetLastError();
}

// ========================================================= pass reduction

constexpr int kRedCtas = 256;
constexpr int kRedThreads = 256;

struct RedSmem {
    double d[2][kRedThreads / 32];
    unsigned long long u[2][kRedThreads / 32];
    unsigned long long c[4][kRedThreads / 32];
};

// Neumaier step.
__device__ __forceinline__ void nsum(double &s, double &c, double x)
{
    double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
}

__device__ void reduce_parts_block(const TilePart *parts, uint64_t begin, uint64_t end, TilePart &out, RedSmem &S)
{
    double s = 0.0, cc = 0.0, mind = DBL_MAX;
    unsigned long long dsum = 0, dxor = 0, nu = 0, nr = 0, ne = 0, np = 0;
    for (uint64_t i = begin + threadIdx.x; i < end; i += blockDim.x) {
        const TilePart &tp = parts[i];
        nsum(s, cc, tp.e2);
        mind = fmin(mind, tp.min_den);
        dsum += tp.dsum;
        dxor ^= tp.dxor;
        nu += tp.n_unique;
        nr += tp.n_in_ref;
        ne += tp.n_ext;
        np += tp.n_pos;
    }
    double v = s + cc;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        v += __shfl_down_sync(0xffffffffu, v, off);
        mind = fmin(mind, __shfl_down_sync(0xffffffffu, mind, off));
        dsum += __shfl_down_sync(0xffffffffu, dsum, off);
        dxor ^= __shfl_down_sync(0xffffffffu, dxor, off);
        nu += __shfl_down_sync(0xffffffffu, nu, off);
        nr += __shfl_down_sync(0xffffffffu, nr, off);
        ne += __shfl_down_sync(0xffffffffu, ne, off);
        np += __shfl_down_sync(0xffffffffu, np, off);
    }
    if (lane == 0) {
        S.d[0][warp] = v;
        S.d[1][warp] = mind;
        S.u[0][warp] = dsum;
        S.u[1][warp] = dxor;
        S.c[0][warp] = nu;
        S.c[1][warp] = nr;
        S.c[2][warp] = ne;
        S.c[3][warp] = np;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, ac = 0.0, m = DBL_MAX;
        unsigned long long x0 = 0, x1 = 0, c0 = 0, c1 = 0, c2 = 0, c3 = 0;
        for (int w = 0; w < nw; ++w) {
            nsum(a, ac, S.d[0][w]);
            m = fmin(m, S.d[1][w]);
            x0 += S.u[0][w];
            x1 ^= S.u[1][w];
            c0 += S.c[0][w];
            c1 += S.c[1][w];
            c2 += S.c[2][w];
            c3 += S.c[3][w];
        }
        out.e2 = a + ac;
        out.min_den = m;
        out.dsum = x0;
        out.dxor = x1;
        // counts of one chunk can exceed 32 bits: carried in the u64 fields below
        out.n_unique = (uint32_t)c0;
        out.n_in_ref = (uint32_t)c1;
        out.n_ext = (uint32_t)c2;
        out.n_pos = (uint32_t)c3;
        S.c[0][0] = c0;
        S.c[1][0] = c1;
        S.c[2][0] = c2;
        S.c[3][0] = c3;
    }
    __syncthreads();
}

struct ChunkPart {
    double e2, min_den;
    unsigned long long dsum, dxor, nu, nr, ne, np;
};

__global__ void __launch_bounds__(kRedThreads) pass_chunk_kernel(const TilePart *__restrict__ parts, uint64_t n,
                                                                 ChunkPart *__restrict__ out)
{
    __shared__ RedSmem S;
    uint64_t per = (n + gridDim.x - 1) / gridDim.x;
    uint64_t b = blockIdx.x * per, e = b + per < n ? b + per : n;
    if (b > n) b = n;
    TilePart tp;
    reduce_parts_block(parts, b, e, tp, S);
    if (threadIdx.x == 0) {
        ChunkPart c;
        c.e2 = tp.e2;
        c.min_den = tp.min_den;
        c.dsum = tp.dsum;
        c.dxor = tp.dxor;
        c.nu = S.c[0][0];
        c.nr = S.c[1][0];
        c.ne = S.c[2][0];
        c.np = S.c[3][0];
        out[blockIdx.x] = c;
    }
}

__global__ void pass_final_kernel(const ChunkPart *__restrict__ chunks, int nchunks,
                                  const unsigned long long *__restrict__ tile_off, uint64_t n_tiles,
                                  unsigned long long expected, RunAcc *acc)
{
    if (threadIdx.x != 0) return;
    double s = 0.0, c = 0.0, m = DBL_MAX;
    unsigned long long d0 = 0, d1 = 0, nu = 0, nr = 0, ne = 0, np = 0;
    for (int i = 0; i < nchunks; ++i) {
        nsum(s, c, chunks[i].e2);
        m = fmin(m, chunks[i].min_den);
        d0 += chunks[i].dsum;
        d1 ^= chunks[i].dxor;
        nu += chunks[i].nu;
        nr += chunks[i].nr;
        ne += chunks[i].ne;
        np += chunks[i].np;
    }
    nsum(acc->e2_s, acc->e2_c, s + c);
    acc->min_den = fmin(acc->min_den, m);
    acc->dsum += d0;
    acc->dxor ^= d1;
    acc->n_unique += nu;
    acc->n_in_ref += nr;
    acc->n_ext += ne;
    acc->n_pos += np;
    unsigned long long got = tile_off[n_tiles];
    acc->n_terms += got;
    if (got != expected) acc->err |= kErrCount;
}

cudaError_t launch_pass_reduce(const TilePart *parts, uint64_t n_tiles, TilePart *chunk_tmp,
                               const unsigned long long *tile_off, unsigned long long expected_terms,
                               RunAcc *acc, cudaStream_t s)
{
    ChunkPart *ch = reinterpret_cast<ChunkPart *>(chunk_tmp);
    pass_chunk_kernel<<<kRedCtas, kRedThreads, 0, s>>>(parts, n_tiles, ch);
    pass_final_kernel<<<1, 32, 0, s>>>(ch, kRedCtas, tile_off, n_tiles, expected_terms, acc);
    return cudaGetLastError();
}

__global__ void acc_init_kernel(RunAcc *acc)
{
    RunAcc a;
    a.e2_s = 0.0;
    a.e2_c = 0.0;
    a.min_den = DBL_MAX;
    a.n_terms = a.n_unique = a.n_in_ref = a.n_ext = a.dsum = a.dxor = a.n_pos = 0;
    a.err = 0;
    a.n_big = 0;
    *acc = a;
}

cudaError_t launch_acc_init(RunAcc *acc, cudaStream_t s)
{
    acc_init_kernel<<<1, 1, 0, s>>>(acc);
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
    off = al(off + (size_t)p.n_sb * (8 + 8 + 4));
    p.smem_pairs = (int)off;
    off = al(off + (size_t)(kMaxOrb * (kMaxOrb - 1) / 2) * 2);
    p.smem_vec = (int)off;
    off = al(off + (size_t)(kGenThreads / 32) * kMaxOrb * 8);
    p.smem_hist = (int)off;
    if (mode == kModeClassCount) off = al(off + (size_t)kNumClasses * 4);
    p.smem_bytes = (int)off;
}

cudaError_t launch_gen(GenMode mode, const GenParams &p, uint64_t n_dets, cudaStream_t s)
{
    if (n_dets == 0) return cudaSuccess;
    const void *fn = nullptr;
    switch (mode) {
    case kModeClassCount: fn = (const void *)gen_kernel<kModeClassCount>; break;
    case kModeTileCount: fn = (const void *)gen_kernel<kModeTileCount>; break;
    case kModeEmit: fn = (const void *)gen_kernel<kModeEmit>; break;
    case kModeDetTerms: fn = (const void *)gen_kernel<kModeDetTerms>; break;
    }
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, p.smem_bytes);
    if (e != cudaSuccess) return e;
    switch (mode) {
    case kModeClassCount: gen_kernel<kModeClassCount><<<(unsigned)n_dets, kGenThreads, p.smem_bytes, s>>>(p); break;
    case kModeTileCount: gen_kernel<kModeTileCount><<<(unsigned)n_dets, kGenThreads, p.smem_bytes, s>>>(p); break;
    case kModeEmit: gen_kernel<kModeEmit><<<(unsigned)n_dets, kGenThreads, p.smem_bytes, s>>>(p); break;
    case kModeDetTerms: gen_kernel<kModeDetTerms><<<(unsigned)n_dets, kGenThreads, p.smem_bytes, s>>>(p); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_diag(const SysDev &sys, const uint64_t *keys, uint64_t n, double *out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    diag_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sys, keys, n, out);
    return cudaGetLastError();
}

}  // namespace pt2
