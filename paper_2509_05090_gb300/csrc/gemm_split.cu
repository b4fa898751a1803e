// Split-precision contraction engine for the CTMRG step: FP64 GEMMs evaluated
// as sums of BF16 x BF16 tcgen05 products with FP32 accumulation in TMEM and
// exact integer recombination (no FP64 arithmetic on the hot loop).
//
// Slicing.  Every row of A (and every column of B) is put on its own
// power-of-two grid: with E = the exponent of the row's largest magnitude,
// x * 2^(-E) lies in (-1, 1) and F = round(x 2^(-E) 2^P), P = 7 + 8 (T-1), is
// split into T balanced base-256 digits d_0 .. d_{T-1} (|d| <= 128), so
// x ~= 2^E sum_i d_i 2^(-7-8i).  The digits are small integers, exact in BF16.
//
// Products.  Level t collects the slice pairs i + j = t (pairs with i + j >= T
// are dropped, relative error ~ T 2^(-8T) of the row/column maxima).  A digit
// product is at most 2^14 and a level holds t + 1 pairs, so over a K chunk of
// 256 a level-t FP32 accumulator holds an exact integer for t <= 3; lower
// levels are accurate far beyond 2^-40.  After every chunk the levels are read
// out of TMEM, rounded to integers and combined as
// S = sum_t S_t 2^(8 (T-1-t)) in int64; the chunks of one CTA are summed in
// registers, split-K CTAs with 64-bit integer atomics (exact, so the result
// does not depend on the order).  The FP64 output is S 2^(E_A + E_B - 14 -
// 8 (T-1)), built from the integer with integer instructions.
//
// Kernel.  Tile 128 x NT (NT = 64 or 96), K staged 64 at a time.  The slicing
// pre-pass writes each operand tile in the exact shared-memory image the MMA
// expects (K-major, 128-byte swizzle: row r of a 128-byte-wide tile at
// (r/8)*1024 + (r%8)*128, 16-byte chunk c at (c ^ (r%8))*16), so one bulk
// asynchronous copy (cp.async.bulk, the TMA engine) moves a whole tile.
// Warp 0 issues the copies, warp 1 the tcgen05.mma instructions (one thread),
// warps 2..9 drain TMEM with tcgen05.ld.  All waits are bounded; on expiry the
// kernel raises an error flag, stops issuing work, frees its TMEM and returns.
#include <cuda_bf16.h>

#include <vector>

#include "ctm_internal.h"

namespace {

constexpr int SP_BM = 128;       // tile rows = TMEM lanes
constexpr int SP_BK = 64;        // K per packed tile (128-byte rows)
constexpr int SP_KT_PER_CHUNK = 4;   // 4 x 64 = 256 K per exact chunk
constexpr int SP_ASLOTS = 4;
constexpr int SP_BSLOTS = 2;
constexpr int SP_THREADS = 320;  // 10 warps
constexpr long long SP_SPIN = 4000000LL;   // x ~200 ns sleep: ~1 s

__device__ __forceinline__ long long off2(const Idx2 &x, int i)
{
    if (x.s1 == 0) return (long long)i * x.s2;   // plain strided dimension: no division
    int hi = i / x.div;
    int lo = i - hi * x.div;
    return (long long)hi * x.s1 + (long long)lo * x.s2;
}

// byte offset of element (r, k) in a packed (rows x 64) BF16 tile, K-major 128B swizzle
__device__ __forceinline__ int sw128_off(int r, int k)
{
    return (r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 3) ^ (r & 7))) << 4) + ((k & 7) << 1);
}

// ---------------------------------------------------------------- pre-pass
// e[r] = exponent E with max_k |X(r,k)| < 2^E (0 for an all-zero row); one warp per row.
__global__ void split_rowexp_kernel(int R, int K, const double *X, Idx2 rmap, Idx2 kmap, int *e)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= R) return;
    const long long ro = off2(rmap, warp);
    double m = 0.0;
    for (int k = lane; k < K; k += 32) m = fmax(m, fabs(X[ro + off2(kmap, k)]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) {
        int E = 0;
        if (m > 0.0 && isfinite(m)) frexp(m, &E);
        e[warp] = E;
    }
}

// Digits of one value: F = round(x 2^(P - E)) from the IEEE fields, integer ops only.
__device__ __forceinline__ long long fixed_point(double x, int E, int P)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    int ex = (int)((b >> 52) & 0x7FF);
    if (ex == 0) return 0;                         // zero or subnormal (far below the row grid)
    long long mant = (long long)((b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52));
    int s = ex - 1075 - E + P;                     // x = mant 2^(ex - 1075)
    long long F;
    if (s >= 0) F = mant << s;                     // |x 2^(P-E)| < 2^P, no overflow
    else if (s <= -64) F = 0;
    else F = (mant + (1LL << (-s - 1))) >> (-s);   // round half up on the magnitude
    return (b >> 63) ? -F : F;
}

// Pack T digit slices of X (R x K via maps) into [T][rowTiles][kTiles][rowsT x 64] swizzled tiles.
// One thread per (row, 8-wide K chunk): it writes one 16-byte chunk per slice.
__global__ void split_pack_kernel(int R, int K, int rowsT, int rowTiles, int kTiles, int T, const double *X,
                                  Idx2 rmap, Idx2 kmap, const int *e, unsigned char *out)
{
    const long long units = (long long)rowTiles * rowsT * kTiles * 8;
    const long long tile_bytes = (long long)rowsT * SP_BK * 2;
    const long long slice_bytes = tile_bytes * rowTiles * kTiles;
    const int P = 7 + 8 * (T - 1);
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < units;
         u += (long long)gridDim.x * blockDim.x) {
        const int c8 = (int)(u % (kTiles * 8));
        const int r = (int)(u / (kTiles * 8));
        const int k0 = c8 * 8;
        long long F[8];
        if (r < R) {
            const int E = e[r];
            const long long ro = off2(rmap, r);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                int k = k0 + q;
                F[q] = (k < K) ? fixed_point(X[ro + off2(kmap, k)], E, P) : 0;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) F[q] = 0;
        }
        const long long tile = (long long)(r / rowsT) * kTiles + (k0 / SP_BK);
        unsigned char *base = out + tile * tile_bytes + sw128_off(r % rowsT, k0 % SP_BK);
        // balanced base-256 digits, least significant slice first
        for (int t = T - 1; t >= 0; --t) {
            __align__(16) __nv_bfloat16 v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                long long d;
                if (t > 0) {
                    d = F[q] & 255;
                    if (d >= 128) d -= 256;
                    F[q] = (F[q] - d) >> 8;
                } else {
                    d = F[q];
                }
                v[q] = __float2bfloat16_rn((float)d);
            }
            *reinterpret_cast<uint4 *>(base + (long long)t * slice_bytes) = *reinterpret_cast<uint4 *>(v);
        }
    }
}

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: false (and the abort flag raised) after ~1 s
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag)
{
    long long it = 0;
    while (!mbar_try(bar, parity)) {
        if (*abort_flag) return false;
        if (++it > SP_SPIN) {
            *abort_flag = 1;
            return false;
        }
        __nanosleep(128);
    }
    return true;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);   // start address
    d |= (uint64_t)1 << 16;                   // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset: 8-row groups are 1024 B apart
    d |= (uint64_t)1 << 46;                   // descriptor version (sm_100 family)
    d |= (uint64_t)2 << 61;                   // 128-byte swizzle
    return d;
}
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// int64 -> nearest double times 2^scale, integer instructions only (|S| < 2^63).
__device__ __forceinline__ double scaled_int_to_double(long long S, int scale)
{
    if (S == 0) return 0.0;
    unsigned long long sign = 0, m = (unsigned long long)S;
    if (S < 0) {
        sign = 1ULL << 63;
        m = (unsigned long long)(-S);
    }
    int lz = __clzll(m);
    int top = 63 - lz;                 // index of the leading bit
    unsigned long long mant;
    int e2 = top;
    if (top > 52) {
        int sh = top - 52;
        unsigned long long half = 1ULL << (sh - 1);
        unsigned long long rem = m & ((1ULL << sh) - 1);
        mant = m >> sh;
        if (rem > half || (rem == half && (mant & 1))) {   // round half to even
            ++mant;
            if (mant >> 53) {
                mant >>= 1;
                ++e2;
            }
        }
    } else {
        mant = m << (52 - top);
    }
    int be = e2 + scale + 1023;
    if (be <= 0) return 0.0;            // underflow: far below FP64 resolution of any result here
    if (be >= 2047) return __longlong_as_double((long long)(sign | (0x7FFULL << 52)));
    return __longlong_as_double((long long)(sign | ((unsigned long long)be << 52) | (mant & 0xFFFFFFFFFFFFFULL)));
}

struct SplitArgs {
    int M, N, K, T;
    int mTiles, nTiles, kTiles;
    int chunks_per_split, ksplit;
    const unsigned char *Apk, *Bpk;
    long long a_slice_bytes, b_slice_bytes;
    const int *eA, *eB;
    double *C;
    Idx2 Cm, Cn;
    unsigned long long *partial;     // ksplit > 1: M x N int64 accumulator
    int *err;
};

template <int NT>
__global__ void __launch_bounds__(SP_THREADS, 1) gemm_split_kernel(SplitArgs a)
{
    constexpr int A_TILE = SP_BM * SP_BK * 2;   // 16 KB
    constexpr int B_TILE = NT * SP_BK * 2;
    constexpr int HALF = NT / 2;
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint64_t bars[SP_ASLOTS * 2 + SP_BSLOTS * 2 + 3];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;

    unsigned char *sm = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *Asm = sm;                                   // SP_ASLOTS x A_TILE
    unsigned char *Bsm = sm + SP_ASLOTS * A_TILE;              // SP_BSLOTS x (T x B_TILE)
    const int T = a.T;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t bar0 = smem_u32(bars);
    auto A_full = [&](int s) { return bar0 + 8u * s; };
    auto A_empty = [&](int s) { return bar0 + 8u * (SP_ASLOTS + s); };
    auto B_full = [&](int s) { return bar0 + 8u * (2 * SP_ASLOTS + s); };
    auto B_empty = [&](int s) { return bar0 + 8u * (2 * SP_ASLOTS + SP_BSLOTS + s); };
    const uint32_t ACC_FULL = bar0 + 8u * (2 * SP_ASLOTS + 2 * SP_BSLOTS);
    const uint32_t ACC_EMPTY = ACC_FULL + 8u;
    const uint32_t DRAIN = ACC_FULL + 16u;

    const int nt = blockIdx.x, mt = blockIdx.y, ks = blockIdx.z;
    const int total_chunks = (a.kTiles + SP_KT_PER_CHUNK - 1) / SP_KT_PER_CHUNK;
    const int c_beg = ks * a.chunks_per_split;
    const int c_end = min(total_chunks, c_beg + a.chunks_per_split);
    volatile int *abort_flag = &abort_sh;

    if (threadIdx.x == 0) {
        abort_sh = 0;
        for (int s = 0; s < SP_ASLOTS; ++s) {
            mbar_init(A_full(s), 1);
            mbar_init(A_empty(s), 1);
        }
        for (int s = 0; s < SP_BSLOTS; ++s) {
            mbar_init(B_full(s), 1);
            mbar_init(B_empty(s), 1);
        }
        mbar_init(ACC_FULL, 1);
        mbar_init(ACC_EMPTY, 8);
        mbar_init(DRAIN, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    if (warp == 0) {
        // ------------------------------------------------ producer: bulk copies
        if (lane == 0) {
            int u = 0, b = 0;
            for (int c = c_beg; c < c_end && !*abort_flag; ++c) {
                const int kt0 = c * SP_KT_PER_CHUNK, kt1 = min(a.kTiles, kt0 + SP_KT_PER_CHUNK);
                for (int kt = kt0; kt < kt1; ++kt) {
                    const int sb = b % SP_BSLOTS;
                    if (!mbar_wait(B_empty(sb), ((b / SP_BSLOTS) & 1) ^ 1, abort_flag)) break;
                    mbar_expect_tx(B_full(sb), (uint32_t)(T * B_TILE));
                    for (int j = 0; j < T; ++j) {
                        const unsigned char *src =
                            a.Bpk + j * a.b_slice_bytes + ((long long)nt * a.kTiles + kt) * B_TILE;
                        bulk_g2s(smem_u32(Bsm + (sb * T + j) * B_TILE), src, B_TILE, B_full(sb));
                    }
                    ++b;
                    for (int i = 0; i < T; ++i) {
                        const int sa = u % SP_ASLOTS;
                        if (!mbar_wait(A_empty(sa), ((u / SP_ASLOTS) & 1) ^ 1, abort_flag)) break;
                        mbar_expect_tx(A_full(sa), (uint32_t)A_TILE);
                        const unsigned char *src =
                            a.Apk + i * a.a_slice_bytes + ((long long)mt * a.kTiles + kt) * A_TILE;
                        bulk_g2s(smem_u32(Asm + sa * A_TILE), src, A_TILE, A_full(sa));
                        ++u;
                    }
                    if (*abort_flag) break;
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer (one thread)
        if (lane == 0) {
            // kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16 (bits 7-9, 10-12 = 1),
            // both K-major, N >> 3 at bit 17, M >> 4 at bit 24
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) |
                                   ((uint32_t)(SP_BM >> 4) << 24);
            int u = 0, b = 0, chunk = 0;
            for (int c = c_beg; c < c_end && !*abort_flag; ++c, ++chunk) {
                if (!mbar_wait(ACC_EMPTY, (chunk & 1) ^ 1, abort_flag)) break;
                tc_fence_after();
                uint32_t started = 0;   // bit t: level t already written in this chunk
                const int kt0 = c * SP_KT_PER_CHUNK, kt1 = min(a.kTiles, kt0 + SP_KT_PER_CHUNK);
                for (int kt = kt0; kt < kt1; ++kt) {
                    const int sb = b % SP_BSLOTS;
                    if (!mbar_wait(B_full(sb), (b / SP_BSLOTS) & 1, abort_flag)) break;
                    tc_fence_after();
                    const int kvalid = min(SP_BK, a.K - kt * SP_BK);
                    const int ksteps = (kvalid + 15) / 16;
                    for (int i = 0; i < T; ++i) {
                        const int sa = u % SP_ASLOTS;
                        if (!mbar_wait(A_full(sa), (u / SP_ASLOTS) & 1, abort_flag)) break;
                        tc_fence_after();
                        const uint64_t ad = sdesc_sw128(smem_u32(Asm + sa * A_TILE));
                        for (int j = 0; j < T - i; ++j) {
                            const int t = i + j;
                            const uint64_t bd = sdesc_sw128(smem_u32(Bsm + (sb * T + j) * B_TILE));
                            for (int kk = 0; kk < ksteps; ++kk) {
                                const uint32_t acc = (started >> t) & 1u;
                                mma_bf16(tmem + (uint32_t)(t * NT), ad + 2ull * kk, bd + 2ull * kk, idesc, acc);
                                started |= 1u << t;
                            }
                        }
                        mma_commit(A_empty(sa));
                        ++u;
                    }
                    mma_commit(B_empty(sb));
                    ++b;
                    if (*abort_flag) break;
                }
                mma_commit(ACC_FULL);
            }
            // every MMA this thread issued has completed once DRAIN flips (bounded wait)
            mma_commit(DRAIN);
            {
                volatile int never = 0;
                long long it = 0;
                while (!mbar_try(DRAIN, 0) && ++it < SP_SPIN) __nanosleep(128);
                (void)never;
            }
        }
    } else {
        // ------------------------------------------------ epilogue warps 2..9
        const int sub = warp & 3;              // TMEM sub-partition this warp may read
        const int half = (warp - 2) >> 2;      // which half of the NT columns
        const uint32_t lane_base = (uint32_t)(32 * sub) << 16;
        long long acc[HALF];
#pragma unroll
        for (int q = 0; q < HALF; ++q) acc[q] = 0;
        int chunk = 0;
        for (int c = c_beg; c < c_end; ++c, ++chunk) {
            // one lane polls, the warp follows it, so tcgen05.ld below runs converged
            int ok = 0;
            if (lane == 0) ok = mbar_wait(ACC_FULL, chunk & 1, abort_flag) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            tc_fence_after();
            for (int t = 0; t < T; ++t) {
                const int sh = 8 * (T - 1 - t);
#pragma unroll
                for (int g = 0; g < HALF / 16; ++g) {
                    float v[16];
                    tmem_ld16(tmem + lane_base + (uint32_t)(t * NT + half * HALF + 16 * g), v);
#pragma unroll
                    for (int q = 0; q < 16; ++q) acc[16 * g + q] += (long long)__float2ll_rn(v[q]) << sh;
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(ACC_EMPTY);
        }
        if (!*abort_flag) {
            const int m = mt * SP_BM + 32 * sub + lane;
            if (m < a.M) {
                const int sc_m = a.eA[m] - 14 - 8 * (T - 1);
                const long long om = off2(a.Cm, m);
#pragma unroll
                for (int q = 0; q < HALF; ++q) {
                    const int n = nt * NT + half * HALF + q;
                    if (n < a.N) {
                        if (a.ksplit == 1)
                            a.C[om + off2(a.Cn, n)] = scaled_int_to_double(acc[q], sc_m + a.eB[n]);
                        else
                            atomicAdd(&a.partial[(size_t)m * a.N + n], (unsigned long long)acc[q]);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (abort_sh && threadIdx.x == 0)
        for (int i = 0; i < 2000; ++i) __nanosleep(100);   // let bulk copies still in flight land
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
    if (threadIdx.x == 0 && abort_sh) atomicExch(a.err, 2);
}

__global__ void split_finalize_kernel(int M, int N, int T, const unsigned long long *partial, const int *eA,
                                      const int *eB, double *C, Idx2 Cm, Idx2 Cn)
{
    const long long total = (long long)M * N;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(t / N), n = (int)(t - (long long)m * N);
        C[off2(Cm, m) + off2(Cn, n)] =
            scaled_int_to_double((long long)partial[t], eA[m] + eB[n] - 14 - 8 * (T - 1));
    }
}

int pick_nt(int N, int T)
{
    if (T * 96 > 512) return 64;
    long long w64 = (long long)((N + 63) / 64) * 64, w96 = (long long)((N + 95) / 96) * 96;
    return (w96 <= w64) ? 96 : 64;
}

// At least 120 KB, so a second CTA never shares the SM (each CTA holds all 512 TMEM columns).
template <int NT>
size_t split_smem_bytes(int T)
{
    size_t b = 1024 + (size_t)SP_ASLOTS * SP_BM * SP_BK * 2 + (size_t)SP_BSLOTS * T * NT * SP_BK * 2;
    return b < 120 * 1024 ? 120 * 1024 : b;
}

}  // namespace

int split_supported_T(int T) { return T >= 2 && T <= 5; }

SplitPlan split_plan(int M, int N, int K, int T, int nt_override, int ks_override)
{
    SplitPlan p{};
    p.NT = (nt_override == 64 || (nt_override == 96 && T * 96 <= 512)) ? nt_override : pick_nt(N, T);
    p.mTiles = (M + SP_BM - 1) / SP_BM;
    p.nTiles = (N + p.NT - 1) / p.NT;
    p.kTiles = (K + SP_BK - 1) / SP_BK;
    const int chunks = (p.kTiles + SP_KT_PER_CHUNK - 1) / SP_KT_PER_CHUNK;
    const long long tiles = (long long)p.mTiles * p.nTiles;
    int ks = 1;
    const int sms = device_sm_count();
    if (ks_override > 0) {
        ks = ks_override;
    } else if (tiles < sms && chunks > 1) {
        ks = (int)((sms + tiles - 1) / tiles);
    }
    if (ks > chunks) ks = chunks;
    if (ks < 1) ks = 1;
    p.chunks_per_split = (chunks + ks - 1) / ks;
    p.ksplit = (chunks + p.chunks_per_split - 1) / p.chunks_per_split;
    p.a_pack_bytes = (size_t)T * p.mTiles * p.kTiles * SP_BM * SP_BK * 2;
    p.b_pack_bytes = (size_t)T * p.nTiles * p.kTiles * p.NT * SP_BK * 2;
    p.partial_bytes = p.ksplit > 1 ? (size_t)M * N * 8 : 0;
    return p;
}

SplitPlan split_plan_caps(int M, int N, int K, int T)
{
    SplitPlan c = split_plan(M, N, K, T);
    for (int nt : {64, 96}) {
        SplitPlan p = split_plan(M, N, K, T, nt, 0);
        if (p.b_pack_bytes > c.b_pack_bytes) c.b_pack_bytes = p.b_pack_bytes;
    }
    const int kTiles = (K + SP_BK - 1) / SP_BK;
    if (kTiles > SP_KT_PER_CHUNK) c.partial_bytes = (size_t)M * N * 8;   // any split-K candidate
    return c;
}

cudaError_t split_prepare()
{
    cudaError_t e = cudaFuncSetAttribute(gemm_split_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)split_smem_bytes<64>(5));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(gemm_split_kernel<96>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)split_smem_bytes<96>(5));
}

static cudaError_t gemm_split_run(const GemmF64 &g, int T, SplitWork w, cudaStream_t st, cudaEvent_t *ev,
                                  SplitPlan p, const SplitOpts *opt = nullptr)
{
    const bool reuse_a = opt && opt->reuse_a;
    bool pack_b = true;
    if (opt && opt->b_pk) {
        if (p.b_pack_bytes > opt->b_cap) return cudaErrorInvalidValue;
        pack_b = (*opt->b_state != p.NT);
        w.Bpk = opt->b_pk;
        w.b_pack_cap = opt->b_cap;
        w.eB = opt->b_e;
    }
    if (p.a_pack_bytes > w.a_pack_cap || p.b_pack_bytes > w.b_pack_cap || p.partial_bytes > w.partial_cap ||
        g.M > w.e_cap || g.N > w.e_cap)
        return cudaErrorInvalidValue;
    cudaError_t e;
    // exponents: rows of A, columns of B
    if (!reuse_a) {
        CTM_COUNT_LAUNCH(1);
        split_rowexp_kernel<<<(g.M * 32 + 255) / 256, 256, 0, st>>>(g.M, g.K, g.A, g.Am, g.Ak, w.eA);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (pack_b) {
        CTM_COUNT_LAUNCH(1);
        split_rowexp_kernel<<<(g.N * 32 + 255) / 256, 256, 0, st>>>(g.N, g.K, g.B, g.Bn, g.Bk, w.eB);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    auto grid_of = [](long long units) {
        long long b = (units + 255) / 256;
        long long cap = 16LL * device_sm_count();
        return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
    };
    long long ua = (long long)p.mTiles * SP_BM * p.kTiles * 8, ub = (long long)p.nTiles * p.NT * p.kTiles * 8;
    if (!reuse_a) {
        CTM_COUNT_LAUNCH(1);
        split_pack_kernel<<<grid_of(ua), 256, 0, st>>>(g.M, g.K, SP_BM, p.mTiles, p.kTiles, T, g.A, g.Am, g.Ak,
                                                       w.eA, w.Apk);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (pack_b) {
        CTM_COUNT_LAUNCH(1);
        split_pack_kernel<<<grid_of(ub), 256, 0, st>>>(g.N, g.K, p.NT, p.nTiles, p.kTiles, T, g.B, g.Bn, g.Bk,
                                                       w.eB, w.Bpk);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (opt && opt->b_pk) *opt->b_state = p.NT;
    }
    if (p.ksplit > 1) {
        e = cudaMemsetAsync(w.partial, 0, p.partial_bytes, st);
        if (e != cudaSuccess) return e;
    }
    SplitArgs a{g.M,
                g.N,
                g.K,
                T,
                p.mTiles,
                p.nTiles,
                p.kTiles,
                p.chunks_per_split,
                p.ksplit,
                w.Apk,
                w.Bpk,
                (long long)p.mTiles * p.kTiles * SP_BM * SP_BK * 2,
                (long long)p.nTiles * p.kTiles * p.NT * SP_BK * 2,
                w.eA,
                w.eB,
                g.C,
                g.Cm,
                g.Cn,
                (unsigned long long *)w.partial,
                w.err};
    dim3 grid(p.nTiles, p.mTiles, p.ksplit);
    CTM_COUNT_LAUNCH(1);
    if (ev) cudaEventRecord(ev[0], st);
    if (p.NT == 96)
        gemm_split_kernel<96><<<grid, SP_THREADS, split_smem_bytes<96>(T), st>>>(a);
    else
        gemm_split_kernel<64><<<grid, SP_THREADS, split_smem_bytes<64>(T), st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], st);
    if (p.ksplit > 1) {
        long long total = (long long)g.M * g.N;
        CTM_COUNT_LAUNCH(1);
        split_finalize_kernel<<<grid_of(total), 256, 0, st>>>(g.M, g.N, T, (const unsigned long long *)w.partial,
                                                              w.eA, w.eB, g.C, g.Cm, g.Cn);
        e = cudaGetLastError();
    }
    return e;
}

// ---------------------------------------------------------------- autotuner
// For each new (M, N, K, T) the first eager call times every candidate plan
// (N tile 64 / 96, K-split auto, 1, 2x, 1/2x) end to end on the real operands
// with CUDA events, keeps the fastest, and re-runs it so the output is valid.
// The choice is cached for the process; captured calls use the cache or the
// default plan.
#include <map>
#include <mutex>
#include <tuple>

namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_tune;
}  // namespace

cudaError_t gemm_split(const GemmF64 &g, int T, SplitWork w, cudaStream_t st, cudaEvent_t *ev,
                       const SplitOpts *opt)
{
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    if (!split_supported_T(T) || g.alpha != 1.0 || g.beta != 0.0) return cudaErrorInvalidValue;
    const auto key = std::make_tuple(g.M, g.N, g.K, T);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end())
            return gemm_split_run(g, T, w, st, ev, split_plan(g.M, g.N, g.K, T, it->second.first, it->second.second),
                                  opt);
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (!w.autotune || cs != cudaStreamCaptureStatusNone)
        return gemm_split_run(g, T, w, st, ev, split_plan(g.M, g.N, g.K, T), opt);
    SplitPlan base = split_plan(g.M, g.N, g.K, T);
    const int chunks = (base.kTiles + SP_KT_PER_CHUNK - 1) / SP_KT_PER_CHUNK;
    std::vector<std::pair<int, int>> cands;
    for (int nt : {64, 96}) {
        if (nt == 96 && T * 96 > 512) continue;
        for (int ks : {base.ksplit, 1, 2 * base.ksplit, base.ksplit / 2}) {
            if (ks < 1 || ks > chunks) continue;
            std::pair<int, int> c{nt, ks};
            bool dup = false;
            for (auto &o : cands) dup |= (o == c);
            if (!dup) cands.push_back(c);
        }
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return cudaErrorUnknown;
    float best = 1e30f;
    std::pair<int, int> best_c{base.NT, base.ksplit};
    for (auto &cnd : cands) {
        SplitPlan p = split_plan(g.M, g.N, g.K, T, cnd.first, cnd.second);
        if (p.a_pack_bytes > w.a_pack_cap || p.b_pack_bytes > w.b_pack_cap || p.partial_bytes > w.partial_cap) continue;
        float ms = 0.f, tot = 0.f;
        for (int rep = 0; rep < 2; ++rep) {   // first run warms caches and the instruction stream
            cudaEventRecord(e0, st);
            cudaError_t e = gemm_split_run(g, T, w, st, nullptr, p);
            cudaEventRecord(e1, st);
            if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return e != cudaSuccess ? e : cudaErrorUnknown;
            }
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep) tot = ms;
        }
        if (tot < best) {
            best = tot;
            best_c = cnd;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = best_c;
    }
    // the candidates re-packed both operands into the work buffers: a cached B is
    // re-packed by this final run, a reused A is freshly packed already
    SplitOpts fin{};
    if (opt) {
        fin = *opt;
        fin.reuse_a = 0;
        if (fin.b_state) *fin.b_state = 0;
    }
    return gemm_split_run(g, T, w, st, ev, split_plan(g.M, g.N, g.K, T, best_c.first, best_c.second),
                          opt ? &fin : nullptr);
}

int split_autotuned_shapes() { return (int)g_tune.size(); }
