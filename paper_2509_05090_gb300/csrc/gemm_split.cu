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
// 8 (T-1)): the int64 -> FP64 conversion instruction and an exact shift of the
// exponent field.
//
// Kernel.  Tile 128 x NT (NT = 64 or 96), K staged 64 at a time; one MMA covers up to
// 256 / NT slice pairs (N = up to 256), since narrow MMAs run far below the tensor peak.  The slicing
// pre-pass writes each operand tile in the exact shared-memory image the MMA
// expects (K-major, 128-byte swizzle: row r of a 128-byte-wide tile at
// (r/8)*1024 + (r%8)*128, 16-byte chunk c at (c ^ (r%8))*16), so one bulk
// asynchronous copy (cp.async.bulk, the TMA engine) moves a whole tile.
// Warp 0 issues the copies, warp 1 the tcgen05.mma instructions (one thread),
// warps 2..17 drain TMEM with tcgen05.ld (four per TMEM sub-partition, a
// quarter of the tile's columns each) and write the tile out through shared
// memory.  All waits are bounded; on expiry the
// kernel raises an error flag, stops issuing work, frees its TMEM and returns.
#include <cuda_bf16.h>

#include <vector>

#include "ctm_internal.h"

namespace {

constexpr int SP_BM = 128;       // tile rows = TMEM lanes
constexpr int SP_BK = 64;        // K per packed tile (128-byte rows)
constexpr int SP_KT_PER_CHUNK = 4;   // 4 x 64 = 256 K per exact chunk
constexpr int SP_BSLOTS = 2;     // B ring: all T slices of a K tile per slot
// Per tile width: A-slice ring depth (the next K tile's slices in flight while the
// current one is multiplied, within 227 KB with T = 5 B slices x 2), epilogue warps
// (four or two per TMEM sub-partition), TMEM columns (T NT <= the allocation) and
// CTAs per SM.  NT = 48 is the two-CTAs-per-SM shape: 256 TMEM columns and ~109 KB
// of shared memory each, so one CTA's epilogue overlaps the other's loads and MMAs.
template <int NT>
struct SpCfg {
    static constexpr int ASLOTS = NT == 96 ? 6 : (NT == 64 ? 8 : 3);
    static constexpr int EPI_WARPS = NT == 48 ? 8 : 16;
    static constexpr int EPI_THREADS = 32 * EPI_WARPS;
    static constexpr int THREADS = 64 + EPI_THREADS;   // producers, MMA issuer, epilogue
    static constexpr int TMEM_COLS = NT == 48 ? 256 : 512;
    static constexpr int MIN_BLOCKS = NT == 48 ? 2 : 1;
};
// The deep-ring variant of the 48-wide tile (plan code SP_DEEP_CODE): one CTA per SM
// whose A ring takes the shared memory a second CTA would have used, so a K-heavy
// contraction (the packed n x n operand streamed past a narrow B) keeps 160 KB of A
// copies in flight per SM instead of 96 KB.
constexpr int SP_DEEP_CODE = 148;
constexpr size_t SP_SMEM_MAX = 232448;   // 227 KB of dynamic shared memory per CTA
template <int T>
struct SpDeep {
    static constexpr size_t B_RING = (size_t)2 * T * 48 * 64 * 2;
    static constexpr int A = (int)((SP_SMEM_MAX - 1024 - B_RING) / (128 * 64 * 2)) < 12
                                 ? (int)((SP_SMEM_MAX - 1024 - B_RING) / (128 * 64 * 2))
                                 : 12;
};
constexpr unsigned SP_SUSPEND_NS = 2000;        // try_wait suspend-time hint: woken at phase completion
constexpr unsigned long long SP_WAIT_NS = 1000000000ULL;   // give up a wait after ~1 s

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
// Row grids.  e[r] holds the largest high word of |X(r, k)| over k: for
// non-negative doubles the integer order of the high words is the numeric order
// of their exponents, which is all the grid needs, so no FP64 instruction is
// used.  E = exp_of_word(e[r]) satisfies max_k |X(r,k)| < 2^E (frexp's
// convention); zero, subnormal-only and inf/NaN rows get E = 0.
__device__ __forceinline__ unsigned abs_hi_word(double x) { return (unsigned)__double2hiint(x) & 0x7FFFFFFFu; }
__device__ __forceinline__ int exp_of_word(int w)
{
    const int ex = w >> 20;
    return (ex == 0 || ex == 0x7FF) ? 0 : ex - 1022;
}

// one warp per row (rows whose K index is contiguous or irregular)
__global__ void split_rowexp_kernel(int R, int K, const double *X, Idx2 rmap, Idx2 kmap, int *e)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= R) return;
    const long long ro = off2(rmap, warp);
    unsigned m = 0;
    for (int k = lane; k < K; k += 32) m = max(m, abs_hi_word(X[ro + off2(kmap, k)]));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) e[warp] = (int)m;
}

// Transposed operands (row index unit-stride, K index strided): one thread per
// row over a K range, lanes along the contiguous rows; the K ranges combine with
// atomicMax into e[], which the caller has zeroed.
constexpr int SP_COLEXP_K = 32;
__global__ void split_colexp_kernel(int R, int K, const double *X, long long kstride, int *e)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int k0 = blockIdx.y * SP_COLEXP_K, k1 = min(K, k0 + SP_COLEXP_K);
    unsigned m = 0;
    for (int k = k0; k < k1; ++k) m = max(m, abs_hi_word(X[(long long)k * kstride + r]));
    if (m) atomicMax(e + r, (int)m);
}

// Digit slicing with T fixed at compile time.  P = 7 + 8 (T-1) fraction bits
// on the row grid; B = 128 (256^(T-1) + ... + 256 + 1) biases the fixed-point
// value F (|F| <= 2^P < B) to G = F + B >= 0, and then byte j of G minus 128 is
// the balanced digit of weight 256^j for j < T-1 (each in [-128, 127]) and
// G >> 8 (T-1) minus 128 the top digit (in [-128, 128]): the same digits as
// repeatedly taking the balanced low byte and shifting.
template <int T>
struct SplitDigits {
    static constexpr int P = 7 + 8 * (T - 1);
    static constexpr unsigned long long B = 128ULL * (((1ULL << (8 * T)) - 1) / 255);
};

// Right shift, less one guard bit, that puts a value of biased exponent field ex
// on the grid of a row with exponent E: x = mant 2^(ex - 1075), so
// F = round(x 2^(P - E)) = ((mant >> sh) + 1) >> 1 with sh = rs - ex,
// rs = E + 1074 - P (rounding half up on the magnitude).
__device__ __forceinline__ int grid_shift(int E, int P) { return E + 1074 - P; }

// G = F + B of one value from its IEEE fields, integer operations only.  Zero
// and subnormal values (far below any row grid) give F = 0, as do values more
// than 63 bits below it; sh < 0 happens only on rows whose grid is undefined
// (E = 0 for an inf/NaN row) and gives F = 0 too.
template <int T>
__device__ __forceinline__ unsigned long long biased_fixed(double x, int rs)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)(b >> 52) & 0x7FF;
    const int sh = rs - ex;
    const unsigned long long mant = (b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
    unsigned long long F = ((mant >> (sh & 63)) + 1) >> 1;
    if (ex == 0 || (unsigned)sh > 63u) F = 0;
    const unsigned long long m = (unsigned long long)((long long)b >> 63);   // all ones if negative
    return (F ^ m) - m + SplitDigits<T>::B;
}

// BF16 pair {lo, hi} in one word (lo in the low half).  The inputs are integers of
// at most 8 significant bits, so the conversion is exact.
__device__ __forceinline__ uint32_t bf16x2_of(float lo, float hi)
{
    uint32_t w;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(w) : "f"(hi), "f"(lo));
    return w;
}

// The digit of slice t (t = 0 most significant, weight 256^(T-1-t)) of a biased
// word, as an exact FP32 integer: the digit byte u placed under the exponent of
// 2^23 reads as 2^23 + u, and subtracting 2^23 + 128 leaves u - 128 (one byte
// permute and one FP32 add; the top digit, up to 9 bits, is added instead).
template <int T>
__device__ __forceinline__ float slice_digit(unsigned long long G, int t)
{
    if (t == 0) return __uint_as_float(0x4B000000u + (uint32_t)(G >> (8 * (T - 1)))) - 8388736.0f;
    return __uint_as_float(__byte_perm((uint32_t)G, 0x4B000000u, 0x7650u | (unsigned)(T - 1 - t))) - 8388736.0f;
}

// Slices of 8 consecutive-K values: slice t's 16-byte chunk goes to base + t * slice_bytes.
template <int T>
__device__ __forceinline__ void write_digit_chunks(const unsigned long long *G, unsigned char *base,
                                                   long long slice_bytes)
{
#pragma unroll
    for (int t = 0; t < T; ++t) {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) w[q] = bf16x2_of(slice_digit<T>(G[2 * q], t), slice_digit<T>(G[2 * q + 1], t));
        *reinterpret_cast<uint4 *>(base + (long long)t * slice_bytes) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Pack T digit slices of X (R x K via maps) into [T][rowTiles][kTiles][rowsT x 64] swizzled tiles.
// One thread per (row, 8-wide K chunk): it writes one 16-byte chunk per slice.
template <int T>
__global__ void split_pack_kernel(int R, int K, int rowsT, int rowTiles, int kTiles, const double *X, Idx2 rmap,
                                  Idx2 kmap, const int *e, unsigned char *out)
{
    const long long units = (long long)rowTiles * rowsT * kTiles * 8;
    const long long tile_bytes = (long long)rowsT * SP_BK * 2;
    const long long slice_bytes = tile_bytes * rowTiles * kTiles;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < units;
         u += (long long)gridDim.x * blockDim.x) {
        const int c8 = (int)(u % (kTiles * 8));
        const int r = (int)(u / (kTiles * 8));
        const int k0 = c8 * 8;
        unsigned long long G[8];
        if (r < R) {
            const int rs = grid_shift(exp_of_word(e[r]), SplitDigits<T>::P);
            const long long ro = off2(rmap, r);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                int k = k0 + q;
                G[q] = (k < K) ? biased_fixed<T>(X[ro + off2(kmap, k)], rs) : SplitDigits<T>::B;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) G[q] = SplitDigits<T>::B;
        }
        const long long tile = (long long)(r / rowsT) * kTiles + (k0 / SP_BK);
        write_digit_chunks<T>(G, out + tile * tile_bytes + sw128_off(r % rowsT, k0 % SP_BK), slice_bytes);
    }
}

// Exponent and digits in one kernel for an operand whose K index is contiguous
// (X(r, k) = X[off(r) + k]) but whose rows are not 16-byte aligned pairs: one
// warp per row scans the row for its exponent word, then packs it in 8-wide
// chunks (the second read of the row hits L1/L2); rows past R up to the padded
// tile count are written as zero digits.
template <int T>
__global__ void __launch_bounds__(256) split_rowpack_kernel(int R, int K, int rowsT, int rowsTotal, int kTiles,
                                                            const double *X, Idx2 rmap, int *e, unsigned char *out,
                                                            long long slice_bytes)
{
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= rowsTotal) return;
    const long long tile_bytes = (long long)rowsT * SP_BK * 2;
    unsigned char *row_base = out + (long long)(r / rowsT) * kTiles * tile_bytes;
    unsigned long long G[8];
    if (r < R) {
        const double *x = X + off2(rmap, r);
        unsigned m0 = 0, m1 = 0, m2 = 0, m3 = 0;
        int k = lane;
        for (; k + 96 < K; k += 128) {
            m0 = max(m0, abs_hi_word(x[k]));
            m1 = max(m1, abs_hi_word(x[k + 32]));
            m2 = max(m2, abs_hi_word(x[k + 64]));
            m3 = max(m3, abs_hi_word(x[k + 96]));
        }
        for (; k < K; k += 32) m0 = max(m0, abs_hi_word(x[k]));
        unsigned m = max(max(m0, m1), max(m2, m3));
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) e[r] = (int)m;
        const int rs = grid_shift(exp_of_word((int)m), SplitDigits<T>::P);
        for (int c8 = lane; c8 < kTiles * 8; c8 += 32) {
            const int k0 = c8 * 8;
#pragma unroll
            for (int q = 0; q < 8; ++q) G[q] = (k0 + q < K) ? biased_fixed<T>(x[k0 + q], rs) : SplitDigits<T>::B;
            write_digit_chunks<T>(G, row_base + (long long)(k0 / SP_BK) * tile_bytes + sw128_off(r % rowsT, k0 % SP_BK),
                                  slice_bytes);
        }
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) G[q] = SplitDigits<T>::B;
        for (int c8 = lane; c8 < kTiles * 8; c8 += 32) {
            const int k0 = c8 * 8;
            write_digit_chunks<T>(G, row_base + (long long)(k0 / SP_BK) * tile_bytes + sw128_off(r % rowsT, k0 % SP_BK),
                                  slice_bytes);
        }
    }
}

// Packing of a contiguous-K operand read once, held in registers: a group of
// WPR warps owns one row; at step j warp w of the group loads the 64-wide K
// tile kt = j WPR + w as one double2 per lane (512 contiguous bytes per warp
// instruction), the group reduces the exponent word through shared memory, and
// each lane writes its two digits of every slice as one 32-bit word, so one
// store instruction fills the tile's whole 128-byte swizzled row of that
// slice.  Needs K even, 16-byte aligned rows and NV WPR >= kTiles; rows from R
// up to rowsTotal and columns from K up to the tile edge get zero digits.
template <int NV, int T>
__global__ void __launch_bounds__(512, 1) split_rowpack_reg_kernel(int R, int K, int rowsT, int rowsTotal, int kTiles,
                                                                int WPR, const double *X, Idx2 rmap, int *e,
                                                                unsigned char *out, long long slice_bytes)
{
    __shared__ unsigned s_m[16];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = warp / WPR, w = warp - g * WPR;
    const int r = blockIdx.x * (blockDim.x / (32 * WPR)) + g;
    const bool live = r < R;
    const double *x = live ? X + off2(rmap, r) : X;
    double2 v[NV];
    unsigned m = 0;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const int k = ((j * WPR + w) << 6) + 2 * lane;
        v[j] = make_double2(0.0, 0.0);
        if (live && k < K) v[j] = *reinterpret_cast<const double2 *>(x + k);
    }
#pragma unroll
    for (int j = 0; j < NV; ++j) m = max(m, max(abs_hi_word(v[j].x), abs_hi_word(v[j].y)));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) s_m[warp] = m;
    __syncthreads();
    if (r >= rowsTotal) return;
    m = 0;
    for (int i = 0; i < WPR; ++i) m = max(m, s_m[g * WPR + i]);
    if (live && w == 0 && lane == 0) e[r] = (int)m;
    const int rs = grid_shift(exp_of_word((int)m), SplitDigits<T>::P);
    const long long tile_bytes = (long long)rowsT * SP_BK * 2;
    unsigned char *row_base = out + (long long)(r / rowsT) * kTiles * tile_bytes + sw128_off(r % rowsT, 2 * lane);
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const int kt = j * WPR + w;
        if (kt < kTiles) {
            const unsigned long long G0 = biased_fixed<T>(v[j].x, rs), G1 = biased_fixed<T>(v[j].y, rs);
            unsigned char *dst = row_base + (long long)kt * tile_bytes;
#pragma unroll
            for (int t = 0; t < T; ++t)
                *reinterpret_cast<uint32_t *>(dst + (long long)t * slice_bytes) =
                    bf16x2_of(slice_digit<T>(G0, t), slice_digit<T>(G1, t));
        }
    }
}

// The same packing for a transposed operand, X(r, k) = X[k * kstride + r]: a
// block stages 32 rows x one 64-wide K tile through shared memory, reading with
// the lanes along the contiguous rows and writing the swizzled chunks as above.
template <int T>
__global__ void __launch_bounds__(256) split_pack_t_kernel(int R, int K, int rowsT, int rowsTotal, int kTiles,
                                                           const double *X, long long kstride, const int *e,
                                                           unsigned char *out, long long slice_bytes)
{
    __shared__ unsigned long long Gs[32][SP_BK + 1];
    const int r0 = blockIdx.x * 32, kt = blockIdx.y;
    {
        const int r = threadIdx.x & 31, kg = threadIdx.x >> 5;
        const int gr = r0 + r;
        const int rs = grid_shift(gr < R ? exp_of_word(e[gr]) : 0, SplitDigits<T>::P);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int kl = kg * 8 + q, k = kt * SP_BK + kl;
            Gs[r][kl] = (gr < R && k < K) ? biased_fixed<T>(X[(long long)k * kstride + gr], rs) : SplitDigits<T>::B;
        }
    }
    __syncthreads();
    const int r = threadIdx.x >> 3, c8 = threadIdx.x & 7;
    const int gr = r0 + r;
    if (gr >= rowsTotal) return;   // past the last padded tile (rowsT need not divide by 32)
    unsigned long long G[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) G[q] = Gs[r][c8 * 8 + q];
    const long long tile = (long long)(gr / rowsT) * kTiles + kt;
    write_digit_chunks<T>(G, out + tile * ((long long)rowsT * SP_BK * 2) + sw128_off(gr % rowsT, c8 * 8), slice_bytes);
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
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(SP_SUSPEND_NS)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait.  try_wait suspends the thread until the phase completes (or the
// hint expires), so a waiting producer / MMA thread resumes without a sleep
// quantum; after ~1 s of global time it gives up: false, abort flag raised.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag)
{
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if ((it & 15) == 0 && global_ns() - t0 > SP_WAIT_NS) {
            *abort_flag = 1;
            return false;
        }
    }
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

// 8 consecutive TMEM columns of this warp's 32 lanes; completes at tmem_wait_ld().
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t *r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// int64 -> nearest double (round half to even, the conversion instruction) times
// 2^scale, the scaling done exactly on the exponent field; results below the
// normal range flush to zero and above it go to infinity.
__device__ __forceinline__ double scaled_int_to_double(long long S, int scale)
{
    const double d = __ll2double_rn(S);
    const int hi = __double2hiint(d), lo = __double2loint(d);
    const int be = ((hi >> 20) & 0x7FF) + scale;
    if (S == 0 || be <= 0) return 0.0;   // far below FP64 resolution of any result here
    if (be >= 2047) return __hiloint2double((hi & (int)0x80000000) | 0x7FF00000, 0);
    return __hiloint2double((hi & ~0x7FF00000) | (be << 20), lo);
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

template <int NT, int T, bool DEEP = false>
__global__ void __launch_bounds__(SpCfg<NT>::THREADS, DEEP ? 1 : SpCfg<NT>::MIN_BLOCKS) gemm_split_kernel(SplitArgs a)
{
    constexpr int A_TILE = SP_BM * SP_BK * 2;   // 16 KB
    constexpr int B_TILE = NT * SP_BK * 2;
    constexpr int QW = NT / (SpCfg<NT>::EPI_WARPS / 4);   // columns per epilogue warp
    constexpr int SP_ASLOTS = DEEP ? SpDeep<T>::A : SpCfg<NT>::ASLOTS;
    constexpr int SP_EPI_WARPS = SpCfg<NT>::EPI_WARPS;
    constexpr int SP_EPI_THREADS = SpCfg<NT>::EPI_THREADS;
    constexpr int TMEM_COLS = SpCfg<NT>::TMEM_COLS;
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint64_t bars[SP_ASLOTS * 2 + SP_BSLOTS * 2 + 3];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;

    unsigned char *sm = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *Asm = sm;                                   // SP_ASLOTS x A_TILE
    unsigned char *Bsm = sm + SP_ASLOTS * A_TILE;              // SP_BSLOTS x (T x B_TILE)
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
        mbar_init(ACC_EMPTY, SP_EPI_WARPS);
        mbar_init(DRAIN, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    if (warp == 0) {
        // ------------------------------------------------ producers: bulk copies
        // lane 0 streams the B tiles (all T slices of a K tile per slot), lane 1 the
        // A slices; each blocks only on its own ring, so the A stream runs ahead of a
        // full B ring instead of queueing behind it
        if (lane == 0) {
            int b = 0;
            for (int c = c_beg; c < c_end && !*abort_flag; ++c) {
                const int kt0 = c * SP_KT_PER_CHUNK, kt1 = min(a.kTiles, kt0 + SP_KT_PER_CHUNK);
                for (int kt = kt0; kt < kt1; ++kt, ++b) {
                    const int sb = b % SP_BSLOTS;
                    if (!mbar_wait(B_empty(sb), ((b / SP_BSLOTS) & 1) ^ 1, abort_flag)) break;
                    mbar_expect_tx(B_full(sb), (uint32_t)(T * B_TILE));
                    for (int j = 0; j < T; ++j) {
                        const unsigned char *src =
                            a.Bpk + j * a.b_slice_bytes + ((long long)nt * a.kTiles + kt) * B_TILE;
                        bulk_g2s(smem_u32(Bsm + (sb * T + j) * B_TILE), src, B_TILE, B_full(sb));
                    }
                }
            }
        } else if (lane == 1) {
            int u = 0;
            for (int c = c_beg; c < c_end && !*abort_flag; ++c) {
                const int kt0 = c * SP_KT_PER_CHUNK, kt1 = min(a.kTiles, kt0 + SP_KT_PER_CHUNK);
                for (int kt = kt0; kt < kt1 && !*abort_flag; ++kt) {
                    for (int i = 0; i < T; ++i, ++u) {
                        const int sa = u % SP_ASLOTS;
                        if (!mbar_wait(A_empty(sa), ((u / SP_ASLOTS) & 1) ^ 1, abort_flag)) break;
                        mbar_expect_tx(A_full(sa), (uint32_t)A_TILE);
                        const unsigned char *src =
                            a.Apk + i * a.a_slice_bytes + ((long long)mt * a.kTiles + kt) * A_TILE;
                        bulk_g2s(smem_u32(Asm + sa * A_TILE), src, A_TILE, A_full(sa));
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer (one thread)
        if (lane == 0) {
            // kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16 (bits 7-9, 10-12 = 1),
            // both K-major, N >> 3 at bit 17, M >> 4 at bit 24
            const uint32_t idesc0 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(SP_BM >> 4) << 24);
            // The T B slices of a K tile are consecutive NT-row tiles of one 128-byte-swizzled
            // operand and the level accumulators consecutive NT-column blocks of TMEM, so
            // A_i times slices j0 .. j0+G-1 is one MMA of N = G NT (<= 256) into levels i+j0 ..
            constexpr int G = 256 / NT;
            // descriptors of ring slot 0; slot s is (s * tile bytes) >> 4 further on
            const uint64_t ad0 = sdesc_sw128(smem_u32(Asm)), bd0 = sdesc_sw128(smem_u32(Bsm));
            int u = 0, b = 0, chunk = 0;
            for (int c = c_beg; c < c_end && !*abort_flag; ++c, ++chunk) {
                if (!mbar_wait(ACC_EMPTY, (chunk & 1) ^ 1, abort_flag)) break;
                tc_fence_after();
                const int kt0 = c * SP_KT_PER_CHUNK, kt1 = min(a.kTiles, kt0 + SP_KT_PER_CHUNK);
                for (int kt = kt0; kt < kt1; ++kt) {
                    const int sb = b % SP_BSLOTS;
                    if (!mbar_wait(B_full(sb), (b / SP_BSLOTS) & 1, abort_flag)) break;
                    tc_fence_after();
                    const int kvalid = min(SP_BK, a.K - kt * SP_BK);
                    const int ksteps = (kvalid + 15) / 16;
                    // level t = i + j is first written by (i = 0, kk = 0) of the chunk's first K tile
                    const uint32_t acc0 = (kt == kt0) ? 0u : 1u;
                    const uint64_t bdb = bd0 + (uint64_t)((sb * T * B_TILE) >> 4);
#pragma unroll
                    for (int i = 0; i < T; ++i) {
                        const int sa = u % SP_ASLOTS;
                        if (!mbar_wait(A_full(sa), (u / SP_ASLOTS) & 1, abort_flag)) break;
                        tc_fence_after();
                        const uint64_t ad = ad0 + (uint64_t)((sa * A_TILE) >> 4);
#pragma unroll
                        for (int j0 = 0; j0 < T - i; j0 += G) {
                            const int nj = (T - i - j0 < G) ? T - i - j0 : G;
                            const uint32_t idesc = idesc0 | ((uint32_t)((nj * NT) >> 3) << 17);
                            const uint32_t d = tmem + (uint32_t)((i + j0) * NT);
                            const uint64_t bd = bdb + (uint64_t)((j0 * B_TILE) >> 4);
                            if (ksteps == SP_BK / 16) {
#pragma unroll
                                for (int kk = 0; kk < SP_BK / 16; ++kk)
                                    mma_bf16(d, ad + 2ull * kk, bd + 2ull * kk, idesc, (i == 0 && kk == 0) ? acc0 : 1u);
                            } else {
                                for (int kk = 0; kk < ksteps; ++kk)
                                    mma_bf16(d, ad + 2ull * kk, bd + 2ull * kk, idesc, (i == 0 && kk == 0) ? acc0 : 1u);
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
                const unsigned long long t0 = global_ns();
                while (!mbar_try(DRAIN, 0) && global_ns() - t0 < SP_WAIT_NS) {
                }
            }
        }
    } else {
        // ------------------------------------------------ epilogue warps 2..17
        const int sub = warp & 3;              // TMEM sub-partition this warp may read
        const int part = (warp - 2) >> 2;      // which slice of the NT columns
        const uint32_t lane_base = (uint32_t)(32 * sub) << 16;
        long long acc[QW];
#pragma unroll
        for (int q = 0; q < QW; ++q) acc[q] = 0;
        int chunk = 0;
        for (int c = c_beg; c < c_end; ++c, ++chunk) {
            // one lane polls, the warp follows it, so tcgen05.ld below runs converged
            int ok = 0;
            if (lane == 0) ok = mbar_wait(ACC_FULL, chunk & 1, abort_flag) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            tc_fence_after();
            // one level at a time: all its column groups in flight, then one wait.
            // A level holds an integer below 2^31 in magnitude (exact for t <= 3),
            // so a 32-bit conversion suffices.
            for (int t = 0; t < T; ++t) {
                const int sh = 8 * (T - 1 - t);
                uint32_t r[QW];
#pragma unroll
                for (int g = 0; g < QW / 8; ++g)
                    tmem_ld8(tmem + lane_base + (uint32_t)(t * NT + part * QW + 8 * g), r + 8 * g);
                tmem_wait_ld();
#pragma unroll
                for (int q = 0; q < QW; ++q) acc[q] += (long long)__float2int_rn(__uint_as_float(r[q])) << sh;
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(ACC_EMPTY);
        }
        // Output through shared memory.  Once the last accumulator is drained every
        // copy has landed and every MMA has completed, so the operand ring is free:
        // the epilogue warps stage the tile there (FP64 bits, or the int64 sum for
        // split-K) with the row and column offsets of the output maps, then write it
        // out with the lanes running along whichever output index is contiguous.
        constexpr int PITCH = NT + 1;
        long long *stage = reinterpret_cast<long long *>(sm);
        long long *row_off = stage + SP_BM * PITCH;
        long long *col_off = row_off + SP_BM;
        int *row_sc = reinterpret_cast<int *>(col_off + NT);   // exponent scales of the output
        int *col_sc = row_sc + SP_BM;
        const int ew = warp - 2, et = threadIdx.x - 64;   // epilogue warp / thread index
        const int m0 = mt * SP_BM, n0 = nt * NT;
        const int rows = min(SP_BM, a.M - m0), cols = min(NT, a.N - n0);
        const bool fin = a.ksplit == 1;   // FP64 output here, else int64 sums to the split-K buffer
        if (!*abort_flag) {
            // the raw sums go to shared memory; they are converted in the write-out,
            // where the accumulator registers are free and a batch of values converts
            // at once instead of one long dependent chain per value
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const int r = 32 * sub + lane;
            const int m = m0 + r;
            if (m < a.M) {
                if (part == 0) {
                    row_off[r] = fin ? off2(a.Cm, m) : (long long)m * a.N;
                    row_sc[r] = fin ? exp_of_word(__ldg(a.eA + m)) - 14 - 8 * (T - 1) : 0;
                }
#pragma unroll
                for (int q = 0; q < QW; ++q) {
                    const int c = part * QW + q;
                    if (n0 + c < a.N) stage[r * PITCH + c] = acc[q];
                }
            }
            for (int c = et; c < cols; c += SP_EPI_THREADS) {
                col_off[c] = fin ? off2(a.Cn, n0 + c) : (long long)(n0 + c);
                col_sc[c] = fin ? exp_of_word(__ldg(a.eB + n0 + c)) : 0;
            }
        }
        asm volatile("bar.sync 1, %0;" ::"n"(SP_EPI_THREADS) : "memory");
        if (!*abort_flag) {
            // Write-out in groups of WU rows (columns): the staged values, offsets and
            // scales of a group are read from shared memory before its stores.
            constexpr int WU = 4;
            const bool along_n = (a.ksplit > 1) || a.Cn.s2 == 1 || a.Cm.s2 != 1;
            if (along_n) {
                constexpr int NCH = (NT + 31) / 32;   // 32-column chunks of a row
                long long co[NCH];
                int cs[NCH];
#pragma unroll
                for (int j = 0; j < NCH; ++j) {
                    const bool in = lane + 32 * j < cols;
                    co[j] = in ? col_off[lane + 32 * j] : 0;
                    cs[j] = in ? col_sc[lane + 32 * j] : 0;
                }
                for (int rb = ew; rb < rows; rb += WU * SP_EPI_WARPS) {
                    long long ro[WU], v[WU][NCH];
                    int rsc[WU];
#pragma unroll
                    for (int w = 0; w < WU; ++w) {
                        const int r = rb + w * SP_EPI_WARPS;
                        ro[w] = r < rows ? row_off[r] : 0;
                        rsc[w] = r < rows ? row_sc[r] : 0;
#pragma unroll
                        for (int j = 0; j < NCH; ++j)
                            v[w][j] = (r < rows && lane + 32 * j < cols) ? stage[r * PITCH + lane + 32 * j] : 0;
                    }
#pragma unroll
                    for (int w = 0; w < WU; ++w) {
                        if (rb + w * SP_EPI_WARPS >= rows) break;
#pragma unroll
                        for (int j = 0; j < NCH; ++j) {
                            if (lane + 32 * j >= cols) continue;
                            if (fin) a.C[ro[w] + co[j]] = scaled_int_to_double(v[w][j], rsc[w] + cs[j]);
                            else atomicAdd(&a.partial[ro[w] + co[j]], (unsigned long long)v[w][j]);
                        }
                    }
                }
            } else {
                constexpr int NRC = SP_BM / 32;   // 32-row chunks of a column
                long long ro[NRC];
                int rsc[NRC];
#pragma unroll
                for (int j = 0; j < NRC; ++j) {
                    const bool in = lane + 32 * j < rows;
                    ro[j] = in ? row_off[lane + 32 * j] : 0;
                    rsc[j] = in ? row_sc[lane + 32 * j] : 0;
                }
                for (int cb = ew; cb < cols; cb += WU * SP_EPI_WARPS) {
                    long long co[WU], v[WU][NRC];
                    int cs[WU];
#pragma unroll
                    for (int w = 0; w < WU; ++w) {
                        const int c = cb + w * SP_EPI_WARPS;
                        co[w] = c < cols ? col_off[c] : 0;
                        cs[w] = c < cols ? col_sc[c] : 0;
#pragma unroll
                        for (int j = 0; j < NRC; ++j)
                            v[w][j] = (c < cols && lane + 32 * j < rows) ? stage[(lane + 32 * j) * PITCH + c] : 0;
                    }
#pragma unroll
                    for (int w = 0; w < WU; ++w) {
                        if (cb + w * SP_EPI_WARPS >= cols) break;
#pragma unroll
                        for (int j = 0; j < NRC; ++j)
                            if (lane + 32 * j < rows) a.C[ro[j] + co[w]] = scaled_int_to_double(v[w][j], rsc[j] + cs[w]);
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
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
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
            scaled_int_to_double((long long)partial[t], exp_of_word(eA[m]) + exp_of_word(eB[n]) - 14 - 8 * (T - 1));
    }
}

int pick_nt(int N, int T)
{
    if (T * 96 > 512) return 64;
    long long w64 = (long long)((N + 63) / 64) * 64, w96 = (long long)((N + 95) / 96) * 96;
    return (w96 <= w64) ? 96 : 64;
}

// A one-CTA-per-SM shape asks for at least 120 KB, so a second CTA never shares the SM
// (it holds all 512 TMEM columns); the NT = 48 shape fits two per SM.
template <int NT, bool DEEP = false>
size_t split_smem_bytes(int T)
{
    const int aslots = DEEP ? (T == 2 ? SpDeep<2>::A : T == 3 ? SpDeep<3>::A : T == 4 ? SpDeep<4>::A : SpDeep<5>::A)
                            : SpCfg<NT>::ASLOTS;
    size_t b = 1024 + (size_t)aslots * SP_BM * SP_BK * 2 + (size_t)SP_BSLOTS * T * NT * SP_BK * 2;
    const size_t out_stage = 1024 + (size_t)SP_BM * (NT + 1) * 8 + (size_t)(SP_BM + NT) * 12;   // epilogue reuse
    if (b < out_stage) b = out_stage;
    if ((DEEP || SpCfg<NT>::MIN_BLOCKS == 1) && b < 120 * 1024) b = 120 * 1024;
    return b;
}

}  // namespace

int split_supported_T(int T) { return T >= 2 && T <= 5; }

SplitPlan split_plan(int M, int N, int K, int T, int nt_override, int ks_override)
{
    SplitPlan p{};
    if (nt_override == SP_DEEP_CODE && T * 48 <= 256) {
        p.deep = 1;
        nt_override = 48;
    }
    p.NT = (nt_override == 64 || (nt_override == 96 && T * 96 <= 512) || (nt_override == 48 && T * 48 <= 256))
               ? nt_override
               : pick_nt(N, T);
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
    for (int nt : {48, 64, 96}) {
        SplitPlan p = split_plan(M, N, K, T, nt, 0);
        if (p.b_pack_bytes > c.b_pack_bytes) c.b_pack_bytes = p.b_pack_bytes;
    }
    const int kTiles = (K + SP_BK - 1) / SP_BK;
    if (kTiles > SP_KT_PER_CHUNK) c.partial_bytes = (size_t)M * N * 8;   // any split-K candidate
    return c;
}

template <int NT, int T, bool DEEP = false>
static cudaError_t split_attr()
{
    return cudaFuncSetAttribute(gemm_split_kernel<NT, T, DEEP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)split_smem_bytes<NT, DEEP>(T));
}

cudaError_t split_prepare()
{
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = split_attr<64, 2>();
    if (e == cudaSuccess) e = split_attr<64, 3>();
    if (e == cudaSuccess) e = split_attr<64, 4>();
    if (e == cudaSuccess) e = split_attr<64, 5>();
    if (e == cudaSuccess) e = split_attr<96, 2>();
    if (e == cudaSuccess) e = split_attr<96, 3>();
    if (e == cudaSuccess) e = split_attr<96, 4>();
    if (e == cudaSuccess) e = split_attr<96, 5>();
    if (e == cudaSuccess) e = split_attr<48, 2>();
    if (e == cudaSuccess) e = split_attr<48, 3>();
    if (e == cudaSuccess) e = split_attr<48, 4>();
    if (e == cudaSuccess) e = split_attr<48, 5>();
    if (e == cudaSuccess) e = split_attr<48, 2, true>();
    if (e == cudaSuccess) e = split_attr<48, 3, true>();
    if (e == cudaSuccess) e = split_attr<48, 4, true>();
    if (e == cudaSuccess) e = split_attr<48, 5, true>();
    return e;
}

// Exponents and digit slices of one operand X(r, k) (rows of A, columns of B).
// A transposed operand -- unit-stride rows, strided K -- is read with the lanes
// along its rows; everything else one row per warp / thread chunk along K.
// ---------------------------------------------------------------- transposed operands, one launch
// Exponents and digits of a transposed operand X(r, k) = X[k * kstride + r] in
// one launch: a cluster of CS CTAs spans K for one group of 32 rows (lanes along
// the contiguous rows, warp kg on the 8-wide chunk kg of each 64-wide K tile).
// CTA c holds the K tiles kt = c + CS i, i < KC, in registers; the row maxima of
// the cluster's CTAs are combined through distributed shared memory between
// cluster barriers (hardware barriers: every thread of every CTA reaches both),
// then each held tile is converted and written through shared memory so that
// eight consecutive threads store one row's 128 bytes.  Rows from R up to
// rowsTotal get zero digits.  Needs CS KC >= kTiles, KC <= KCMAX, CS <= 8.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
__device__ __forceinline__ unsigned ld_cluster_u32(const void *local, unsigned rank)
{
    uint32_t ra, v;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(smem_u32(local)), "r"(rank));
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(ra) : "memory");
    return v;
}

template <int T, int KCMAX>
__global__ void __launch_bounds__(256, 1) split_pack_tc_kernel(int R, int K, int rowsT, int rowsTotal, int kTiles,
                                                               int KC, const double *X, long long kstride, int *e,
                                                               unsigned char *out, long long slice_bytes)
{
    __shared__ unsigned long long Gs[32][SP_BK + 1];
    __shared__ unsigned s_part[8][32];
    __shared__ unsigned s_cta[32];
    __shared__ unsigned s_row[32];
    const int lane = threadIdx.x & 31, kg = threadIdx.x >> 5;
    const int CS = gridDim.x, c = blockIdx.x;   // the cluster spans the grid's x extent
    const int r0 = blockIdx.y * 32, gr = r0 + lane;
    double v[KCMAX][8];
    unsigned m = 0;
#pragma unroll
    for (int i = 0; i < KCMAX; ++i) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = (c + CS * i) * SP_BK + kg * 8 + q;
            v[i][q] = (i < KC && gr < R && k < K) ? X[(long long)k * kstride + gr] : 0.0;
            m = max(m, abs_hi_word(v[i][q]));
        }
    }
    s_part[kg][lane] = m;
    __syncthreads();
    if (kg == 0) {
        unsigned mm = 0;
        for (int w = 0; w < 8; ++w) mm = max(mm, s_part[w][lane]);
        s_cta[lane] = mm;
    }
    cluster_arrive();
    cluster_wait();   // every CTA's s_cta is written
    if (kg == 0) {
        unsigned mm = 0;
        for (int p = 0; p < CS; ++p) mm = max(mm, ld_cluster_u32(&s_cta[lane], (unsigned)p));
        s_row[lane] = mm;
        if (c == 0 && gr < R) e[gr] = (int)mm;
    }
    cluster_arrive();   // this CTA's remote reads are done; waited for before exit
    __syncthreads();
    const int rs = grid_shift(exp_of_word((int)s_row[lane]), SplitDigits<T>::P);
    const int rw = threadIdx.x >> 3, c8 = threadIdx.x & 7;
    const int grw = r0 + rw;
#pragma unroll
    for (int i = 0; i < KCMAX; ++i) {
        const int kt = c + CS * i;
        if (i < KC && kt < kTiles) {   // uniform over the CTA
#pragma unroll
            for (int q = 0; q < 8; ++q) Gs[lane][kg * 8 + q] = biased_fixed<T>(v[i][q], rs);
            __syncthreads();
            if (grw < rowsTotal) {
                unsigned long long G[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) G[q] = Gs[rw][c8 * 8 + q];
                const long long tile = (long long)(grw / rowsT) * kTiles + kt;
                write_digit_chunks<T>(G, out + tile * ((long long)rowsT * SP_BK * 2) + sw128_off(grw % rowsT, c8 * 8),
                                      slice_bytes);
            }
            __syncthreads();
        }
    }
    cluster_wait();
}

template <int T, int KCMAX>
static cudaError_t launch_pack_tc(int R, int K, int rowsT, int rowsTotal, int kTiles, int CS, int KC, const double *X,
                                  long long kstride, int *e, unsigned char *pk, long long slice_bytes, cudaStream_t st)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(CS, (rowsTotal + 31) / 32, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, split_pack_tc_kernel<T, KCMAX>, R, K, rowsT, rowsTotal, kTiles, KC, X, kstride, e,
                              pk, slice_bytes);
}

template <int T>
static cudaError_t split_prepass_t(int R, int K, const double *X, Idx2 rmap, Idx2 kmap, int rowsT, int rowTiles,
                                   int kTiles, int *e, unsigned char *pk, cudaStream_t st)
{
    const long long slice_bytes = (long long)rowTiles * kTiles * rowsT * SP_BK * 2;
    const int KC = (kTiles + 7) / 8;
    int CS = 1;
    while (CS * KC < kTiles) CS *= 2;   // <= 8 for kTiles <= 64
    // one launch for transposed operands whose clusters fit in one wave (one CTA
    // per SM at this register count); wider ones convert faster at full occupancy.
    // (For the n x chi projector operands the clusters cover only a few row groups,
    // but the two-launch path, fully parallel, measured slower: 0.254 -> 0.274 ms of
    // pre-pass per step at D = 6, chi = 72.)
    if (rmap.s1 == 0 && rmap.s2 == 1 && kmap.s1 == 0 && kmap.s2 != 1 && kTiles <= 64 &&
        (long long)(rowTiles * rowsT + 31) / 32 * CS <= device_sm_count()) {
        CTM_COUNT_LAUNCH(1);
        cudaError_t e1 = KC <= 2 ? launch_pack_tc<T, 2>(R, K, rowsT, rowTiles * rowsT, kTiles, CS, KC, X, kmap.s2, e, pk,
                                                        slice_bytes, st)
                                 : launch_pack_tc<T, 8>(R, K, rowsT, rowTiles * rowsT, kTiles, CS, KC, X, kmap.s2, e, pk,
                                                        slice_bytes, st);
        return e1 != cudaSuccess ? e1 : cudaGetLastError();
    }
    if (rmap.s1 == 0 && rmap.s2 == 1 && kmap.s1 == 0 && kmap.s2 != 1) {
        cudaError_t e0 = cudaMemsetAsync(e, 0, sizeof(int) * (size_t)R, st);
        if (e0 != cudaSuccess) return e0;
        CTM_COUNT_LAUNCH(2);
        split_colexp_kernel<<<dim3((R + 127) / 128, (K + SP_COLEXP_K - 1) / SP_COLEXP_K), 128, 0, st>>>(R, K, X,
                                                                                                       kmap.s2, e);
        split_pack_t_kernel<T><<<dim3((rowTiles * rowsT + 31) / 32, kTiles), 256, 0, st>>>(
            R, K, rowsT, rowTiles * rowsT, kTiles, X, kmap.s2, e, pk, slice_bytes);
        return cudaGetLastError();
    }
    if (kmap.s1 == 0 && kmap.s2 == 1) {
        const int rows = rowTiles * rowsT;
        CTM_COUNT_LAUNCH(1);
        const bool pairs = ((uintptr_t)X & 15) == 0 && (K & 1) == 0 && (rmap.s1 & 1) == 0 && (rmap.s2 & 1) == 0;
        if (pairs && kTiles <= 128) {
            int nv = 1;
            while (nv < 8 && (kTiles + nv - 1) / nv > 8) nv *= 2;
            const int wpr = (kTiles + nv - 1) / nv;        // <= 16 warps per row
            const int rpb = wpr >= 8 ? 1 : 8 / wpr;         // rows per block
            const int blocks = (rows + rpb - 1) / rpb, threads = 32 * wpr * rpb;
#define CTM_ROWPACK(NVV)                                                                                              \
    split_rowpack_reg_kernel<NVV, T><<<blocks, threads, 0, st>>>(R, K, rowsT, rows, kTiles, wpr, X, rmap, e, pk,       \
                                                                 slice_bytes)
            if (nv == 1) CTM_ROWPACK(1);
            else if (nv == 2) CTM_ROWPACK(2);
            else if (nv == 4) CTM_ROWPACK(4);
            else CTM_ROWPACK(8);
#undef CTM_ROWPACK
            return cudaGetLastError();
        }
        split_rowpack_kernel<T><<<(rows + 7) / 8, 256, 0, st>>>(R, K, rowsT, rows, kTiles, X, rmap, e, pk,
                                                                slice_bytes);
        return cudaGetLastError();
    }
    CTM_COUNT_LAUNCH(2);
    split_rowexp_kernel<<<(R * 32 + 255) / 256, 256, 0, st>>>(R, K, X, rmap, kmap, e);
    const long long units = (long long)rowTiles * rowsT * kTiles * 8;
    long long blocks = (units + 255) / 256, cap = 64LL * device_sm_count();
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    split_pack_kernel<T><<<(int)blocks, 256, 0, st>>>(R, K, rowsT, rowTiles, kTiles, X, rmap, kmap, e, pk);
    return cudaGetLastError();
}

static cudaError_t split_prepass(int R, int K, const double *X, Idx2 rmap, Idx2 kmap, int rowsT, int rowTiles,
                                 int kTiles, int T, int *e, unsigned char *pk, cudaStream_t st)
{
    switch (T) {
    case 2: return split_prepass_t<2>(R, K, X, rmap, kmap, rowsT, rowTiles, kTiles, e, pk, st);
    case 3: return split_prepass_t<3>(R, K, X, rmap, kmap, rowsT, rowTiles, kTiles, e, pk, st);
    case 4: return split_prepass_t<4>(R, K, X, rmap, kmap, rowsT, rowTiles, kTiles, e, pk, st);
    case 5: return split_prepass_t<5>(R, K, X, rmap, kmap, rowsT, rowTiles, kTiles, e, pk, st);
    default: return cudaErrorInvalidValue;
    }
}

static cudaError_t gemm_split_run(const GemmF64 &g, int T, SplitWork w, cudaStream_t st, cudaEvent_t *ev,
                                  SplitPlan p, const SplitOpts *opt = nullptr)
{
    bool pack_a = !(opt && opt->reuse_a);
    if (opt && opt->a_pk) {
        if (p.a_pack_bytes > opt->a_cap) return cudaErrorInvalidValue;
        w.Apk = opt->a_pk;
        w.a_pack_cap = opt->a_cap;
        w.eA = opt->a_e;
        pack_a = opt->a_fill != 0;
    }
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
    if (ev) cudaEventRecord(ev[2], st);   // before the operand pre-pass (profiling)
    if (pack_a) {
        e = split_prepass(g.M, g.K, g.A, g.Am, g.Ak, SP_BM, p.mTiles, p.kTiles, T, w.eA, w.Apk, st);
        if (e != cudaSuccess) return e;
    }
    if (pack_b) {
        e = split_prepass(g.N, g.K, g.B, g.Bn, g.Bk, p.NT, p.nTiles, p.kTiles, T, w.eB, w.Bpk, st);
        if (e != cudaSuccess) return e;
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
#define CTM_SPLIT_LAUNCH(nt, t) \
    if (p.NT == nt && T == t && !p.deep)                                                                    \
        gemm_split_kernel<nt, t><<<grid, SpCfg<nt>::THREADS, split_smem_bytes<nt>(t), st>>>(a);       \
    if (p.NT == nt && T == t && p.deep && nt == 48)                                                         \
        gemm_split_kernel<48, t, true><<<grid, SpCfg<48>::THREADS, split_smem_bytes<48, true>(t), st>>>(a);
    CTM_SPLIT_LAUNCH(64, 2)
    CTM_SPLIT_LAUNCH(64, 3)
    CTM_SPLIT_LAUNCH(64, 4)
    CTM_SPLIT_LAUNCH(64, 5)
    CTM_SPLIT_LAUNCH(96, 2)
    CTM_SPLIT_LAUNCH(96, 3)
    CTM_SPLIT_LAUNCH(96, 4)
    CTM_SPLIT_LAUNCH(96, 5)
    CTM_SPLIT_LAUNCH(48, 2)
    CTM_SPLIT_LAUNCH(48, 3)
    CTM_SPLIT_LAUNCH(48, 4)
    CTM_SPLIT_LAUNCH(48, 5)
#undef CTM_SPLIT_LAUNCH
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], st);
    if (p.ksplit > 1) {
        const long long total = (long long)g.M * g.N;
        long long blocks = (total + 255) / 256, cap = 16LL * device_sm_count();
        if (blocks > cap) blocks = cap;
        CTM_COUNT_LAUNCH(1);
        split_finalize_kernel<<<(int)blocks, 256, 0, st>>>(g.M, g.N, T, (const unsigned long long *)w.partial,
                                                              w.eA, w.eB, g.C, g.Cm, g.Cn);
        e = cudaGetLastError();
    }
    return e;
}

// ---------------------------------------------------------------- autotuner
// For each new (M, N, K, T) the first eager call times every candidate plan
// (N tile 64 / 96, K-split auto, 1, 2x, 1/2x, one wave) end to end on the real operands
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
    const int tkey[4] = {g.M, g.N, g.K, T};
    int tval[2];
    if (w.autotune && tune_cache_lookup("split", tkey, 4, tval, 2)) {
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune[key] = {tval[0], tval[1]};
        }
        return gemm_split_run(g, T, w, st, ev, split_plan(g.M, g.N, g.K, T, tval[0], tval[1]), opt);
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (!w.autotune || cs != cudaStreamCaptureStatusNone)
        return gemm_split_run(g, T, w, st, ev, split_plan(g.M, g.N, g.K, T), opt);
    SplitPlan base = split_plan(g.M, g.N, g.K, T);
    const int chunks = (base.kTiles + SP_KT_PER_CHUNK - 1) / SP_KT_PER_CHUNK;
    std::vector<std::pair<int, int>> cands;
    for (int nt : {48, 64, 96, SP_DEEP_CODE}) {
        if ((nt == 96 && T * 96 > 512) || ((nt == 48 || nt == SP_DEEP_CODE) && T * 48 > 256)) continue;
        // the deep ring pays off only for long K streams: at K of a few thousand it can win
        // alone yet slow the step, whose concurrent corner update and corner spectrum
        // then find every SM held by one 226 KB CTA (measured 1053 against ~1130 steps/s
        // at D = 6, chi = 72); it was chosen at K = 8192 (D = 8, chi = 128)
        if (nt == SP_DEEP_CODE && (chunks < 2 || g.K < 4096)) continue;
        // auto, none, 2x, 1/2x, and the most splits that still fit one wave of CTAs
        const int ntw = nt == SP_DEEP_CODE ? 48 : nt;   // tile width of the candidate
        const int one_wave = (int)(device_sm_count() / ((long long)base.mTiles * ((g.N + ntw - 1) / ntw)));
        for (int ks : {base.ksplit, 1, 2 * base.ksplit, base.ksplit / 2, one_wave}) {
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
        tot = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {   // first run warms caches; the fastest of three counts
            cudaEventRecord(e0, st);
            cudaError_t e = gemm_split_run(g, T, w, st, nullptr, p);
            cudaEventRecord(e1, st);
            if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return e != cudaSuccess ? e : cudaErrorUnknown;
            }
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep && ms < tot) tot = ms;
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
    tval[0] = best_c.first;
    tval[1] = best_c.second;
    tune_cache_store("split", tkey, 4, tval, 2);
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

// ---------------------------------------------------------------- split TF32
// C = A B with A = A_hi + A_lo and B = B_hi + B_lo (TF32 values in FP32 containers, after
// the exact power-of-two scaling of each row of A and column of B by 2^-E, E from the
// exponent pre-pass above), the products A_hi B_hi + A_hi B_lo + A_lo B_hi (T = 2) or
// A_hi B_hi alone (T = 1) by tcgen05.mma.kind::tf32 into FP32 accumulators in TMEM, so
// the result has about FP32 accuracy.  A K tile is 32 wide: 128-byte rows of four-byte
// elements, so tiles, rings, bulk copies, the 128-byte swizzle and the 32-byte advance of
// the operand descriptors per MMA (K = 8) are those of the BF16 path, byte for byte.  The
// CTA accumulates its whole K range in TMEM (two levels: A_hi [B_hi | B_lo] as one MMA of
// N = 2 NT, then A_lo B_hi into the second level) and drains it once; the epilogue adds the
// levels in FP32 and builds the FP64 result and its scale on the exponent field with integer
// arithmetic.  Split-K partial results meet in an FP64 buffer through atomics.
namespace {

constexpr int TF_BK = 32;            // K per packed tile
constexpr int TF_NT = 64;            // tile N
constexpr int TF_ASLOTS = 4;         // A ring (16 KB slots)
constexpr int TF_EPI_WARPS = 8;      // two per TMEM sub-partition, NT / 2 columns each
constexpr int TF_THREADS = 64 + 32 * TF_EPI_WARPS;
constexpr int TF_KT_PER_CHUNK = 4;   // split-K granularity: 128 K

// byte offset of element (r, k) in a packed (rows x 32) four-byte tile, K-major 128B swizzle
__device__ __forceinline__ int sw128_off32(int r, int k)
{
    return (r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 2) ^ (r & 7))) << 4) + ((k & 3) << 2);
}

// x 2^-E (exact, on the exponent field; |x| < 2^E) rounded to FP32, then hi = that value
// rounded to TF32 (10 fraction bits, ties away from zero) and lo = the exact remainder
// rounded to TF32.  Values more than 2^-1022 below the row's scale become zero.
__device__ __forceinline__ void tf32_split(double x, int E, uint32_t &hi, uint32_t &lo)
{
    const int hw = __double2hiint(x), lw = __double2loint(x);
    const int ex = (hw >> 20) & 0x7FF;
    hi = 0u;
    lo = 0u;
    if (ex == 0 || ex == 0x7FF || ex - E <= 0) return;
    const double xs = __hiloint2double(hw - (E << 20), lw);
    const float f = __double2float_rn(xs);
    const uint32_t hb = (__float_as_uint(f) + 0x1000u) & 0xFFFFE000u;
    const float r = f - __uint_as_float(hb);
    hi = hb;
    lo = (__float_as_uint(r) + 0x1000u) & 0xFFFFE000u;
}

// the FP32 value with bits b times 2^scale, as a double, by integer arithmetic (subnormal
// FP32 values, far below the scales of the row and the column, become zero)
__device__ __forceinline__ double scaled_f32_to_double(uint32_t b, int scale)
{
    const uint32_t mag = b & 0x7FFFFFFFu;
    const int ef = (int)(mag >> 23);
    if (ef == 0) return 0.0;
    const int be = ef - 127 + 1023 + scale;
    if (be <= 0) return 0.0;
    const uint32_t sgn = b & 0x80000000u;
    if (be >= 2047) return __hiloint2double((int)(sgn | 0x7FF00000u), 0);
    const uint32_t m = mag & 0x7FFFFFu;
    return __hiloint2double((int)(sgn | ((uint32_t)be << 20) | (m >> 3)), (int)(m << 29));
}

// Operand pre-pass: one block per 32 rows x one 32-wide K tile.  The loads run along
// whichever index of X is contiguous (rfast: the rows), the hi/lo words are staged in
// shared memory, and one warp stores each row's 128 bytes (its 16-byte chunks permuted
// within the row as the swizzle asks).  Rows from R up to the padded tile grid get zeros.
template <int T>
__global__ void __launch_bounds__(256) tf32_pack_kernel(int R, int K, int rowsT, int rowsTotal, int kTiles,
                                                        const double *X, Idx2 rmap, Idx2 kmap, const int *e, int rfast,
                                                        unsigned char *out, long long slice_bytes)
{
    __shared__ uint32_t Hs[32][33], Ls[32][33];
    __shared__ int Es[32];
    const int r0 = blockIdx.x * 32, kt = blockIdx.y;
    const int tid = threadIdx.x;
    if (tid < 32) Es[tid] = (r0 + tid < R) ? exp_of_word(e[r0 + tid]) : 0;
    __syncthreads();
    for (int q = tid; q < 32 * TF_BK; q += 256) {
        const int i = rfast ? (q & 31) : (q >> 5);
        const int j = rfast ? (q >> 5) : (q & 31);
        const int gr = r0 + i, gk = kt * TF_BK + j;
        uint32_t hi = 0u, lo = 0u;
        if (gr < R && gk < K) tf32_split(X[off2(rmap, gr) + off2(kmap, gk)], Es[i], hi, lo);
        Hs[i][j] = hi;
        Ls[i][j] = lo;
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    for (int i = warp; i < 32; i += 8) {
        const int gr = r0 + i;
        if (gr >= rowsTotal) break;
        const long long tile = (long long)(gr / rowsT) * kTiles + kt;
        unsigned char *dst = out + tile * ((long long)rowsT * TF_BK * 4) + sw128_off32(gr % rowsT, lane);
        *(uint32_t *)dst = Hs[i][lane];
        if (T == 2) *(uint32_t *)(dst + slice_bytes) = Ls[i][lane];
    }
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

size_t tf32_smem_bytes(int T)
{
    size_t b = 1024 + (size_t)TF_ASLOTS * SP_BM * TF_BK * 4 + (size_t)SP_BSLOTS * T * TF_NT * TF_BK * 4;
    const size_t stage = 1024 + (size_t)SP_BM * (TF_NT + 1) * 4 + (size_t)(SP_BM + TF_NT) * 12;
    return b > stage ? b : stage;
}

template <int T>
__global__ void __launch_bounds__(TF_THREADS, 2) gemm_tf32_kernel(SplitArgs a)
{
    constexpr int NT = TF_NT;
    constexpr int A_TILE = SP_BM * TF_BK * 4;   // 16 KB
    constexpr int B_TILE = NT * TF_BK * 4;      // 8 KB
    constexpr int QW = NT / (TF_EPI_WARPS / 4);  // columns per epilogue thread
    constexpr int TMEM_COLS = T == 1 ? 64 : 128;
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint64_t bars[TF_ASLOTS * 2 + SP_BSLOTS * 2 + 2];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;

    unsigned char *sm = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *Asm = sm;
    unsigned char *Bsm = sm + TF_ASLOTS * A_TILE;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t bar0 = smem_u32(bars);
    auto A_full = [&](int s) { return bar0 + 8u * s; };
    auto A_empty = [&](int s) { return bar0 + 8u * (TF_ASLOTS + s); };
    auto B_full = [&](int s) { return bar0 + 8u * (2 * TF_ASLOTS + s); };
    auto B_empty = [&](int s) { return bar0 + 8u * (2 * TF_ASLOTS + SP_BSLOTS + s); };
    const uint32_t ACC_FULL = bar0 + 8u * (2 * TF_ASLOTS + 2 * SP_BSLOTS);
    const uint32_t DRAIN = ACC_FULL + 8u;

    const int nt = blockIdx.x, mt = blockIdx.y, ks = blockIdx.z;
    const int kt_beg = ks * a.chunks_per_split * TF_KT_PER_CHUNK;
    const int kt_end = min(a.kTiles, kt_beg + a.chunks_per_split * TF_KT_PER_CHUNK);
    volatile int *abort_flag = &abort_sh;

    if (threadIdx.x == 0) {
        abort_sh = 0;
        for (int s = 0; s < TF_ASLOTS; ++s) {
            mbar_init(A_full(s), 1);
            mbar_init(A_empty(s), 1);
        }
        for (int s = 0; s < SP_BSLOTS; ++s) {
            mbar_init(B_full(s), 1);
            mbar_init(B_empty(s), 1);
        }
        mbar_init(ACC_FULL, 1);
        mbar_init(DRAIN, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    if (warp == 0) {
        // ------------------------------------------------ producers: bulk copies
        if (lane == 0) {
            int b = 0;
            for (int kt = kt_beg; kt < kt_end && !*abort_flag; ++kt, ++b) {
                const int sb = b % SP_BSLOTS;
                if (!mbar_wait(B_empty(sb), ((b / SP_BSLOTS) & 1) ^ 1, abort_flag)) break;
                mbar_expect_tx(B_full(sb), (uint32_t)(T * B_TILE));
                for (int j = 0; j < T; ++j) {
                    const unsigned char *src = a.Bpk + j * a.b_slice_bytes + ((long long)nt * a.kTiles + kt) * B_TILE;
                    bulk_g2s(smem_u32(Bsm + (sb * T + j) * B_TILE), src, B_TILE, B_full(sb));
                }
            }
        } else if (lane == 1) {
            int u = 0;
            for (int kt = kt_beg; kt < kt_end && !*abort_flag; ++kt) {
                for (int i = 0; i < T; ++i, ++u) {
                    const int sa = u % TF_ASLOTS;
                    if (!mbar_wait(A_empty(sa), ((u / TF_ASLOTS) & 1) ^ 1, abort_flag)) break;
                    mbar_expect_tx(A_full(sa), (uint32_t)A_TILE);
                    const unsigned char *src = a.Apk + i * a.a_slice_bytes + ((long long)mt * a.kTiles + kt) * A_TILE;
                    bulk_g2s(smem_u32(Asm + sa * A_TILE), src, A_TILE, A_full(sa));
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer (one thread)
        if (lane == 0) {
            // kind::tf32: D = F32 (bits 4-5 = 1), A = B = TF32 (bits 7-9, 10-12 = 2), both
            // K-major, N >> 3 at bit 17, M >> 4 at bit 24
            const uint32_t idesc0 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(SP_BM >> 4) << 24);
            const uint64_t ad0 = sdesc_sw128(smem_u32(Asm)), bd0 = sdesc_sw128(smem_u32(Bsm));
            int u = 0, b = 0;
            for (int kt = kt_beg; kt < kt_end && !*abort_flag; ++kt, ++b) {
                const int sb = b % SP_BSLOTS;
                if (!mbar_wait(B_full(sb), (b / SP_BSLOTS) & 1, abort_flag)) break;
                tc_fence_after();
                const uint64_t bdb = bd0 + (uint64_t)((sb * T * B_TILE) >> 4);
#pragma unroll
                for (int i = 0; i < T; ++i, ++u) {
                    const int sa = u % TF_ASLOTS;
                    if (!mbar_wait(A_full(sa), (u / TF_ASLOTS) & 1, abort_flag)) break;
                    tc_fence_after();
                    const uint64_t ad = ad0 + (uint64_t)((sa * A_TILE) >> 4);
                    // A_hi times [B_hi | B_lo] into levels 0 .. T-1; A_lo times B_hi into level 1
                    const int n = (i == 0) ? T * NT : NT;
                    const uint32_t idesc = idesc0 | ((uint32_t)(n >> 3) << 17);
                    const uint32_t d = tmem + (uint32_t)(i * NT);
#pragma unroll
                    for (int kk = 0; kk < TF_BK / 8; ++kk)
                        mma_tf32(d, ad + 2ull * kk, bdb + 2ull * kk, idesc, (kt == kt_beg && kk == 0 && i == 0) ? 0u : 1u);
                    mma_commit(A_empty(sa));
                }
                mma_commit(B_empty(sb));
            }
            mma_commit(ACC_FULL);
            mma_commit(DRAIN);
            {
                const unsigned long long t0 = global_ns();
                while (!mbar_try(DRAIN, 0) && global_ns() - t0 < SP_WAIT_NS) {
                }
            }
        }
    } else {
        // ------------------------------------------------ epilogue warps
        const int sub = warp & 3;
        const int part = (warp - 2) >> 2;
        const uint32_t lane_base = (uint32_t)(32 * sub) << 16;
        uint32_t v[QW];
        int ok = 0;
        if (lane == 0) ok = mbar_wait(ACC_FULL, 0, abort_flag) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (ok) {
            tc_fence_after();
#pragma unroll
            for (int g = 0; g < QW / 8; ++g) tmem_ld8(tmem + lane_base + (uint32_t)(part * QW + 8 * g), v + 8 * g);
            tmem_wait_ld();
            if (T == 2) {
                uint32_t w[QW];
#pragma unroll
                for (int g = 0; g < QW / 8; ++g)
                    tmem_ld8(tmem + lane_base + (uint32_t)(NT + part * QW + 8 * g), w + 8 * g);
                tmem_wait_ld();
#pragma unroll
                for (int q = 0; q < QW; ++q) v[q] = __float_as_uint(__uint_as_float(v[q]) + __uint_as_float(w[q]));
            }
            tc_fence_before();
        }
        // stage the FP32 sums in the (now idle) operand ring, then write them out along the
        // contiguous output index
        constexpr int PITCH = NT + 1;
        uint32_t *stage = reinterpret_cast<uint32_t *>(sm);
        long long *row_off = reinterpret_cast<long long *>(sm + (((size_t)SP_BM * PITCH * 4 + 15) & ~(size_t)15));
        long long *col_off = row_off + SP_BM;
        int *row_sc = reinterpret_cast<int *>(col_off + NT);
        int *col_sc = row_sc + SP_BM;
        const int et = threadIdx.x - 64, ew = warp - 2;
        const int m0 = mt * SP_BM, n0 = nt * NT;
        const int rows = min(SP_BM, a.M - m0), cols = min(NT, a.N - n0);
        const bool fin = a.ksplit == 1;
        if (!*abort_flag) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const int r = 32 * sub + lane;
            if (m0 + r < a.M) {
                if (part == 0) {
                    row_off[r] = fin ? off2(a.Cm, m0 + r) : (long long)(m0 + r) * a.N;
                    row_sc[r] = exp_of_word(__ldg(a.eA + m0 + r));
                }
#pragma unroll
                for (int q = 0; q < QW; ++q) {
                    const int c = part * QW + q;
                    if (n0 + c < a.N) stage[r * PITCH + c] = v[q];
                }
            }
            for (int c = et; c < cols; c += 32 * TF_EPI_WARPS) {
                col_off[c] = fin ? off2(a.Cn, n0 + c) : (long long)(n0 + c);
                col_sc[c] = exp_of_word(__ldg(a.eB + n0 + c));
            }
        }
        asm volatile("bar.sync 1, %0;" ::"n"(32 * TF_EPI_WARPS) : "memory");
        if (!*abort_flag) {
            double *part_buf = reinterpret_cast<double *>(a.partial);
            const bool along_n = !fin || a.Cn.s2 == 1 || a.Cm.s2 != 1;
            if (along_n) {
                for (int r = ew; r < rows; r += TF_EPI_WARPS) {
                    const long long ro = row_off[r];
                    const int rs = row_sc[r];
                    for (int c = lane; c < cols; c += 32) {
                        const double x = scaled_f32_to_double(stage[r * PITCH + c], rs + col_sc[c]);
                        if (fin) a.C[ro + col_off[c]] = x;
                        else atomicAdd(part_buf + ro + col_off[c], x);
                    }
                }
            } else {
                for (int c = ew; c < cols; c += TF_EPI_WARPS) {
                    const long long co = col_off[c];
                    const int cs = col_sc[c];
                    for (int r = lane; r < rows; r += 32)
                        a.C[row_off[r] + co] = scaled_f32_to_double(stage[r * PITCH + c], row_sc[r] + cs);
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
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
    if (threadIdx.x == 0 && abort_sh) atomicExch(a.err, 2);
}

// split-K: the FP64 partial sums (already scaled) to the output maps
__global__ void tf32_finalize_kernel(int M, int N, const double *partial, double *C, Idx2 Cm, Idx2 Cn)
{
    const long long total = (long long)M * N;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(t / N), n = (int)(t - (long long)m * N);
        C[off2(Cm, m) + off2(Cn, n)] = partial[t];
    }
}

}  // namespace

SplitPlan tf32_plan(int M, int N, int K, int T)
{
    SplitPlan p{};
    p.NT = TF_NT;
    p.deep = 0;
    p.mTiles = (M + SP_BM - 1) / SP_BM;
    p.nTiles = (N + TF_NT - 1) / TF_NT;
    p.kTiles = (K + TF_BK - 1) / TF_BK;
    const int chunks = (p.kTiles + TF_KT_PER_CHUNK - 1) / TF_KT_PER_CHUNK;
    const long long tiles = (long long)p.mTiles * p.nTiles;
    const int slots = 2 * device_sm_count();   // two CTAs per SM
    int ks = 1;
    if (tiles < slots && chunks > 1) ks = (int)((slots + tiles - 1) / tiles);
    if (ks > chunks) ks = chunks;
    p.chunks_per_split = (chunks + ks - 1) / ks;
    p.ksplit = (chunks + p.chunks_per_split - 1) / p.chunks_per_split;
    p.a_pack_bytes = (size_t)T * p.mTiles * p.kTiles * SP_BM * TF_BK * 4;
    p.b_pack_bytes = (size_t)T * p.nTiles * p.kTiles * TF_NT * TF_BK * 4;
    p.partial_bytes = p.ksplit > 1 ? (size_t)M * N * 8 : 0;
    return p;
}

SplitPlan tf32_plan_caps(int M, int N, int K, int T) { return tf32_plan(M, N, K, T); }

int tf32_supported_T(int T) { return T == 1 || T == 2; }

cudaError_t tf32_prepare()
{
    cudaError_t e = cudaFuncSetAttribute(gemm_tf32_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tf32_smem_bytes(1));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gemm_tf32_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tf32_smem_bytes(2));
    return e;
}

// exponents of the rows of X(r, k) (the largest high word of |X| along k)
static cudaError_t tf32_exponents(int R, int K, const double *X, Idx2 rmap, Idx2 kmap, int *e, cudaStream_t st)
{
    if (rmap.s1 == 0 && rmap.s2 == 1 && kmap.s1 == 0 && kmap.s2 != 1) {
        cudaError_t e0 = cudaMemsetAsync(e, 0, sizeof(int) * (size_t)R, st);
        if (e0 != cudaSuccess) return e0;
        CTM_COUNT_LAUNCH(1);
        split_colexp_kernel<<<dim3((R + 127) / 128, (K + SP_COLEXP_K - 1) / SP_COLEXP_K), 128, 0, st>>>(R, K, X,
                                                                                                       kmap.s2, e);
        return cudaGetLastError();
    }
    CTM_COUNT_LAUNCH(1);
    split_rowexp_kernel<<<(R * 32 + 255) / 256, 256, 0, st>>>(R, K, X, rmap, kmap, e);
    return cudaGetLastError();
}

static cudaError_t tf32_pack(int R, int K, const double *X, Idx2 rmap, Idx2 kmap, int rowsT, int rowTiles, int kTiles,
                             int T, const int *e, unsigned char *out, cudaStream_t st)
{
    const int rowsTotal = rowTiles * rowsT;
    const long long slice_bytes = (long long)rowsTotal * kTiles * TF_BK * 4;
    const int rfast = (rmap.s1 == 0 && rmap.s2 == 1 && !(kmap.s1 == 0 && kmap.s2 == 1)) ? 1 : 0;
    const dim3 grid((rowsTotal + 31) / 32, kTiles);
    CTM_COUNT_LAUNCH(1);
    if (T == 1)
        tf32_pack_kernel<1><<<grid, 256, 0, st>>>(R, K, rowsT, rowsTotal, kTiles, X, rmap, kmap, e, rfast, out,
                                                  slice_bytes);
    else
        tf32_pack_kernel<2><<<grid, 256, 0, st>>>(R, K, rowsT, rowsTotal, kTiles, X, rmap, kmap, e, rfast, out,
                                                  slice_bytes);
    return cudaGetLastError();
}

cudaError_t gemm_tf32(const GemmF64 &g, int T, SplitWork w, cudaStream_t st, cudaEvent_t *ev)
{
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    if (!tf32_supported_T(T) || g.alpha != 1.0 || g.beta != 0.0) return cudaErrorInvalidValue;
    const SplitPlan p = tf32_plan(g.M, g.N, g.K, T);
    if (p.a_pack_bytes > w.a_pack_cap || p.b_pack_bytes > w.b_pack_cap || p.partial_bytes > w.partial_cap ||
        g.M > w.e_cap || g.N > w.e_cap)
        return cudaErrorInvalidValue;
    cudaError_t e;
    if (ev) cudaEventRecord(ev[2], st);
    if ((e = tf32_exponents(g.M, g.K, g.A, g.Am, g.Ak, w.eA, st)) != cudaSuccess) return e;
    if ((e = tf32_pack(g.M, g.K, g.A, g.Am, g.Ak, SP_BM, p.mTiles, p.kTiles, T, w.eA, w.Apk, st)) != cudaSuccess)
        return e;
    if ((e = tf32_exponents(g.N, g.K, g.B, g.Bn, g.Bk, w.eB, st)) != cudaSuccess) return e;
    if ((e = tf32_pack(g.N, g.K, g.B, g.Bn, g.Bk, TF_NT, p.nTiles, p.kTiles, T, w.eB, w.Bpk, st)) != cudaSuccess)
        return e;
    if (p.ksplit > 1 && (e = cudaMemsetAsync(w.partial, 0, p.partial_bytes, st)) != cudaSuccess) return e;
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
                (long long)p.mTiles * p.kTiles * SP_BM * TF_BK * 4,
                (long long)p.nTiles * p.kTiles * TF_NT * TF_BK * 4,
                w.eA,
                w.eB,
                g.C,
                g.Cm,
                g.Cn,
                (unsigned long long *)w.partial,
                w.err};
    dim3 grid(p.nTiles, p.mTiles, p.ksplit);
    if (ev) cudaEventRecord(ev[0], st);
    CTM_COUNT_LAUNCH(1);
    if (T == 1) gemm_tf32_kernel<1><<<grid, TF_THREADS, tf32_smem_bytes(1), st>>>(a);
    else gemm_tf32_kernel<2><<<grid, TF_THREADS, tf32_smem_bytes(2), st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], st);
    if (p.ksplit > 1) {
        const long long total = (long long)g.M * g.N;
        long long blocks = (total + 255) / 256, cap = 16LL * device_sm_count();
        if (blocks > cap) blocks = cap;
        CTM_COUNT_LAUNCH(1);
        tf32_finalize_kernel<<<(int)blocks, 256, 0, st>>>(g.M, g.N, (const double *)w.partial, g.C, g.Cm, g.Cn);
        e = cudaGetLastError();
    }
    return e;
}
