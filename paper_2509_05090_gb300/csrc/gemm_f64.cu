// FP64 tensor-contraction GEMM for the plain-precision CTMRG step.
//
// Every contraction of the step (enlarged corner, Sec. II.B Fig. 3c; reduced
// corner and corner renormalisation, Fig. 3a,d; edge renormalisation,
// Fig. 3b) is a GEMM over fused tensor indices.  Operands and outputs are
// addressed through two-level index maps (Idx2) so that the permuted 4-index
// layouts are read and written in place, with no transpose kernels.
//
// Tiles from 32 x 32 to 72 x 72 outputs per CTA (the bond dimensions divide
// them), a strided micro-tile per thread so a warp's shared-memory reads are
// conflict-free, K staged through shared memory with a register prefetch of the
// next K tile; the tile and the K split are chosen per shape from a wave model.
#include "ctm_internal.h"

namespace {

__device__ __forceinline__ long long off2(const Idx2 &x, int i)
{
    if (x.s1 == 0) return (long long)i * x.s2;   // plain strided dimension: no division
    int hi = i / x.div;
    int lo = i - hi * x.div;
    return (long long)hi * x.s1 + (long long)lo * x.s2;
}

// BM x BN outputs per CTA, (BM/MT) x (BN/MT) threads with an MT x MT micro-tile
// each (rows ty + TY*i, columns tx + TX*j), K staged BK at a time.  GB300's FP64
// pipe is narrow enough that shared-memory bandwidth never binds, so the small
// tiles use 2 x 2 micro-tiles: more threads per CTA to hide the FP64 latency.  The tile
// shape is picked per GEMM so that the bond dimensions (chi = 72, D2 = 36 ...)
// divide it without padding waste.  When the K map has unit stride the A tile
// is fetched K-fastest, otherwise M-fastest (likewise N/K for B), so
// consecutive threads touch consecutive addresses whenever the layout allows.
template <int BM, int BN, int BK, int MT>
__global__ void __launch_bounds__((BM / MT) * (BN / MT)) gemm_f64_kernel(GemmF64 g, int a_kfast, int b_nfast,
                                                                         int kchunk, double *partial)
{
    constexpr int TY = BM / MT, TX = BN / MT, NT = TY * TX;
    constexpr int EA = (BM * BK + NT - 1) / NT, EB = (BN * BK + NT - 1) / NT;
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(g.K, kbeg + kchunk);

    double acc[MT][MT];
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < MT; ++j) acc[i][j] = 0.0;

    double ra[EA], rb[EB];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int e = 0; e < EA; ++e) {
            int lin = tid + e * NT;
            double v = 0.0;
            if (lin < BM * BK) {
                int mm, kk;
                if (a_kfast) { kk = lin % BK; mm = lin / BK; }
                else { mm = lin % BM; kk = lin / BM; }
                int m = m0 + mm, k = k0 + kk;
                if (m < g.M && k < kend) v = g.A[off2(g.Am, m) + off2(g.Ak, k)];
            }
            ra[e] = v;
        }
#pragma unroll
        for (int e = 0; e < EB; ++e) {
            int lin = tid + e * NT;
            double v = 0.0;
            if (lin < BN * BK) {
                int nn, kb;
                if (b_nfast) { nn = lin % BN; kb = lin / BN; }
                else { kb = lin % BK; nn = lin / BK; }
                int n = n0 + nn, k2 = k0 + kb;
                if (n < g.N && k2 < kend) v = g.B[off2(g.Bk, k2) + off2(g.Bn, n)];
            }
            rb[e] = v;
        }
    };
    auto stash = [&]() {
#pragma unroll
        for (int e = 0; e < EA; ++e) {
            int lin = tid + e * NT;
            if (lin < BM * BK) {
                int mm, kk;
                if (a_kfast) { kk = lin % BK; mm = lin / BK; }
                else { mm = lin % BM; kk = lin / BM; }
                As[kk][mm] = ra[e];
            }
        }
#pragma unroll
        for (int e = 0; e < EB; ++e) {
            int lin = tid + e * NT;
            if (lin < BN * BK) {
                int nn, kb;
                if (b_nfast) { nn = lin % BN; kb = lin / BN; }
                else { kb = lin % BK; nn = lin / BK; }
                Bs[kb][nn] = rb[e];
            }
        }
    };

    if (kbeg < kend) fetch(kbeg);
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        __syncthreads();
        stash();
        __syncthreads();
        if (k0 + BK < kend) fetch(k0 + BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[MT], b[MT];
#pragma unroll
            for (int i = 0; i < MT; ++i) a[i] = As[kk][ty + TY * i];
#pragma unroll
            for (int j = 0; j < MT; ++j) b[j] = Bs[kk][tx + TX * j];
#pragma unroll
            for (int i = 0; i < MT; ++i)
#pragma unroll
                for (int j = 0; j < MT; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
    }

#pragma unroll
    for (int i = 0; i < MT; ++i) {
        int m = m0 + ty + TY * i;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < MT; ++j) {
            int n = n0 + tx + TX * j;
            if (n >= g.N) continue;
            if (partial) {
                partial[((size_t)blockIdx.z * g.M + m) * g.N + n] = acc[i][j];
            } else {
                long long o = off2(g.Cm, m) + off2(g.Cn, n);
                double v = g.alpha * acc[i][j];
                if (g.beta != 0.0) v += g.beta * g.C[o];
                g.C[o] = v;
            }
        }
    }
}

struct TileCfg {
    int bm, bn, bk, mt;
};
constexpr TileCfg kTiles[] = {{64, 64, 16, 4}, {72, 72, 12, 4}, {64, 32, 16, 4}, {72, 36, 12, 4},
                              {32, 64, 16, 4}, {36, 72, 12, 4}, {64, 72, 12, 4}, {72, 64, 16, 4},
                              {32, 32, 16, 2}, {36, 36, 12, 2}};

// Deterministic split-K reduction: fixed summation order over the splits.
__global__ void splitk_reduce_kernel(GemmF64 g, int ksplit, const double *partial)
{
    long long total = (long long)g.M * g.N;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int z = 0; z < ksplit; ++z) s += partial[(size_t)z * total + t];
        int m = (int)(t / g.N), n = (int)(t - (long long)m * g.N);
        long long o = off2(g.Cm, m) + off2(g.Cn, n);
        double v = g.alpha * s;
        if (g.beta != 0.0) v += g.beta * g.C[o];
        g.C[o] = v;
    }
}

}  // namespace

unsigned long long g_ctm_launches = 0;

int device_sm_count()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

static long long ceil_to(long long x, long long b) { return (x + b - 1) / b * b; }

// Tile and K-split choice.  The FP64 pipe of one SM is the bottleneck, so the
// cost of a (tile, split) pair is the number of waves of CTAs times the padded
// work of one CTA (small tiles also re-read operands more often, charged
// lightly).  Split-K candidates (only when the caller gave scratch): enough
// splits for two CTAs per SM, and the most splits that still fit one wave.
struct TilePick {
    TileCfg t;
    int ksplit;
};

static TilePick pick_tile_split(int M, int N, int K, bool splitk_ok)
{
    const long long sms = device_sm_count();
    TilePick best{kTiles[0], 1};
    double best_cost = 1e300;
    for (const TileCfg &t : kTiles) {
        const long long tiles = ((M + t.bm - 1) / t.bm) * (long long)((N + t.bn - 1) / t.bn);
        long long cand[3] = {1, 1, 1};
        int nc = 1;
        if (splitk_ok && tiles < 2 * sms && K >= 4 * t.bk) {
            long long maxs = K / (2 * t.bk);
            if (maxs > 64) maxs = 64;
            long long s2 = (2 * sms + tiles - 1) / tiles, s1 = sms / tiles;
            cand[nc++] = s2 < maxs ? s2 : maxs;
            cand[nc++] = s1 < maxs ? s1 : maxs;
        }
        for (int ci = 0; ci < nc; ++ci) {
            const long long s = cand[ci] < 1 ? 1 : cand[ci];
            const long long kchunk = ceil_to((K + s - 1) / s, t.bk);
            const long long s_eff = (K + kchunk - 1) / kchunk;
            const long long ctas = tiles * s_eff;
            const long long waves = (ctas + sms - 1) / sms;
            double cost = (double)waves * t.bm * t.bn * kchunk * (1.0 + 8.0 / t.bm + 8.0 / t.bn);
            if (s_eff > 1) cost += (double)M * N * s_eff / (double)sms;   // the split-K reduction
            if (cost < best_cost * 0.999) {
                best_cost = cost;
                best = TilePick{t, (int)s_eff};
            }
        }
    }
    return best;
}

static TileCfg pick_tile(int M, int N, int K, bool splitk_ok) { return pick_tile_split(M, N, K, splitk_ok).t; }

int gemm_f64_pick_split(int M, int N, int K) { return pick_tile_split(M, N, K, true).ksplit; }

template <int BM, int BN, int BK, int MT>
static cudaError_t launch_tile(const GemmF64 &g, int ksplit, double *scratch, cudaStream_t st)
{
    int a_kfast = (g.Ak.s2 == 1 && g.Ak.div >= g.K) ? 1 : 0;
    int b_nfast = (g.Bn.s2 == 1 && g.Bn.div >= g.N) ? 1 : 0;
    if (ksplit < 1 || !scratch) ksplit = 1;
    int kchunk = (g.K + ksplit - 1) / ksplit;
    kchunk = ((kchunk + BK - 1) / BK) * BK;
    if (kchunk <= 0) kchunk = BK;
    ksplit = (g.K + kchunk - 1) / kchunk;
    if (ksplit < 1) ksplit = 1;
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, ksplit);
    constexpr int NT = (BM / MT) * (BN / MT);
    if (ksplit == 1) {
        CTM_COUNT_LAUNCH(1);
        gemm_f64_kernel<BM, BN, BK, MT><<<grid, NT, 0, st>>>(g, a_kfast, b_nfast, kchunk, nullptr);
        return cudaGetLastError();
    }
    CTM_COUNT_LAUNCH(2);
    gemm_f64_kernel<BM, BN, BK, MT><<<grid, NT, 0, st>>>(g, a_kfast, b_nfast, kchunk, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    long long total = (long long)g.M * g.N;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4 * device_sm_count()) blocks = 4 * device_sm_count();
    splitk_reduce_kernel<<<blocks, 256, 0, st>>>(g, ksplit, scratch);
    return cudaGetLastError();
}

cudaError_t gemm_f64(const GemmF64 &g, int ksplit, double *scratch, size_t scratch_elems, cudaStream_t st)
{
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    // never let the split-K partials outgrow the scratch the caller owns
    const size_t per_split = (size_t)g.M * (size_t)g.N;
    if (ksplit > 1 && (!scratch || (size_t)ksplit * per_split > scratch_elems))
        ksplit = scratch ? (int)(scratch_elems / per_split) : 1;
    if (ksplit < 1) ksplit = 1;
    TileCfg t = pick_tile(g.M, g.N, g.K, ksplit > 1);
#define CTM_TILE(a, b, c, d) \
    if (t.bm == a && t.bn == b && t.bk == c && t.mt == d) return launch_tile<a, b, c, d>(g, ksplit, scratch, st);
    CTM_TILE(64, 64, 16, 4)
    CTM_TILE(72, 72, 12, 4)
    CTM_TILE(64, 32, 16, 4)
    CTM_TILE(72, 36, 12, 4)
    CTM_TILE(32, 64, 16, 4)
    CTM_TILE(36, 72, 12, 4)
    CTM_TILE(64, 72, 12, 4)
    CTM_TILE(72, 64, 16, 4)
    CTM_TILE(32, 32, 16, 2)
    CTM_TILE(36, 36, 12, 2)
#undef CTM_TILE
    return cudaErrorInvalidValue;
}
