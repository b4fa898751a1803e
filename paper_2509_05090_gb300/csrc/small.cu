// Bandwidth- and latency-bound kernels of the CTMRG step: C3v projection and
// double layer (Sec. II.A, App. A, Fig. 1b), environment initialisation,
// warm start of the reduced corner, corner re-symmetrisation and
// normalisation (Fig. 3a), edge normalisation, the corner-spectrum
// convergence test, and the final bond-energy contraction (Eq. 1, Eq. 4).
// All FP64.
#include <math.h>

#include <atomic>
#include <cooperative_groups.h>
#include <mutex>

#include "ctm_internal.h"

namespace {

__device__ __forceinline__ double block_sum(double v, double *red)
{
    // block-wide reduction (any block size up to 1024; red: >= 32 doubles): warp
    // sums, then warp 0 reduces the per-warp sums with shuffles -- short FP64 chains
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double s = (lane < nw) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) red[32] = s;
    }
    __syncthreads();
    return red[32];
}

// a0: A_sym = (1/6) sum over the six permutations of the virtual legs, then
// unit Frobenius norm.  One CTA; the tensor is at most a few thousand entries.
__global__ void c3v_project_kernel(int d, int D, const double *Ain, double *Aout, int symmetrize)
{
    extern __shared__ double sA[];
    __shared__ double red[33];
    const int D3 = D * D * D, tot = d * D3;
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
        int s = t / D3, r = t % D3;
        int i = r / (D * D), j = (r / D) % D, k = r % D;
        const double *As = Ain + (size_t)s * D3;
        double v;
        if (symmetrize)
            v = (As[(i * D + j) * D + k] + As[(i * D + k) * D + j] + As[(j * D + i) * D + k] +
                 As[(j * D + k) * D + i] + As[(k * D + i) * D + j] + As[(k * D + j) * D + i]) / 6.0;
        else
            v = As[r];
        sA[t] = v;
    }
    __syncthreads();
    double ss = 0.0;
    for (int t = threadIdx.x; t < tot; t += blockDim.x) ss += sA[t] * sA[t];
    ss = block_sum(ss, red);
    double f = (symmetrize && ss > 0.0) ? 1.0 / sqrt(ss) : 1.0;
    for (int t = threadIdx.x; t < tot; t += blockDim.x) Aout[t] = sA[t] * f;
}

// a1: a[(ii')][(jj')][(kk')] = sum_s K[s,i,j,k] B[s,i',j',k'].
__global__ void double_layer_kernel(int d, int D, const double *K, const double *B, double *a)
{
    const int D2 = D * D, D3 = D * D * D;
    const long long tot = (long long)D2 * D2 * D2;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x) {
        int u = (int)(t / (D2 * D2)), v = (int)((t / D2) % D2), w = (int)(t % D2);
        int i = u / D, i2 = u % D, j = v / D, j2 = v % D, k = w / D, k2 = w % D;
        double s = 0.0;
        for (int p = 0; p < d; ++p)
            s = fma(K[(size_t)p * D3 + (i * D + j) * D + k], B[(size_t)p * D3 + (i2 * D + j2) * D + k2], s);
        a[t] = s;
    }
}

// Open layers for the bond-energy contraction: b[(s,t)][u][v][w] = A[s]... (x) A[t]...
__global__ void open_layers_kernel(int d, int D, const double *A, double *b)
{
    const int D2 = D * D, D3 = D * D * D;
    const long long per = (long long)D2 * D2 * D2;
    const long long tot = per * d * d;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x) {
        int p = (int)(t / per);
        long long r = t - p * per;
        int s = p / d, q = p % d;
        int u = (int)(r / (D2 * D2)), v = (int)((r / D2) % D2), w = (int)(r % D2);
        int i = u / D, i2 = u % D, j = v / D, j2 = v % D, k = w / D, k2 = w % D;
        b[t] = A[(size_t)s * D3 + (i * D + j) * D + k] * A[(size_t)q * D3 + (i2 * D + j2) * D + k2];
    }
}

// Initial environment: C = I, T[a][u][b] = delta_ab t_u, t_u = sum_{v,w} a[u][(vv)][(ww)],
// Q = first chi columns of I_n.
__global__ void init_env_kernel(int chi, int D, const double *a, double *C, double *T, double *Q)
{
    const int D2 = D * D;
    const long long n = (long long)chi * D2;
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = tid; t < (long long)chi * chi; t += stride) C[t] = ((t / chi) == (t % chi)) ? 1.0 : 0.0;
    for (long long t = tid; t < n * chi; t += stride) Q[t] = ((t / chi) == (t % chi)) ? 1.0 : 0.0;
    for (long long t = tid; t < (long long)chi * D2 * chi; t += stride) {
        int al = (int)(t / ((long long)D2 * chi));
        int u = (int)((t / chi) % D2);
        int be = (int)(t % chi);
        double v = 0.0;
        if (al == be)
            for (int p = 0; p < D; ++p)
                for (int q = 0; q < D; ++q) v += a[((size_t)u * D2 + p * D + p) * D2 + q * D + q];
        T[t] = v;
    }
}

// Reduced-corner warm start: Qs = Q diag(sgn C_jj), sgn(0) = +1.
__global__ void warm_start_kernel(long long n, int chi, const double *Q, const double *C, double *Qs)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n * chi;
         t += (long long)gridDim.x * blockDim.x) {
        int j = (int)(t % chi);
        double v = Q[t];
        Qs[t] = (C[(size_t)j * chi + j] < 0.0) ? -v : v;
    }
}

// a5 tail: C' = (Cr + Cr^T)/2, then unit Frobenius norm, over several blocks (the FP64 work of one SM would
// bind): partial sums of squares, then every block derives the factor from the
// partials with one warp and scales its share.
__global__ void corner_sym_sumsq_kernel(int chi, const double *Cr, double *partials)
{
    __shared__ double red[33];
    double ss = 0.0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < chi * chi; t += gridDim.x * blockDim.x) {
        const int i = t / chi, j = t - i * chi;
        const double v = 0.5 * (Cr[t] + Cr[(size_t)j * chi + i]);
        ss = fma(v, v, ss);
    }
    ss = block_sum(ss, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = ss;
}
__global__ void corner_sym_scale_kernel(int chi, const double *Cr, const double *partials, int np, double *Cn)
{
    __shared__ double f;
    if (threadIdx.x < 32) {
        double s = 0.0;
        for (int i = threadIdx.x; i < np; i += 32) s += partials[i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) f = s > 0.0 ? 1.0 / sqrt(s) : 1.0;
    }
    __syncthreads();
    const double h = 0.5 * f;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < chi * chi; t += gridDim.x * blockDim.x) {
        const int i = t / chi, j = t - i * chi;
        Cn[t] = (Cr[t] + Cr[(size_t)j * chi + i]) * h;
    }
}

// Frobenius normalisation of a large array: per-block partial sums of squares...
__global__ void sumsq_partial_kernel(long long count, const double *x, double *partials)
{
    __shared__ double red[33];
    double s = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
         t += (long long)gridDim.x * blockDim.x)
        s = fma(x[t], x[t], s);
    s = block_sum(s, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// ... then every block re-sums the partials in the same order and scales its share.
__global__ void scale_by_partials_kernel(long long count, double *x, const double *partials, int np)
{
    __shared__ double f;
    if (threadIdx.x < 32) {   // one warp sums the partials: short chains, then shuffles
        double s = 0.0;
        for (int i = threadIdx.x; i < np; i += 32) s += partials[i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) f = s > 0.0 ? 1.0 / sqrt(s) : 1.0;
    }
    __syncthreads();
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
         t += (long long)gridDim.x * blockDim.x)
        x[t] *= f;
}

// a7: corner spectrum and delta, in three launches.
// (1) Householder tridiagonalisation of the symmetric corner -> diagonal d and squared
//     off-diagonal e^2 (global work buffer): one CTA with the corner in shared memory
//     below TRI_CLUSTER_MIN, a thread-block cluster holding it by rows from there;
// (2) one warp per eigenvalue: multisection on [-|C|_F, |C|_F], each
//     lane evaluating the Sturm count at one of 32 points per round
//     (5 bits per round instead of 1).  The count is the number of sign
//     changes of p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2}, kept in range by
//     exact power-of-two rescaling -- no division on the dependent chain;
// (3) one CTA: |lambda| sorted descending by rank, unit 2-norm, delta.
constexpr int SPEC_WARPS = 1;   // one eigenvalue per CTA: the chi Sturm chains spread over chi SMs
constexpr int TRI_THREADS = 256;
constexpr size_t SPEC_SM_ALONE_BYTES = 220 * 1024;   // within the 224 KB opt-in of spectrum_prepare
constexpr int TRI_FULL_MAX = 160;   // the full corner in shared memory up to here, its lower triangle beyond
constexpr int TRI_SMEM_MAX = 224;   // the lower triangle of a 224 x 224 corner: 197 KB of shared memory
constexpr int SPEC_MAX_CHI = 512;   // beyond TRI_SMEM_MAX the lower triangle lives in the work buffer (L2)
// From here up the reduction runs over a thread-block cluster where the device schedules one
// (its per-column cost hardly depends on chi, so it overtakes the one-CTA kernels early;
// the benchmark's chi = 72 and the batch's instances keep the one-CTA kernel)
constexpr int TRI_CLUSTER_MIN = 97;

// offset (doubles) of the global lower triangle in the spectrum's work buffer, after
// d, e^2 (2 chi) and the eigenvalues (chi)
__host__ __device__ inline size_t tri_global_off(int chi) { return (size_t)3 * chi + 8; }

__global__ void __launch_bounds__(TRI_THREADS) tridiag_kernel(int chi, const double *C, double *work)
{
    extern __shared__ double sm[];
    __shared__ double red[33];
    __shared__ double sh_beta, sh_alpha;
    // odd row pitch: the mat-vec's lanes read down a column, conflict-free
    const int ld = chi | 1;
    double *A = sm;                      // chi x ld
    double *v = A + chi * ld;            // chi
    double *p = v + chi;                 // chi
    const int tid = threadIdx.x;
    for (int t = tid; t < chi * chi; t += blockDim.x) {
        int i = t / chi, j = t % chi;
        A[i * ld + j] = 0.5 * (C[t] + C[(size_t)j * chi + i]);
    }
    __syncthreads();
    for (int kc = 0; kc + 2 < chi; ++kc) {
        const int b0 = kc + 1, m = chi - b0;
        // x = the column below the diagonal, kept in v (v_0 = x_0 until alpha is known)
        double part = 0.0;
        for (int i = tid; i < m; i += blockDim.x) {
            const double x = A[(b0 + i) * ld + kc];
            v[i] = x;
            if (i > 0) part += x * x;
        }
        const double tail = block_sum(part, red);   // its barriers also publish v
        if (tail == 0.0) continue;                  // already tridiagonal in this column
        const double x0 = v[0];
        // the last thread (outside the mat-vec rows) derives the reflector while the
        // others form y = A x; then A v = y - alpha A e_0 with v = x - alpha e_0
        if (tid == (int)blockDim.x - 1) {
            const double nrm = sqrt(tail + x0 * x0);
            const double alpha = (x0 >= 0.0) ? -nrm : nrm;
            sh_alpha = alpha;
            sh_beta = 1.0 / (nrm * (nrm + fabs(x0)));
        }
        for (int i = tid; i < m; i += blockDim.x) {
            const double *row = A + (b0 + i) * ld + b0;
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
            int j = 0;
            for (; j + 3 < m; j += 4) {
                s0 = fma(row[j], v[j], s0);
                s1 = fma(row[j + 1], v[j + 1], s1);
                s2 = fma(row[j + 2], v[j + 2], s2);
                s3 = fma(row[j + 3], v[j + 3], s3);
            }
            for (; j < m; ++j) s0 = fma(row[j], v[j], s0);
            p[i] = (s0 + s1) + (s2 + s3);
        }
        __syncthreads();
        const double beta = sh_beta, alpha = sh_alpha;
        for (int i = tid; i < m; i += blockDim.x) p[i] = beta * fma(-alpha, A[(b0 + i) * ld + b0], p[i]);
        if (tid == 0) v[0] = x0 - alpha;
        __syncthreads();
        double pv = 0.0;
        for (int i = tid; i < m; i += blockDim.x) pv += p[i] * v[i];
        pv = block_sum(pv, red);
        const double Kf = 0.5 * beta * pv;
        for (int i = tid; i < m; i += blockDim.x) p[i] -= Kf * v[i];   // p <- w
        __syncthreads();
        for (int t = tid; t < m * m; t += blockDim.x) {
            int i = t / m, j = t % m;
            A[(b0 + i) * ld + b0 + j] -= v[i] * p[j] + p[i] * v[j];
        }
        if (tid == 0) {
            A[b0 * ld + kc] = alpha;
            A[kc * ld + b0] = alpha;
        }
        __syncthreads();
    }
    for (int i = tid; i < chi; i += blockDim.x) {
        work[i] = A[i * ld + i];
        double e = (i + 1 < chi) ? A[(i + 1) * ld + i] : 0.0;
        work[chi + i] = e * e;
    }
}

// The same reduction with only the lower triangle stored (packed rows; the mat-vec reads
// the upper part through the symmetry), for corners too large for the full matrix:
// chi > TRI_FULL_MAX.  GA: the triangle lives in the work buffer (global memory, L2
// resident: 1 MB at chi = 512) instead of shared memory, for chi > TRI_SMEM_MAX; the
// steps are the same, and __syncthreads orders the block's global accesses as it does
// its shared ones.
__device__ __forceinline__ int lo_off(int i, int j) { return i * (i + 1) / 2 + j; }   // i >= j

template <bool GA>
__global__ void __launch_bounds__(TRI_THREADS) tridiag_packed_kernel(int chi, const double *C, double *work)
{
    extern __shared__ double sm[];
    __shared__ double red[33];
    __shared__ double sh_beta, sh_alpha;
    double *A = GA ? work + tri_global_off(chi) : sm;         // chi (chi + 1) / 2
    double *v = GA ? sm : A + (size_t)chi * (chi + 1) / 2;    // chi
    double *p = v + chi;                                      // chi
    const int tid = threadIdx.x;
    for (int t = tid; t < chi * chi; t += blockDim.x) {
        const int i = t / chi, j = t % chi;
        if (j <= i) A[lo_off(i, j)] = 0.5 * (C[t] + C[(size_t)j * chi + i]);
    }
    __syncthreads();
    for (int kc = 0; kc + 2 < chi; ++kc) {
        const int b0 = kc + 1, m = chi - b0;
        double part = 0.0;
        for (int i = tid; i < m; i += blockDim.x) {
            const double x = A[lo_off(b0 + i, kc)];
            v[i] = x;
            if (i > 0) part += x * x;
        }
        const double tail = block_sum(part, red);
        if (tail == 0.0) continue;
        const double x0 = v[0];
        if (tid == (int)blockDim.x - 1) {
            const double nrm = sqrt(tail + x0 * x0);
            const double alpha = (x0 >= 0.0) ? -nrm : nrm;
            sh_alpha = alpha;
            sh_beta = 1.0 / (nrm * (nrm + fabs(x0)));
        }
        for (int i = tid; i < m; i += blockDim.x) {
            const int r = b0 + i;
            const double *row = A + lo_off(r, b0);   // A[r][b0 + j] for j <= i
            double s0 = 0.0, s1 = 0.0;
            int j = 0;
            for (; j + 1 <= i; j += 2) {
                s0 = fma(row[j], v[j], s0);
                s1 = fma(row[j + 1], v[j + 1], s1);
            }
            if (j <= i) s0 = fma(row[j], v[j], s0);
            for (j = i + 1; j < m; ++j) s1 = fma(A[lo_off(b0 + j, r)], v[j], s1);   // A[r][b0+j] = A[b0+j][r]
            p[i] = s0 + s1;
        }
        __syncthreads();
        const double beta = sh_beta, alpha = sh_alpha;
        for (int i = tid; i < m; i += blockDim.x) p[i] = beta * fma(-alpha, A[lo_off(b0 + i, b0)], p[i]);
        if (tid == 0) v[0] = x0 - alpha;
        __syncthreads();
        double pv = 0.0;
        for (int i = tid; i < m; i += blockDim.x) pv += p[i] * v[i];
        pv = block_sum(pv, red);
        const double Kf = 0.5 * beta * pv;
        for (int i = tid; i < m; i += blockDim.x) p[i] -= Kf * v[i];   // p <- w
        __syncthreads();
        for (int t = tid; t < m * m; t += blockDim.x) {
            const int i = t / m, j = t % m;
            if (j <= i) A[lo_off(b0 + i, b0 + j)] -= v[i] * p[j] + p[i] * v[j];
        }
        if (tid == 0) A[lo_off(b0, kc)] = alpha;
        __syncthreads();
    }
    for (int i = tid; i < chi; i += blockDim.x) {
        work[i] = A[lo_off(i, i)];
        double e = (i + 1 < chi) ? A[lo_off(i + 1, i)] : 0.0;
        work[chi + i] = e * e;
    }
}

// The reduction spread over a thread-block cluster, for chi >= TRI_CLUSTER_MIN: the
// symmetric corner is distributed by rows (row i, all chi entries, on CTA i % CS), so
// each CTA's mat-vec and rank-2 update touch only its own shared memory.  Per column kc
// the CTA owning row kc (= column kc) stores d_kc = A[kc][kc] and writes the row's
// trailing part x into every CTA's column buffer (distributed shared memory); after a
// cluster barrier every CTA derives the same reflector from the same bits (alpha =
// -sign(x_0)|x|, v = x - alpha e_0, beta = 1/(|x|(|x| + |x_0|))), forms p_i = beta (A v)_i
// for its rows and writes p_i into every CTA's p buffer; after a second barrier every
// CTA forms w = p - (beta/2)(p^T v) v and updates its rows, A_ij -= v_i w_j + w_i v_j.
// e_kc = alpha.  The two buffers alternate by column parity, so a broadcast never
// overwrites one still being read (every CTA passes the next column's first barrier
// only after finishing the current column).  Cluster barriers are hardware barriers:
// nothing spins.
constexpr int TRI_CL_THREADS = 512;   // the largest block tri_cluster_threads gives
constexpr int TRI_CL_SMEM_MAX = 226 * 1024;   // dynamic, below the 227 KB opt-in less the static part

// one warp per local row (4 to 16 warps): fewer threads make the per-column barriers cheaper
__host__ __device__ inline int tri_cluster_threads(int chi, int cs)
{
    const int w = (chi + cs - 1) / cs;
    return 32 * (w < 4 ? 4 : w > 16 ? 16 : w);
}

__host__ __device__ inline size_t tri_cluster_smem_bytes(int chi, int cs)
{
    return sizeof(double) * ((size_t)((chi + cs - 1) / cs) * chi + 5 * (size_t)chi);
}

template <int CS>
__global__ void __launch_bounds__(TRI_CL_THREADS, 1) tridiag_cluster_kernel(int chi, const double *C, double *work)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ double sm[];
    __shared__ double red[33];
    const int rank = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int nloc = (chi - rank + CS - 1) / CS;   // rows rank, rank + CS, ...
    const int nmax = (chi + CS - 1) / CS;
    double *A = sm;                           // nmax x chi, full rows
    double *vb = A + (size_t)nmax * chi;      // 2 x chi: the pivot row's trailing part, by parity
    double *pb = vb + 2 * (size_t)chi;        // 2 x chi: p, by parity
    double *w = pb + 2 * (size_t)chi;         // chi
    for (int t = tid; t < nloc * chi; t += blockDim.x) {
        const int l = t / chi, j = t % chi, i = rank + CS * l;
        A[t] = 0.5 * (C[(size_t)i * chi + j] + C[(size_t)j * chi + i]);
    }
    cl.sync();   // every CTA of the cluster is running before the first remote store
    for (int kc = 0; kc + 2 < chi; ++kc) {
        const int b0 = kc + 1, m = chi - b0;
        double *v = vb + (size_t)(kc & 1) * chi;
        double *p = pb + (size_t)(kc & 1) * chi;
        if (kc % CS == rank) {
            const double *row = A + (size_t)(kc / CS) * chi;
            if (tid == 0) work[kc] = row[kc];
            for (int t = tid; t < m * CS; t += blockDim.x) {
                const int r = t / m, j = t % m;
                double *dst = cl.map_shared_rank(v, r);
                dst[j] = row[b0 + j];
            }
        }
        cl.sync();
        // |x|^2 below the pivot by warp 0 in a fixed order (the same bits in every CTA)
        if (warp == 0) {
            double t = 0.0;
            for (int i = 1 + lane; i < m; i += 32) t = fma(v[i], v[i], t);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) red[32] = t;
        }
        __syncthreads();
        const double tail = red[32];
        const double x0 = v[0];
        if (tail == 0.0) {   // already reduced in this column (the same decision in every CTA)
            if (rank == 0 && tid == 0) work[chi + kc] = x0 * x0;
            continue;
        }
        const double nrm = sqrt(tail + x0 * x0);
        const double alpha = (x0 >= 0.0) ? -nrm : nrm;
        const double beta = 1.0 / (nrm * (nrm + fabs(x0)));
        const double v0 = x0 - alpha;
        if (rank == 0 && tid == 0) work[chi + kc] = alpha * alpha;
        int lf = b0 - rank;                    // first local row with i >= b0
        lf = lf > 0 ? (lf + CS - 1) / CS : 0;
        for (int l = lf + warp; l < nloc; l += nwarps) {
            const int i = rank + CS * l;
            const double *row = A + (size_t)l * chi + b0;
            double s0 = 0.0, s1 = 0.0;
            for (int j = lane; j < m; j += 64) {
                s0 = fma(row[j], j == 0 ? v0 : v[j], s0);
                if (j + 32 < m) s1 = fma(row[j + 32], v[j + 32], s1);
            }
            double sum = s0 + s1;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (lane < CS) {
                double *dst = cl.map_shared_rank(p, lane);
                dst[i - b0] = beta * sum;
            }
        }
        cl.sync();
        if (warp == 0) {
            double t = 0.0;
            for (int j = lane; j < m; j += 32) t = fma(p[j], j == 0 ? v0 : v[j], t);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) red[32] = t;
        }
        __syncthreads();
        const double Kf = 0.5 * beta * red[32];
        for (int j = tid; j < m; j += blockDim.x) w[j] = p[j] - Kf * (j == 0 ? v0 : v[j]);
        __syncthreads();
        for (int l = lf + warp; l < nloc; l += nwarps) {
            const int ii = rank + CS * l - b0;
            const double vi = ii == 0 ? v0 : v[ii], wi = w[ii];
            double *row = A + (size_t)l * chi + b0;
            for (int j = lane; j < m; j += 32) row[j] -= vi * w[j] + wi * (j == 0 ? v0 : v[j]);
        }
        __syncthreads();   // this CTA's rows are final for the column before its next broadcast
    }
    // the last 2 x 2 block (chi >= TRI_CLUSTER_MIN here): d_{chi-2}, d_{chi-1}, e_{chi-2}
    for (int i = chi - 2; i < chi; ++i)
        if (i % CS == rank && tid == 0) {
            const double *row = A + (size_t)(i / CS) * chi;
            work[i] = row[i];
            if (i == chi - 1) {
                work[2 * chi - 2] = row[chi - 2] * row[chi - 2];
                work[2 * chi - 1] = 0.0;
            }
        }
    cl.sync();   // no CTA leaves while another may still write into its shared memory
}

// Number of eigenvalues of the tridiagonal (d, e2) below x: the sign changes of
// p_i = (d_i - x) p_{i-1} - e2_{i-1} p_{i-2}.  Only the recurrence itself is FP64
// arithmetic (three operations per step -- GB300's FP64 pipe is narrow); the zero
// test, the sign comparison and the range check read the bit pattern with integer
// instructions, and the rare rescaling is by exact powers of two.
__device__ __forceinline__ int sturm_count(int chi, const double *d, const double *e2, double x, double tiny)
{
    double pm = 1.0, p = d[0] - x;
    if (p == 0.0) p = -tiny;
    int cnt = (p < 0.0);
    int hp = __double2hiint(p);
    for (int i = 1; i < chi; ++i) {
        double pn = fma(d[i] - x, p, -e2[i - 1] * pm);
        int hn = __double2hiint(pn);
        if (((hn & 0x7FFFFFFF) | __double2loint(pn)) == 0) {   // +-0
            pn = (hp < 0) ? tiny : -tiny;
            hn = __double2hiint(pn);
        }
        cnt += ((hn ^ hp) < 0);   // sign bits differ
        pm = p;
        p = pn;
        const int ex = (hn >> 20) & 0x7FF;
        if (ex > 1023 + 500) {
            p *= 0x1p-500;
            pm *= 0x1p-500;
            hn = __double2hiint(p);
        } else if (ex < 1023 - 500) {
            p *= 0x1p+500;
            pm *= 0x1p+500;
            hn = __double2hiint(p);
        }
        hp = hn;
    }
    return cnt;
}

__global__ void bisect_kernel(int chi, const double *work, double *lam)
{
    extern __shared__ double sm[];
    double *d = sm, *e2 = sm + chi;   // 2 chi
    for (int i = threadIdx.x; i < chi; i += blockDim.x) {
        d[i] = work[i];
        e2[i] = work[chi + i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int ei = blockIdx.x * SPEC_WARPS + (threadIdx.x >> 5);
    if (ei >= chi) return;
    // every eigenvalue lies in [-|T|_F, |T|_F] (the Frobenius norm bounds the
    // spectral radius; it is the corner's, unchanged by the orthogonal reduction):
    // one square root instead of per-row Gershgorin radii
    double f2 = 0.0;
    for (int i = 0; i < chi; ++i) f2 = fma(d[i], d[i], f2) + 2.0 * e2[i];
    const double scale = fmax(sqrt(f2), 1e-300);
    double lo = -scale * (1.0 + 1e-12), hi = scale * (1.0 + 1e-12);
    const double tiny = 1e-290 * scale;
    for (int round = 0; round < 16; ++round) {
        if (hi - lo <= 4e-16 * scale) break;
        double x = lo + (hi - lo) * (double)(lane + 1) / 33.0;
        int cnt = sturm_count(chi, d, e2, x, tiny);
        unsigned below = __ballot_sync(0xffffffffu, cnt <= ei);   // a prefix of lanes
        int L = __popc(below);
        double xl = __shfl_sync(0xffffffffu, x, (L > 0) ? L - 1 : 0);
        double xh = __shfl_sync(0xffffffffu, x, (L < 32) ? L : 31);
        double nlo = (L > 0) ? xl : lo;
        double nhi = (L < 32) ? xh : hi;
        lo = nlo;
        hi = nhi;
    }
    if (lane == 0) lam[ei] = 0.5 * (lo + hi);
}

// stride 2: the chi x stride eigenvalues come in equal pairs (a Hermitian corner through
// its real embedding); every second one of the sorted magnitudes is kept.
__global__ void spectrum_finish_kernel(int chi, int stride, const double *lam_in, double *s_new, const double *s_old,
                                       double *delta)
{
    __shared__ double red[33];
    __shared__ double lam[SPEC_MAX_CHI], srt[SPEC_MAX_CHI];
    const int tid = threadIdx.x, nall = chi * stride;
    for (int i = tid; i < nall; i += blockDim.x) lam[i] = fabs(lam_in[i]);
    __syncthreads();
    for (int i = tid; i < nall; i += blockDim.x) {
        double ai = lam[i];
        int rank = 0;
        for (int j = 0; j < nall; ++j) {
            double aj = lam[j];
            rank += (aj > ai) || (aj == ai && j < i);
        }
        srt[rank] = ai;
    }
    __syncthreads();
    double ss = 0.0;
    for (int i = tid; i < chi; i += blockDim.x) ss += srt[i * stride] * srt[i * stride];
    ss = block_sum(ss, red);
    const double f = ss > 0.0 ? 1.0 / sqrt(ss) : 0.0;
    for (int i = tid; i < chi; i += blockDim.x) lam[i] = srt[i * stride] * f;
    __syncthreads();
    for (int i = tid; i < chi; i += blockDim.x) srt[i] = lam[i];
    __syncthreads();
    double dd = 0.0;
    for (int i = tid; i < chi; i += blockDim.x) {
        double x = srt[i] - s_old[i];
        dd += x * x;
    }
    dd = block_sum(dd, red);
    for (int i = tid; i < chi; i += blockDim.x) s_new[i] = srt[i];
    if (tid == 0) *delta = sqrt(dd);
}

__global__ void spectrum_init_kernel(int chi, double *s)
{
    for (int i = threadIdx.x; i < chi; i += blockDim.x) s[i] = 1.0 / sqrt((double)chi);
}

// Eq. (1): rho[(sA sB)][(tA tB)] = raw[(sB tB)][(sA tA)] / trace; e_a = tr(rho h_a);
// E_site = (1/2) sum_a e_a.  out: e_x, e_y, e_z, E_site, then rho (d^4).
__global__ void bond_energy_kernel(int d, const double *raw, const double *h, double *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int dd = d * d;
    double z = 0.0;
    for (int sA = 0; sA < d; ++sA)
        for (int sB = 0; sB < d; ++sB) z += raw[(sB * d + sB) * dd + (sA * d + sA)];
    double *rho = out + 4;
    for (int sA = 0; sA < d; ++sA)
        for (int sB = 0; sB < d; ++sB)
            for (int tA = 0; tA < d; ++tA)
                for (int tB = 0; tB < d; ++tB)
                    rho[(sA * d + sB) * dd + tA * d + tB] = raw[(sB * d + tB) * dd + (sA * d + tA)] / z;
    double es = 0.0;
    for (int a = 0; a < 3; ++a) {
        double e = 0.0;
        for (int r = 0; r < dd; ++r)
            for (int c = 0; c < dd; ++c) e += rho[r * dd + c] * h[(size_t)a * dd * dd + c * dd + r];
        out[a] = e;
        es += e;
    }
    out[3] = 0.5 * es;
}

__global__ void check_finite_kernel(long long count, const double *x, int *flag)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
         t += (long long)gridDim.x * blockDim.x)
        if (!isfinite(x[t])) *flag = 1;
}

int grid_for(long long count, int per_sm = 8)
{
    long long b = (count + 255) / 256;
    long long cap = (long long)per_sm * device_sm_count();
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

}  // namespace

cudaError_t launch_c3v_project_normalize(int d, int D, const double *Ain, double *Aout, int symmetrize,
                                         cudaStream_t st)
{
    size_t smem = sizeof(double) * (size_t)d * D * D * D;
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(c3v_project_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    CTM_COUNT_LAUNCH(1);
    c3v_project_kernel<<<1, 256, smem, st>>>(d, D, Ain, Aout, symmetrize);
    return cudaGetLastError();
}

cudaError_t launch_double_layer(int d, int D, const double *K, const double *B, double *a, cudaStream_t st)
{
    long long tot = (long long)D * D * D * D * D * D;
    CTM_COUNT_LAUNCH(1);
    double_layer_kernel<<<grid_for(tot), 256, 0, st>>>(d, D, K, B, a);
    return cudaGetLastError();
}

cudaError_t launch_open_layers(int d, int D, const double *A, double *b, cudaStream_t st)
{
    long long tot = (long long)D * D * D * D * D * D * d * d;
    CTM_COUNT_LAUNCH(1);
    open_layers_kernel<<<grid_for(tot), 256, 0, st>>>(d, D, A, b);
    return cudaGetLastError();
}

cudaError_t launch_init_env(int chi, int D, const double *a, double *C, double *T, double *Q, cudaStream_t st)
{
    long long tot = (long long)chi * D * D * chi;
    CTM_COUNT_LAUNCH(1);
    init_env_kernel<<<grid_for(tot), 256, 0, st>>>(chi, D, a, C, T, Q);
    return cudaGetLastError();
}

cudaError_t launch_warm_start(int n, int chi, const double *Q, const double *C, double *Qs, cudaStream_t st)
{
    CTM_COUNT_LAUNCH(1);
    warm_start_kernel<<<grid_for((long long)n * chi), 256, 0, st>>>(n, chi, Q, C, Qs);
    return cudaGetLastError();
}

cudaError_t launch_corner_sym_normalize(int chi, const double *Cr, double *Cn, double *partials, cudaStream_t st)
{
    int nb = (chi * chi + 255) / 256;
    if (nb > CORNER_NORM_BLOCKS) nb = CORNER_NORM_BLOCKS;
    CTM_COUNT_LAUNCH(2);
    corner_sym_sumsq_kernel<<<nb, 256, 0, st>>>(chi, Cr, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    corner_sym_scale_kernel<<<nb, 256, 0, st>>>(chi, Cr, partials, nb, Cn);
    return cudaGetLastError();
}

cudaError_t launch_normalize(long long count, double *x, double *partials, int nblocks, cudaStream_t st)
{
    CTM_COUNT_LAUNCH(1);
    sumsq_partial_kernel<<<nblocks, 256, 0, st>>>(count, x, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    CTM_COUNT_LAUNCH(1);
    scale_by_partials_kernel<<<nblocks, 256, 0, st>>>(count, x, partials, nblocks);
    return cudaGetLastError();
}

// Cluster size for the distributed reduction of a chi x chi corner (chi >= TRI_CLUSTER_MIN):
// 16 CTAs where the device schedules such clusters with this shared memory, else 8,
// else 0 (the single-CTA reduction from global memory).  Decided once per chi.
static std::mutex g_tri_mu;
static signed char g_tri_cs[SPEC_MAX_CHI + 1];   // 0: not decided, -1: none, else the size
static std::atomic<bool> g_tri_cluster_ok{false}; // the cluster kernels' attributes were accepted

template <int CS>
static int tri_cluster_fits(int chi)
{
    const size_t smem = tri_cluster_smem_bytes(chi, CS);
    if (smem > TRI_CL_SMEM_MAX) return 0;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(CS, 1, 1);
    cfg.blockDim = dim3(tri_cluster_threads(chi, CS), 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, tridiag_cluster_kernel<CS>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nc > 0;
}

static int tri_cluster_size(int chi)
{
    if (chi < TRI_CLUSTER_MIN || chi > SPEC_MAX_CHI || !g_tri_cluster_ok) return 0;
    std::lock_guard<std::mutex> lk(g_tri_mu);
    if (!g_tri_cs[chi]) g_tri_cs[chi] = tri_cluster_fits<16>(chi) ? 16 : tri_cluster_fits<8>(chi) ? 8 : -1;
    return g_tri_cs[chi] > 0 ? g_tri_cs[chi] : 0;
}

static cudaError_t launch_tridiag_cluster(int cs, int chi, const double *C, double *work, cudaStream_t st)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(cs, 1, 1);
    cfg.blockDim = dim3(tri_cluster_threads(chi, cs), 1, 1);
    cfg.dynamicSmemBytes = tri_cluster_smem_bytes(chi, cs);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cs == 16 ? cudaLaunchKernelEx(&cfg, tridiag_cluster_kernel<16>, chi, C, work)
                    : cudaLaunchKernelEx(&cfg, tridiag_cluster_kernel<8>, chi, C, work);
}

size_t spectrum_work_doubles(int chi)
{
    return tri_global_off(chi) + (chi > TRI_SMEM_MAX ? (size_t)chi * (chi + 1) / 2 : 0);
}

// bisection of the tridiagonal in work (n = chi x stride eigenvalues), then the sorted,
// normalised magnitudes (every stride-th) and delta
static cudaError_t spectrum_tail(int chi, int stride, double *work, double *s_new, const double *s_old, double *delta,
                                 cudaStream_t st)
{
    const int n = chi * stride;
    CTM_COUNT_LAUNCH(2);
    bisect_kernel<<<(n + SPEC_WARPS - 1) / SPEC_WARPS, 32 * SPEC_WARPS, 2 * sizeof(double) * n, st>>>(n, work,
                                                                                                      work + 2 * n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    spectrum_finish_kernel<<<1, 256, 0, st>>>(chi, stride, work + 2 * n, s_new, s_old, delta);
    return cudaGetLastError();
}

static cudaError_t launch_tridiag(int chi, const double *C, double *work, cudaStream_t st, bool reserve_sm);

cudaError_t launch_spectrum_pairs(int chi, const double *E, double *s_new, const double *s_old, double *delta,
                                  double *work, cudaStream_t st)
{
    if (2 * chi > SPEC_MAX_CHI || !work) return cudaErrorInvalidValue;
    cudaError_t e = launch_tridiag(2 * chi, E, work, st, false);
    if (e != cudaSuccess) return e;
    return spectrum_tail(chi, 2, work, s_new, s_old, delta, st);
}

cudaError_t launch_spectrum(int chi, const double *C, double *s_new, const double *s_old, double *delta,
                            double *work, cudaStream_t st, bool reserve_sm)
{
    if (chi > SPEC_MAX_CHI || !work) return cudaErrorInvalidValue;
    cudaError_t e = launch_tridiag(chi, C, work, st, reserve_sm);
    if (e != cudaSuccess) return e;
    return spectrum_tail(chi, 1, work, s_new, s_old, delta, st);
}

// step one of the spectrum: the tridiagonal (d, e^2) of the symmetric chi x chi matrix C in work
static cudaError_t launch_tridiag(int chi, const double *C, double *work, cudaStream_t st, bool reserve_sm)
{
    // reserve_sm: the tridiagonalisation runs beside a lone instance's step for ~0.4 ms on
    // one SM; asking for (nearly) all of the SM's shared memory keeps the step's CTAs off
    // that SM, whose CTAs it would otherwise slow (a grid-synchronous QR waits for its
    // slowest CTA): measured 0.892 -> 0.872 ms per step at D = 6, chi = 72.  (Not inside a
    // batch, where many spectra run at once.)
    const bool full = chi <= TRI_FULL_MAX, global = chi > TRI_SMEM_MAX;
    size_t smem = sizeof(double) * ((full ? (size_t)chi * (chi | 1) : global ? 0 : (size_t)chi * (chi + 1) / 2) +
                                    2 * (size_t)chi);
    if (reserve_sm && smem < SPEC_SM_ALONE_BYTES) smem = SPEC_SM_ALONE_BYTES;
    CTM_COUNT_LAUNCH(1);
    cudaError_t e = cudaSuccess;
    const int cs = tri_cluster_size(chi);
    if (cs) e = launch_tridiag_cluster(cs, chi, C, work, st);
    else if (full) tridiag_kernel<<<1, TRI_THREADS, smem, st>>>(chi, C, work);
    else if (!global) tridiag_packed_kernel<false><<<1, TRI_THREADS, smem, st>>>(chi, C, work);
    else tridiag_packed_kernel<true><<<1, TRI_THREADS, smem, st>>>(chi, C, work);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_spectrum_from_tridiag(int chi, double *work, double *s_new, const double *s_old, double *delta,
                                        cudaStream_t st)
{
    if (chi > SPEC_MAX_CHI || !work) return cudaErrorInvalidValue;
    return spectrum_tail(chi, 1, work, s_new, s_old, delta, st);
}

cudaError_t launch_spectrum_init(int chi, double *s, cudaStream_t st)
{
    CTM_COUNT_LAUNCH(1);
    spectrum_init_kernel<<<1, 256, 0, st>>>(chi, s);
    return cudaGetLastError();
}

cudaError_t launch_bond_energy(int d, const double *rho_raw, const double *h, double *out, cudaStream_t st)
{
    CTM_COUNT_LAUNCH(1);
    bond_energy_kernel<<<1, 32, 0, st>>>(d, rho_raw, h, out);
    return cudaGetLastError();
}

cudaError_t launch_check_finite(long long count, const double *x, int *flag, cudaStream_t st)
{
    CTM_COUNT_LAUNCH(1);
    check_finite_kernel<<<grid_for(count), 256, 0, st>>>(count, x, flag);
    return cudaGetLastError();
}

cudaError_t spectrum_prepare()
{
    cudaError_t e = cudaFuncSetAttribute(tridiag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 224 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(tridiag_packed_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 224 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(tridiag_packed_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 224 * 1024);
    if (e != cudaSuccess) return e;
    // the cluster reduction is optional: where the device refuses these attributes the
    // single-CTA reduction from global memory serves
    const bool ok = cudaFuncSetAttribute(tridiag_cluster_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TRI_CL_SMEM_MAX) == cudaSuccess &&
                    cudaFuncSetAttribute(tridiag_cluster_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TRI_CL_SMEM_MAX) == cudaSuccess &&
                    cudaFuncSetAttribute(tridiag_cluster_kernel<16>, cudaFuncAttributeNonPortableClusterSizeAllowed,
                                         1) == cudaSuccess;
    if (!ok) cudaGetLastError();
    g_tri_cluster_ok = ok;
    return cudaSuccess;
}
