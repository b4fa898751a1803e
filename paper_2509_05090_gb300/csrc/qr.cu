// Householder QR of the reduced corner Y (n x k, tall and skinny), Sec. II.B,
// Fig. 3(d): Y = Q R with Q serving as the isometric projector and the gauge
// fixed so that diag(R) >= 0.  Always FP64.
//
// One cooperative launch over G <= #SM CTAs.  CTA c keeps its block of rows of
// Y (and later of Q) in shared memory for the whole factorisation.  Per column
// j every CTA forms the partial dot products x^T a_kk over its rows (x = the
// column below the diagonal) and adds them into one k-vector with FP64
// atomics; after one grid barrier every CTA reads the k sums and row j, derives
// the reflector (alpha = -sign(x_0)|x|, v = x - alpha e_0, tau = 2/v^T v)
// redundantly, and applies it to its own rows:  v^T a_kk = x^T a_kk - alpha a_jk.
// So a column costs one grid barrier.  The reflectors v_j (unnormalised,
// tau_j = 2 / v_j^T v_j) are written out and Q = H_0 ... H_{k-1} [I; 0] is formed
// in compact-WY form without further barriers: with S = V^T V, the triangular
// factor satisfies T^{-1} = striu(S) + diag(S)/2 (the "UT" form of the
// product of reflectors), so Q = E - V W with W = T V_top^T (one small
// triangular solve) -- two GEMMs and two small kernels.  Columns with
// R_jj < 0 are negated (gauge diag(R) >= 0).  The grid size of the
// factorisation is tuned once per shape by timing a few rows-per-CTA choices.
//
// The grid barrier is a counter/generation pair in global memory; its spin is
// bounded (about a second) and on expiry sets an error flag that the host
// reports as CTM_ETIMEOUT instead of hanging.
#include <cooperative_groups.h>

#include "ctm_internal.h"

namespace {

constexpr int QR_THREADS = 256;
constexpr long long QR_SPIN_LIMIT = 20000000LL;   // x ~64 ns sleep: ~1.3 s

// Grid barrier number `epoch` (1, 2, ...): one release-add per CTA on a
// monotonic counter; the CTA that completes G*epoch arrivals publishes the epoch
// with a release store, the others poll it with acquire loads.  No reset, no
// extra fences; the poll is bounded.
__device__ __forceinline__ bool grid_barrier(unsigned *count, unsigned *flag, unsigned G, unsigned epoch, int *err)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned old;
        asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(count) : "memory");
        if (old == G * epoch - 1) {
            asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(flag), "r"(epoch) : "memory");
        } else {
            long long it = 0;
            unsigned f;
            for (;;) {
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(f) : "l"(flag) : "memory");
                if ((int)(f - epoch) >= 0) break;
                if (++it > QR_SPIN_LIMIT) {
                    atomicExch(err, 1);
                    break;
                }
                if (it > 64) __nanosleep(32);
            }
        }
    }
    __syncthreads();
    return *((volatile int *)err) == 0;
}

struct QrArgs {
    int n, k, G, rows_per;
    const double *Y;
    double *Q, *R;
    double *V;        // n x k reflectors (written)
    double *ta;       // 2 x k: tau, alpha (written by CTA 0)
    double *sbuf;     // 3 x k, rotating accumulators
    double *rowbuf;   // 2 x k
    unsigned *bar;
    int *err;
};

__global__ void __launch_bounds__(QR_THREADS) qr_kernel(QrArgs a)
{
    extern __shared__ double sm[];
    const int k = a.k;
    const int c = blockIdx.x;
    const int r0 = c * a.rows_per;
    const int r1 = min(a.n, r0 + a.rows_per);
    const int nr = max(0, r1 - r0);
    double *Ys = sm;                          // rows_per x k
    double *sv = Ys + (size_t)a.rows_per * k; // k
    double *rj = sv + k;                      // k
    double *cf = rj + k;                      // k
    double *taus = cf + k;                    // k
    double *v0s = taus + k;                   // k
    double *alps = v0s + k;                   // k
    const int tid = threadIdx.x;

    for (int t = tid; t < nr * k; t += blockDim.x) Ys[t] = a.Y[(size_t)r0 * k + t];
    __syncthreads();

    int step = 0;   // rotating-buffer counter
    // ---------------------------------------------------------- factorisation
    for (int j = 0; j < k; ++j, ++step) {
        double *acc = a.sbuf + (step % 3) * k;
        const int rs = max(r0, j) - r0;   // first local row taking part
        // x^T a_kk over this CTA's rows: P lanes per column split the rows, two
        // accumulators each, so the dependent FP64 chain is short; then shuffles
        const int ncols = k - j;
        int P = 1;
        while (P < 32 && P * 2 * ncols <= (int)blockDim.x) P *= 2;
        for (int base = 0; base < ncols * P; base += blockDim.x) {
            const int t = base + tid;
            const int kk = j + t / P, part = t % P;
            double s0 = 0.0, s1 = 0.0;
            if (t < ncols * P) {
                int r = rs + part;
                for (; r + P < nr; r += 2 * P) {
                    s0 = fma(Ys[r * k + j], Ys[r * k + kk], s0);
                    s1 = fma(Ys[(r + P) * k + j], Ys[(r + P) * k + kk], s1);
                }
                if (r < nr) s0 = fma(Ys[r * k + j], Ys[r * k + kk], s0);
            }
            double s = s0 + s1;
            for (int o = P >> 1; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, P);
            if (t < ncols * P && part == 0 && rs < nr) atomicAdd(&acc[kk], s);
        }
        if (j >= r0 && j < r1)
            for (int kk = j + tid; kk < k; kk += blockDim.x) a.rowbuf[(j & 1) * k + kk] = Ys[(j - r0) * k + kk];
        if (!grid_barrier(a.bar, a.bar + 1, a.G, (unsigned)(step + 1), a.err)) return;
        // thread 0 derives the reflector (alpha = -sign(x_0)|x|, v_0 = x_0 - alpha,
        // tau = 2 / v^T v = 1 / (|x| (|x| + |x_0|))) while the others fetch the sums
        if (tid == 0) {
            const double nrm2 = ((volatile double *)acc)[j], x0 = ((volatile double *)a.rowbuf)[(j & 1) * k + j];
            const double nrm = sqrt(nrm2);
            double tau = 0.0, alpha = x0, v0 = 0.0;
            if (nrm > 0.0) {
                alpha = (x0 >= 0.0) ? -nrm : nrm;
                v0 = x0 - alpha;
                tau = 1.0 / (nrm * (nrm + fabs(x0)));
            }
            taus[j] = tau;
            v0s[j] = v0;
            alps[j] = (nrm > 0.0) ? alpha : 0.0;
        }
        for (int kk = j + 1 + tid; kk < k; kk += blockDim.x) {
            sv[kk] = ((volatile double *)acc)[kk];
            rj[kk] = ((volatile double *)a.rowbuf)[(j & 1) * k + kk];
        }
        if (c == 0) {
            double *z = a.sbuf + ((step + 2) % 3) * k;
            for (int kk = tid; kk < k; kk += blockDim.x) z[kk] = 0.0;
        }
        __syncthreads();
        const double tau = taus[j], v0 = v0s[j], alpha = alps[j];
        for (int kk = j + 1 + tid; kk < k; kk += blockDim.x) cf[kk] = tau * (sv[kk] - alpha * rj[kk]);
        if (c == 0) {
            for (int kk = tid; kk < k; kk += blockDim.x) {
                double v = 0.0;
                if (kk == j) v = alpha;
                else if (kk > j) v = rj[kk] - v0 * (tau * (sv[kk] - alpha * rj[kk]));
                a.R[(size_t)j * k + kk] = v;
            }
        }
        __syncthreads();
        if (tau != 0.0) {
            const int ncol = k - j - 1;
            const int rows = nr - rs;
            for (int t = tid; t < rows * ncol; t += blockDim.x) {
                int r = rs + t / ncol;
                int kk = j + 1 + t % ncol;
                double vr = (r0 + r == j) ? v0 : Ys[r * k + j];
                Ys[r * k + kk] -= vr * cf[kk];
            }
        }
        __syncthreads();
    }

    // ---------------------------------------------------------- reflectors out
    for (int t = tid; t < nr * k; t += blockDim.x) {
        const int r = r0 + t / k, j = t % k;
        double v = 0.0;
        if (r == j) v = v0s[j];
        else if (r > j) v = Ys[t];
        if (taus[j] == 0.0) v = 0.0;
        a.V[(size_t)r0 * k + t] = v;
    }
    if (c == 0) {
        for (int j = tid; j < k; j += blockDim.x) {
            a.ta[j] = taus[j];
            a.ta[k + j] = alps[j];
        }
        __syncthreads();
        for (int t = tid; t < k * k; t += blockDim.x) {
            int rr = t / k;
            if (alps[rr] < 0.0) a.R[t] = -a.R[t];
        }
    }
    (void)step;
}

// W = U^{-1} V_top^T with U = striu(S) + diag(S)/2 (unit diagonal where tau = 0).
// One CTA, blocked from the bottom in row blocks of QR_WB: for a block, every
// (row, column) pair first sums the already solved rows below the block -- all
// independent, one pass -- and then the QR_WB x QR_WB diagonal block is solved
// row by row (short chains).  U (full, shared), the reciprocal diagonal and W
// live in shared memory; the only divisions are the k reciprocals.
constexpr int QR_WB = 8;

__device__ __forceinline__ int up_off(int k, int i, int j) { return i * k - (i * (i - 1)) / 2 + (j - i); }

__global__ void qr_wy_solve_kernel(int k, const double *S, const double *V, const double *ta, double *W)
{
    extern __shared__ double sm[];
    double *Ws = sm;                              // k x k
    double *Us = Ws + (size_t)k * k;              // upper triangle of S, packed by rows (k (k+1) / 2)
    double *rd = Us + (size_t)k * (k + 1) / 2;    // k
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
        const int i = t / k, j = t % k;
        if (j >= i) Us[up_off(k, i, j)] = S[t];
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) rd[i] = (ta[i] == 0.0) ? 1.0 : 2.0 / S[(size_t)i * k + i];
    __syncthreads();
    for (int i1 = k; i1 > 0; i1 -= QR_WB) {
        const int i0 = i1 - QR_WB > 0 ? i1 - QR_WB : 0;
        const int rows = i1 - i0;
        // rhs for the block: V_top^T[i][col] - sum_{j >= i1} U[i][j] W[j][col]
        for (int t = threadIdx.x; t < rows * k; t += blockDim.x) {
            const int i = i0 + t / k, col = t % k;
            const double *u = Us + up_off(k, i, i) - i;   // u[j] = U[i][j] for j >= i
            double s0 = 0.0, s1 = 0.0;
            int j = i1;
            for (; j + 1 < k; j += 2) {
                s0 = fma(u[j], Ws[j * k + col], s0);
                s1 = fma(u[j + 1], Ws[(j + 1) * k + col], s1);
            }
            if (j < k) s0 = fma(u[j], Ws[j * k + col], s0);
            Ws[i * k + col] = V[(size_t)col * k + i] - (s0 + s1);
        }
        __syncthreads();
        // the diagonal block, bottom row first
        for (int i = i1 - 1; i >= i0; --i) {
            const double *u = Us + up_off(k, i, i) - i;
            for (int col = threadIdx.x; col < k; col += blockDim.x) {
                double s = Ws[i * k + col];
                for (int j = i + 1; j < i1; ++j) s = fma(-u[j], Ws[j * k + col], s);
                Ws[i * k + col] = s * rd[i];
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) W[t] = Ws[t];
}

// Q <- diag-sign gauge of (E - V W): Q holds -V W on entry.
__global__ void qr_form_q_kernel(long long n, int k, const double *ta, double *Q)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n * k;
         t += (long long)gridDim.x * blockDim.x) {
        const long long r = t / k;
        const int c = (int)(t % k);
        double q = Q[t] + (r == c ? 1.0 : 0.0);
        Q[t] = (ta[k + c] < 0.0) ? -q : q;
    }
}

size_t qr_smem_bytes(int rows_per, int k) { return sizeof(double) * ((size_t)rows_per * k + 6 * (size_t)k); }

int qr_layout(int n, int k, int rows_min, int *G_out, int *rows_out)
{
    int sms = device_sm_count();
    int rows_per = (n + sms - 1) / sms;
    if (rows_per < rows_min) rows_per = rows_min;
    if (rows_per < 1) rows_per = 1;
    int G = (n + rows_per - 1) / rows_per;
    *G_out = G;
    *rows_out = rows_per;
    return qr_smem_bytes(rows_per, k) <= 200 * 1024;
}

}  // namespace

size_t qr_scratch_doubles(int k) { return (size_t)5 * k + 8; }

int qr_supported(int n, int k)
{
    int G, rp;
    return n >= k && k >= 1 && k <= 128 && qr_layout(n, k, 1, &G, &rp);
}

size_t qr_sk_doubles(int n, int k)
{
    const size_t a = 64 * (size_t)k * k, b = 4 * (size_t)n * k;   // split-K partials of V^T V and of V W
    return a > b ? a : b;
}

size_t qr_wy_doubles(int n, int k) { return (size_t)n * k + 3 * (size_t)k * k + 2 * (size_t)k + qr_sk_doubles(n, k); }

static cudaError_t qr_factor_launch(int n, int k, int rows_per, const double *Y, double *R, QrScratch s, cudaStream_t st)
{
    const int G = (n + rows_per - 1) / rows_per;
    const size_t smem = qr_smem_bytes(rows_per, k);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qr_kernel, QR_THREADS, smem);
    if (per_sm * device_sm_count() < G) return cudaErrorCooperativeLaunchTooLarge;
    cudaError_t e = cudaMemsetAsync(s.sbuf, 0, sizeof(double) * 3 * k, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(s.bar, 0, sizeof(unsigned) * 2, st);
    if (e != cudaSuccess) return e;
    QrArgs a{n, k, G, rows_per, Y, nullptr, R, s.V, s.ta, s.sbuf, s.rowbuf, s.bar, s.err};
    void *args[] = {&a};
    CTM_COUNT_LAUNCH(1);
    return cudaLaunchCooperativeKernel((void *)qr_kernel, dim3(G), dim3(QR_THREADS), args, smem, st);
}

#include <map>
#include <mutex>
#include <utility>
static std::mutex g_qr_mu;
static std::map<std::pair<int, int>, int> g_qr_rows;   // (n, k) -> rows per CTA, for rows_min == 1

// rows per CTA: tuned once per (n, k) by timing the factorisation (eager calls only)
static int qr_pick_rows(int n, int k, const double *Y, double *R, QrScratch s, cudaStream_t st)
{
    int G, rp0;
    qr_layout(n, k, s.rows_min > 0 ? s.rows_min : 1, &G, &rp0);
    if (s.rows_min > 1) return rp0;
    {
        std::lock_guard<std::mutex> lk(g_qr_mu);
        auto it = g_qr_rows.find({n, k});
        if (it != g_qr_rows.end()) return it->second;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs != cudaStreamCaptureStatusNone) return rp0;
    int best = rp0;
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return rp0;
    // fewer rows than rp0 puts several CTAs on an SM (the launch checks they all fit)
    for (int rp : {rp0, 8, 12, 16, 24, 32, 48, 64, 96, 128}) {
        if ((rp < rp0 && rp * 2 < rp0) || (rp != rp0 && rp < 8) || qr_smem_bytes(rp, k) > 200 * 1024) continue;
        float ms = 0.f;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, st);
            cudaError_t e = qr_factor_launch(n, k, rp, Y, R, s, st);
            cudaEventRecord(e1, st);
            if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                ms = 1e30f;
                cudaGetLastError();
                break;
            }
            cudaEventElapsedTime(&ms, e0, e1);
        }
        int herr = 0;
        cudaMemcpy(&herr, s.err, sizeof(int), cudaMemcpyDeviceToHost);
        if (herr) break;   // a bounded wait expired: keep the default, the caller will report it
        if (ms < best_ms) {
            best_ms = ms;
            best = rp;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lk(g_qr_mu);
    g_qr_rows[{n, k}] = best;
    return best;
}

cudaError_t qr_householder(int n, int k, const double *Y, double *Q, double *R, QrScratch s, cudaStream_t st)
{
    int G, rp;
    if (!qr_supported(n, k) || !s.V) return cudaErrorInvalidValue;
    if (!qr_layout(n, k, s.rows_min > 0 ? s.rows_min : 1, &G, &rp) && !qr_layout(n, k, 1, &G, &rp))
        return cudaErrorInvalidValue;
    const int rows_per = qr_pick_rows(n, k, Y, R, s, st);
    cudaError_t e = qr_factor_launch(n, k, rows_per, Y, R, s, st);
    if (e != cudaSuccess) return e;
    // S = V^T V
    GemmF64 gs{k, k, n, s.V, idx_lin(1), idx_lin(k), s.V, idx_lin(k), idx_lin(1), s.S, idx_lin(k), idx_lin(1), 1.0,
               0.0};
    if ((e = gemm_f64(gs, gemm_f64_pick_split(k, k, n), s.sk, s.sk_elems, st)) != cudaSuccess) return e;
    CTM_COUNT_LAUNCH(2);
    qr_wy_solve_kernel<<<1, 512, sizeof(double) * ((size_t)k * k + (size_t)k * (k + 1) / 2 + k), st>>>(
        k, s.S, s.V, s.ta, s.W);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // Q = -V W, then + E and the sign gauge
    GemmF64 gq{n, k, k, s.V, idx_lin(k), idx_lin(1), s.W, idx_lin(k), idx_lin(1), Q, idx_lin(k), idx_lin(1), -1.0,
               0.0};
    if ((e = gemm_f64(gq, gemm_f64_pick_split(n, k, k), s.sk, s.sk_elems, st)) != cudaSuccess) return e;
    long long tot = (long long)n * k;
    int blocks = (int)((tot + 255) / 256);
    if (blocks > 8 * device_sm_count()) blocks = 8 * device_sm_count();
    qr_form_q_kernel<<<blocks, 256, 0, st>>>(n, k, s.ta, Q);
    return cudaGetLastError();
}

cudaError_t qr_prepare()
{
    cudaError_t e = cudaFuncSetAttribute(qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(qr_wy_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}
