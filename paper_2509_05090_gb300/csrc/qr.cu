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
// Applying reflector j to the trailing columns and forming the partial sums of
// column j+1 is one pass over the CTA's rows, so a column costs one grid barrier
// and one sweep of the shared-memory block.  The reflectors v_j (unnormalised,
// tau_j = 2 / v_j^T v_j) are written out and Q = H_0 ... H_{k-1} [I; 0] is formed
// in compact-WY form without further barriers: with S = V^T V, the triangular
// factor satisfies T^{-1} = striu(S) + diag(S)/2 (the "UT" form of the
// product of reflectors), so Q = E - V W with W = T V_top^T (one small
// triangular solve) -- two GEMMs and two small kernels.  Columns with
// R_jj < 0 are negated (gauge diag(R) >= 0).  The grid size of the
// factorisation is tuned once per shape by timing a few rows-per-CTA choices.
//
// The grid barrier is one monotonic counter in global memory; its spin is
// bounded (about a second) and on expiry sets an error flag that the host
// reports as CTM_ETIMEOUT instead of hanging.
#include <cooperative_groups.h>

#include "ctm_internal.h"

namespace {

constexpr int QR_THREADS = 512;
constexpr long long QR_SPIN_LIMIT = 20000000LL;   // x ~64 ns sleep: ~1.3 s

// Grid barrier number `epoch` (1, 2, ...): every CTA adds 1 to a monotonic
// counter with a release reduction (no value returned) and polls the counter
// with acquire loads until it reaches G * epoch.  No reset, no separate flag;
// the poll is bounded.
__device__ __forceinline__ bool grid_barrier(unsigned *count, unsigned G, unsigned epoch, int *err)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
        const unsigned target = G * epoch;
        long long it = 0;
        unsigned f;
        for (;;) {
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(f) : "l"(count) : "memory");
            if ((int)(f - target) >= 0) break;
            if (++it > QR_SPIN_LIMIT) {
                atomicExch(err, 1);
                break;
            }
            if (it > 64) __nanosleep(32);
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

    // Column sums x_j^T a_kk (rows >= j of the current trailing block) over this
    // CTA's rows, kk = j .. k-1, into acc: P lanes per column split the rows, two
    // accumulators each, so the dependent FP64 chains stay short; then shuffles.
    // With upd != 0 the trailing columns kk > j are first updated by the previous
    // reflector (a_kk -= v cf_kk, v = column j-1) in the same pass, and the
    // owner of row j publishes it for the next pivot.
    auto col_pass = [&](int j, double *acc, int upd) {
        const int rs = max(r0, j) - r0;
        const int ncols = k - j;
        int P = 1;
        while (P < 32 && P * 2 * ncols <= (int)blockDim.x) P *= 2;
        for (int base = 0; base < ncols * P; base += blockDim.x) {
            const int t = base + tid;
            const int kk = j + t / P, part = t % P;
            double s0 = 0.0, s1 = 0.0;
            if (t < ncols * P) {
                const double cfk = (upd && kk > j) ? cf[kk] : 0.0;
                int r = rs + part;
                for (; r + P < nr; r += 2 * P) {
                    const int r2 = r + P;
                    double x0 = Ys[r * k + kk], x1 = Ys[r2 * k + kk];
                    if (upd && kk > j) {
                        x0 = fma(-Ys[r * k + j - 1], cfk, x0);
                        x1 = fma(-Ys[r2 * k + j - 1], cfk, x1);
                        Ys[r * k + kk] = x0;
                        Ys[r2 * k + kk] = x1;
                    }
                    s0 = fma(Ys[r * k + j], x0, s0);
                    s1 = fma(Ys[r2 * k + j], x1, s1);
                    if (r0 + r == j) a.rowbuf[(j & 1) * k + kk] = x0;
                    if (r0 + r2 == j) a.rowbuf[(j & 1) * k + kk] = x1;
                }
                if (r < nr) {
                    double x0 = Ys[r * k + kk];
                    if (upd && kk > j) {
                        x0 = fma(-Ys[r * k + j - 1], cfk, x0);
                        Ys[r * k + kk] = x0;
                    }
                    s0 = fma(Ys[r * k + j], x0, s0);
                    if (r0 + r == j) a.rowbuf[(j & 1) * k + kk] = x0;
                }
            }
            double sum = s0 + s1;
            for (int o = P >> 1; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o, P);
            if (t < ncols * P && part == 0 && rs < nr) atomicAdd(&acc[kk], sum);
        }
    };

    int step = 0;   // rotating-buffer counter
    // ---------------------------------------------------------- factorisation
    col_pass(0, a.sbuf, 0);
    for (int j = 0; j < k; ++j, ++step) {
        double *acc = a.sbuf + (step % 3) * k;
        if (!grid_barrier(a.bar, a.G, (unsigned)(step + 1), a.err)) return;
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
        if (j + 1 < k) {
            // H_j on column j+1 (rows below the pivot: row j itself is R's and
            // never read again), then the fused update + column sums for j+1
            const int rs1 = max(r0, j + 1) - r0;
            const double cf1 = cf[j + 1];
            for (int r = rs1 + tid; r < nr; r += blockDim.x) {
                const double x = fma(-Ys[r * k + j], cf1, Ys[r * k + j + 1]);
                Ys[r * k + j + 1] = x;
                if (r0 + r == j + 1) a.rowbuf[((j + 1) & 1) * k + j + 1] = x;
            }
            __syncthreads();
            col_pass(j + 1, a.sbuf + ((step + 1) % 3) * k, 1);
        }
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
// The k right-hand sides are independent: CTA b solves columns [8b, 8b + 8).
// Rows are blocked by QR_WB = 8 from the bottom; every CTA first inverts the
// diagonal 8 x 8 blocks of U (all blocks at once, one thread per block column),
// then per row block sums the already solved rows below it (independent dot
// products split over QR_WL lanes) and applies the block inverse (8-term dots).
// So the dependent FP64 chains per block are short and the CTA syncs twice per
// block.  U (packed upper triangle), the block inverses and the CTA's W columns
// live in shared memory.
constexpr int QR_WB = 8;      // row block (and diagonal inverse) size
constexpr int QR_WC = 8;      // right-hand-side columns per CTA
constexpr int QR_WL = 4;      // lanes per dot product in the block update
constexpr int QR_WY_THREADS = 256;

__device__ __forceinline__ int up_off(int k, int i, int j) { return i * k - (i * (i - 1)) / 2 + (j - i); }

size_t qr_wy_smem_bytes(int k)
{
    const int nb = (k + QR_WB - 1) / QR_WB;
    return sizeof(double) * ((size_t)k * (k + 1) / 2 + (size_t)nb * QR_WB * QR_WB + (size_t)k * QR_WC + k);
}

__global__ void __launch_bounds__(QR_WY_THREADS) qr_wy_solve_kernel(int k, const double *S, const double *V,
                                                                    const double *ta, double *W)
{
    extern __shared__ double sm[];
    const int nb = (k + QR_WB - 1) / QR_WB;
    double *Us = sm;                                   // k (k+1) / 2
    double *Di = Us + (size_t)k * (k + 1) / 2;         // nb x 8 x 8 block inverses
    double *Wc = Di + (size_t)nb * QR_WB * QR_WB;      // k x QR_WC
    double *rd = Wc + (size_t)k * QR_WC;               // k reciprocal diagonal
    const int c0 = blockIdx.x * QR_WC;
    const int ncol = min(QR_WC, k - c0);
    const int tid = threadIdx.x;
    for (int t = tid; t < k * k; t += blockDim.x) {
        const int i = t / k, j = t % k;
        if (j > i) Us[up_off(k, i, j)] = S[t];
        else if (j == i) Us[up_off(k, i, i)] = (ta[i] == 0.0) ? 1.0 : 0.5 * S[t];
    }
    for (int t = tid; t < k * QR_WC; t += blockDim.x) {
        const int i = t / QR_WC, cc = t % QR_WC;
        Wc[t] = (cc < ncol) ? V[(size_t)(c0 + cc) * k + i] : 0.0;
    }
    __syncthreads();
    for (int i = tid; i < k; i += blockDim.x) rd[i] = 1.0 / Us[up_off(k, i, i)];
    __syncthreads();
    // block inverses: thread (b, c) back-substitutes D_b x = e_c
    for (int t = tid; t < nb * QR_WB; t += blockDim.x) {
        const int bb = t / QR_WB, cl = t % QR_WB;
        const int i0 = bb * QR_WB, bs = min(QR_WB, k - i0);
        double *D = Di + bb * QR_WB * QR_WB;
        if (cl < bs) {
            double x[QR_WB];
#pragma unroll
            for (int r = QR_WB - 1; r >= 0; --r) {
                double v = 0.0;
                if (r <= cl) {
                    v = (r == cl) ? 1.0 : 0.0;
#pragma unroll
                    for (int j = r + 1; j < QR_WB; ++j)
                        if (j <= cl) v = fma(-Us[up_off(k, i0 + r, i0 + j)], x[j], v);
                    v *= rd[i0 + r];
                }
                x[r] = v;
            }
#pragma unroll
            for (int r = 0; r < QR_WB; ++r) D[r * QR_WB + cl] = x[r];
        } else {
#pragma unroll
            for (int r = 0; r < QR_WB; ++r) D[r * QR_WB + cl] = 0.0;
        }
    }
    __syncthreads();
    for (int bb = nb - 1; bb >= 0; --bb) {
        const int i0 = bb * QR_WB, i1 = min(k, i0 + QR_WB);
        // rhs of the block: Wc[i][cc] -= sum_{j >= i1} U[i][j] Wc[j][cc]
        for (int t = tid; t < QR_WB * QR_WC * QR_WL; t += blockDim.x) {
            const int lane = t % QR_WL, pc = t / QR_WL;
            const int i = i0 + pc / QR_WC, cc = pc % QR_WC;
            double s0 = 0.0, s1 = 0.0;
            if (i < i1) {
                const double *u = Us + up_off(k, i, i) - i;   // u[j] = U[i][j] for j >= i
                int j = i1 + lane;
                for (; j + QR_WL < k; j += 2 * QR_WL) {
                    s0 = fma(u[j], Wc[j * QR_WC + cc], s0);
                    s1 = fma(u[j + QR_WL], Wc[(j + QR_WL) * QR_WC + cc], s1);
                }
                if (j < k) s0 = fma(u[j], Wc[j * QR_WC + cc], s0);
            }
            double sum = s0 + s1;
#pragma unroll
            for (int o = QR_WL / 2; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o, QR_WL);
            if (lane == 0 && i < i1) Wc[i * QR_WC + cc] -= sum;
        }
        __syncthreads();
        // apply the block inverse
        double wv = 0.0;
        const int r = tid / QR_WC, cc = tid % QR_WC;
        if (tid < QR_WB * QR_WC && i0 + r < i1) {
            const double *D = Di + bb * QR_WB * QR_WB + r * QR_WB;
#pragma unroll
            for (int j = 0; j < QR_WB; ++j)
                if (i0 + j < i1) wv = fma(D[j], Wc[(i0 + j) * QR_WC + cc], wv);
        }
        __syncthreads();
        if (tid < QR_WB * QR_WC && i0 + r < i1) Wc[(i0 + r) * QR_WC + cc] = wv;
        __syncthreads();
    }
    for (int t = tid; t < k * QR_WC; t += blockDim.x) {
        const int i = t / QR_WC, cc = t % QR_WC;
        if (cc < ncol) W[(size_t)i * k + c0 + cc] = Wc[t];
    }
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
    qr_wy_solve_kernel<<<(k + QR_WC - 1) / QR_WC, QR_WY_THREADS, qr_wy_smem_bytes(k), st>>>(k, s.S, s.V, s.ta, s.W);
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
