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
// So a column costs one grid barrier.  Q = H_0 H_1 ... H_{k-1} [I; 0] is then
// accumulated backwards the same way, and columns with R_jj < 0 are negated.
//
// The grid barrier is a counter/generation pair in global memory; its spin is
// bounded (about a second) and on expiry sets an error flag that the host
// reports as CTM_ETIMEOUT instead of hanging.
#include <cooperative_groups.h>

#include "ctm_internal.h"

namespace {

constexpr int QR_THREADS = 256;
constexpr long long QR_SPIN_LIMIT = 20000000LL;   // x ~64 ns sleep: ~1.3 s

__device__ __forceinline__ bool grid_barrier(unsigned *count, unsigned *gen, unsigned G, int *err)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = gen;
        unsigned my = *vgen;
        __threadfence();
        unsigned arrived = atomicAdd(count, 1u);
        if (arrived == G - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            long long it = 0;
            while (*vgen == my) {
                if (++it > QR_SPIN_LIMIT) {
                    atomicExch(err, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *((volatile int *)err) == 0;
}

struct QrArgs {
    int n, k, G, rows_per;
    const double *Y;
    double *Q, *R;
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
    double *Qs = Ys + (size_t)a.rows_per * k; // rows_per x k
    double *sv = Qs + (size_t)a.rows_per * k; // k
    double *rj = sv + k;                      // k
    double *cf = rj + k;                      // k
    double *taus = cf + k;                    // k
    double *v0s = taus + k;                   // k
    double *alps = v0s + k;                   // k
    const int tid = threadIdx.x;

    for (int t = tid; t < nr * k; t += blockDim.x) Ys[t] = a.Y[(size_t)r0 * k + t];
    __syncthreads();

    int step = 0;   // rotating-buffer counter shared by both phases
    // ---------------------------------------------------------- factorisation
    for (int j = 0; j < k; ++j, ++step) {
        double *acc = a.sbuf + (step % 3) * k;
        const int rs = max(r0, j) - r0;   // first local row taking part
        for (int kk = j + tid; kk < k; kk += blockDim.x) {
            double s = 0.0;
            for (int r = rs; r < nr; ++r) s = fma(Ys[r * k + j], Ys[r * k + kk], s);
            if (rs < nr) atomicAdd(&acc[kk], s);
        }
        if (j >= r0 && j < r1)
            for (int kk = j + tid; kk < k; kk += blockDim.x) a.rowbuf[(j & 1) * k + kk] = Ys[(j - r0) * k + kk];
        if (!grid_barrier(a.bar, a.bar + 1, a.G, a.err)) return;
        for (int kk = j + tid; kk < k; kk += blockDim.x) {
            sv[kk] = ((volatile double *)acc)[kk];
            rj[kk] = ((volatile double *)a.rowbuf)[(j & 1) * k + kk];
        }
        if (c == 0) {
            double *z = a.sbuf + ((step + 2) % 3) * k;
            for (int kk = tid; kk < k; kk += blockDim.x) z[kk] = 0.0;
        }
        __syncthreads();
        if (tid == 0) {
            double nrm2 = sv[j], x0 = rj[j];
            double nrm = sqrt(nrm2);
            double tau = 0.0, alpha = x0, v0 = 0.0;
            if (nrm > 0.0) {
                alpha = (x0 >= 0.0) ? -nrm : nrm;
                v0 = x0 - alpha;
                tau = 1.0 / (nrm * (nrm + fabs(x0)));   // 2 / v^T v, v^T v = 2|x|(|x| + |x_0|)
            }
            taus[j] = tau;
            v0s[j] = v0;
            alps[j] = (nrm > 0.0) ? alpha : 0.0;
        }
        __syncthreads();
        const double tau = taus[j], v0 = v0s[j], alpha = alps[j];
        for (int kk = j + 1 + tid; kk < k; kk += blockDim.x) cf[kk] = tau * (sv[kk] - alpha * rj[kk]);
        __syncthreads();
        if (c == 0) {
            for (int kk = tid; kk < k; kk += blockDim.x) {
                double v = 0.0;
                if (kk == j) v = alpha;
                else if (kk > j) v = rj[kk] - v0 * cf[kk];
                a.R[(size_t)j * k + kk] = v;
            }
        }
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

    // ---------------------------------------------------------- Q = H_0..H_{k-1} [I;0]
    for (int t = tid; t < nr * k; t += blockDim.x) {
        int r = t / k, cc = t % k;
        Qs[t] = (r0 + r == cc) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int j = k - 1; j >= 0; --j) {
        const double tau = taus[j];
        if (tau == 0.0) continue;       // uniform across CTAs
        const double v0 = v0s[j];
        double *acc = a.sbuf + (step % 3) * k;
        const int rs = max(r0, j) - r0;
        for (int kk = j + tid; kk < k; kk += blockDim.x) {
            double s = 0.0;
            for (int r = rs; r < nr; ++r) {
                double vr = (r0 + r == j) ? v0 : Ys[r * k + j];
                s = fma(vr, Qs[r * k + kk], s);
            }
            if (rs < nr) atomicAdd(&acc[kk], s);
        }
        if (!grid_barrier(a.bar, a.bar + 1, a.G, a.err)) return;
        for (int kk = j + tid; kk < k; kk += blockDim.x) sv[kk] = tau * ((volatile double *)acc)[kk];
        if (c == 0) {
            double *z = a.sbuf + ((step + 2) % 3) * k;
            for (int kk = tid; kk < k; kk += blockDim.x) z[kk] = 0.0;
        }
        __syncthreads();
        const int ncol = k - j;
        const int rows = nr - rs;
        for (int t = tid; t < rows * ncol; t += blockDim.x) {
            int r = rs + t / ncol;
            int kk = j + t % ncol;
            double vr = (r0 + r == j) ? v0 : Ys[r * k + j];
            Qs[r * k + kk] -= vr * sv[kk];
        }
        __syncthreads();
        ++step;
    }

    // ---------------------------------------------------------- gauge diag(R) >= 0
    for (int t = tid; t < nr * k; t += blockDim.x) {
        int cc = t % k;
        double v = Qs[t];
        a.Q[(size_t)r0 * k + t] = (alps[cc] < 0.0) ? -v : v;
    }
    if (c == 0) {
        __syncthreads();
        for (int t = tid; t < k * k; t += blockDim.x) {
            int rr = t / k;
            if (alps[rr] < 0.0) a.R[t] = -a.R[t];
        }
    }
}

size_t qr_smem_bytes(int rows_per, int k) { return sizeof(double) * ((size_t)2 * rows_per * k + 6 * (size_t)k); }

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
    return n >= k && k >= 1 && qr_layout(n, k, 1, &G, &rp);
}

cudaError_t qr_householder(int n, int k, const double *Y, double *Q, double *R, QrScratch s, cudaStream_t st)
{
    int G, rows_per;
    if (!qr_layout(n, k, s.rows_min > 0 ? s.rows_min : 1, &G, &rows_per)) {
        if (!qr_layout(n, k, 1, &G, &rows_per)) return cudaErrorInvalidValue;
    }
    size_t smem = qr_smem_bytes(rows_per, k);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qr_kernel, QR_THREADS, smem);
    if (per_sm * device_sm_count() < G) return cudaErrorCooperativeLaunchTooLarge;
    cudaError_t e = cudaMemsetAsync(s.sbuf, 0, sizeof(double) * 3 * k, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(s.bar, 0, sizeof(unsigned) * 2, st);
    if (e != cudaSuccess) return e;
    QrArgs a{n, k, G, rows_per, Y, Q, R, s.sbuf, s.rowbuf, s.bar, s.err};
    void *args[] = {&a};
    CTM_COUNT_LAUNCH(1);
    return cudaLaunchCooperativeKernel((void *)qr_kernel, dim3(G), dim3(QR_THREADS), args, smem, st);
}

cudaError_t qr_prepare()
{
    return cudaFuncSetAttribute(qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}
