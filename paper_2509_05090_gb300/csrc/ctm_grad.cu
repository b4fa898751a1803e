// Hand-written adjoint of the QR-based CTMRG step and of the bond energy
// (Sec. II.D: the energy gradient through k tracked CTMRG steps after detached
// warm-up steps, here computed without automatic differentiation).
//
// Forward: warm-up steps (detached), then k tracked steps whose input
// environments (C, T, Q_prev) are checkpointed, then the energy.  Backward:
// the energy's adjoint gives (C-bar, T-bar, Q-bar) of the last environment;
// for t = k-1 .. 0 the step is recomputed from its checkpoint and its adjoint
// maps the output cotangents (C'-bar, T'-bar, Q-bar) to the input cotangents
// while accumulating a-bar.  Every contraction's adjoint is two FP64 GEMMs over
// the same fused-index maps as the forward.  The QR adjoint (thin QR, R unused
// downstream) is Y-bar = (Q-bar + Q copyltu(-Q-bar^T Q)) R^{-T}, with the
// triangular solve regularised as 1/R_ii -> R_ii / (R_ii^2 + eps^2),
// eps = 1e-13 |R_00|.  Finally a-bar and the open-layer cotangent give A-bar,
// taken back through the C3v projection and the normalisation.
// The warm-start sign S = diag(sgn C_ii) is piecewise constant (no gradient).
#include <math.h>
#include <string.h>

#include "ctm_ctx.h"

namespace {

constexpr int GB = 256;   // reduction blocks

__device__ __forceinline__ double block_sum256(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    __syncthreads();
    return s;
}

// partials[2*b] = sum x^2, partials[2*b+1] = sum x*g over block b's share
__global__ void nrm_dot_partial_kernel(long long count, const double *x, const double *g, double *partials)
{
    __shared__ double red[32];
    double s = 0.0, t = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        s = fma(x[i], x[i], s);
        t = fma(x[i], g[i], t);
    }
    s = block_sum256(s, red);
    t = block_sum256(t, red);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = s;
        partials[2 * blockIdx.x + 1] = t;
    }
}

// y = x / |x| forward; given g = dL/dy: dL/dx = g/|x| - x <x,g>/|x|^3
__global__ void normalize_backward_kernel(long long count, const double *x, const double *g, double *out,
                                          const double *partials, int np)
{
    __shared__ double nrm, dot;
    if (threadIdx.x == 0) {
        double s = 0.0, t = 0.0;
        for (int i = 0; i < np; ++i) {
            s += partials[2 * i];
            t += partials[2 * i + 1];
        }
        nrm = sqrt(s);
        dot = t;
    }
    __syncthreads();
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    const double c3 = dot * inv * inv * inv;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = g[i] * inv - x[i] * c3;
}

// C' = sym(Cr)/|sym(Cr)|: Cr-bar from C'-bar.  One CTA.
__global__ void corner_backward_kernel(int chi, const double *Cr, const double *Cpb, double *Crb)
{
    __shared__ double red[32];
    double ss = 0.0, sd = 0.0;
    for (int t = threadIdx.x; t < chi * chi; t += blockDim.x) {
        int i = t / chi, j = t % chi;
        double cs = 0.5 * (Cr[t] + Cr[j * chi + i]);
        ss += cs * cs;
        sd += cs * Cpb[t];
    }
    ss = block_sum256(ss, red);
    sd = block_sum256(sd, red);
    const double nrm = sqrt(ss);
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    const double dot = sd * inv;   // <C', C'-bar>
    for (int t = threadIdx.x; t < chi * chi; t += blockDim.x) {
        int i = t / chi, j = t % chi;
        double cs_t = 0.5 * (Cr[t] + Cr[j * chi + i]);
        double gst = (Cpb[t] - cs_t * inv * dot) * inv;
        double gst2 = (Cpb[j * chi + i] - cs_t * inv * dot) * inv;   // C_s symmetric: C_s[j][i] = cs_t
        Crb[t] = 0.5 * (gst + gst2);
    }
}

// Z <- copyltu(Z): lower triangle mirrored to the upper one.  One CTA, in place.
__global__ void copyltu_kernel(int k, double *Z)
{
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
        int i = t / k, j = t % k;
        if (j > i) Z[t] = Z[j * k + i];
    }
}

// Ybar[r,:] = B[r,:] R^{-T}: back substitution of R x = B[r,:]^T per row (R upper triangular),
// with the diagonal regularised.  R in shared memory; one thread per row.
__global__ void trisolve_rows_kernel(long long n, int k, const double *R, const double *B, double *X)
{
    extern __shared__ double sR[];
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) sR[t] = R[t];
    __syncthreads();
    const double eps = 1e-13 * fabs(sR[0]);
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        const double *b = B + r * k;
        double *x = X + r * k;
        for (int i = k - 1; i >= 0; --i) {
            double s = b[i];
            for (int j = i + 1; j < k; ++j) s -= sR[i * k + j] * x[j];
            const double d = sR[i * k + i];
            x[i] = s * d / (d * d + eps * eps);
        }
    }
}

__global__ void sign_cols_kernel(long long n, int k, const double *X, const double *C, double *Y)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n * k;
         t += (long long)gridDim.x * blockDim.x) {
        int j = (int)(t % k);
        Y[t] = (C[(size_t)j * k + j] < 0.0) ? -X[t] : X[t];
    }
}

// Energy: E_site = (1/2) sum_a sum_{rc} rho[r][c] h_a[c][r], rho[(sA sB)][(tA tB)] = raw[(sB tB)][(sA tA)]/Z.
// rawb = dE/draw; out[0] = E_site.
__global__ void rho_backward_kernel(int d, const double *raw, const double *h, double *rawb, double *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int dd = d * d;
    double Z = 0.0;
    for (int sA = 0; sA < d; ++sA)
        for (int sB = 0; sB < d; ++sB) Z += raw[(sB * d + sB) * dd + sA * d + sA];
    // rhob[r][c] = (1/2) sum_a h_a[c][r]; E = <rhob, rho>
    double E = 0.0;
    for (int r = 0; r < dd; ++r)
        for (int cc = 0; cc < dd; ++cc) {
            int sA = r / d, sB = r % d, tA = cc / d, tB = cc % d;
            double rho = raw[(sB * d + tB) * dd + sA * d + tA] / Z;
            double hb = 0.0;
            for (int a = 0; a < 3; ++a) hb += h[(size_t)a * dd * dd + cc * dd + r];
            E += 0.5 * hb * rho;
        }
    for (int r = 0; r < dd; ++r)
        for (int cc = 0; cc < dd; ++cc) {
            int sA = r / d, sB = r % d, tA = cc / d, tB = cc % d;
            double hb = 0.0;
            for (int a = 0; a < 3; ++a) hb += h[(size_t)a * dd * dd + cc * dd + r];
            double g = (0.5 * hb - (r == cc ? E : 0.0)) / Z;
            rawb[(sB * d + tB) * dd + sA * d + tA] = g;
        }
    out[0] = E;
}

// Y1o-bar[ab][pB][z] = sum_pA rawb[pB][pA] G2[ab][pA][z];  G2-bar[ab][pA][z] = sum_pB rawb[pB][pA] Y1o[ab][pB][z]
__global__ void raw_backward_kernel(long long nab, int dd, int D2, const double *rawb, const double *Y1o,
                                    const double *G2, double *Y1ob, double *G2b)
{
    __shared__ double rb[81];
    for (int i = threadIdx.x; i < dd * dd; i += blockDim.x) rb[i] = rawb[i];
    __syncthreads();
    const long long row = (long long)dd * D2;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nab * D2;
         t += (long long)gridDim.x * blockDim.x) {
        long long ab = t / D2;
        int z = (int)(t - ab * D2);
        const double *y = Y1o + ab * row + z;
        const double *g = G2 + ab * row + z;
        for (int p = 0; p < dd; ++p) {
            double sy = 0.0, sg = 0.0;
            for (int q = 0; q < dd; ++q) {
                sy += rb[p * dd + q] * g[(size_t)q * D2];
                sg += rb[q * dd + p] * y[(size_t)q * D2];
            }
            Y1ob[ab * row + (long long)p * D2 + z] = sy;
            G2b[ab * row + (long long)p * D2 + z] = sg;
        }
    }
}

// A-bar from the double layer a = sum_s A (x) A and the open layers b[(s,t)] = A[s] (x) A[t]:
// Ab[s,ijk] = sum_{i'j'k'} ( ab[(ii')(jj')(kk')] + ab[(i'i)(j'j)(k'k)] ) A[s,i'j'k']
//           + sum_t sum_{i'j'k'} ( bb[(s,t)][(ii')..] A[t,i'j'k'] + bb[(t,s)][(i'i)..] A[t,i'j'k'] )
__global__ void layers_backward_kernel(int d, int D, const double *A, const double *ab, const double *bb, double *Ab)
{
    const int D2 = D * D, D3 = D * D * D;
    const long long D6 = (long long)D2 * D2 * D2;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < d * D3; t += gridDim.x * blockDim.x) {
        const int s = t / D3, r = t % D3;
        const int i = r / (D * D), j = (r / D) % D, k = r % D;
        double acc = 0.0;
        for (int q = 0; q < D3; ++q) {
            const int i2 = q / (D * D), j2 = (q / D) % D, k2 = q % D;
            const long long o1 = ((long long)(i * D + i2) * D2 + (j * D + j2)) * D2 + (k * D + k2);
            const long long o2 = ((long long)(i2 * D + i) * D2 + (j2 * D + j)) * D2 + (k2 * D + k);
            acc += (ab[o1] + ab[o2]) * A[(size_t)s * D3 + q];
            for (int u = 0; u < d; ++u)
                acc += bb[(long long)(s * d + u) * D6 + o1] * A[(size_t)u * D3 + q] +
                       bb[(long long)(u * d + s) * D6 + o2] * A[(size_t)u * D3 + q];
        }
        Ab[t] = acc;
    }
}

// a0 backward: A = P(Araw)/|P(Araw)| (P = average over the 6 leg permutations, self-adjoint):
// Araw-bar = P( Ab/|P Araw| - A <A, Ab>/|P Araw| ).  One CTA.
__global__ void project_backward_kernel(int d, int D, const double *Araw, const double *A, const double *Ab,
                                        double *out, int symmetrize)
{
    extern __shared__ double g[];
    __shared__ double red[32];
    const int D3 = D * D * D, tot = d * D3;
    if (!symmetrize) {
        for (int t = threadIdx.x; t < tot; t += blockDim.x) out[t] = Ab[t];
        return;
    }
    double ss = 0.0, dot = 0.0;
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
        int s = t / D3, r = t % D3;
        int i = r / (D * D), j = (r / D) % D, k = r % D;
        const double *As = Araw + (size_t)s * D3;
        double v = (As[(i * D + j) * D + k] + As[(i * D + k) * D + j] + As[(j * D + i) * D + k] +
                    As[(j * D + k) * D + i] + As[(k * D + i) * D + j] + As[(k * D + j) * D + i]) / 6.0;
        ss += v * v;
        dot += A[t] * Ab[t];
    }
    ss = block_sum256(ss, red);
    dot = block_sum256(dot, red);
    const double inv = ss > 0.0 ? 1.0 / sqrt(ss) : 0.0;
    for (int t = threadIdx.x; t < tot; t += blockDim.x) g[t] = (Ab[t] - A[t] * dot) * inv;
    __syncthreads();
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
        int s = t / D3, r = t % D3;
        int i = r / (D * D), j = (r / D) % D, k = r % D;
        const double *gs = g + (size_t)s * D3;
        out[t] = (gs[(i * D + j) * D + k] + gs[(i * D + k) * D + j] + gs[(j * D + i) * D + k] +
                  gs[(j * D + k) * D + i] + gs[(k * D + i) * D + j] + gs[(k * D + j) * D + i]) / 6.0;
    }
}

int grid_of(long long count)
{
    long long b = (count + 255) / 256;
    long long cap = 8LL * device_sm_count();
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

// ---------------------------------------------------------------- workspace
struct GradBufs {
    double *ck;            // (k+1) checkpoints of (C, T, Q)
    double *X2, *Mb, *Xb, *H3b, *H1b;                 // n x n
    double *G, *Gb, *Wb, *MQb, *Qb, *Yb, *Bq, *Qsb, *Qnext, *Qs_keep;   // n x chi
    double *Y1b, *H2, *H2b;                           // chi^2 D2
    double *Crb, *Cpb, *Cb, *Zm, *P[5], *P5b, *Chb, *tmp;   // chi x chi
    double *Tr, *Trb, *Tpb, *Tb;                      // chi D2 chi
    double *ab, *bb, *Abar;
    double *Y1ob, *G2b;                               // chi^2 d^2 D2
    double *rawb, *scal, *part;
    double *sk;                                       // split-K partials of the adjoint GEMMs
    size_t sk_elems;
    size_t ck_stride;
};

size_t grad_layout(const ctm_ctx *c, int k, GradBufs *g, char *base)
{
    const long long chi = c->chi, D2 = c->D2, n = c->n, d = c->d;
    size_t off = 0;
    auto td = [&](long long count) -> double * {
        double *p = base ? (double *)(base + off) : nullptr;
        off += align_up(sizeof(double) * (size_t)(count > 0 ? count : 1));
        return p;
    };
    GradBufs b;
    b.ck_stride = (size_t)(chi * chi + chi * D2 * chi + n * chi);
    b.ck = td((long long)(k + 1) * (long long)b.ck_stride);
    b.X2 = td(n * n);
    b.Mb = td(n * n);
    b.Xb = td(n * n);
    b.H3b = td(n * n);
    b.H1b = td(n * n);
    b.G = td(n * chi);
    b.Gb = td(n * chi);
    b.Wb = td(n * chi);
    b.MQb = td(n * chi);
    b.Qb = td(n * chi);
    b.Yb = td(n * chi);
    b.Bq = td(n * chi);
    b.Qsb = td(n * chi);
    b.Qnext = td(n * chi);
    b.Qs_keep = td(n * chi);
    b.Y1b = td(chi * chi * D2);
    b.H2 = td(chi * chi * D2);
    b.H2b = td(chi * chi * D2);
    b.Crb = td(chi * chi);
    b.Cpb = td(chi * chi);
    b.Cb = td(chi * chi);
    b.Zm = td(chi * chi);
    for (int i = 0; i < 5; ++i) b.P[i] = td(chi * chi);
    b.P5b = td(chi * chi);
    b.Chb = td(chi * chi);
    b.tmp = td(chi * chi);
    b.Tr = td(chi * D2 * chi);
    b.Trb = td(chi * D2 * chi);
    b.Tpb = td(chi * D2 * chi);
    b.Tb = td(chi * D2 * chi);
    b.ab = td(D2 * D2 * D2);
    b.bb = td(d * d * D2 * D2 * D2);
    b.Abar = td(d * c->D * c->D * c->D);
    b.Y1ob = td(chi * chi * d * d * D2);
    b.G2b = td(chi * chi * d * d * D2);
    b.rawb = td(d * d * d * d);
    b.scal = td(16);
    b.part = td(2 * GB);
    long long ske = 8 * n * chi;
    if (64 * chi * chi > ske) ske = 64 * chi * chi;
    if (16 * D2 * D2 * D2 > ske) ske = 16 * D2 * D2 * D2;
    if (ske < (1LL << 20)) ske = 1LL << 20;
    b.sk = td(ske);
    b.sk_elems = (size_t)ske;
    if (g) *g = b;
    return off;
}

#define CK(expr)                                 \
    do {                                         \
        cudaError_t _e = (expr);                 \
        if (_e != cudaSuccess) return CTM_ECUDA; \
    } while (0)

// C(m,n) = alpha A(m,k) B(k,n) + beta C(m,n), FP64
struct G64 {
    ctm_ctx *c;
    const GradBufs *b;
    cudaError_t operator()(int M, int N, int K, const double *A, Idx2 Am, Idx2 Ak, const double *B, Idx2 Bk, Idx2 Bn,
                           double *C, Idx2 Cm, Idx2 Cn, double alpha = 1.0, double beta = 0.0) const
    {
        GemmF64 g{M, N, K, A, Am, Ak, B, Bk, Bn, C, Cm, Cn, alpha, beta};
        return gemm_f64(g, gemm_f64_pick_split(M, N, K), b->sk, b->sk_elems, c->stream);
    }
};

inline Idx2 L(long long s) { return idx_lin(s); }
inline Idx2 S2(int div, long long hi, long long lo) { return idx_split(div, hi, lo); }

// Forward of one step from (C, T, Qp), keeping every intermediate the adjoint needs:
// W, X' (c->X), Y1, M, Qs, Y, Q (c->Qn), R, MQ, Cr, H1' (X2), H2, H3' (c->H), Tr (unnormalised).
int step_forward_keep(ctm_ctx *c, GradBufs &b, const double *C, const double *T, const double *Qp)
{
    const int chi = c->chi, D2 = c->D2;
    const long long n = c->n;
    G64 G{c, &b};
    cudaStream_t st = c->stream;
    CK(G((int)n, chi, chi, T, L(chi), L(1), C, L(chi), L(1), c->W, L(chi), L(1)));
    CK(G((int)n, (int)n, chi, c->W, L(chi), L(1), T, L(1), L(chi), c->X, S2(D2, (long long)chi * D2 * D2, D2),
         S2(D2, (long long)D2 * D2, 1)));
    CK(G(chi * chi, D2, D2 * D2, c->X, L((long long)D2 * D2), L(1), c->a, L(D2), L(1), c->Y1, L(D2), L(1)));
    CK(G(chi * chi, D2 * D2, D2, c->Y1, L(D2), L(1), c->a, L((long long)D2 * D2), L(1), c->M,
         S2(chi, (long long)D2 * n, D2), S2(D2, 1, n)));
    CK(launch_warm_start((int)n, chi, Qp, C, c->Qs, st));
    CK(G((int)n, chi, (int)n, c->M, L(n), L(1), c->Qs, L(chi), L(1), c->Y, L(chi), L(1)));
    QrScratch qs = ctmi::qr_scratch(c);
    CK(qr_householder((int)n, chi, c->Y, c->Qn, c->R, qs, st));
    CK(G((int)n, chi, (int)n, c->M, L(n), L(1), c->Qn, L(chi), L(1), c->MQ, L(chi), L(1)));
    CK(G(chi, chi, (int)n, c->Qn, L(1), L(chi), c->MQ, L(chi), L(1), c->Cr, L(chi), L(1)));
    CK(G((int)n, (int)n, chi, T, L(chi), L(1), c->Qn, L(n), L(1), b.X2, S2(D2, (long long)chi * D2 * D2, D2),
         S2(chi, 1, (long long)D2 * D2)));
    CK(G(chi * chi, D2, D2 * D2, b.X2, L((long long)D2 * D2), L(1), c->a, L(D2), L(1), b.H2, L(D2), L(1)));
    CK(G(chi * chi, D2 * D2, D2, b.H2, L(D2), L(1), c->a, L((long long)D2 * D2), L(1), c->H,
         S2(chi, (long long)D2 * D2 * chi, 1), S2(D2, chi, (long long)D2 * chi)));
    CK(G(chi, (int)n, (int)n, c->Qn, L(1), L(chi), c->H, L(n), L(1), b.Tr, L(n), L(1)));
    return CTM_OK;
}

// Adjoint of the projector part: given Qbar (total cotangent of Q) and Mbar (partial),
// run the QR backward and Y = M Qs, adding to Mbar and writing Qsbar-with-sign into Qp_bar.
int projector_backward(ctm_ctx *c, GradBufs &b, const double *Cprev, double *Qp_bar)
{
    const int chi = c->chi;
    const long long n = c->n;
    G64 G{c, &b};
    cudaStream_t st = c->stream;
    // Zm = copyltu(-Qbar^T Q)
    CK(G(chi, chi, (int)n, b.Qb, L(1), L(chi), c->Qn, L(chi), L(1), b.Zm, L(chi), L(1), -1.0, 0.0));
    copyltu_kernel<<<1, 256, 0, st>>>(chi, b.Zm);
    CK(cudaGetLastError());
    // Bq = Qbar + Q Zm
    CK(cudaMemcpyAsync(b.Bq, b.Qb, sizeof(double) * n * chi, cudaMemcpyDeviceToDevice, st));
    CK(G((int)n, chi, chi, c->Qn, L(chi), L(1), b.Zm, L(chi), L(1), b.Bq, L(chi), L(1), 1.0, 1.0));
    // Ybar = Bq R^{-T}
    trisolve_rows_kernel<<<grid_of(n), 256, sizeof(double) * chi * chi, st>>>(n, chi, c->R, b.Bq, b.Yb);
    CK(cudaGetLastError());
    // Y = M Qs: Mbar += Ybar Qs^T ; Qs_bar = M^T Ybar ; Qp_bar = Qs_bar S
    CK(G((int)n, (int)n, chi, b.Yb, L(chi), L(1), c->Qs, L(1), L(chi), b.Mb, L(n), L(1), 1.0, 1.0));
    CK(G((int)n, chi, (int)n, c->M, L(1), L(n), b.Yb, L(chi), L(1), b.Qsb, L(chi), L(1)));
    sign_cols_kernel<<<grid_of(n * chi), 256, 0, st>>>(n, chi, b.Qsb, Cprev, Qp_bar);
    CK(cudaGetLastError());
    return CTM_OK;
}

// Adjoint of the enlarged corner: Mbar (and an optional extra X'-bar already in Xb when xb_init)
// -> abar, Tbar (+=), Cbar (=).
int corner_chain_backward(ctm_ctx *c, GradBufs &b, const double *C, const double *T, bool xb_init)
{
    const int chi = c->chi, D2 = c->D2;
    const long long n = c->n;
    G64 G{c, &b};
    // M = Y1 a (permuted): Y1bar, abar[z,(x,y)]
    CK(G(chi * chi, D2, D2 * D2, b.Mb, S2(chi, (long long)D2 * n, D2), S2(D2, 1, n), c->a, L(1), L((long long)D2 * D2),
         b.Y1b, L(D2), L(1)));
    CK(G(D2, D2 * D2, chi * chi, c->Y1, L(1), L(D2), b.Mb, S2(chi, (long long)D2 * n, D2), S2(D2, 1, n), b.ab,
         L((long long)D2 * D2), L(1), 1.0, 1.0));
    // Y1 = X' a: X'bar (+= when the energy already wrote one), abar[(u,l),z]
    CK(G(chi * chi, D2 * D2, D2, b.Y1b, L(D2), L(1), c->a, L(1), L(D2), b.Xb, L((long long)D2 * D2), L(1), 1.0,
         xb_init ? 1.0 : 0.0));
    CK(G(D2 * D2, D2, chi * chi, c->X, L(1), L((long long)D2 * D2), b.Y1b, L(D2), L(1), b.ab, L(D2), L(1), 1.0, 1.0));
    // X' = W T^T: Wbar, Tbar += X'bar^T-part W
    CK(G((int)n, chi, (int)n, b.Xb, S2(D2, (long long)chi * D2 * D2, D2), S2(D2, (long long)D2 * D2, 1), T, L(chi),
         L(1), b.Wb, L(chi), L(1)));
    CK(G((int)n, chi, (int)n, b.Xb, S2(D2, (long long)D2 * D2, 1), S2(D2, (long long)chi * D2 * D2, D2), c->W, L(chi),
         L(1), b.Tb, L(chi), L(1), 1.0, 1.0));
    // W = T C: Tbar += Wbar C^T, Cbar = T^T Wbar
    CK(G((int)n, chi, chi, b.Wb, L(chi), L(1), C, L(1), L(chi), b.Tb, L(chi), L(1), 1.0, 1.0));
    CK(G(chi, chi, (int)n, T, L(1), L(chi), b.Wb, L(chi), L(1), b.Cb, L(chi), L(1)));
    return CTM_OK;
}

// Adjoint of one step: inputs Cpb (C'-bar), Tpb (T'-bar), Qnext (Q-bar from the next use of Q);
// outputs Cb, Tb, Qp_bar (into Qnext for the previous step) and accumulates ab.
int step_backward(ctm_ctx *c, GradBufs &b, const double *C, const double *T)
{
    const int chi = c->chi, D2 = c->D2;
    const long long n = c->n, nT = (long long)chi * D2 * chi;
    G64 G{c, &b};
    cudaStream_t st = c->stream;
    // T' = Tr/|Tr|
    nrm_dot_partial_kernel<<<GB, 256, 0, st>>>(nT, b.Tr, b.Tpb, b.part);
    normalize_backward_kernel<<<GB, 256, 0, st>>>(nT, b.Tr, b.Tpb, b.Trb, b.part, GB);
    CK(cudaGetLastError());
    // Qbar = Qnext + H3' Trb^T ; H3'bar = Q Trb
    CK(cudaMemcpyAsync(b.Qb, b.Qnext, sizeof(double) * n * chi, cudaMemcpyDeviceToDevice, st));
    CK(G((int)n, chi, (int)n, c->H, L(n), L(1), b.Trb, L(1), L(n), b.Qb, L(chi), L(1), 1.0, 1.0));
    CK(G((int)n, (int)n, chi, c->Qn, L(chi), L(1), b.Trb, L(n), L(1), b.H3b, L(n), L(1)));
    // H3' = H2 a: H2bar, abar[z,(x,y)]
    CK(G(chi * chi, D2, D2 * D2, b.H3b, S2(chi, (long long)D2 * D2 * chi, 1), S2(D2, chi, (long long)D2 * chi), c->a,
         L(1), L((long long)D2 * D2), b.H2b, L(D2), L(1)));
    CK(G(D2, D2 * D2, chi * chi, b.H2, L(1), L(D2), b.H3b, S2(chi, (long long)D2 * D2 * chi, 1),
         S2(D2, chi, (long long)D2 * chi), b.ab, L((long long)D2 * D2), L(1), 1.0, 1.0));
    // H2 = H1' a: H1'bar, abar[(u,w),z]
    CK(G(chi * chi, D2 * D2, D2, b.H2b, L(D2), L(1), c->a, L(1), L(D2), b.H1b, L((long long)D2 * D2), L(1)));
    CK(G(D2 * D2, D2, chi * chi, b.X2, L(1), L((long long)D2 * D2), b.H2b, L(D2), L(1), b.ab, L(D2), L(1), 1.0, 1.0));
    // H1' = T Q_r: Tbar = H1'bar Q ; Qbar += T^T H1'bar
    CK(G((int)n, chi, (int)n, b.H1b, S2(D2, (long long)chi * D2 * D2, D2), S2(chi, 1, (long long)D2 * D2), c->Qn,
         L(1), L(n), b.Tb, L(chi), L(1)));
    CK(G(chi, (int)n, (int)n, T, L(1), L(chi), b.H1b, S2(D2, (long long)chi * D2 * D2, D2),
         S2(chi, 1, (long long)D2 * D2), b.Qb, L(n), L(1), 1.0, 1.0));
    // C' = sym(Cr)/|.|
    corner_backward_kernel<<<1, 256, 0, st>>>(chi, c->Cr, b.Cpb, b.Crb);
    CK(cudaGetLastError());
    // Cr = Q^T MQ: Qbar += MQ Crb^T ; MQbar = Q Crb
    CK(G((int)n, chi, chi, c->MQ, L(chi), L(1), b.Crb, L(1), L(chi), b.Qb, L(chi), L(1), 1.0, 1.0));
    CK(G((int)n, chi, chi, c->Qn, L(chi), L(1), b.Crb, L(chi), L(1), b.MQb, L(chi), L(1)));
    // MQ = M Q: Mbar = MQbar Q^T ; Qbar += M^T MQbar
    CK(G((int)n, (int)n, chi, b.MQb, L(chi), L(1), c->Qn, L(1), L(chi), b.Mb, L(n), L(1)));
    CK(G((int)n, chi, (int)n, c->M, L(1), L(n), b.MQb, L(chi), L(1), b.Qb, L(chi), L(1), 1.0, 1.0));
    int rc = projector_backward(c, b, C, b.Qnext);
    if (rc != CTM_OK) return rc;
    return corner_chain_backward(c, b, C, T, false);
}

}  // namespace

using namespace ctmi;

extern "C" size_t ctm_grad_workspace_bytes(const ctm_ctx *c, int k_tracked)
{
    if (!c || k_tracked < 1) return 0;
    return grad_layout(c, k_tracked, nullptr, nullptr);
}

extern "C" int ctm_grad(ctm_ctx *c, int warmup, int k_tracked, const double *h_dev, void *gws, size_t gws_bytes,
                        double *energy_host, double *dA_dev)
{
    if (!c || !h_dev || !gws || !dA_dev || warmup < 0 || k_tracked < 1) return CTM_EINVAL;
    if (c->d * c->d > 9 || c->cfg.corner_mode != 0) return CTM_EUNSUPPORTED;
    if ((uintptr_t)gws % 256 != 0) return CTM_EINVAL;
    if (gws_bytes < grad_layout(c, k_tracked, nullptr, nullptr)) return CTM_ENOMEM;
    GradBufs b;
    grad_layout(c, k_tracked, &b, (char *)gws);
    if (sizeof(double) * (size_t)c->chi * c->chi > 200 * 1024) return CTM_EUNSUPPORTED;
    if (cudaFuncSetAttribute(trisolve_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
            cudaSuccess ||
        cudaFuncSetAttribute(project_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
            cudaSuccess)
        return CTM_ECUDA;
    const int chi = c->chi, D2 = c->D2, d = c->d, dd = d * d;
    const long long n = c->n, nC = (long long)chi * chi, nT = (long long)chi * D2 * chi, nQ = n * chi;
    cudaStream_t st = c->stream;
    G64 G{c, &b};
    if (join_side(c) != CTM_OK) return CTM_ECUDA;
    // ---- forward: detached warm-up, then tracked steps with checkpoints, both in the
    // context's precision (split-BF16 contractions with the FP64 QR on a split context)
    if (warmup > 0) {
        int rc = ctm_step(c, warmup, nullptr);
        if (rc != CTM_OK) return rc;
    }
    auto ck = [&](int t) { return b.ck + (size_t)t * b.ck_stride; };
    int rc = CTM_OK;
    for (int t = 0; t <= k_tracked && rc == CTM_OK; ++t) {
        double *p = ck(t);
        if (cudaMemcpyAsync(p, c->C, sizeof(double) * nC, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(p + nC, c->T, sizeof(double) * nT, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(p + nC + nT, c->Q, sizeof(double) * nQ, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            rc = CTM_ECUDA;
        if (rc == CTM_OK && t < k_tracked) rc = ctm_step(c, 1, nullptr);
    }
    if (rc != CTM_OK) return rc;
    if (join_side(c) != CTM_OK) return CTM_ECUDA;

    // ---- energy forward from the last checkpoint, keeping intermediates
    const double *Ck = ck(k_tracked), *Tk = ck(k_tracked) + nC, *Qk = ck(k_tracked) + nC + nT;
    CK(cudaMemsetAsync(b.ab, 0, sizeof(double) * D2 * D2 * D2, st));
    CK(cudaMemsetAsync(b.bb, 0, sizeof(double) * dd * D2 * D2 * D2, st));
    CK(G((int)n, chi, chi, Tk, L(chi), L(1), Ck, L(chi), L(1), c->W, L(chi), L(1)));
    CK(G((int)n, (int)n, chi, c->W, L(chi), L(1), Tk, L(1), L(chi), c->X, S2(D2, (long long)chi * D2 * D2, D2),
         S2(D2, (long long)D2 * D2, 1)));
    CK(G(chi * chi, D2, D2 * D2, c->X, L((long long)D2 * D2), L(1), c->a, L(D2), L(1), c->Y1, L(D2), L(1)));
    CK(G(chi * chi, D2 * D2, D2, c->Y1, L(D2), L(1), c->a, L((long long)D2 * D2), L(1), c->M,
         S2(chi, (long long)D2 * n, D2), S2(D2, 1, n)));
    CK(launch_warm_start((int)n, chi, Qk, Ck, c->Qs, st));
    CK(G((int)n, chi, (int)n, c->M, L(n), L(1), c->Qs, L(chi), L(1), c->Y, L(chi), L(1)));
    {
        QrScratch qs = ctmi::qr_scratch(c);
        CK(qr_householder((int)n, chi, c->Y, c->Qn, c->R, qs, st));
    }
    CK(G((int)n, chi, (int)n, c->M, L(n), L(1), c->Qn, L(chi), L(1), c->MQ, L(chi), L(1)));
    CK(G(chi, chi, (int)n, c->Qn, L(1), L(chi), c->MQ, L(chi), L(1), c->Cr, L(chi), L(1)));
    CK(launch_corner_sym_normalize(chi, c->Cr, b.P[0], c->norm_part, st));   // P1 = Ch
    for (int p = 1; p < 5; ++p)
        CK(G(chi, chi, chi, b.P[p - 1], L(chi), L(1), b.P[0], L(chi), L(1), b.P[p], L(chi), L(1)));
    CK(G((int)n, chi, chi, c->Qn, L(chi), L(1), b.P[4], L(chi), L(1), b.G, L(chi), L(1)));
    CK(G((int)n, (int)n, chi, b.G, L(chi), L(1), c->Qn, L(1), L(chi), c->H, L(n), L(1)));   // Em
    CK(launch_open_layers(d, c->D, c->A, c->b, st));
    const long long D3 = (long long)D2 * D2 * D2;
    CK(G(chi * chi, dd * D2, D2 * D2, c->X, L((long long)D2 * D2), L(1), c->b, L(D2), S2(D2, D3, 1), c->Y1o,
         L((long long)dd * D2), L(1)));
    CK(G(chi * chi, dd * D2, D2 * D2, c->H, S2(chi, (long long)D2 * n, D2), S2(D2, 1, n), c->b, L(1),
         S2(D2, D3, (long long)D2 * D2), c->G2, L((long long)dd * D2), L(1)));
    CK(rho_reduce(c));
    rho_backward_kernel<<<1, 32, 0, st>>>(d, c->rho_raw, h_dev, b.rawb, b.scal);
    CK(cudaGetLastError());

    // ---- energy backward
    raw_backward_kernel<<<grid_of((long long)chi * chi * D2), 256, 0, st>>>((long long)chi * chi, dd, D2, b.rawb, c->Y1o,
                                                                          c->G2, b.Y1ob, b.G2b);
    CK(cudaGetLastError());
    // G2 = Em' b: Em-bar (into H3b), b-bar
    CK(G(chi * chi, D2 * D2, dd * D2, b.G2b, L((long long)dd * D2), L(1), c->b, L((long long)D2 * D2), L(1), b.H3b,
         S2(chi, (long long)D2 * n, D2), S2(D2, 1, n)));
    CK(G(dd * D2, D2 * D2, chi * chi, b.G2b, L(1), L((long long)dd * D2), c->H, S2(chi, (long long)D2 * n, D2),
         S2(D2, 1, n), b.bb, L((long long)D2 * D2), L(1), 1.0, 1.0));
    // Y1o = X' b: X'-bar (first write), b-bar
    CK(G(chi * chi, D2 * D2, dd * D2, b.Y1ob, L((long long)dd * D2), L(1), c->b, S2(D2, D3, 1), L(D2), b.Xb,
         L((long long)D2 * D2), L(1)));
    CK(G(D2 * D2, dd * D2, chi * chi, c->X, L(1), L((long long)D2 * D2), b.Y1ob, L((long long)dd * D2), L(1), b.bb,
         L(D2), S2(D2, D3, 1), 1.0, 1.0));
    // Em = G Q^T: Gbar = Em-bar Q ; Qbar = Em-bar^T G
    CK(G((int)n, chi, (int)n, b.H3b, L(n), L(1), c->Qn, L(chi), L(1), b.Gb, L(chi), L(1)));
    CK(G((int)n, chi, (int)n, b.H3b, L(1), L(n), b.G, L(chi), L(1), b.Qb, L(chi), L(1)));
    // G = Q P5: Qbar += Gbar P5^T ; P5bar = Q^T Gbar
    CK(G((int)n, chi, chi, b.Gb, L(chi), L(1), b.P[4], L(1), L(chi), b.Qb, L(chi), L(1), 1.0, 1.0));
    CK(G(chi, chi, (int)n, c->Qn, L(1), L(chi), b.Gb, L(chi), L(1), b.P5b, L(chi), L(1)));
    // P5 = Ch^5: Chbar = sum_k P_k P5bar P_{4-k}  (P_0 = I)
    CK(G(chi, chi, chi, b.P5b, L(chi), L(1), b.P[3], L(chi), L(1), b.Chb, L(chi), L(1)));
    for (int kk = 1; kk <= 3; ++kk) {
        CK(G(chi, chi, chi, b.P[kk - 1], L(chi), L(1), b.P5b, L(chi), L(1), b.tmp, L(chi), L(1)));
        CK(G(chi, chi, chi, b.tmp, L(chi), L(1), b.P[3 - kk], L(chi), L(1), b.Chb, L(chi), L(1), 1.0, 1.0));
    }
    CK(G(chi, chi, chi, b.P[3], L(chi), L(1), b.P5b, L(chi), L(1), b.Chb, L(chi), L(1), 1.0, 1.0));
    // Ch = sym(Cr)/|.| ; Cr = Q^T MQ ; MQ = M Q
    corner_backward_kernel<<<1, 256, 0, st>>>(chi, c->Cr, b.Chb, b.Crb);
    CK(cudaGetLastError());
    CK(G((int)n, chi, chi, c->MQ, L(chi), L(1), b.Crb, L(1), L(chi), b.Qb, L(chi), L(1), 1.0, 1.0));
    CK(G((int)n, chi, chi, c->Qn, L(chi), L(1), b.Crb, L(chi), L(1), b.MQb, L(chi), L(1)));
    CK(G((int)n, (int)n, chi, b.MQb, L(chi), L(1), c->Qn, L(1), L(chi), b.Mb, L(n), L(1)));
    CK(G((int)n, chi, (int)n, c->M, L(1), L(n), b.MQb, L(chi), L(1), b.Qb, L(chi), L(1), 1.0, 1.0));
    CK(cudaMemsetAsync(b.Tb, 0, sizeof(double) * nT, st));
    if ((rc = projector_backward(c, b, Ck, b.Qnext)) != CTM_OK) return rc;
    if ((rc = corner_chain_backward(c, b, Ck, Tk, true)) != CTM_OK) return rc;

    // ---- tracked steps, last to first
    for (int t = k_tracked - 1; t >= 0; --t) {
        CK(cudaMemcpyAsync(b.Cpb, b.Cb, sizeof(double) * nC, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(b.Tpb, b.Tb, sizeof(double) * nT, cudaMemcpyDeviceToDevice, st));
        const double *Ct = ck(t), *Tt = ck(t) + nC, *Qt = ck(t) + nC + nT;
        if ((rc = step_forward_keep(c, b, Ct, Tt, Qt)) != CTM_OK) return rc;
        if ((rc = step_backward(c, b, Ct, Tt)) != CTM_OK) return rc;
    }

    // ---- layers and projection
    layers_backward_kernel<<<grid_of((long long)d * c->D * c->D * c->D), 256, 0, st>>>(d, c->D, c->A, b.ab, b.bb,
                                                                                     b.Abar);
    CK(cudaGetLastError());
    const size_t psm = sizeof(double) * (size_t)d * c->D * c->D * c->D;
    project_backward_kernel<<<1, 256, psm, st>>>(d, c->D, c->Araw, c->A, b.Abar, dA_dev, c->cfg.symmetrize);
    CK(cudaGetLastError());
    // the context keeps the environment after the tracked steps
    CK(cudaMemcpyAsync(c->C, Ck, sizeof(double) * nC, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(c->T, Tk, sizeof(double) * nT, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(c->Q, Qk, sizeof(double) * nQ, cudaMemcpyDeviceToDevice, st));
    double E = 0.0;
    CK(cudaMemcpyAsync(&E, b.scal, sizeof(double), cudaMemcpyDeviceToHost, st));
    if ((rc = read_status(c)) != CTM_OK) return rc;
    if (!isfinite(E)) return CTM_ENONFINITE;
    if (energy_host) *energy_host = E;
    return CTM_OK;
}
