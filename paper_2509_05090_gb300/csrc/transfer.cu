// Transfer-matrix spectrum of the environment (Sec. II.C, Fig. 4a, Eq. 3).
//
// Every sector is a quadrant of an effective square lattice of radial dimers
// d[u,w,x,y] = sum_z aB[u,w,z] aA[z,x,y] and the edge T a half-infinite strip of
// it, so one column of the plane -- an edge, one dimer, the opposite edge -- is
//   TM[(a,y,b),(g,w,h)] = sum_{u,x,z} T[a,u,g] aB[u,w,z] aA[z,x,y] T[b,x,h],
// a (chi D2 chi)-square matrix that advances one Bravais vector along the edge.
// Its leading eigenvalues give the correlation length xi = -1/ln(lambda_1) and
// the gap ln(lambda_1/lambda_2) of the finite-correlation-length extrapolation
// (lambda_i = |lambda_i'| / |lambda_0'|).
//
// The matrix is never formed.  TM v is four contractions through the step's
// contraction engine (FP64 or split-BF16, the context's precision):
//   P1[a,u,(w,h)] = T[(a,u),g] v[g,(w,h)]          (the context's X buffer)
//   P2[(a,h),z]   = P1[a,u,w,h] aB[(u,w),z]        (Y1)
//   P3[a,y,x,h]   = P2[(a,h),z] aA[z,(x,y)]        (H; written in the order step 4 reads)
//   out[(a,y),b]  = P3[(a,y),(x,h)] T[b,(x,h)]
// Subspace iteration keeps m vectors orthonormal (Cholesky QR, twice, through the
// FP64 GEMM); every few iterations the Rayleigh quotient H = V^T TM V (m x m) is
// reduced to Hessenberg form and its eigenvalues found by complex-shifted QR
// iterations in one device thread, and the iteration stops when the leading
// magnitudes, normalised by the largest, change by less than the tolerance.
#include <math.h>

#include "ctm_ctx.h"

#define CK(expr)                                 \
    do {                                         \
        cudaError_t _e = (expr);                 \
        if (_e != cudaSuccess) return CTM_ECUDA; \
    } while (0)

namespace {

constexpr int TR_MAXV = SUBSPACE_MAXV;

struct cplx {
    double re, im;
};
__device__ inline cplx cadd(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
__device__ inline cplx csub(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
__device__ inline cplx cmul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ inline cplx cconj(cplx a) { return {a.re, -a.im}; }
__device__ inline double cabs2(cplx a) { return a.re * a.re + a.im * a.im; }
__device__ inline cplx csqrt_(cplx a)
{
    const double r = sqrt(sqrt(cabs2(a)));
    const double t = 0.5 * atan2(a.im, a.re);
    return {r * cos(t), r * sin(t)};
}

// Uniform [-1, 1) from a counter (splitmix64 finaliser): deterministic start vectors.
__device__ inline double hash_uniform(unsigned long long i)
{
    unsigned long long z = i + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

__global__ void tr_init_kernel(long long count, double *V)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
         t += (long long)gridDim.x * blockDim.x)
        V[t] = hash_uniform((unsigned long long)t);
}

// G = R^T R (Cholesky, R upper) of the m x m Gram matrix, then Rinv = R^-1.  A
// non-positive pivot (dependent vectors) is replaced by a tiny positive one so the
// iteration continues; flag[0] counts such pivots.
__global__ void tr_chol_kernel(int m, const double *G, double *Rinv, int *flag)
{
    if (threadIdx.x != 0) return;
    double R[TR_MAXV][TR_MAXV], X[TR_MAXV][TR_MAXV];
    double scale = 0.0;
    for (int i = 0; i < m; ++i) scale = fmax(scale, G[i * m + i]);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) R[i][j] = 0.0;
    for (int j = 0; j < m; ++j) {
        double s = G[j * m + j];
        for (int k = 0; k < j; ++k) s -= R[k][j] * R[k][j];
        if (!(s > 1e-28 * scale)) {
            s = 1e-28 * (scale > 0.0 ? scale : 1.0);
            atomicAdd(flag, 1);
        }
        R[j][j] = sqrt(s);
        for (int i = j + 1; i < m; ++i) {
            double t = G[j * m + i];
            for (int k = 0; k < j; ++k) t -= R[k][j] * R[k][i];
            R[j][i] = t / R[j][j];
        }
    }
    for (int j = m - 1; j >= 0; --j)   // back substitution, column by column of the inverse
        for (int i = m - 1; i >= 0; --i) {
            double t = (i == j) ? 1.0 : 0.0;
            for (int k = i + 1; k < m; ++k) t -= R[i][k] * X[k][j];
            X[i][j] = (i <= j) ? t / R[i][i] : 0.0;
        }
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) Rinv[i * m + j] = X[i][j];
}

// Eigenvalue magnitudes of the m x m matrix H (descending) into lam[0..m).
// Householder reduction to upper Hessenberg form, then QR iterations on the complex
// Hessenberg matrix with the Wilkinson shift of the trailing 2 x 2 block (the
// eigenvalue nearer the corner entry), a Givens rotation per subdiagonal entry,
// and deflation once a subdiagonal entry is negligible against its neighbours.
__global__ void tr_eig_kernel(int m, const double *Hin, double *lam, int *flag)
{
    if (threadIdx.x != 0) return;
    double A[TR_MAXV][TR_MAXV];
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) A[i][j] = Hin[i * m + j];
    for (int k = 0; k + 2 < m; ++k) {   // Hessenberg: zero A[k+2..][k]
        double nrm = 0.0;
        for (int i = k + 1; i < m; ++i) nrm += A[i][k] * A[i][k];
        nrm = sqrt(nrm);
        if (nrm == 0.0) continue;
        double v[TR_MAXV];
        const double alpha = A[k + 1][k] >= 0.0 ? -nrm : nrm;
        for (int i = 0; i < m; ++i) v[i] = 0.0;
        v[k + 1] = A[k + 1][k] - alpha;
        for (int i = k + 2; i < m; ++i) v[i] = A[i][k];
        double vv = 0.0;
        for (int i = k + 1; i < m; ++i) vv += v[i] * v[i];
        if (vv == 0.0) continue;
        const double tau = 2.0 / vv;
        for (int j = 0; j < m; ++j) {   // A <- (I - tau v v^T) A
            double s = 0.0;
            for (int i = k + 1; i < m; ++i) s += v[i] * A[i][j];
            s *= tau;
            for (int i = k + 1; i < m; ++i) A[i][j] -= s * v[i];
        }
        for (int i = 0; i < m; ++i) {   // A <- A (I - tau v v^T)
            double s = 0.0;
            for (int j = k + 1; j < m; ++j) s += A[i][j] * v[j];
            s *= tau;
            for (int j = k + 1; j < m; ++j) A[i][j] -= s * v[j];
        }
    }
    cplx Z[TR_MAXV][TR_MAXV];
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) Z[i][j] = {(j + 1 >= i) ? A[i][j] : 0.0, 0.0};
    double out[TR_MAXV];
    int hi = m - 1, iters = 0;
    while (hi >= 0) {
        if (hi == 0) {
            out[0] = sqrt(cabs2(Z[0][0]));
            break;
        }
        // deflation: the lowest negligible subdiagonal entry at or above hi
        int lo = hi;
        while (lo > 0) {
            const double s = sqrt(cabs2(Z[lo - 1][lo - 1])) + sqrt(cabs2(Z[lo][lo]));
            const double sub = sqrt(cabs2(Z[lo][lo - 1]));
            if (sub <= 2.3e-16 * s || sub == 0.0) {
                Z[lo][lo - 1] = {0.0, 0.0};
                break;
            }
            --lo;
        }
        if (lo == hi) {   // Z[hi][hi] is an eigenvalue
            out[hi] = sqrt(cabs2(Z[hi][hi]));
            --hi;
            iters = 0;
            continue;
        }
        if (++iters > 400) {   // no convergence: report the diagonal as it stands
            for (int i = 0; i <= hi; ++i) out[i] = sqrt(cabs2(Z[i][i]));
            atomicAdd(flag, 1);
            break;
        }
        // Wilkinson shift from the trailing 2 x 2 block of the active window
        const cplx a = Z[hi - 1][hi - 1], b = Z[hi - 1][hi], c = Z[hi][hi - 1], d = Z[hi][hi];
        const cplx half_tr = {0.5 * (a.re + d.re), 0.5 * (a.im + d.im)};
        const cplx disc = csqrt_(cadd(cmul(csub(half_tr, a), csub(half_tr, a)), cmul(b, c)));
        const cplx e1 = cadd(half_tr, disc), e2 = csub(half_tr, disc);
        cplx mu = (cabs2(csub(e1, d)) < cabs2(csub(e2, d))) ? e1 : e2;
        if (iters % 11 == 10) mu = cadd(d, {sqrt(cabs2(c)), 0.0});   // exceptional shift
        for (int i = lo; i <= hi; ++i) Z[i][i] = csub(Z[i][i], mu);
        // QR of the window by Givens rotations G_k acting on rows k, k+1
        cplx cs[TR_MAXV], sn[TR_MAXV];
        for (int k = lo; k < hi; ++k) {
            const cplx x = Z[k][k], y = Z[k + 1][k];
            const double r = sqrt(cabs2(x) + cabs2(y));
            cplx cc = {1.0, 0.0}, ss = {0.0, 0.0};
            if (r > 0.0) {
                cc = {x.re / r, x.im / r};
                ss = {y.re / r, y.im / r};
            }
            cs[k] = cc;
            sn[k] = ss;
            // [conj(cc) conj(ss); -ss cc] applied to rows k, k+1 (columns k..m-1)
            for (int j = k; j < m; ++j) {
                const cplx u = Z[k][j], w = Z[k + 1][j];
                Z[k][j] = cadd(cmul(cconj(cc), u), cmul(cconj(ss), w));
                Z[k + 1][j] = csub(cmul(cc, w), cmul(ss, u));
            }
        }
        // R Q: apply the adjoint rotations on the right (columns k, k+1, rows 0..k+1)
        for (int k = lo; k < hi; ++k) {
            const cplx cc = cs[k], ss = sn[k];
            for (int i = 0; i <= k + 1 && i < m; ++i) {
                const cplx u = Z[i][k], w = Z[i][k + 1];
                Z[i][k] = cadd(cmul(u, cc), cmul(w, ss));
                Z[i][k + 1] = csub(cmul(w, cconj(cc)), cmul(u, cconj(ss)));
            }
        }
        for (int i = lo; i <= hi; ++i) Z[i][i] = cadd(Z[i][i], mu);
    }
    for (int i = 1; i < m; ++i) {   // descending (insertion sort)
        const double x = out[i];
        int j = i - 1;
        while (j >= 0 && out[j] < x) {
            out[j + 1] = out[j];
            --j;
        }
        out[j + 1] = x;
    }
    for (int i = 0; i < m; ++i) lam[i] = out[i];
}

}  // namespace

namespace ctmi {

// out = TM v (one vector of length chi D2 chi, layout [chi][D2][chi]).
static cudaError_t transfer_apply(ctm_ctx *c, const double *v, double *out)
{
    const int chi = c->chi, D2 = c->D2;
    const long long n = c->n;
    GemmF64 g;
    // P1[(a,u)][(w,h)] = sum_g T[(a,u),g] v[g,(w,h)]
    g = GemmF64{(int)n, D2 * chi, chi, c->T, idx_lin(chi), idx_lin(1), v, idx_lin((long long)D2 * chi), idx_lin(1),
                c->X, idx_lin((long long)D2 * chi), idx_lin(1), 1.0, 0.0};
    cudaError_t e = run_gemm(c, g);
    if (e != cudaSuccess) return e;
    // P2[(a,h)][z] = sum_{(u,w)} P1[a][u][w][h] aB[(u,w)][z]
    g = GemmF64{chi * chi, D2, D2 * D2, c->X, idx_split(chi, (long long)D2 * D2 * chi, 1),
                idx_split(D2, (long long)D2 * chi, chi), c->a, idx_lin(D2), idx_lin(1), c->Y1, idx_lin(D2), idx_lin(1),
                1.0, 0.0};
    if ((e = run_gemm(c, g, GEMM_B_IS_A_LZ)) != cudaSuccess) return e;
    // P3[a][y][x][h] = sum_z P2[(a,h)][z] aA[z][(x,y)]
    g = GemmF64{chi * chi, D2 * D2, D2, c->Y1, idx_lin(D2), idx_lin(1), c->a, idx_lin((long long)D2 * D2), idx_lin(1),
                c->H, idx_split(chi, (long long)D2 * D2 * chi, 1), idx_split(D2, chi, (long long)D2 * chi), 1.0, 0.0};
    if ((e = run_gemm(c, g)) != cudaSuccess) return e;
    // out[(a,y)][b] = sum_{(x,h)} P3[(a,y)][(x,h)] T[b][(x,h)]
    g = GemmF64{(int)n, chi, D2 * chi, c->H, idx_lin((long long)D2 * chi), idx_lin(1), c->T, idx_lin(1),
                idx_lin((long long)D2 * chi), out, idx_lin(chi), idx_lin(1), 1.0, 0.0};
    return run_gemm(c, g);
}

static size_t subspace_layout(long long N, int m, char *base, double **V, double **W, double **G, double **Rinv,
                              double **H, double **lam, int **flag)
{
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off += align_up(bytes);
        return p;
    };
    *V = (double *)take(sizeof(double) * (size_t)N * m);
    *W = (double *)take(sizeof(double) * (size_t)N * m);
    *G = (double *)take(sizeof(double) * m * m);
    *Rinv = (double *)take(sizeof(double) * m * m);
    *H = (double *)take(sizeof(double) * m * m);
    *lam = (double *)take(sizeof(double) * TR_MAXV);
    *flag = (int *)take(64);
    return off;
}

// V <- orthonormal basis of span(W) (Cholesky QR twice), W used as scratch.
static cudaError_t orthonormalise(const SubspaceWork &s, int m, long long N, double *W, double *V, double *G,
                                  double *Rinv, int *flag)
{
    cudaStream_t st = s.stream;
    double *src = W, *dst = V;
    for (int pass = 0; pass < 2; ++pass) {
        // G = src^T src (m x m over N), vectors stored one after another
        GemmF64 g{m, m, (int)N, src, idx_lin(N), idx_lin(1), src, idx_lin(1), idx_lin(N), G, idx_lin(m), idx_lin(1),
                  1.0, 0.0};
        cudaError_t e = gemm_f64(g, gemm_f64_pick_split(m, m, (int)N), s.splitk, s.splitk_elems, st);
        if (e != cudaSuccess) return e;
        CTM_COUNT_LAUNCH(1);
        tr_chol_kernel<<<1, 32, 0, st>>>(m, G, Rinv, flag);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        // dst = src Rinv: row r of the (N x m) matrix whose column j is vector j
        g = GemmF64{(int)N, m, m, src, idx_lin(1), idx_lin(N), Rinv, idx_lin(m), idx_lin(1), dst, idx_lin(1),
                    idx_lin(N), 1.0, 0.0};
        if ((e = gemm_f64(g, 1, s.splitk, s.splitk_elems, st)) != cudaSuccess) return e;
        double *t = src;
        src = dst;
        dst = t;
    }
    // after two passes the result is in W; copy to V
    return cudaMemcpyAsync(V, W, sizeof(double) * (size_t)N * m, cudaMemcpyDeviceToDevice, st);
}

}  // namespace ctmi

using namespace ctmi;

size_t subspace_workspace_bytes(long long N, int m)
{
    double *V, *W, *G, *Rinv, *H, *lam;
    int *flag;
    return subspace_layout(N, m, nullptr, &V, &W, &G, &Rinv, &H, &lam, &flag);
}

int subspace_spectrum(const SubspaceWork &s, long long N, int m, int nev, int pairs, int max_iter, double tol,
                      void *tws, const std::function<cudaError_t(const double *, double *)> &apply, double *mags,
                      int *iters_out)
{
    if (m < 2 || m > TR_MAXV || nev < 1 || pairs * (nev - 1) >= m || max_iter < 1) return CTM_EINVAL;
    double *V, *W, *G, *Rinv, *H, *lam;
    int *flag;
    subspace_layout(N, m, (char *)tws, &V, &W, &G, &Rinv, &H, &lam, &flag);
    cudaStream_t st = s.stream;
    CK(cudaMemsetAsync(flag, 0, sizeof(int), st));
    CTM_COUNT_LAUNCH(1);
    tr_init_kernel<<<256, 256, 0, st>>>(N * m, W);
    CK(cudaGetLastError());
    CK(orthonormalise(s, m, N, W, V, G, Rinv, flag));
    double prev[TR_MAXV], cur[TR_MAXV];
    for (int i = 0; i < m; ++i) prev[i] = -1.0;
    const int check = 5;
    int it = 0;
    bool done = false;
    while (it < max_iter && !done) {
        for (int j = 0; j < m; ++j) CK(apply(V + (size_t)j * N, W + (size_t)j * N));
        ++it;
        if (it % check == 0 || it == max_iter) {
            // Rayleigh quotient H = V^T (Op V) and its eigenvalue magnitudes
            GemmF64 g{m, m, (int)N, V, idx_lin(N), idx_lin(1), W, idx_lin(1), idx_lin(N), H, idx_lin(m), idx_lin(1),
                      1.0, 0.0};
            CK(gemm_f64(g, gemm_f64_pick_split(m, m, (int)N), s.splitk, s.splitk_elems, st));
            CTM_COUNT_LAUNCH(1);
            tr_eig_kernel<<<1, 32, 0, st>>>(m, H, lam, flag);
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(cur, lam, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
            int err = 0;
            if (s.err) CK(cudaMemcpyAsync(&err, s.err, sizeof(int), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if (err) return CTM_ETIMEOUT;
            // converged when every kept magnitude, normalised by the largest, moved by less
            // than tol (absolute: magnitudes far below lambda_0 carry FP64 noise of order
            // 1e-16 lambda_0)
            done = true;
            for (int i = 0; i < nev; ++i) {
                const int k = i * pairs;
                if (!isfinite(cur[k])) return CTM_ENONFINITE;
                const double a = cur[k] / cur[0], b = prev[k] / (prev[0] > 0.0 ? prev[0] : 1.0);
                if (!(fabs(a - b) <= tol)) done = false;
            }
            for (int i = 0; i < m; ++i) prev[i] = cur[i];
        }
        if (!done) CK(orthonormalise(s, m, N, W, V, G, Rinv, flag));
    }
    if (!(cur[0] > 0.0)) return CTM_ENONFINITE;
    for (int i = 0; i < nev; ++i) mags[i] = cur[i * pairs] / cur[0];
    if (iters_out) *iters_out = it;
    return done ? CTM_OK : CTM_ENOTCONVERGED;
}

static int transfer_vectors(int nev) { return nev + 5 < TR_MAXV ? nev + 5 : TR_MAXV; }

extern "C" size_t ctm_transfer_workspace_bytes(const ctm_ctx *c, int nev)
{
    if (!c || nev < 2 || nev > TR_MAXV - 2) return 0;
    return subspace_workspace_bytes((long long)c->chi * c->D2 * c->chi, transfer_vectors(nev));
}

extern "C" int ctm_transfer_spectrum(ctm_ctx *c, int nev, int max_iter, double tol, void *tws, size_t tws_bytes,
                                     double *lambda_host, double *xi_host, double *gap_host, int *iters_out)
{
    if (!c || !tws || !lambda_host || nev < 2 || nev > TR_MAXV - 2 || max_iter < 1) return CTM_EINVAL;
    if ((uintptr_t)tws % 256 != 0) return CTM_EINVAL;
    if (tws_bytes < ctm_transfer_workspace_bytes(c, nev)) return CTM_ENOMEM;
    if (tol <= 0.0) tol = 1e-12;
    if (join_side(c) != CTM_OK) return CTM_ECUDA;
    const long long N = (long long)c->chi * c->D2 * c->chi;
    SubspaceWork sw{c->stream, c->splitk, c->splitk_elems, c->err};
    int rc = subspace_spectrum(sw, N, transfer_vectors(nev), nev, 1, max_iter, tol, tws,
                               [c](const double *v, double *out) { return transfer_apply(c, v, out); }, lambda_host,
                               iters_out);
    if (rc != CTM_OK && rc != CTM_ENOTCONVERGED) return rc;
    if (xi_host) *xi_host = lambda_host[1] > 0.0 ? -1.0 / log(lambda_host[1]) : 0.0;
    if (gap_host) *gap_host = (nev >= 3 && lambda_host[2] > 0.0) ? log(lambda_host[1] / lambda_host[2]) : INFINITY;
    return rc;
}
