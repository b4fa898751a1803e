/*
 * ctm_oracle.c -- plain, slow, FP64 CPU oracle for one QR-based C3v CTMRG step
 * on the honeycomb lattice (arXiv 2509.05090).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU
 * baseline leg may load this library.  It shares no code with the CUDA path:
 * every loop below is written out directly from the paper's definitions, with
 * no blocking, fusion or reordering beyond pairwise contraction of a tensor
 * network.
 *
 * Threads.  Where a loop nest writes disjoint outputs, its outermost output
 * loop is shared among OpenMP threads (when built with -fopenmp).  Every output
 * element is still accumulated by one thread in the loop order written here, so
 * the results do not depend on the thread count (bit for bit).
 *
 * Index conventions (all arrays row-major double):
 *   A[s][i][j][k]            site tensor, d x D x D x D                (Fig. 1a)
 *   a[u][v][w], u = i*D + i'  double-layer tensor, D2 = D*D per leg    (Fig. 1b)
 *   C[g][h]                  corner, chi x chi                          (Fig. 3a)
 *   T[a][u][g]               edge: a = outer side (crosses the sector
 *                            boundary), u = end leg toward the apex,
 *                            g = corner side                            (Fig. 3b)
 *   M[(a,y)][(b,x)]          enlarged corner, n x n, n = chi*D2, fused
 *                            index a*D2 + y (chi index slow)            (Fig. 3c)
 *   Q[r][j]                  projector n x chi; R chi x chi             (Fig. 3d)
 *
 * Sector wiring (Fig. 1c,d; the drawings are not in the text, this is the
 * reading the tests pin with the honeycomb Ising model): a 60-degree sector is
 * a quadrant of radial dimers.  The apex dimer's outer site (tensor aB, legs
 * u, l, z) touches the ends of the two edges; its inner site (aA, legs z, x, y)
 * carries the two open legs of the new corner.  z is the radial bond.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX3(a, b, c, nb, nc) (((size_t)(a) * (nb) + (b)) * (nc) + (c))

static double *orc_alloc(size_t n)
{
    double *p = (double *)calloc(n ? n : 1, sizeof(double));
    return p;
}

/* Number of threads for the parallel loops (<= 0: the OpenMP default); returns
 * the count now in effect (1 without OpenMP). */
int orc_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* a0: C3v (A1) projection, Appendix A: A_sym = (1/|G|) sum_g T_g(A).  For the
 * trivial irrep U_g = I and real tensors, the six group elements act as the six
 * permutations of the three virtual legs.                                    */
void orc_c3v_project(int d, int D, const double *A, double *out)
{
    for (int s = 0; s < d; ++s)
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j)
                for (int k = 0; k < D; ++k) {
                    const double *As = A + (size_t)s * D * D * D;
                    double v = As[IDX3(i, j, k, D, D)] + As[IDX3(i, k, j, D, D)] +
                               As[IDX3(j, i, k, D, D)] + As[IDX3(j, k, i, D, D)] +
                               As[IDX3(k, i, j, D, D)] + As[IDX3(k, j, i, D, D)];
                    out[(size_t)s * D * D * D + IDX3(i, j, k, D, D)] = v / 6.0;
                }
}

double orc_frobenius(long n, const double *x)
{
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += x[i] * x[i];
    return sqrt(s);
}

void orc_scale(long n, double *x, double f)
{
    for (long i = 0; i < n; ++i) x[i] *= f;
}

/* ------------------------------------------------------------------------ */
/* a1: double layer, Fig. 1(b): a[(ii'),(jj'),(kk')] = sum_s K[s,i,j,k] B[s,i',j',k'].
 * K is the ket layer and B the bra layer (real tensors: B = A).  With d = 1 and
 * single physical slices this also builds the "open" layer A[s] (x) A[s'].    */
void orc_double_layer(int d, int D, const double *K, const double *B, double *a)
{
    int D2 = D * D;
    size_t D3 = (size_t)D * D * D;
    memset(a, 0, sizeof(double) * (size_t)D2 * D2 * D2);
    for (int s = 0; s < d; ++s)
        for (int i = 0; i < D; ++i)
            for (int i2 = 0; i2 < D; ++i2)
                for (int j = 0; j < D; ++j)
                    for (int j2 = 0; j2 < D; ++j2)
                        for (int k = 0; k < D; ++k)
                            for (int k2 = 0; k2 < D; ++k2) {
                                int u = i * D + i2, v = j * D + j2, w = k * D + k2;
                                a[IDX3(u, v, w, D2, D2)] +=
                                    K[s * D3 + IDX3(i, j, k, D, D)] * B[s * D3 + IDX3(i2, j2, k2, D, D)];
                            }
}

/* ------------------------------------------------------------------------ */
/* plain matrix products                                                      */
/* C[m x n] = A[m x k] B[k x n]                                               */
void orc_matmul(int m, int k, int n, const double *A, const double *B, double *C)
{
    memset(C, 0, sizeof(double) * (size_t)m * n);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m; ++i)
        for (int p = 0; p < k; ++p) {
            double aip = A[(size_t)i * k + p];
            for (int j = 0; j < n; ++j) C[(size_t)i * n + j] += aip * B[(size_t)p * n + j];
        }
}

/* C[m x n] = A^T B with A stored k x m, B stored k x n.  Each C[i][j] sums its
 * products over p in ascending order.                                        */
void orc_matmul_tn(int m, int k, int n, const double *A, const double *B, double *C)
{
    memset(C, 0, sizeof(double) * (size_t)m * n);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m; ++i)
        for (int p = 0; p < k; ++p) {
            double api = A[(size_t)p * m + i];
            for (int j = 0; j < n; ++j) C[(size_t)i * n + j] += api * B[(size_t)p * n + j];
        }
}

/* ------------------------------------------------------------------------ */
/* a2: enlarged corner, Fig. 3(c) with the sector reading above:
 *   X[a,u,l,b]  = sum_{g,h} T[a,u,g] C[g,h] T[b,l,h]
 *   Y1[a,b,z]   = sum_{u,l} X[a,u,l,b] aB[u,l,z]
 *   M[(a,y),(b,x)] = sum_z Y1[a,b,z] aA[z,x,y]                              */
void orc_enlarged_corner(int chi, int D2, const double *C, const double *T,
                         const double *aB, const double *aA, double *M)
{
    size_t n = (size_t)chi * D2;
    double *W = orc_alloc(n * chi);          /* W[a,u,h] = sum_g T[a,u,g] C[g,h] */
    double *X = orc_alloc((size_t)chi * D2 * D2 * chi);
    double *Y1 = orc_alloc((size_t)chi * chi * D2);
    orc_matmul((int)n, chi, chi, T, C, W);
#pragma omp parallel for schedule(static)
    for (int a = 0; a < chi; ++a)
        for (int u = 0; u < D2; ++u)
            for (int l = 0; l < D2; ++l)
                for (int b = 0; b < chi; ++b) {
                    double s = 0.0;
                    for (int h = 0; h < chi; ++h)
                        s += W[IDX3(a, u, h, D2, chi)] * T[IDX3(b, l, h, D2, chi)];
                    X[(((size_t)a * D2 + u) * D2 + l) * chi + b] = s;
                }
#pragma omp parallel for schedule(static)
    for (int a = 0; a < chi; ++a)
        for (int b = 0; b < chi; ++b)
            for (int z = 0; z < D2; ++z) {
                double s = 0.0;
                for (int u = 0; u < D2; ++u)
                    for (int l = 0; l < D2; ++l)
                        s += X[(((size_t)a * D2 + u) * D2 + l) * chi + b] * aB[IDX3(u, l, z, D2, D2)];
                Y1[IDX3(a, b, z, chi, D2)] = s;
            }
#pragma omp parallel for schedule(static)
    for (int a = 0; a < chi; ++a)
        for (int y = 0; y < D2; ++y)
            for (int b = 0; b < chi; ++b)
                for (int x = 0; x < D2; ++x) {
                    double s = 0.0;
                    for (int z = 0; z < D2; ++z)
                        s += Y1[IDX3(a, b, z, chi, D2)] * aA[IDX3(z, x, y, D2, D2)];
                    M[((size_t)a * D2 + y) * n + (size_t)b * D2 + x] = s;
                }
    free(W);
    free(X);
    free(Y1);
}

/* ------------------------------------------------------------------------ */
/* a4: Householder QR of Y (n x k, n >= k), Fig. 3(d).  Returns the thin factors
 * Q (n x k, orthonormal columns) and R (k x k, upper triangular), then fixes the
 * gauge so that diag(R) >= 0 (sign(0) = +1): Q <- Q S, R <- S R.
 * Unblocked: one reflector per column, applied to the remaining columns, then
 * Q = H_0 H_1 ... H_{k-1} [I; 0] by backward accumulation.                  */
void orc_householder_qr(int n, int k, const double *Y, double *Q, double *R)
{
    double *A = orc_alloc((size_t)n * k);
    double *V = orc_alloc((size_t)n * k);    /* V[:, j] reflector j (rows >= j) */
    double *tau = orc_alloc((size_t)k);
    memcpy(A, Y, sizeof(double) * (size_t)n * k);
    for (int j = 0; j < k; ++j) {
        double nrm2 = 0.0;
        for (int r = j; r < n; ++r) nrm2 += A[(size_t)r * k + j] * A[(size_t)r * k + j];
        double nrm = sqrt(nrm2);
        if (nrm == 0.0) {
            tau[j] = 0.0;
            continue;
        }
        double x0 = A[(size_t)j * k + j];
        double alpha = (x0 >= 0.0) ? -nrm : nrm;   /* reflect x onto alpha e_0 */
        double vtv = 0.0;
        for (int r = j; r < n; ++r) {
            double v = A[(size_t)r * k + j] - (r == j ? alpha : 0.0);
            V[(size_t)r * k + j] = v;
            vtv += v * v;
        }
        tau[j] = 2.0 / vtv;
        /* each column is updated by one thread in the written order (bit-identical for any
         * thread count) */
#pragma omp parallel for schedule(static)
        for (int c = j; c < k; ++c) {
            double w = 0.0;
            for (int r = j; r < n; ++r) w += V[(size_t)r * k + j] * A[(size_t)r * k + c];
            for (int r = j; r < n; ++r) A[(size_t)r * k + c] -= tau[j] * w * V[(size_t)r * k + j];
        }
    }
    /* R = upper triangle */
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) R[(size_t)i * k + j] = (j >= i) ? A[(size_t)i * k + j] : 0.0;
    /* Q = H_0 ... H_{k-1} E, E = first k columns of I_n */
    memset(Q, 0, sizeof(double) * (size_t)n * k);
    for (int j = 0; j < k; ++j) Q[(size_t)j * k + j] = 1.0;
    for (int j = k - 1; j >= 0; --j) {
        if (tau[j] == 0.0) continue;
#pragma omp parallel for schedule(static)
        for (int c = 0; c < k; ++c) {
            double w = 0.0;
            for (int r = j; r < n; ++r) w += V[(size_t)r * k + j] * Q[(size_t)r * k + c];
            for (int r = j; r < n; ++r) Q[(size_t)r * k + c] -= tau[j] * w * V[(size_t)r * k + j];
        }
    }
    /* gauge: diag(R) >= 0 */
    for (int j = 0; j < k; ++j) {
        if (R[(size_t)j * k + j] < 0.0) {
            for (int r = 0; r < n; ++r) Q[(size_t)r * k + j] = -Q[(size_t)r * k + j];
            for (int c = 0; c < k; ++c) R[(size_t)j * k + c] = -R[(size_t)j * k + c];
        }
    }
    free(A);
    free(V);
    free(tau);
}

/* ------------------------------------------------------------------------ */
/* a5: corner renormalisation, Fig. 3(a): C' = Q^T M Q, then the mirror
 * re-symmetrisation C' <- (C' + C'^T)/2 and unit Frobenius norm.  Returns the
 * norm before normalisation.                                                 */
double orc_corner_update(int n, int chi, const double *M, const double *Q, double *Cn)
{
    double *MQ = orc_alloc((size_t)n * chi);
    double *Cr = orc_alloc((size_t)chi * chi);
    orc_matmul(n, n, chi, M, Q, MQ);
    orc_matmul_tn(chi, n, chi, Q, MQ, Cr);
    for (int i = 0; i < chi; ++i)
        for (int j = 0; j < chi; ++j)
            Cn[(size_t)i * chi + j] = 0.5 * (Cr[(size_t)i * chi + j] + Cr[(size_t)j * chi + i]);
    double nrm = orc_frobenius((long)chi * chi, Cn);
    if (nrm > 0.0) orc_scale((long)chi * chi, Cn, 1.0 / nrm);
    free(MQ);
    free(Cr);
    return nrm;
}

/* Cheap corner variant: the QR of the reduced corner Y = M Q_prev S gives
 * Q^T M Q_prev = R S (S = diag(sgn Cprev_jj), sgn(0) = +1), which is Q^T M Q once
 * Q = Q_prev; C' = sym(R S), unit Frobenius norm.  Returns the norm before
 * normalisation.                                                             */
double orc_corner_from_r(int chi, const double *R, const double *Cprev, double *Cn)
{
    for (int i = 0; i < chi; ++i)
        for (int j = 0; j < chi; ++j) {
            double si = Cprev[(size_t)i * chi + i] < 0.0 ? -1.0 : 1.0;
            double sj = Cprev[(size_t)j * chi + j] < 0.0 ? -1.0 : 1.0;
            Cn[(size_t)i * chi + j] = 0.5 * (R[(size_t)i * chi + j] * sj + R[(size_t)j * chi + i] * si);
        }
    double nrm = orc_frobenius((long)chi * chi, Cn);
    if (nrm > 0.0) orc_scale((long)chi * chi, Cn, 1.0 / nrm);
    return nrm;
}

/* ------------------------------------------------------------------------ */
/* a6: edge renormalisation, Fig. 3(b).  The edge grows by one radial dimer at
 * its apex end; both of its long sides are compressed with the same Q:
 *   T'[i,x,j] = sum Q[(a,y),i] T[a,u,g] aB[u,w,z] aA[z,x,y] Q[(g,w),j]
 * evaluated pairwise as
 *   H1[a,u,w,j] = sum_g T[a,u,g] Q[(g,w),j]
 *   H2[a,j,z]   = sum_{u,w} H1[a,u,w,j] aB[u,w,z]
 *   H3[a,j,x,y] = sum_z H2[a,j,z] aA[z,x,y]
 *   T'[i,x,j]   = sum_{a,y} Q[(a,y),i] H3[a,j,x,y]
 * then unit Frobenius norm.  Returns the norm before normalisation.           */
double orc_edge_update(int chi, int D2, const double *T, const double *aB, const double *aA,
                       const double *Q, double *Tn)
{
    size_t n = (size_t)chi * D2;
    double *H1 = orc_alloc((size_t)chi * D2 * D2 * chi);
    double *H2 = orc_alloc((size_t)chi * chi * D2);
    double *H3 = orc_alloc((size_t)chi * chi * D2 * D2);
#pragma omp parallel for schedule(static)
    for (int a = 0; a < chi; ++a)
        for (int u = 0; u < D2; ++u)
            for (int w = 0; w < D2; ++w)
                for (int j = 0; j < chi; ++j) {
                    double s = 0.0;
                    for (int g = 0; g < chi; ++g)
                        s += T[IDX3(a, u, g, D2, chi)] * Q[((size_t)g * D2 + w) * chi + j];
                    H1[(((size_t)a * D2 + u) * D2 + w) * chi + j] = s;
                }
#pragma omp parallel for schedule(static)
    for (int a = 0; a < chi; ++a)
        for (int j = 0; j < chi; ++j)
            for (int z = 0; z < D2; ++z) {
                double s = 0.0;
                for (int u = 0; u < D2; ++u)
                    for (int w = 0; w < D2; ++w)
                        s += H1[(((size_t)a * D2 + u) * D2 + w) * chi + j] * aB[IDX3(u, w, z, D2, D2)];
                H2[IDX3(a, j, z, chi, D2)] = s;
            }
#pragma omp parallel for schedule(static)
    for (int a = 0; a < chi; ++a)
        for (int j = 0; j < chi; ++j)
            for (int x = 0; x < D2; ++x)
                for (int y = 0; y < D2; ++y) {
                    double s = 0.0;
                    for (int z = 0; z < D2; ++z) s += H2[IDX3(a, j, z, chi, D2)] * aA[IDX3(z, x, y, D2, D2)];
                    H3[(((size_t)a * chi + j) * D2 + x) * D2 + y] = s;
                }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < chi; ++i)
        for (int x = 0; x < D2; ++x)
            for (int j = 0; j < chi; ++j) {
                double s = 0.0;
                for (int a = 0; a < chi; ++a)
                    for (int y = 0; y < D2; ++y)
                        s += Q[((size_t)a * D2 + y) * chi + i] * H3[(((size_t)a * chi + j) * D2 + x) * D2 + y];
                Tn[IDX3(i, x, j, D2, chi)] = s;
            }
    double nrm = orc_frobenius((long)(chi * (size_t)D2 * chi), Tn);
    if (nrm > 0.0) orc_scale((long)(chi * (size_t)D2 * chi), Tn, 1.0 / nrm);
    (void)n;
    free(H1);
    free(H2);
    free(H3);
    return nrm;
}

/* ------------------------------------------------------------------------ */
/* Transfer matrix of the converged environment (Sec. II.C, Fig. 4a).  With the
 * sector reading above every sector is a quadrant of an effective square lattice
 * of radial dimers d[u,w,x,y] = sum_z aB[u,w,z] aA[z,x,y], and the edge T is a
 * half-infinite strip of it.  One column of the plane is an edge, one dimer and
 * the opposite edge; it maps the boundary index (g,w,h) on one side to (a,y,b)
 * on the other, one Bravais vector along the edge direction:
 *   TM[(a,y,b),(g,w,h)] = sum_{u,x,z} T[a,u,g] aB[u,w,z] aA[z,x,y] T[b,x,h].
 * Index fusion: (a,y,b) -> (a*D2 + y)*chi + b.
 *
 * orc_transfer_apply: out = TM v for v[g][w][h], pairwise in the order
 *   P1[a,u,w,h] = sum_g T[a,u,g] v[g,w,h]
 *   P2[a,h,z]   = sum_{u,w} P1[a,u,w,h] aB[u,w,z]
 *   P3[a,x,y,h] = sum_z P2[a,h,z] aA[z,x,y]
 *   out[a,y,b]  = sum_{x,h} P3[a,x,y,h] T[b,x,h].                             */
void orc_transfer_apply(int chi, int D2, const double *T, const double *aB, const double *aA, const double *v,
                        double *out)
{
    size_t cd = (size_t)chi * D2;
    double *P1 = orc_alloc(cd * D2 * chi);
    double *P2 = orc_alloc((size_t)chi * chi * D2);
    double *P3 = orc_alloc(cd * D2 * chi);
#pragma omp parallel for schedule(static)
    for (int a = 0; a < chi; ++a)
        for (int u = 0; u < D2; ++u)
            for (int w = 0; w < D2; ++w)
                for (int h = 0; h < chi; ++h) {
                    double s = 0.0;
                    for (int g = 0; g < chi; ++g) s += T[IDX3(a, u, g, D2, chi)] * v[IDX3(g, w, h, D2, chi)];
                    P1[(((size_t)a * D2 + u) * D2 + w) * chi + h] = s;
                }
#pragma omp parallel for schedule(static)
    for (int a = 0; a < chi; ++a)
        for (int h = 0; h < chi; ++h)
            for (int z = 0; z < D2; ++z) {
                double s = 0.0;
                for (int u = 0; u < D2; ++u)
                    for (int w = 0; w < D2; ++w)
                        s += P1[(((size_t)a * D2 + u) * D2 + w) * chi + h] * aB[IDX3(u, w, z, D2, D2)];
                P2[IDX3(a, h, z, chi, D2)] = s;
            }
#pragma omp parallel for schedule(static)
    for (int a = 0; a < chi; ++a)
        for (int x = 0; x < D2; ++x)
            for (int y = 0; y < D2; ++y)
                for (int h = 0; h < chi; ++h) {
                    double s = 0.0;
                    for (int z = 0; z < D2; ++z) s += P2[IDX3(a, h, z, chi, D2)] * aA[IDX3(z, x, y, D2, D2)];
                    P3[(((size_t)a * D2 + x) * D2 + y) * chi + h] = s;
                }
#pragma omp parallel for schedule(static)
    for (int a = 0; a < chi; ++a)
        for (int y = 0; y < D2; ++y)
            for (int b = 0; b < chi; ++b) {
                double s = 0.0;
                for (int x = 0; x < D2; ++x)
                    for (int h = 0; h < chi; ++h)
                        s += P3[(((size_t)a * D2 + x) * D2 + y) * chi + h] * T[IDX3(b, x, h, D2, chi)];
                out[IDX3(a, y, b, D2, chi)] = s;
            }
    free(P1);
    free(P2);
    free(P3);
}

/* The dense transfer matrix (small cases): column c of TM is TM e_c.          */
void orc_transfer_matrix(int chi, int D2, const double *T, const double *aB, const double *aA, double *TM)
{
    size_t N = (size_t)chi * D2 * chi;
    double *e = orc_alloc(N), *col = orc_alloc(N);
    for (size_t c = 0; c < N; ++c) {
        memset(e, 0, sizeof(double) * N);
        e[c] = 1.0;
        orc_transfer_apply(chi, D2, T, aB, aA, e, col);
        for (size_t r = 0; r < N; ++r) TM[r * N + c] = col[r];
    }
    free(e);
    free(col);
}

/* ------------------------------------------------------------------------ */
/* Symmetric eigen-decomposition by the cyclic Jacobi method (rotations in row
 * order, sweeps until the off-diagonal mass is negligible).  w gets the
 * eigenvalues (unsorted), V (may be NULL) the eigenvectors as columns.        */
int orc_sym_eig(int n, const double *S, double *w, double *V)
{
    double *A = orc_alloc((size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) A[(size_t)i * n + j] = 0.5 * (S[(size_t)i * n + j] + S[(size_t)j * n + i]);
    if (V) {
        memset(V, 0, sizeof(double) * (size_t)n * n);
        for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    }
    int sweep;
    for (sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double x = A[(size_t)i * n + j] * A[(size_t)i * n + j];
                tot += x;
                if (i != j) off += x;
            }
        if (off <= 1e-34 * tot || off == 0.0) break;
        int rotated = 0;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[(size_t)p * n + q];
                double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                /* an off-diagonal entry below half an ulp of the diagonal pair is
                 * already zero to working precision */
                if (fabs(apq) <= 1.1e-16 * sqrt(fabs(app * aqq)) || apq == 0.0) continue;
                rotated = 1;
                /* rotation angle that zeroes A[p][q]: tan(2 theta) = 2 apq / (aqq - app) */
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int r = 0; r < n; ++r) { /* columns p, q */
                    double arp = A[(size_t)r * n + p], arq = A[(size_t)r * n + q];
                    A[(size_t)r * n + p] = c * arp - s * arq;
                    A[(size_t)r * n + q] = s * arp + c * arq;
                }
                for (int r = 0; r < n; ++r) { /* rows p, q */
                    double apr = A[(size_t)p * n + r], aqr = A[(size_t)q * n + r];
                    A[(size_t)p * n + r] = c * apr - s * aqr;
                    A[(size_t)q * n + r] = s * apr + c * aqr;
                }
                if (V)
                    for (int r = 0; r < n; ++r) {
                        double vrp = V[(size_t)r * n + p], vrq = V[(size_t)r * n + q];
                        V[(size_t)r * n + p] = c * vrp - s * vrq;
                        V[(size_t)r * n + q] = s * vrp + c * vrq;
                    }
            }
        if (!rotated) break;
    }
    for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
    free(A);
    return sweep;
}

/* a7: corner spectrum for the convergence test: singular values of the
 * symmetric corner (= |eigenvalues|), sorted descending, unit 2-norm.         */
void orc_corner_spectrum(int chi, const double *C, double *s)
{
    double *w = orc_alloc((size_t)chi);
    orc_sym_eig(chi, C, w, NULL);
    for (int i = 0; i < chi; ++i) w[i] = fabs(w[i]);
    for (int i = 0; i < chi; ++i) /* selection sort, descending */
        for (int j = i + 1; j < chi; ++j)
            if (w[j] > w[i]) {
                double t = w[i];
                w[i] = w[j];
                w[j] = t;
            }
    double nrm = 0.0;
    for (int i = 0; i < chi; ++i) nrm += w[i] * w[i];
    nrm = sqrt(nrm);
    for (int i = 0; i < chi; ++i) s[i] = nrm > 0.0 ? w[i] / nrm : 0.0;
    free(w);
}

/* ------------------------------------------------------------------------ */
/* Conventional projector, Fig. 3(c) (cross-check only): the chi eigenvectors of
 * the symmetric enlarged corner with the largest |eigenvalue|; each column's
 * largest-magnitude entry is made positive.                                  */
void orc_evd_projector(int n, int chi, const double *M, double *P)
{
    double *w = orc_alloc((size_t)n);
    double *V = orc_alloc((size_t)n * n);
    int *idx = (int *)calloc((size_t)n, sizeof(int));
    orc_sym_eig(n, M, w, V);
    for (int i = 0; i < n; ++i) idx[i] = i;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (fabs(w[idx[j]]) > fabs(w[idx[i]])) {
                int t = idx[i];
                idx[i] = idx[j];
                idx[j] = t;
            }
    for (int c = 0; c < chi; ++c) {
        int e = idx[c];
        int imax = 0;
        for (int r = 0; r < n; ++r)
            if (fabs(V[(size_t)r * n + e]) > fabs(V[(size_t)imax * n + e])) imax = r;
        double sg = V[(size_t)imax * n + e] < 0.0 ? -1.0 : 1.0;
        for (int r = 0; r < n; ++r) P[(size_t)r * chi + c] = sg * V[(size_t)r * n + e];
    }
    free(w);
    free(V);
    free(idx);
}

/* ------------------------------------------------------------------------ */
/* a8: nearest-neighbour reduced density matrix, Eq. (1) and Fig. 5(b).  The
 * plane is six sectors; one sector's apex dimer (inner site A, outer site B)
 * has its physical legs open.  With the projector Q of the current
 * environment, Ch = sym(Q^T M Q) and Coo[ss'] = Q^T M^{oo}[ss'] Q,
 *   rho[(sA,sB),(sA',sB')] = tr(Ch^5 Coo) / sum_{sA,sB} tr(Ch^5 Coo[(sA sB),(sA sB)]).
 * M^{oo} is the enlarged corner built with the open layers
 * A[sB] (x) A[sB'] on the outer site and A[sA] (x) A[sA'] on the inner site.
 * A is the (projected, normalised) single-layer tensor.  rho is d^2 x d^2.   */
void orc_rho(int d, int D, int chi, const double *A, const double *C, const double *T,
             const double *Q, double *rho)
{
    int D2 = D * D;
    size_t n = (size_t)chi * D2;
    size_t D3 = (size_t)D * D * D;
    size_t D6 = (size_t)D2 * D2 * D2;
    double *a = orc_alloc(D6);
    double *M = orc_alloc(n * n);
    double *MQ = orc_alloc(n * chi);
    double *Ch = orc_alloc((size_t)chi * chi);
    double *Cr = orc_alloc((size_t)chi * chi);
    double *P5 = orc_alloc((size_t)chi * chi);
    double *tmp = orc_alloc((size_t)chi * chi);
    double *bA = orc_alloc(D6), *bB = orc_alloc(D6);
    orc_double_layer(d, D, A, A, a);
    orc_enlarged_corner(chi, D2, C, T, a, a, M);
    orc_matmul((int)n, (int)n, chi, M, Q, MQ);
    orc_matmul_tn(chi, (int)n, chi, Q, MQ, Cr);
    for (int i = 0; i < chi; ++i)
        for (int j = 0; j < chi; ++j)
            Ch[(size_t)i * chi + j] = 0.5 * (Cr[(size_t)i * chi + j] + Cr[(size_t)j * chi + i]);
    double nrm = orc_frobenius((long)chi * chi, Ch);
    orc_scale((long)chi * chi, Ch, 1.0 / nrm);
    /* P5 = Ch^5 */
    memcpy(P5, Ch, sizeof(double) * chi * chi);
    for (int p = 0; p < 4; ++p) {
        orc_matmul(chi, chi, chi, P5, Ch, tmp);
        memcpy(P5, tmp, sizeof(double) * chi * chi);
    }
    int dd = d * d;
    for (int sA = 0; sA < d; ++sA)
        for (int sB = 0; sB < d; ++sB)
            for (int tA = 0; tA < d; ++tA)
                for (int tB = 0; tB < d; ++tB) {
                    orc_double_layer(1, D, A + sA * D3, A + tA * D3, bA);
                    orc_double_layer(1, D, A + sB * D3, A + tB * D3, bB);
                    orc_enlarged_corner(chi, D2, C, T, bB, bA, M);
                    orc_matmul((int)n, (int)n, chi, M, Q, MQ);
                    orc_matmul_tn(chi, (int)n, chi, Q, MQ, Cr); /* Coo */
                    double tr = 0.0;
                    for (int i = 0; i < chi; ++i)
                        for (int j = 0; j < chi; ++j) tr += P5[(size_t)i * chi + j] * Cr[(size_t)j * chi + i];
                    rho[(size_t)(sA * d + sB) * dd + (tA * d + tB)] = tr;
                }
    double z = 0.0;
    for (int i = 0; i < dd; ++i) z += rho[(size_t)i * dd + i];
    for (int i = 0; i < dd * dd; ++i) rho[i] /= z;
    free(a);
    free(M);
    free(MQ);
    free(Ch);
    free(Cr);
    free(P5);
    free(tmp);
    free(bA);
    free(bB);
}
