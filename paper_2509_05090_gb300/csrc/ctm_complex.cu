// Complex C3v CTMRG (App. A, Sec. II.B, Sec. III.C): site tensors symmetric under
// a complex physical representation of C3v (the E irrep of the Kitaev model, or the
// trivial A1 one), a Hermitian enlarged corner, Householder QR with real diag(R) >= 0,
// C' = sym(Q^H M Q)/|.|, T' = Q^H (T a a) Q/|.|, and the bond energies.
//
// Storage: complex tensors are planar.  A tensor that enters a contraction as the
// right operand holds four planes [Re, Im, -Im, Re] so that each complex product
// C = op(A) op(B) is two real products with the inner dimension doubled,
//   Re C = [Re A | s_A Im A] [Re B ; -s_B Im B],  Im C = [Re A | s_A Im A] [s_B Im B ; Re B]
// (s = -1 for a conjugated operand), every operand a strided view of one plane pair
// and both products sharing the packed left operand.  The complex QR is the real
// Householder QR of the 2 x 2 block embedding [[Re, -Im], [Im, Re]] of the reduced
// corner, whose unique factors (positive diagonal) are the embeddings of the complex
// Q and R; the corner spectrum comes from a Householder reduction of the Hermitian
// corner to a tridiagonal matrix and the bisection of the real path.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <array>
#include <new>
#include <vector>

#include "ctm_internal.h"

struct ctm_complex_ctx {
    ctm_config cfg;
    int irrep;
    int d, D, D2, chi;
    long long n;
    int split_T;
    int tf32_T;   // 1, 2: TF32 products (CTM_FP32_TF32, CTM_SPLIT_TF32)
    cudaStream_t stream;
    double U[3][3][2];      // the rotation paired with the leg cycle (energies of the x, y bonds)
    // planes: P_* is the plane stride of each tensor (elements)
    double *Ain, *A, *a, *aA, *bB, *bA;   // a: the outer site's layer; aA: the apex site's (z leg first)
    long long PA, Pa, Pb;
    double *C, *Cn, *Cr, *T, *Tn, *Q, *Qn, *Qs;
    long long PC, PT, PQ;
    double *Y, *W, *MQ, *R;
    long long PY;
    double *M, *X, *H;
    long long PM;
    double *Y1, *Y1o, *G2;
    long long PY1, PYo;
    double *P5a, *P5b;
    double *Yemb, *Qemb, *Remb;
    double *s, *s_new, *delta, *spec_work;
    double *spec_emb;   // chi > ZSMEM_CHI: the real 2chi x 2chi embedding of the corner
    double *splitk;
    size_t splitk_elems;
    double *qr_sbuf, *qr_rowbuf, *qr_wy;
    double *qr_gpart, *qr_spart;   // deterministic mode: per-CTA partial sums of the embedded QR
    double *qr_slab;               // the embedded QR's row blocks where they do not fit shared memory
    size_t qr_slab_elems;
    int qr_gmax;
    unsigned *qr_bar;
    int *err, *flag;
    double *norm_part;
    double *rho_part, *rho_raw, *hrot, *eout;
    SplitWork sw;
    int steps_done;
    // steps after the first (eager, autotuning) one replay a captured one-step graph
    cudaStream_t own;
    cudaEvent_t ev_in, ev_out;
    // the corner spectrum runs on a side stream beside the edge update
    cudaStream_t side;
    cudaEvent_t ev_fork, ev_join;
    cudaGraphExec_t graph1, graphK;
    unsigned long long graph1_kernels, graphK_kernels;
    int graphK_steps;
    int graph_failed;
    int side_pending;   // a corner spectrum on the side stream not yet joined into the main stream
    // pipelined converge (as in the real path): two graphs of pipe_steps steps whose
    // corner spectra are shifted by one step and whose deltas (and final error flag)
    // go to pinned host memory, ring half 0 and half 1
    cudaGraphExec_t pipe[2];
    int pipe_steps;
    unsigned long long pipe_kernels;
    cudaEvent_t pipe_done[2];
    double *ring_h;
    int *ring_err_h;
    int ring_cap;
    int spec_head, spec_skip;           // while capturing them: see zstep
    double *delta_head, *delta_dst;
};

namespace {

constexpr int ZMAX_D = 3;
// the Hermitian corner of the one-CTA spectrum kernel (two planes) fits one SM's shared
// memory up to chi = 112; beyond, the spectrum runs on the real 2chi x 2chi embedding
// through the real path's reduction (a thread-block cluster), up to chi = 256, where the
// QR of the 2n x 2chi embedding reaches its 512 columns
constexpr int ZSMEM_CHI = 112;
constexpr int ZMAX_CHI = 256;
constexpr int ZNORM_BLOCKS = 128;
constexpr int ZRHO_BLOCKS = 128;
constexpr int ZRHO_MAX_DD = 9;

struct ZGroup {
    double U[6][ZMAX_D][ZMAX_D][2];
    int perm[6][3];
    int anti[6];
};

// ------------------------------------------------------------------ host: the group
struct Cx {
    double re, im;
};
static inline Cx cmul(Cx a, Cx b) { return Cx{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
static inline Cx cadd(Cx a, Cx b) { return Cx{a.re + b.re, a.im + b.im}; }
static inline Cx cconj(Cx a) { return Cx{a.re, -a.im}; }

struct HMat {
    int d;
    Cx v[ZMAX_D][ZMAX_D];
};
static HMat hm_zero(int d)
{
    HMat m;
    m.d = d;
    for (int i = 0; i < ZMAX_D; ++i)
        for (int j = 0; j < ZMAX_D; ++j) m.v[i][j] = Cx{0.0, 0.0};
    return m;
}
static HMat hm_eye(int d)
{
    HMat m = hm_zero(d);
    for (int i = 0; i < d; ++i) m.v[i][i] = Cx{1.0, 0.0};
    return m;
}
static HMat hm_mul(const HMat &a, const HMat &b)
{
    HMat m = hm_zero(a.d);
    for (int i = 0; i < a.d; ++i)
        for (int j = 0; j < a.d; ++j)
            for (int k = 0; k < a.d; ++k) m.v[i][j] = cadd(m.v[i][j], cmul(a.v[i][k], b.v[k][j]));
    return m;
}
static HMat hm_conj(const HMat &a)
{
    HMat m = a;
    for (int i = 0; i < a.d; ++i)
        for (int j = 0; j < a.d; ++j) m.v[i][j] = cconj(a.v[i][j]);
    return m;
}
static HMat hm_scale(const HMat &a, Cx s)
{
    HMat m = a;
    for (int i = 0; i < a.d; ++i)
        for (int j = 0; j < a.d; ++j) m.v[i][j] = cmul(a.v[i][j], s);
    return m;
}
static double hm_dist(const HMat &a, const HMat &b)
{
    double m = 0.0;
    for (int i = 0; i < a.d; ++i)
        for (int j = 0; j < a.d; ++j) m = fmax(m, hypot(a.v[i][j].re - b.v[i][j].re, a.v[i][j].im - b.v[i][j].im));
    return m;
}

// Spin-S matrices in the S^z basis (m = S, S-1, ..., -S) combined along a unit vector:
// e.S = e_x S^x + e_y S^y + e_z S^z.
static HMat spin_along(int d, const double e[3])
{
    const double S = 0.5 * (d - 1);
    HMat m = hm_zero(d);
    for (int k = 0; k < d; ++k) m.v[k][k] = Cx{e[2] * (S - k), 0.0};
    for (int k = 1; k < d; ++k) {
        const double mk = S - k;
        const double sp = sqrt(S * (S + 1.0) - mk * (mk + 1.0));   // <m_k + 1| S^+ |m_k>
        // S^x = (S^+ + S^-)/2, S^y = (S^+ - S^-)/(2i)
        m.v[k - 1][k] = cadd(m.v[k - 1][k], Cx{0.5 * sp * e[0], -0.5 * sp * e[1]});
        m.v[k][k - 1] = cadd(m.v[k][k - 1], Cx{0.5 * sp * e[0], 0.5 * sp * e[1]});
    }
    return m;
}

// exp(i theta H): Taylor series of the scaled argument, then repeated squaring.
static HMat expm_i(const HMat &H, double theta)
{
    double nrm = 0.0;
    for (int i = 0; i < H.d; ++i)
        for (int j = 0; j < H.d; ++j) nrm += hypot(H.v[i][j].re, H.v[i][j].im);
    nrm *= fabs(theta);
    int sq = 0;
    while (nrm > 0.25) {
        nrm *= 0.5;
        ++sq;
    }
    const HMat X = hm_scale(H, Cx{0.0, theta / (double)(1 << sq)});
    HMat sum = hm_eye(H.d), term = hm_eye(H.d);
    for (int k = 1; k <= 24; ++k) {
        term = hm_scale(hm_mul(term, X), Cx{1.0 / k, 0.0});
        for (int i = 0; i < H.d; ++i)
            for (int j = 0; j < H.d; ++j) sum.v[i][j] = cadd(sum.v[i][j], term.v[i][j]);
    }
    for (int s = 0; s < sq; ++s) sum = hm_mul(sum, sum);
    return sum;
}

struct Elem {
    HMat U;
    int perm[3];
    int anti;
};

// g after h: U = U_g op(U_h) (op = conj when g is anti-unitary), legs perm[q] = p_h[p_g[q]].
static Elem compose(const Elem &g, const Elem &h)
{
    Elem r;
    r.U = hm_mul(g.U, g.anti ? hm_conj(h.U) : h.U);
    for (int q = 0; q < 3; ++q) r.perm[q] = h.perm[g.perm[q]];
    r.anti = g.anti ^ h.anti;
    return r;
}
static bool same(const Elem &a, const Elem &b)
{
    return a.anti == b.anti && a.perm[0] == b.perm[0] && a.perm[1] == b.perm[1] && a.perm[2] == b.perm[2] &&
           hm_dist(a.U, b.U) < 1e-12;
}

// App. A: generators of C3v acting on A[s; x, y, z].  The rotation
// U_C3 = (-1)^(d-1) e^{i 2pi/3} exp(i 2pi/3 n.S), n = (1,1,1)/sqrt 3, with the leg
// cycle out[s; i, j, k] = U A[s; k, i, j]; the reflection p_1 (normal m_1 = (1,-1,0)/sqrt 2)
// = K-hat C exp(i pi m_1.S) (anti-unitary; its phase set to 1), with the exchange of
// the x and y legs.  The other elements come from closure.  A1: U = I, no conjugation.
static bool make_group(int d, int irrep, ZGroup *grp, HMat *Urot)
{
    Elem e, r, p;
    e.U = hm_eye(d);
    e.perm[0] = 0, e.perm[1] = 1, e.perm[2] = 2;
    e.anti = 0;
    r = e;
    r.perm[0] = 1, r.perm[1] = 2, r.perm[2] = 0;
    p = e;
    p.perm[0] = 1, p.perm[1] = 0, p.perm[2] = 2;
    if (irrep == 1) {
        const double PI = 3.14159265358979323846;
        const double s3 = 1.0 / sqrt(3.0), s2 = 1.0 / sqrt(2.0);
        const double nvec[3] = {s3, s3, s3}, mvec[3] = {s2, -s2, 0.0};
        const double sgn = (d - 1) % 2 ? -1.0 : 1.0;
        r.U = hm_scale(expm_i(spin_along(d, nvec), 2.0 * PI / 3.0),
                       Cx{sgn * cos(2.0 * PI / 3.0), sgn * sin(2.0 * PI / 3.0)});
        HMat K = hm_zero(d);
        for (int q = 0; q < d; ++q) K.v[q][d - 1 - q] = Cx{(q % 2) ? -1.0 : 1.0, 0.0};
        p.U = hm_mul(K, hm_conj(expm_i(spin_along(d, mvec), PI)));
        p.anti = 1;
    }
    std::vector<Elem> el{e};
    std::vector<Elem> frontier{r, p};
    while (!frontier.empty()) {
        Elem g = frontier.back();
        frontier.pop_back();
        bool found = false;
        for (const Elem &x : el) found = found || same(g, x);
        if (found) continue;
        el.push_back(g);
        if (el.size() > 6) return false;
        const size_t cur = el.size();
        for (size_t i = 0; i < cur; ++i) {
            frontier.push_back(compose(g, el[i]));
            frontier.push_back(compose(el[i], g));
        }
    }
    if (el.size() != 6) return false;
    memset(grp, 0, sizeof(*grp));
    for (int g = 0; g < 6; ++g) {
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                grp->U[g][i][j][0] = el[g].U.v[i][j].re;
                grp->U[g][i][j][1] = el[g].U.v[i][j].im;
            }
        for (int q = 0; q < 3; ++q) grp->perm[g][q] = el[g].perm[q];
        grp->anti[g] = el[g].anti;
    }
    *Urot = r.U;
    return true;
}

// ------------------------------------------------------------------ device kernels
__device__ __forceinline__ long long zoff2(const Idx2 &x, int i)
{
    if (x.s1 == 0) return (long long)i * x.s2;
    const int hi = i / x.div;
    return (long long)hi * x.s1 + (long long)(i - hi * x.div) * x.s2;
}

int zgrid(long long count)
{
    long long b = (count + 255) / 256, cap = 8LL * device_sm_count();
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

// Layout of a planar complex tensor: element t (row-major in the complex index) sits at
// base(t) = (t / row_len) * row_stride + t % row_len, plane p at base(t) + p * P.  Two
// planes hold [Re, Im]; five hold [Re, -Im, Re, Im, Re], so that every pair a real product
// needs -- [Re ; -Im], [Im ; Re], [Re ; Im], [-Im ; Re] -- is two adjacent planes.
// "Plane-stacked": one row (row_len = count), P = count.  "Row-blocked": the planes of
// one row follow each other, P = row_len, row_stride = planes * row_len.
struct ZLay {
    long long row_len, row_stride, P;
    int planes;
};
__host__ __device__ inline ZLay zlay_stacked(long long count, int planes) { return ZLay{count, 0, count, planes}; }
__host__ __device__ inline ZLay zlay_rows(long long row_len, int planes)
{
    return ZLay{row_len, planes * row_len, row_len, planes};
}
__host__ __device__ inline long long zbase(const ZLay &L, long long t)
{
    return L.row_stride ? (t / L.row_len) * L.row_stride + t % L.row_len : t;
}
__host__ __device__ inline int zim_plane(const ZLay &L) { return L.planes == 5 ? 3 : 1; }

__device__ __forceinline__ void zstore(double *x, const ZLay &L, long long t, double re, double im)
{
    const long long b = zbase(L, t);
    if (L.planes == 5) {
        x[b] = re;
        x[b + L.P] = -im;
        x[b + 2 * L.P] = re;
        x[b + 3 * L.P] = im;
        x[b + 4 * L.P] = re;
    } else {
        x[b] = re;
        x[b + L.P] = im;
    }
}

// interleaved (re, im) -> the layout L
__global__ void zc_load_kernel(long long count, const double *src, double *dst, ZLay L)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
         t += (long long)gridDim.x * blockDim.x)
        zstore(dst, L, t, src[2 * t], src[2 * t + 1]);
}

// the layout L -> interleaved
__global__ void zc_interleave_kernel(long long count, const double *src, ZLay L, double *dst)
{
    const int ip = zim_plane(L);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
         t += (long long)gridDim.x * blockDim.x) {
        const long long b = zbase(L, t);
        dst[2 * t] = src[b];
        dst[2 * t + 1] = src[b + ip * L.P];
    }
}

// the other planes of a five-plane tensor from its Re (0) and Im (3) planes
__global__ void zc_complete_kernel(long long count, double *x, ZLay L)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
         t += (long long)gridDim.x * blockDim.x) {
        const long long b = zbase(L, t);
        zstore(x, L, t, x[b], x[b + 3 * L.P]);
    }
}

// App. A: out[s; i0, i1, i2] = (1/6) sum_g sum_t U_g[s, t] X_g[t; legs], X_g = conj(A) for an
// anti-unitary g, and A's leg perm_g[q] carries i_q.
__global__ void zc_project_kernel(int d, int D, const double *A, long long P, ZGroup grp, int symmetrize,
                                  double *out, long long Po)
{
    const int D3 = D * D * D;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < d * D3; t += gridDim.x * blockDim.x) {
        const int s = t / D3, r = t - s * D3;
        if (!symmetrize) {
            out[t] = A[t];
            out[Po + t] = A[P + t];
            continue;
        }
        const int iv[3] = {r / (D * D), (r / D) % D, r % D};
        double re = 0.0, im = 0.0;
        for (int g = 0; g < 6; ++g) {
            int l[3];
            for (int q = 0; q < 3; ++q) l[grp.perm[g][q]] = iv[q];
            const int off = (l[0] * D + l[1]) * D + l[2];
            const double sg = grp.anti[g] ? -1.0 : 1.0;
            for (int u = 0; u < d; ++u) {
                const double ar = A[u * D3 + off], ai = sg * A[P + u * D3 + off];
                const double ur = grp.U[g][s][u][0], ui = grp.U[g][s][u][1];
                re += ur * ar - ui * ai;
                im += ur * ai + ui * ar;
            }
        }
        out[t] = re / 6.0;
        out[Po + t] = im / 6.0;
    }
}

// sum of |x|^2 over a complex tensor of layout L
__global__ void zc_sumsq_kernel(long long count, const double *x, ZLay L, double *partials)
{
    __shared__ double red[8];
    const int ip = zim_plane(L);
    double acc = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
         t += (long long)gridDim.x * blockDim.x) {
        const long long b = zbase(L, t);
        acc += x[b] * x[b] + x[b + ip * L.P] * x[b + ip * L.P];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        partials[blockIdx.x] = s;
    }
}

// x <- x / sqrt(sum of partials), every plane of layout L
__global__ void zc_scale_kernel(long long count, double *x, ZLay L, const double *partials, int nparts)
{
    __shared__ double inv;
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nparts; ++b) s += partials[b];
        inv = s > 0.0 ? 1.0 / sqrt(s) : 1.0;
    }
    __syncthreads();
    const int ip = zim_plane(L);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
         t += (long long)gridDim.x * blockDim.x) {
        const long long b = zbase(L, t);
        zstore(x, L, t, x[b] * inv, x[b + ip * L.P] * inv);
    }
}

// Fig. 1b: a[(ii'),(jj'),(kk')] = sum_s K[s,i,j,k] conj(B[s,i',j',k']) (five planes, stacked).
// rot = 1 cycles the legs of both layers so that the z leg comes first.
__device__ __forceinline__ void zc_layer_entry(int D, long long t, int rot, int &kidx, int &bidx)
{
    const int D2 = D * D;
    const int u = (int)(t / ((long long)D2 * D2)), l = (int)((t / D2) % D2), z = (int)(t % D2);
    const int i = u / D, ip = u % D, j = l / D, jp = l % D, k = z / D, kp = z % D;
    if (!rot) {
        kidx = (i * D + j) * D + k;
        bidx = (ip * D + jp) * D + kp;
    } else {   // legs (z, x, y): the first index is the z leg of A
        kidx = (j * D + k) * D + i;
        bidx = (jp * D + kp) * D + ip;
    }
}

__global__ void zc_double_layer_kernel(int d, int D, const double *A, long long PA, int rot, double *a)
{
    const long long D6 = (long long)D * D * D * D * D * D;
    const int D3 = D * D * D;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < D6;
         t += (long long)gridDim.x * blockDim.x) {
        int ki, bi;
        zc_layer_entry(D, t, rot, ki, bi);
        double re = 0.0, im = 0.0;
        for (int s = 0; s < d; ++s) {
            const double kr = A[s * D3 + ki], kim = A[PA + s * D3 + ki];
            const double br = A[s * D3 + bi], bim = A[PA + s * D3 + bi];
            re += kr * br + kim * bim;
            im += kim * br - kr * bim;
        }
        zstore(a, zlay_stacked(D6, 5), t, re, im);
    }
}

// open layers b[p = s*d + t][(ii'),(jj'),(kk')] = A[s, ...] conj(A[t, ...]) (five planes, stacked)
__global__ void zc_open_layers_kernel(int d, int D, const double *A, long long PA, int rot, double *b)
{
    const long long D6 = (long long)D * D * D * D * D * D;
    const int D3 = D * D * D;
    const long long tot = D6 * d * d;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(t / D6);
        const long long e = t - (long long)p * D6;
        const int s = p / d, tt = p % d;
        int ki, bi;
        zc_layer_entry(D, e, rot, ki, bi);
        const double kr = A[s * D3 + ki], kim = A[PA + s * D3 + ki];
        const double br = A[tt * D3 + bi], bim = A[PA + tt * D3 + bi];
        zstore(b, zlay_stacked(tot, 5), t, kr * br + kim * bim, kim * br - kr * bim);
    }
}

// C = I, T[a][u][b] = delta_ab t_u with t_u = sum_{v,w} a[u][(vv)][(ww)], Q = first chi columns of I
// (C, Q: five planes stacked; T: five planes row-blocked by its rows (a, u))
__global__ void zc_init_env_kernel(int chi, int D, const double *a, long long Pa, double *C, double *T, double *Q)
{
    const int D2 = D * D;
    const long long n = (long long)chi * D2;
    const long long tot = (long long)chi * D2 * chi;
    const int ip = 3;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x) {
        const int al = (int)(t / ((long long)D2 * chi)), u = (int)((t / chi) % D2), be = (int)(t % chi);
        double re = 0.0, im = 0.0;
        if (al == be)
            for (int v = 0; v < D; ++v)
                for (int w = 0; w < D; ++w) {
                    const long long o = ((long long)u * D2 + v * D + v) * D2 + w * D + w;
                    re += a[o];
                    im += a[ip * Pa + o];
                }
        zstore(T, zlay_rows(chi, 5), t, re, im);
    }
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)chi * chi;
         t += (long long)gridDim.x * blockDim.x)
        zstore(C, zlay_stacked((long long)chi * chi, 5), t, (t / chi == t % chi) ? 1.0 : 0.0, 0.0);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n * chi;
         t += (long long)gridDim.x * blockDim.x)
        zstore(Q, zlay_stacked(n * chi, 5), t, (t / chi == t % chi) ? 1.0 : 0.0, 0.0);
}

// Qs = Q diag(sgn Re C_jj) (sgn 0 = +1), every plane of the five (stacked)
__global__ void zc_warm_start_kernel(long long n, int chi, const double *Q, long long PQ, const double *C, double *Qs)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n * chi;
         t += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(t % chi);
        const double sg = C[(long long)j * chi + j] < 0.0 ? -1.0 : 1.0;
        for (int p = 0; p < 5; ++p) Qs[p * PQ + t] = sg * Q[p * PQ + t];
    }
}

// The cheap corner variant: Cr = R S with S = diag(sgn Re C_jj) of the corner that entered the
// step (two planes each)
__global__ void zc_rs_kernel(int chi, const double *R, long long PR, const double *C, double *Cr, long long PCr)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < chi * chi; t += gridDim.x * blockDim.x) {
        const int j = t % chi;
        const double sg = C[(long long)j * chi + j] < 0.0 ? -1.0 : 1.0;
        Cr[t] = sg * R[t];
        Cr[PCr + t] = sg * R[PR + t];
    }
}

// E[(r,c),(j,c')] = [[Re y, -Im y], [Im y, Re y]][c][c'] (2n x 2k, row-major)
__global__ void zc_embed_kernel(long long n, int k, const double *Y, long long PY, double *E)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n * k;
         t += (long long)gridDim.x * blockDim.x) {
        const long long r = t / k;
        const int j = (int)(t % k);
        const double re = Y[t], im = Y[PY + t];
        const long long ld = 2LL * k;
        E[(2 * r) * ld + 2 * j] = re;
        E[(2 * r) * ld + 2 * j + 1] = -im;
        E[(2 * r + 1) * ld + 2 * j] = im;
        E[(2 * r + 1) * ld + 2 * j + 1] = re;
    }
}

// complex factor from the first column of each 2 x 2 block of an embedding
__global__ void zc_extract_kernel(long long n, int k, const double *E, double *Z, long long PZ, int planes)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n * k;
         t += (long long)gridDim.x * blockDim.x) {
        const long long r = t / k;
        const int j = (int)(t % k);
        const long long ld = 2LL * k;
        zstore(Z, zlay_stacked(PZ, planes), t, E[(2 * r) * ld + 2 * j], E[(2 * r + 1) * ld + 2 * j]);
    }
}

// Fig. 3a: Cn = (Cr + Cr^H)/2 normalised (five planes, stacked); one CTA.
__global__ void zc_herm_normalize_kernel(int chi, const double *Cr, long long PCr, double *Cn, long long PC)
{
    __shared__ double red[32];
    __shared__ double inv;
    const int nn = chi * chi;
    double acc = 0.0;
    for (int t = threadIdx.x; t < nn; t += blockDim.x) {
        const int i = t / chi, j = t % chi;
        const double re = 0.5 * (Cr[t] + Cr[j * chi + i]);
        const double im = 0.5 * (Cr[PCr + t] - Cr[PCr + j * chi + i]);
        acc += re * re + im * im;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        inv = s > 0.0 ? 1.0 / sqrt(s) : 1.0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nn; t += blockDim.x) {
        const int i = t / chi, j = t % chi;
        const double re = 0.5 * (Cr[t] + Cr[j * chi + i]) * inv;
        const double im = 0.5 * (Cr[PCr + t] - Cr[PCr + j * chi + i]) * inv;
        zstore(Cn, zlay_stacked(PC, 5), t, re, im);
    }
}

// Sum over the CTA of one value per thread (blockDim a multiple of 32, <= 1024).
__device__ double zblock_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < nw; ++i) s += red[i];
        red[32] = s;
    }
    __syncthreads();
    return red[32];
}

// The corner spectrum, step one: Householder reduction of the Hermitian corner (Re in plane
// 0, Im in plane 3 of its five planes) to tridiagonal form in one CTA's shared memory.  For
// column k with x the part below the diagonal, x_0 = |x_0| e^{i theta}: alpha =
// -e^{i theta} |x|, v = x - alpha e_0, beta = 2 / |v|^2 = 1 / (|x| (|x| + |x_0|)); with
// p = beta A v, K = (beta/2) Re(v^H p) and w = p - K v the update is
// A <- A - v w^H - w v^H.  The result is a Hermitian tridiagonal matrix whose eigenvalues
// are those of the real symmetric one with off-diagonal |e_i|: work receives its diagonal
// and |e_i|^2, which the bisection of the real spectrum takes as they are.
constexpr int ZTRI_THREADS = 256;
size_t ztridiag_smem_bytes(int chi) { return sizeof(double) * ((size_t)2 * chi * (chi | 1) + 4 * (size_t)chi); }
size_t ztridiag_launch_bytes(int chi)
{
    const size_t need = ztridiag_smem_bytes(chi), alone = 220 * 1024;
    return need > alone ? need : alone;
}

__global__ void __launch_bounds__(ZTRI_THREADS) zc_tridiag_kernel(int chi, const double *C, long long PC, double *work)
{
    extern __shared__ double sm[];
    __shared__ double red[33];
    __shared__ double sh_beta, sh_ar, sh_ai;
    const int ld = chi | 1;
    double *Ar = sm, *Ai = Ar + (size_t)chi * ld;
    double *vr = Ai + (size_t)chi * ld, *vi = vr + chi, *pr = vi + chi, *pim = pr + chi;
    const int tid = threadIdx.x;
    const double *Ci = C + 3 * PC;
    for (int t = tid; t < chi * chi; t += blockDim.x) {
        const int i = t / chi, j = t % chi;
        Ar[i * ld + j] = 0.5 * (C[t] + C[j * chi + i]);
        Ai[i * ld + j] = 0.5 * (Ci[t] - Ci[j * chi + i]);
    }
    __syncthreads();
    for (int kc = 0; kc + 2 < chi; ++kc) {
        const int b0 = kc + 1, m = chi - b0;
        double part = 0.0;
        for (int i = tid; i < m; i += blockDim.x) {
            const double xr = Ar[(b0 + i) * ld + kc], xi = Ai[(b0 + i) * ld + kc];
            vr[i] = xr;
            vi[i] = xi;
            if (i > 0) part += xr * xr + xi * xi;
        }
        const double tail = zblock_sum(part, red);   // its barriers also publish v
        if (tail == 0.0) continue;                   // already tridiagonal in this column
        const double x0r = vr[0], x0i = vi[0];
        if (tid == (int)blockDim.x - 1) {
            const double a0 = sqrt(x0r * x0r + x0i * x0i);
            const double nrm = sqrt(tail + a0 * a0);
            const double cr = a0 > 0.0 ? x0r / a0 : 1.0, ci = a0 > 0.0 ? x0i / a0 : 0.0;
            sh_ar = -cr * nrm;
            sh_ai = -ci * nrm;
            sh_beta = 1.0 / (nrm * (nrm + a0));
        }
        // y = A x over the trailing block (v still holds x)
        for (int i = tid; i < m; i += blockDim.x) {
            const double *rr = Ar + (b0 + i) * ld + b0, *ri = Ai + (b0 + i) * ld + b0;
            double sr0 = 0.0, si0 = 0.0, sr1 = 0.0, si1 = 0.0;
            int j = 0;
            for (; j + 1 < m; j += 2) {
                sr0 = fma(rr[j], vr[j], fma(-ri[j], vi[j], sr0));
                si0 = fma(rr[j], vi[j], fma(ri[j], vr[j], si0));
                sr1 = fma(rr[j + 1], vr[j + 1], fma(-ri[j + 1], vi[j + 1], sr1));
                si1 = fma(rr[j + 1], vi[j + 1], fma(ri[j + 1], vr[j + 1], si1));
            }
            if (j < m) {
                sr0 = fma(rr[j], vr[j], fma(-ri[j], vi[j], sr0));
                si0 = fma(rr[j], vi[j], fma(ri[j], vr[j], si0));
            }
            pr[i] = sr0 + sr1;
            pim[i] = si0 + si1;
        }
        __syncthreads();
        const double beta = sh_beta, ar = sh_ar, ai = sh_ai;
        // p = beta (A x - alpha A e_0), then v_0 = x_0 - alpha
        for (int i = tid; i < m; i += blockDim.x) {
            const double er = Ar[(b0 + i) * ld + b0], ei = Ai[(b0 + i) * ld + b0];
            pr[i] = beta * (pr[i] - (ar * er - ai * ei));
            pim[i] = beta * (pim[i] - (ar * ei + ai * er));
        }
        if (tid == 0) {
            vr[0] = x0r - ar;
            vi[0] = x0i - ai;
        }
        __syncthreads();
        double pv = 0.0;   // Re(v^H p)
        for (int i = tid; i < m; i += blockDim.x) pv += vr[i] * pr[i] + vi[i] * pim[i];
        pv = zblock_sum(pv, red);
        const double Kf = 0.5 * beta * pv;
        for (int i = tid; i < m; i += blockDim.x) {   // p <- w
            pr[i] -= Kf * vr[i];
            pim[i] -= Kf * vi[i];
        }
        __syncthreads();
        for (int t = tid; t < m * m; t += blockDim.x) {
            const int i = t / m, j = t % m;
            // v_i conj(w_j) + w_i conj(v_j)
            const double re = vr[i] * pr[j] + vi[i] * pim[j] + pr[i] * vr[j] + pim[i] * vi[j];
            const double im = vi[i] * pr[j] - vr[i] * pim[j] + pim[i] * vr[j] - pr[i] * vi[j];
            Ar[(b0 + i) * ld + b0 + j] -= re;
            Ai[(b0 + i) * ld + b0 + j] -= im;
        }
        if (tid == 0) {
            Ar[b0 * ld + kc] = ar;
            Ai[b0 * ld + kc] = ai;
            Ar[kc * ld + b0] = ar;
            Ai[kc * ld + b0] = -ai;
        }
        __syncthreads();
    }
    for (int i = tid; i < chi; i += blockDim.x) {
        work[i] = Ar[i * ld + i];
        double e2 = 0.0;
        if (i + 1 < chi) {
            const double er = Ar[(i + 1) * ld + i], ei = Ai[(i + 1) * ld + i];
            e2 = er * er + ei * ei;
        }
        work[chi + i] = e2;
    }
}

// raw[pA][pB] = sum_{ab, z} Y1o[ab][pB][z] G2[ab][pA][z] (complex, no conjugation)
__global__ void zc_rho_partial_kernel(long long nab, int dd, int D2, const double *Y1o, const double *G2,
                                      long long P, double *partials)
{
    __shared__ double red[2 * ZRHO_MAX_DD * ZRHO_MAX_DD][8];
    double acc[2 * ZRHO_MAX_DD * ZRHO_MAX_DD];
    for (int i = 0; i < 2 * dd * dd; ++i) acc[i] = 0.0;
    const long long row = (long long)dd * D2;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nab * D2;
         t += (long long)gridDim.x * blockDim.x) {
        const long long ab = t / D2;
        const int z = (int)(t - ab * D2);
        const long long o = ab * row + z;
        for (int pb = 0; pb < dd; ++pb) {
            const double yr = Y1o[o + pb * D2], yi = Y1o[P + o + pb * D2];
            for (int pa = 0; pa < dd; ++pa) {
                const double gr = G2[o + pa * D2], gi = G2[P + o + pa * D2];
                acc[2 * (pa * dd + pb)] += yr * gr - yi * gi;
                acc[2 * (pa * dd + pb) + 1] += yr * gi + yi * gr;
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = 0; i < 2 * dd * dd; ++i) {
        double v = acc[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[i][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 2 * dd * dd) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
        partials[(size_t)blockIdx.x * 2 * dd * dd + threadIdx.x] = s;
    }
}

// Eq. 1: rho[(sA sB)][(tA tB)] = raw[(sA tA)][(sB tB)] / tr; e_a = Re tr(rho h'_a) with the
// rotated bond operators h'_a; out = e_x, e_y, e_z, E_site, then rho (complex, interleaved).
__global__ void zc_energy_kernel(int d, int nparts, const double *partials, const double *hrot, double *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int dd = d * d;
    double raw[2 * ZRHO_MAX_DD * ZRHO_MAX_DD];
    for (int i = 0; i < 2 * dd * dd; ++i) {
        double s = 0.0;
        for (int b = 0; b < nparts; ++b) s += partials[(size_t)b * 2 * dd * dd + i];
        raw[i] = s;
    }
    double zr = 0.0, zi = 0.0;
    for (int sA = 0; sA < d; ++sA)
        for (int sB = 0; sB < d; ++sB) {
            const int o = 2 * ((sA * d + sA) * dd + sB * d + sB);
            zr += raw[o];
            zi += raw[o + 1];
        }
    const double zz = zr * zr + zi * zi;
    double *rho = out + 4;
    for (int sA = 0; sA < d; ++sA)
        for (int sB = 0; sB < d; ++sB)
            for (int tA = 0; tA < d; ++tA)
                for (int tB = 0; tB < d; ++tB) {
                    const int o = 2 * ((sA * d + tA) * dd + sB * d + tB);
                    const int r = 2 * ((sA * d + sB) * dd + tA * d + tB);
                    rho[r] = (raw[o] * zr + raw[o + 1] * zi) / zz;
                    rho[r + 1] = (raw[o + 1] * zr - raw[o] * zi) / zz;
                }
    double es = 0.0;
    for (int a = 0; a < 3; ++a) {
        double e = 0.0;
        for (int r = 0; r < dd; ++r)
            for (int c = 0; c < dd; ++c) {
                const double *h = hrot + 2 * ((size_t)a * dd * dd + c * dd + r);
                e += rho[2 * (r * dd + c)] * h[0] - rho[2 * (r * dd + c) + 1] * h[1];
            }
        out[a] = e;
        es += e;
    }
    out[3] = 0.5 * es;
}

__global__ void zc_check_finite_kernel(long long count, const double *x, int *flag)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
         t += (long long)gridDim.x * blockDim.x)
        if (!isfinite(x[t])) *flag = 1;
}

// ------------------------------------------------------------------ host helpers
#define ZK(expr)                                          \
    do {                                                  \
        cudaError_t _e = (expr);                          \
        if (_e != cudaSuccess) return CTM_ECUDA;          \
    } while (0)

#define ZLAUNCH(kernel, grid, block, ...)                          \
    do {                                                           \
        CTM_COUNT_LAUNCH(1);                                       \
        kernel<<<(grid), (block), 0, c->stream>>>(__VA_ARGS__);    \
        ZK(cudaGetLastError());                                    \
    } while (0)

// A complex contraction C(m,n) = sum_k op(A)(m,k) op(B)(k,n) of planar tensors.  Each
// operand's k map is a plain stride; the plane index is stacked on it (k' = (plane, k)),
// which is again a plain stride when the planes are K strides apart.  A has two planes
// [Re, Im] (a5 = 0) or five (a5 = 1); B has five; C receives Re in plane 0 and Im in
// plane 1 (c5 = 0) or 3 (c5 = 1, the caller completes the other planes).
struct ZGemm {
    int M, N, K;
    const double *A;
    long long PA;
    int a5;
    Idx2 Am, Ak;
    int conjA;
    const double *B;
    long long PB;
    Idx2 Bk, Bn;
    int conjB;
    double *C;
    long long PC;
    int c5;
    Idx2 Cm, Cn;
};

int real_gemm(ctm_complex_ctx *c, const GemmF64 &g, int reuse_a)
{
    if (c->tf32_T > 0) return gemm_tf32(g, c->tf32_T, c->sw, c->stream, nullptr) == cudaSuccess ? CTM_OK : CTM_ECUDA;
    if (c->split_T > 0) {
        SplitOpts o{};
        o.reuse_a = reuse_a;
        return gemm_split(g, c->split_T, c->sw, c->stream, nullptr, &o) == cudaSuccess ? CTM_OK : CTM_ECUDA;
    }
    return gemm_f64(g, gemm_f64_pick_split(g.M, g.N, g.K), c->splitk, c->splitk_elems, c->stream) == cudaSuccess
               ? CTM_OK
               : CTM_ECUDA;
}

static Idx2 zkmap(int K, long long P, long long s2)
{
    if (P == (long long)K * s2) return idx_lin(s2);   // the two planes are one strided run
    return Idx2{K, P, s2};
}

// reuse_a: the left operand is that of the previous zgemm call, unchanged since (its
// packed slices are still in the split engine's work buffers)
int zgemm(ctm_complex_ctx *c, const ZGemm &z, int reuse_a = 0)
{
    if (z.Ak.s1 != 0 || z.Bk.s1 != 0) return CTM_EINVAL;
    if (z.conjA && !z.a5) return CTM_EINVAL;
    // A' = [Re A | s_A Im A]: planes (2, 3) of five, (0, 1) conjugated, or (0, 1) of two
    const double *Ap = z.A + ((z.a5 && !z.conjA) ? 2 * z.PA : 0);
    const Idx2 Ak2 = zkmap(z.K, z.PA, z.Ak.s2);
    // B planes [Re, -Im, Re, Im, Re]: Re C takes [Re ; -s_B Im] = planes (0, 1), or (2, 3)
    // conjugated; Im C takes [s_B Im ; Re] = planes (3, 4), or (1, 2) conjugated
    const double *Br = z.B + (z.conjB ? 2 : 0) * z.PB;
    const double *Bi = z.B + (z.conjB ? 1 : 3) * z.PB;
    const Idx2 Bk2 = zkmap(z.K, z.PB, z.Bk.s2);
    GemmF64 gr{z.M, z.N, 2 * z.K, Ap, z.Am, Ak2, Br, Bk2, z.Bn, z.C, z.Cm, z.Cn, 1.0, 0.0};
    GemmF64 gi{z.M, z.N, 2 * z.K, Ap, z.Am, Ak2, Bi, Bk2, z.Bn, z.C + (z.c5 ? 3 : 1) * z.PC, z.Cm, z.Cn, 1.0, 0.0};
    int rc = real_gemm(c, gr, reuse_a);
    if (rc != CTM_OK) return rc;
    return real_gemm(c, gi, 1);
}

int znormalize(ctm_complex_ctx *c, long long count, double *x, ZLay L)
{
    int nb = zgrid(count);
    if (nb > ZNORM_BLOCKS) nb = ZNORM_BLOCKS;
    ZLAUNCH(zc_sumsq_kernel, nb, 256, count, x, L, c->norm_part);
    ZLAUNCH(zc_scale_kernel, zgrid(count), 256, count, x, L, c->norm_part, nb);
    return CTM_OK;
}

QrScratch zqr_scratch(ctm_complex_ctx *c)
{
    const long long k = 2LL * c->chi;
    QrScratch q;
    memset(&q, 0, sizeof(q));
    q.sbuf = c->qr_sbuf;
    q.rowbuf = c->qr_rowbuf;
    q.bar = c->qr_bar;
    q.err = c->err;
    q.rows_min = 1;
    q.V = c->qr_wy;
    q.S = q.V + k * k;
    q.W = q.S + k * k;
    q.ta = q.W + k * k;
    q.gpart = c->qr_gpart;
    q.spart = c->qr_spart;
    q.gmax = c->qr_gmax;
    q.yslab = c->qr_slab;
    q.yslab_elems = c->qr_slab_elems;
    q.force_slab = false;
    return q;
}

// (M, N, K) of the real products (K doubled) of the step and the energy
std::vector<std::array<int, 3>> zshapes(const ctm_complex_ctx *c)
{
    const int chi = c->chi, D2 = c->D2, n = (int)c->n, dd = c->d * c->d;
    return {{n, chi, 2 * chi},          {n, n, 2 * chi},          {chi * chi, D2, 2 * D2 * D2},
            {chi * chi, D2 * D2, 2 * D2}, {n, chi, 2 * n},          {chi, chi, 2 * n},
            {n, chi, 2 * chi},          {chi, chi, 2 * chi},      {chi * chi, dd * D2, 2 * D2 * D2}};
}

size_t zlayout(ctm_complex_ctx *c, char *base)
{
    const long long chi = c->chi, D2 = c->D2, n = c->n, d = c->d, D = c->D;
    const long long D3 = D2 * D2 * D2, dd = d * d, k2 = 2 * chi;
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off += (bytes + 255) & ~(size_t)255;
        return p;
    };
    auto td = [&](long long count) -> double * { return (double *)take(sizeof(double) * (size_t)count); };
    c->PA = d * D * D * D;
    c->Ain = td(2 * c->PA);
    c->A = td(2 * c->PA);
    c->Pa = D3;
    c->a = td(5 * D3);
    c->aA = td(5 * D3);
    c->Pb = dd * D3;
    c->bB = td(5 * c->Pb);
    c->bA = td(5 * c->Pb);
    c->PC = chi * chi;
    c->C = td(5 * c->PC);
    c->Cn = td(5 * c->PC);
    c->Cr = td(2 * c->PC);
    c->R = td(2 * c->PC);
    c->P5a = td(2 * c->PC);
    c->P5b = td(5 * c->PC);
    c->PT = chi * D2 * chi;
    c->T = td(5 * c->PT);
    c->Tn = td(5 * c->PT);
    c->PQ = n * chi;
    c->Q = td(5 * c->PQ);
    c->Qn = td(5 * c->PQ);
    c->Qs = td(5 * c->PQ);
    c->PY = n * chi;
    c->Y = td(2 * c->PY);
    c->W = td(2 * c->PY);
    c->MQ = td(2 * c->PY);
    c->PM = n * n;
    c->M = td(2 * c->PM);
    c->X = td(2 * c->PM);
    c->H = td(2 * c->PM);
    c->PY1 = chi * chi * D2;
    c->Y1 = td(2 * c->PY1);
    c->PYo = chi * chi * dd * D2;
    c->Y1o = td(2 * c->PYo);
    c->G2 = td(2 * c->PYo);
    c->Yemb = td(2 * n * k2);
    c->Qemb = td(2 * n * k2);
    c->Remb = td(k2 * k2);
    c->s = td(chi);
    c->s_new = td(chi);
    c->delta = td(8);
    c->spec_work = td((long long)spectrum_work_doubles(chi > ZSMEM_CHI ? 2 * (int)chi : (int)chi));
    c->spec_emb = chi > ZSMEM_CHI ? td(4 * chi * chi) : nullptr;
    size_t sk = 0;
    for (const auto &sh : zshapes(c)) {
        int s = gemm_f64_pick_split(sh[0], sh[1], sh[2]);
        if (s > 1 && (size_t)s * sh[0] * sh[1] > sk) sk = (size_t)s * sh[0] * sh[1];
    }
    c->splitk_elems = sk;
    c->splitk = td((long long)sk + 1);
    c->qr_sbuf = td((long long)qr_scratch_doubles((int)k2));
    c->qr_rowbuf = td((long long)qr_rowbuf_doubles((int)k2));
    c->qr_wy = td((long long)qr_wy_doubles((int)(2 * n), (int)k2));
    c->qr_slab_elems = qr_slab_doubles((int)(2 * n), (int)k2);
    c->qr_slab = c->qr_slab_elems ? td((long long)c->qr_slab_elems) : nullptr;
    if (c->cfg.deterministic) {
        c->qr_gmax = qr_det_gmax((int)(2 * n));
        c->qr_gpart = td((long long)qr_det_gram_doubles((int)k2, c->qr_gmax));
        c->qr_spart = td((long long)qr_det_s_doubles((int)k2, c->qr_gmax));
    }
    c->qr_bar = (unsigned *)take(64);
    c->err = (int *)take(64);
    c->flag = (int *)take(64);
    c->norm_part = td(ZNORM_BLOCKS);
    c->rho_part = td((long long)ZRHO_BLOCKS * 2 * dd * dd);
    c->rho_raw = td(2 * dd * dd);
    c->hrot = td(3 * 2 * dd * dd);
    c->eout = td(4 + 2 * dd * dd);
    if (c->split_T > 0 || c->tf32_T > 0) {
        size_t ap = 0, bp = 0, pp = 0;
        long long ecap = 0;
        for (const auto &sh : zshapes(c)) {
            SplitPlan pl = c->tf32_T > 0 ? tf32_plan_caps(sh[0], sh[1], sh[2], c->tf32_T)
                                         : split_plan_caps(sh[0], sh[1], sh[2], c->split_T);
            if (pl.a_pack_bytes > ap) ap = pl.a_pack_bytes;
            if (pl.b_pack_bytes > bp) bp = pl.b_pack_bytes;
            if (pl.partial_bytes > pp) pp = pl.partial_bytes;
            if (sh[0] > ecap) ecap = sh[0];
            if (sh[1] > ecap) ecap = sh[1];
        }
        c->sw.Apk = (unsigned char *)take(ap);
        c->sw.a_pack_cap = ap;
        c->sw.Bpk = (unsigned char *)take(bp);
        c->sw.b_pack_cap = bp;
        c->sw.eA = (int *)take(sizeof(int) * (size_t)ecap);
        c->sw.eB = (int *)take(sizeof(int) * (size_t)ecap);
        c->sw.e_cap = (int)ecap;
        c->sw.partial = (void *)take(pp + 8);
        c->sw.partial_cap = pp;
        c->sw.err = c->err;
        c->sw.autotune = 1;
    }
    return off;
}

bool zconfig_ok(const ctm_config *cfg, int irrep)
{
    if (!cfg) return false;
    if (irrep != CTM_IRREP_A1 && irrep != CTM_IRREP_E) return false;
    if (cfg->d < 1 || cfg->d > ZMAX_D) return false;
    if (irrep == CTM_IRREP_E && cfg->d < 2) return false;
    if (cfg->D < 1 || cfg->D > 10) return false;
    if (cfg->chi < 1 || cfg->chi > ZMAX_CHI) return false;
    if (cfg->precision != CTM_FP64 && cfg->precision != CTM_SPLIT_BF16 && cfg->precision != CTM_SPLIT_TF32 &&
        cfg->precision != CTM_FP32_TF32)
        return false;
    if (cfg->precision == CTM_SPLIT_BF16 && !split_supported_T(cfg->n_split)) return false;
    if (cfg->corner_mode != 0 && cfg->corner_mode != 1) return false;
    if (cfg->deterministic != 0 && cfg->deterministic != 1) return false;
    const long long n = (long long)cfg->chi * cfg->D * cfg->D;
    if (n > 12000) return false;
    return qr_supported((int)(2 * n), 2 * cfg->chi) != 0;
}

int zread_status(ctm_complex_ctx *c)
{
    int err = 0;
    ZK(cudaMemcpyAsync(&err, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    ZK(cudaStreamSynchronize(c->stream));
    return err ? CTM_ETIMEOUT : CTM_OK;
}

// ------------------------------------------------------------------ the step
// Layouts of the step's tensors (ZLay): a, aA, C, Q, Qs five planes stacked; T five planes
// row-blocked by its rows (a, u); W [(a,u)][2][h], X [(a,b)][2][(u,l)], Y1 [(a,b)][2][z] and
// M [(a,y)][2][(b,x)] two planes row-blocked (k contiguous for the next contraction); Y, MQ,
// Cr and H two planes stacked (k slowest for the next contraction).
ZLay lay_T(const ctm_complex_ctx *c) { return zlay_rows(c->chi, 5); }

// Fig. 3c: W = T C; X'[a][b][u][l] = sum_h W[(a,u),h] conj(T[(b,l),h]);
// Y1[(a,b)][z] = sum_{u,l} X' a[u,l,z]; M[(a,y)][(b,x)] = sum_z Y1 aA[z,x,y], with aA the double
// layer of the apex site (z leg first; equal to a for a C3-symmetric tensor)
int zenlarged_corner(ctm_complex_ctx *c)
{
    const int chi = c->chi, D2 = c->D2;
    const long long n = c->n, DD = (long long)D2 * D2;
    int rc;
    ZGemm z{(int)n, chi, chi, c->T, chi, 1, idx_lin(5LL * chi), idx_lin(1), 0, c->C, c->PC, idx_lin(chi), idx_lin(1),
            0, c->W, chi, 0, idx_lin(2LL * chi), idx_lin(1)};
    if ((rc = zgemm(c, z)) != CTM_OK) return rc;
    z = ZGemm{(int)n, (int)n, chi, c->W, chi, 0, idx_lin(2LL * chi), idx_lin(1), 0, c->T, chi, idx_lin(1),
              idx_lin(5LL * chi), 1, c->X, DD, 0, idx_split(D2, (long long)chi * 2 * DD, D2), idx_split(D2, 2 * DD, 1)};
    if ((rc = zgemm(c, z)) != CTM_OK) return rc;
    z = ZGemm{chi * chi, D2, D2 * D2, c->X, DD, 0, idx_lin(2 * DD), idx_lin(1), 0, c->a, c->Pa, idx_lin(D2),
              idx_lin(1), 0, c->Y1, D2, 0, idx_lin(2LL * D2), idx_lin(1)};
    if ((rc = zgemm(c, z)) != CTM_OK) return rc;
    z = ZGemm{chi * chi, D2 * D2, D2, c->Y1, D2, 0, idx_lin(2LL * D2), idx_lin(1), 0, c->aA, c->Pa, idx_lin(DD),
              idx_split(D2, 1, D2), 0, c->M, n, 0, idx_split(chi, 2LL * D2 * n, D2), idx_split(D2, 2 * n, 1)};
    return zgemm(c, z);
}

// Fig. 3d: Y = M Q diag(sgn Re C_jj); Y = Q R through the real QR of the embedding
int zprojector(ctm_complex_ctx *c)
{
    const int chi = c->chi;
    const long long n = c->n;
    int rc;
    ZLAUNCH(zc_warm_start_kernel, zgrid(n * chi), 256, n, chi, c->Q, c->PQ, c->C, c->Qs);
    ZGemm z{(int)n, chi, (int)n, c->M, n, 0, idx_lin(2 * n), idx_lin(1), 0, c->Qs, c->PQ, idx_lin(chi), idx_lin(1), 0,
            c->Y, c->PY, 0, idx_lin(chi), idx_lin(1)};
    if ((rc = zgemm(c, z)) != CTM_OK) return rc;
    ZLAUNCH(zc_embed_kernel, zgrid(n * chi), 256, n, chi, c->Y, c->PY, c->Yemb);
    ZK(qr_householder((int)(2 * n), 2 * chi, c->Yemb, c->Qemb, c->Remb, zqr_scratch(c), c->stream));
    ZLAUNCH(zc_extract_kernel, zgrid(n * chi), 256, n, chi, c->Qemb, c->Qn, c->PQ, 5);
    ZLAUNCH(zc_extract_kernel, zgrid((long long)chi * chi), 256, (long long)chi, chi, c->Remb, c->R, c->PC, 2);
    return CTM_OK;
}

// Fig. 3a: Cn = sym(Qn^H M Qn)/|.|, through Cr[i][j] = sum_r MQ[r][j] conj(Qn[r][i])
int zcorner(ctm_complex_ctx *c, double *Cout)
{
    const int chi = c->chi;
    const long long n = c->n;
    int rc;
    // the previous contraction was Y = M Qs (only the QR in between): M is packed already
    ZGemm z{(int)n, chi, (int)n, c->M, n, 0, idx_lin(2 * n), idx_lin(1), 0, c->Qn, c->PQ, idx_lin(chi), idx_lin(1), 0,
            c->MQ, c->PY, 0, idx_lin(chi), idx_lin(1)};
    if ((rc = zgemm(c, z, 1)) != CTM_OK) return rc;
    z = ZGemm{chi, chi, (int)n, c->MQ, c->PY, 0, idx_lin(1), idx_lin(chi), 0, c->Qn, c->PQ, idx_lin(chi), idx_lin(1), 1,
              c->Cr, c->PC, 0, idx_lin(1), idx_lin(chi)};
    if ((rc = zgemm(c, z)) != CTM_OK) return rc;
    ZLAUNCH(zc_herm_normalize_kernel, 1, 1024, chi, c->Cr, c->PC, Cout, c->PC);
    return CTM_OK;
}

// Cheap corner variant (Sec. II.B, Fig. 3d): Cn = sym(R S)/|.|; R S = Qn^H M Q_prev exactly,
// which is Qn^H M Qn at a fixed point
int zcorner_from_r(ctm_complex_ctx *c, double *Cout)
{
    const int chi = c->chi;
    ZLAUNCH(zc_rs_kernel, zgrid((long long)chi * chi), 256, chi, c->R, c->PC, c->C, c->Cr, c->PC);
    ZLAUNCH(zc_herm_normalize_kernel, 1, 1024, chi, c->Cr, c->PC, Cout, c->PC);
    return CTM_OK;
}

// Fig. 3b: T'[i,x,j] = sum conj(Q[(a,y),i]) T[a,u,g] a[u,w,z] aA[z,x,y] Q[(g,w),j], normalised
int zedge(ctm_complex_ctx *c)
{
    const int chi = c->chi, D2 = c->D2;
    const long long n = c->n, DD = (long long)D2 * D2;
    int rc;
    // H1'[a][j][u][w] = sum_g T[(a,u),g] Q[(g,w),j]   (into X, laid out as X')
    ZGemm z{(int)n, (int)n, chi, c->T, chi, 1, idx_lin(5LL * chi), idx_lin(1), 0, c->Qn, c->PQ, idx_lin(n),
            idx_split(D2, 1, chi), 0, c->X, DD, 0, idx_split(D2, (long long)chi * 2 * DD, D2),
            idx_split(D2, 2 * DD, 1)};
    if ((rc = zgemm(c, z)) != CTM_OK) return rc;
    // H2[(a,j)][z] = H1'[(a,j),(u,w)] a[(u,w),z]
    z = ZGemm{chi * chi, D2, D2 * D2, c->X, DD, 0, idx_lin(2 * DD), idx_lin(1), 0, c->a, c->Pa, idx_lin(D2),
              idx_lin(1), 0, c->Y1, D2, 0, idx_lin(2LL * D2), idx_lin(1)};
    if ((rc = zgemm(c, z)) != CTM_OK) return rc;
    // H3'[a][y][x][j] = H2[(a,j),z] a[z,x,y]
    z = ZGemm{chi * chi, D2 * D2, D2, c->Y1, D2, 0, idx_lin(2LL * D2), idx_lin(1), 0, c->aA, c->Pa, idx_lin(DD),
              idx_split(D2, 1, D2), 0, c->H, c->PM, 0, idx_split(chi, DD * chi, 1),
              idx_split(D2, (long long)D2 * chi, chi)};
    if ((rc = zgemm(c, z)) != CTM_OK) return rc;
    // T'[i][(x,j)] = sum_{(a,y)} H3'[(a,y),(x,j)] conj(Q[(a,y),i]), into T's row-blocked layout
    z = ZGemm{(int)n, chi, (int)n, c->H, c->PM, 0, idx_lin(1), idx_lin(n), 0, c->Qn, c->PQ, idx_lin(chi), idx_lin(1), 1,
              c->Tn, chi, 1, idx_split(chi, 5LL * chi, 1), idx_lin(5 * n)};
    if ((rc = zgemm(c, z)) != CTM_OK) return rc;
    return znormalize(c, (long long)chi * D2 * chi, c->Tn, lay_T(c));
}

// The real symmetric embedding of the Hermitian part H = Ar + i Ai of the corner (Re in
// plane 0, Im in plane 3): E = [[Ar, -Ai], [Ai, Ar]] (2chi x 2chi), whose eigenvalues are
// H's, each twice.
__global__ void zc_embed_kernel(int chi, const double *C, long long PC, double *E)
{
    const long long N = 2LL * chi, total = N * N;
    const double *Ci = C + 3 * PC;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(t / N), q = (int)(t % N);
        const int i = r % chi, j = q % chi, br = r / chi, bq = q / chi;
        double v;
        if (br == bq) v = 0.5 * (C[(size_t)i * chi + j] + C[(size_t)j * chi + i]);
        else {
            const double ai = 0.5 * (Ci[(size_t)i * chi + j] - Ci[(size_t)j * chi + i]);
            v = (br == 0) ? -ai : ai;
        }
        E[t] = v;
    }
}

// the corner spectrum of C (five planes): delta against the previous one, on `st`;
// with dst, the delta is also copied there (pinned host memory)
int zspectrum(ctm_complex_ctx *c, const double *Cin, cudaStream_t st, double *dst = nullptr)
{
    const int chi = c->chi;
    if (st != c->stream) {
        ZK(cudaEventRecord(c->ev_fork, c->stream));
        ZK(cudaStreamWaitEvent(st, c->ev_fork, 0));
    }
    if (chi > ZSMEM_CHI) {
        const long long n2 = 4LL * chi * chi;
        CTM_COUNT_LAUNCH(1);
        zc_embed_kernel<<<zgrid(n2), 256, 0, st>>>(chi, Cin, c->PC, c->spec_emb);
        ZK(cudaGetLastError());
        ZK(launch_spectrum_pairs(chi, c->spec_emb, c->s_new, c->s, c->delta, c->spec_work, st));
    } else {
        CTM_COUNT_LAUNCH(1);
        // all but a few KB of the SM's shared memory: the step's CTAs stay off its SM (as for
        // the real corner spectrum)
        zc_tridiag_kernel<<<1, ZTRI_THREADS, ztridiag_launch_bytes(chi), st>>>(chi, Cin, c->PC, c->spec_work);
        ZK(cudaGetLastError());
        ZK(launch_spectrum_from_tridiag(chi, c->spec_work, c->s_new, c->s, c->delta, st));
    }
    ZK(cudaMemcpyAsync(c->s, c->s_new, sizeof(double) * chi, cudaMemcpyDeviceToDevice, st));
    if (dst) ZK(cudaMemcpyAsync(dst, c->delta, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (st != c->stream) ZK(cudaEventRecord(c->ev_join, st));
    return CTM_OK;
}

// One step.  The spectrum of C' runs on the side stream from the corner update on; it is
// joined before the next step's corner update rewrites C', or at the end when join_now.
// In the pipelined graphs (spec_head / spec_skip set while capturing) the first step
// also computes, beside itself, the spectrum of the corner C it starts from (the
// previous graph's last step, whose own spectrum was skipped); C is rewritten only at
// the hand-over, after the corner update that waits for it.
int zstep(ctm_complex_ctx *c, int join_now)
{
    int rc;
    if (c->spec_head) {
        if ((rc = zspectrum(c, c->C, c->side, c->delta_head)) != CTM_OK) return rc;
        c->side_pending = 1;
    }
    if ((rc = zenlarged_corner(c)) != CTM_OK) return rc;
    if ((rc = zprojector(c)) != CTM_OK) return rc;
    if (c->side_pending) {
        ZK(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
        c->side_pending = 0;
    }
    if ((rc = c->cfg.corner_mode ? zcorner_from_r(c, c->Cn) : zcorner(c, c->Cn)) != CTM_OK) return rc;
    if (!c->spec_skip) {
        if ((rc = zspectrum(c, c->Cn, c->side, c->delta_dst)) != CTM_OK) return rc;
        c->side_pending = 1;
    }
    if ((rc = zedge(c)) != CTM_OK) return rc;
    const long long chi = c->chi, D2 = c->D2, n = c->n;
    cudaStream_t st = c->stream;
    if (join_now && c->side_pending) {
        ZK(cudaStreamWaitEvent(st, c->ev_join, 0));
        c->side_pending = 0;
    }
    ZK(cudaMemcpyAsync(c->C, c->Cn, sizeof(double) * 5 * chi * chi, cudaMemcpyDeviceToDevice, st));
    ZK(cudaMemcpyAsync(c->T, c->Tn, sizeof(double) * 5 * chi * D2 * chi, cudaMemcpyDeviceToDevice, st));
    ZK(cudaMemcpyAsync(c->Q, c->Qn, sizeof(double) * 5 * n * chi, cudaMemcpyDeviceToDevice, st));
    c->steps_done++;
    return CTM_OK;
}

int zcheck_env_finite(ctm_complex_ctx *c)
{
    cudaStream_t st = c->stream;
    ZK(cudaMemsetAsync(c->flag, 0, sizeof(int), st));
    ZLAUNCH(zc_check_finite_kernel, zgrid(5 * c->PC), 256, 5 * c->PC, c->C, c->flag);
    ZLAUNCH(zc_check_finite_kernel, zgrid(5 * c->PT), 256, 5 * c->PT, c->T, c->flag);
    int f = 0;
    ZK(cudaMemcpyAsync(&f, c->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    ZK(cudaStreamSynchronize(st));
    return f ? CTM_ENONFINITE : CTM_OK;
}

// ------------------------------------------------------------------ transfer spectrum (f2)
// The column transfer matrix of the complex environment (Sec. II.C),
//   TM[(a,y,b),(g,w,h)] = sum T[a,u,g] aB[u,w,z] aA[z,x,y] conj(T[b,x,h])
// (the opposite edge is the mirror image of T), is applied as the edge update's first
// three contractions with v in place of Q, then a contraction with conj(T) over
// (x, h).  The real path's subspace iteration runs on its real form (vectors
// [Re v | Im v]), whose spectrum holds each magnitude of the complex one twice.

// [Re v | Im v] (N each) -> five planes [Re, -Im, Re, Im, Re] of stride N
__global__ void zc_tr_expand_kernel(long long N, const double *v2, double *v5)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x) {
        const double re = v2[t], im = v2[N + t];
        v5[t] = re;
        v5[N + t] = -im;
        v5[2 * N + t] = re;
        v5[3 * N + t] = im;
        v5[4 * N + t] = re;
    }
}

// T's row-blocked five planes (row r = (b,x) holds 5 chi values) -> plain planes of stride N
__global__ void zc_tr_unblock_kernel(long long N, int chi, const double *T, double *Tp)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 5 * N;
         t += (long long)gridDim.x * blockDim.x) {
        const long long p = t / N, e = t - p * N, r = e / chi, h = e - r * chi;
        Tp[t] = T[r * 5 * chi + p * chi + h];
    }
}

size_t ztransfer_layout(const ctm_complex_ctx *c, int m, char *base, double **Vq, double **Tp, void **sub)
{
    const long long N = (long long)c->chi * c->D2 * c->chi;
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off += (bytes + 255) & ~(size_t)255;
        return p;
    };
    *sub = take(subspace_workspace_bytes(2 * N, m));
    *Vq = (double *)take(sizeof(double) * 5 * (size_t)N);
    *Tp = (double *)take(sizeof(double) * 5 * (size_t)N);
    return off;
}

// out2 = TM v2 for vectors [Re | Im] of length N each
int ztransfer_apply(ctm_complex_ctx *c, const double *v2, double *out2, double *Vq, const double *Tp)
{
    const int chi = c->chi, D2 = c->D2;
    const long long n = c->n, N = n * chi, DD = (long long)D2 * D2;
    int rc;
    ZLAUNCH(zc_tr_expand_kernel, zgrid(N), 256, N, v2, Vq);
    // P1[a][h][u][w] = sum_g T[(a,u),g] v[(g,w),h]   (into X, as H1' of the edge update)
    ZGemm z{(int)n, (int)n, chi, c->T, chi, 1, idx_lin(5LL * chi), idx_lin(1), 0, Vq, N, idx_lin(n),
            idx_split(D2, 1, chi), 0, c->X, DD, 0, idx_split(D2, (long long)chi * 2 * DD, D2),
            idx_split(D2, 2 * DD, 1)};
    if ((rc = zgemm(c, z)) != CTM_OK) return rc;
    // P2[(a,h)][z] = P1[(a,h),(u,w)] aB[(u,w),z]
    z = ZGemm{chi * chi, D2, D2 * D2, c->X, DD, 0, idx_lin(2 * DD), idx_lin(1), 0, c->a, c->Pa, idx_lin(D2),
              idx_lin(1), 0, c->Y1, D2, 0, idx_lin(2LL * D2), idx_lin(1)};
    if ((rc = zgemm(c, z)) != CTM_OK) return rc;
    // P3[a][y][x][h] = P2[(a,h),z] aA[z,x,y]
    z = ZGemm{chi * chi, D2 * D2, D2, c->Y1, D2, 0, idx_lin(2LL * D2), idx_lin(1), 0, c->aA, c->Pa, idx_lin(DD),
              idx_split(D2, 1, D2), 0, c->H, c->PM, 0, idx_split(chi, DD * chi, 1),
              idx_split(D2, (long long)D2 * chi, chi)};
    if ((rc = zgemm(c, z)) != CTM_OK) return rc;
    // out[(a,y)][b] = sum_{(x,h)} P3[(a,y),(x,h)] conj(T[b,(x,h)])
    z = ZGemm{(int)n, chi, (int)n, c->H, c->PM, 0, idx_lin(n), idx_lin(1), 0, Tp, N, idx_lin(1), idx_lin(n), 1,
              out2, N, 0, idx_lin(chi), idx_lin(1)};
    return zgemm(c, z);
}

}  // namespace

extern "C" {

size_t ctm_complex_workspace_bytes(const ctm_config *cfg, int irrep)
{
    if (!zconfig_ok(cfg, irrep)) return 0;
    ctm_complex_ctx c;
    memset(&c, 0, sizeof(c));
    c.cfg = *cfg;
    c.d = cfg->d;
    c.D = cfg->D;
    c.D2 = cfg->D * cfg->D;
    c.chi = cfg->chi;
    c.n = (long long)c.chi * c.D2;
    c.split_T = cfg->precision == CTM_SPLIT_BF16 ? cfg->n_split : 0;
    c.tf32_T = cfg->precision == CTM_SPLIT_TF32 ? 2 : (cfg->precision == CTM_FP32_TF32 ? 1 : 0);
    return zlayout(&c, nullptr);
}

int ctm_complex_init(const ctm_config *cfg, int irrep, const double *A_dev, void *workspace, size_t ws_bytes,
                     void *stream, ctm_complex_ctx **out)
{
    if (!out) return CTM_EINVAL;
    *out = nullptr;
    if (!cfg || !A_dev || !workspace) return CTM_EINVAL;
    if (!zconfig_ok(cfg, irrep)) return CTM_EINVAL;
    if ((uintptr_t)workspace % 256 != 0) return CTM_EINVAL;
    ctm_complex_ctx *c = new (std::nothrow) ctm_complex_ctx;
    if (!c) return CTM_ENOMEM;
    memset(c, 0, sizeof(*c));
    c->cfg = *cfg;
    c->irrep = irrep;
    c->d = cfg->d;
    c->D = cfg->D;
    c->D2 = cfg->D * cfg->D;
    c->chi = cfg->chi;
    c->n = (long long)c->chi * c->D2;
    c->split_T = cfg->precision == CTM_SPLIT_BF16 ? cfg->n_split : 0;
    c->tf32_T = cfg->precision == CTM_SPLIT_TF32 ? 2 : (cfg->precision == CTM_FP32_TF32 ? 1 : 0);
    c->stream = (cudaStream_t)stream;
    if (ws_bytes < zlayout(c, nullptr)) {
        delete c;
        return CTM_ENOMEM;
    }
    zlayout(c, (char *)workspace);
    ZGroup grp;
    HMat Ur;
    if (!make_group(c->d, irrep, &grp, &Ur)) {
        delete c;
        return CTM_EUNSUPPORTED;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            c->U[i][j][0] = (i < c->d && j < c->d) ? Ur.v[i][j].re : 0.0;
            c->U[i][j][1] = (i < c->d && j < c->d) ? Ur.v[i][j].im : 0.0;
        }
    int rc = CTM_OK;
    do {
        if (qr_prepare() != cudaSuccess || spectrum_prepare() != cudaSuccess || split_prepare() != cudaSuccess ||
            tf32_prepare() != cudaSuccess ||
            cudaFuncSetAttribute(zc_tridiag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)ztridiag_launch_bytes(ZSMEM_CHI)) != cudaSuccess) {
            rc = CTM_ECUDA;
            break;
        }
        int prio_least = 0, prio_greatest = 0;
        cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
        if (cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_least) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
            rc = CTM_ECUDA;
            break;
        }
        const long long cnt = c->PA;
        if (cudaMemsetAsync(c->err, 0, sizeof(int), c->stream) != cudaSuccess) { rc = CTM_ECUDA; break; }
        CTM_COUNT_LAUNCH(5);
        zc_load_kernel<<<zgrid(cnt), 256, 0, c->stream>>>(cnt, A_dev, c->Ain, zlay_stacked(cnt, 2));
        zc_project_kernel<<<zgrid(cnt), 256, 0, c->stream>>>(c->d, c->D, c->Ain, cnt, grp, cfg->symmetrize ? 1 : 0,
                                                             c->A, cnt);
        if (cudaGetLastError() != cudaSuccess) { rc = CTM_ECUDA; break; }
        if ((rc = znormalize(c, cnt, c->A, zlay_stacked(cnt, 2))) != CTM_OK) break;
        const long long D6 = c->Pa;
        zc_double_layer_kernel<<<zgrid(D6), 256, 0, c->stream>>>(c->d, c->D, c->A, cnt, 0, c->a);
        zc_double_layer_kernel<<<zgrid(D6), 256, 0, c->stream>>>(c->d, c->D, c->A, cnt, 1, c->aA);
        zc_init_env_kernel<<<zgrid(c->PT), 256, 0, c->stream>>>(c->chi, c->D, c->a, c->Pa, c->C, c->T, c->Q);
        if (cudaGetLastError() != cudaSuccess) { rc = CTM_ECUDA; break; }
        if (launch_spectrum_init(c->chi, c->s, c->stream) != cudaSuccess) { rc = CTM_ECUDA; break; }
        if (cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream) != cudaSuccess) { rc = CTM_ECUDA; break; }
        CTM_COUNT_LAUNCH(1);
        zc_check_finite_kernel<<<zgrid(2 * cnt), 256, 0, c->stream>>>(2 * cnt, c->A, c->flag);
        int f = 0;
        if (cudaMemcpyAsync(&f, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess) {
            rc = CTM_ECUDA;
            break;
        }
        if (f) rc = CTM_ENONFINITE;
    } while (0);
    if (rc != CTM_OK) {
        ctm_complex_destroy(c);
        return rc;
    }
    *out = c;
    return CTM_OK;
}

// Capture nsteps steps on the private stream into graph1 (one step) or graphK (the last
// multi-step count asked for); a launch that cannot be captured leaves graph_failed set
// and the context runs eagerly.  Inside a multi-step graph each step's spectrum overlaps
// the next step up to its corner update; the graph ends joined.
static int zcapture(ctm_complex_ctx *c, int nsteps)
{
    cudaGraphExec_t *exec = nsteps == 1 ? &c->graph1 : &c->graphK;
    if (c->graph_failed) return CTM_OK;
    if (nsteps == 1 ? c->graph1 != nullptr : (c->graphK && c->graphK_steps == nsteps)) return CTM_OK;
    if (*exec) {
        cudaGraphExecDestroy(*exec);
        *exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    const unsigned long long l0 = g_ctm_launches;
    ZK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    const int steps0 = c->steps_done;
    int rc = CTM_OK;
    for (int i = 0; i < nsteps && rc == CTM_OK; ++i) rc = zstep(c, i == nsteps - 1);
    c->steps_done = steps0;
    c->side_pending = 0;
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (rc == CTM_OK && e == cudaSuccess && g) e = cudaGraphInstantiate(exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (rc != CTM_OK || e != cudaSuccess || !*exec) {
        cudaGetLastError();
        *exec = nullptr;
        c->graph_failed = 1;
    } else if (nsteps == 1) {
        c->graph1_kernels = g_ctm_launches - l0;
    } else {
        c->graphK_kernels = g_ctm_launches - l0;
        c->graphK_steps = nsteps;
    }
    g_ctm_launches = l0;
    return CTM_OK;
}

// The two pipelined graphs of k steps (ring halves 0 and 1): slot 0 of a half gets the
// delta of the step before the graph, slot i that of step i (1 <= i < k), and the graph
// ends by copying the error flag.  Leaves pipe_steps = 0 if capturing failed.
static int zcapture_pipe(ctm_complex_ctx *c, int k)
{
    if (c->pipe[0] && c->pipe[1] && c->pipe_steps == k) return CTM_OK;
    c->pipe_steps = 0;
    if (k > c->ring_cap) {
        for (int h = 0; h < 2; ++h)
            if (c->pipe[h]) {
                cudaGraphExecDestroy(c->pipe[h]);
                c->pipe[h] = nullptr;
            }
        if (c->ring_h) cudaFreeHost(c->ring_h);
        c->ring_h = nullptr;
        c->ring_cap = 0;
        ZK(cudaHostAlloc((void **)&c->ring_h, sizeof(double) * 2 * (size_t)k, cudaHostAllocDefault));
        c->ring_cap = k;
    }
    if (!c->ring_err_h) ZK(cudaHostAlloc((void **)&c->ring_err_h, 2 * sizeof(int), cudaHostAllocDefault));
    for (int h = 0; h < 2; ++h) {
        if (!c->pipe_done[h]) ZK(cudaEventCreateWithFlags(&c->pipe_done[h], cudaEventDisableTiming));
        if (c->pipe[h]) {
            cudaGraphExecDestroy(c->pipe[h]);
            c->pipe[h] = nullptr;
        }
        if (c->graph_failed) return CTM_OK;
        double *ring = c->ring_h + (size_t)h * c->ring_cap;
        cudaGraph_t g = nullptr;
        const unsigned long long l0 = g_ctm_launches;
        ZK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        const int steps0 = c->steps_done;
        int rc = CTM_OK;
        for (int i = 0; i < k && rc == CTM_OK; ++i) {
            c->spec_head = i == 0;
            c->delta_head = c->spec_head ? ring : nullptr;
            c->spec_skip = i == k - 1;
            c->delta_dst = c->spec_skip ? nullptr : ring + i + 1;
            rc = zstep(c, i == k - 1);
        }
        c->spec_head = c->spec_skip = 0;
        c->delta_head = c->delta_dst = nullptr;
        if (rc == CTM_OK &&
            cudaMemcpyAsync(c->ring_err_h + h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
            rc = CTM_ECUDA;
        c->steps_done = steps0;
        c->side_pending = 0;
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (rc == CTM_OK && e == cudaSuccess && g) e = cudaGraphInstantiate(&c->pipe[h], g, 0);
        if (g) cudaGraphDestroy(g);
        const unsigned long long captured = g_ctm_launches - l0;
        g_ctm_launches = l0;   // nothing ran yet: replays add the captured kernel count
        if (rc != CTM_OK || e != cudaSuccess || !c->pipe[h]) {
            cudaGetLastError();
            c->pipe[h] = nullptr;
            c->graph_failed = 1;
            return CTM_OK;
        }
        c->pipe_kernels = captured;
    }
    c->pipe_steps = k;
    return CTM_OK;
}

int ctm_complex_step(ctm_complex_ctx *c, int nsteps, double *delta_host)
{
    if (!c || nsteps < 1) return CTM_EINVAL;
    int rc;
    bool done = false;
    if (c->steps_done > 0 && !c->graph_failed) {
        // steps after the first (eager, autotuning) one: one captured graph of nsteps steps,
        // ordered after the caller's stream
        cudaStream_t user = c->stream;
        ZK(cudaEventRecord(c->ev_in, user));
        ZK(cudaStreamWaitEvent(c->own, c->ev_in, 0));
        c->stream = c->own;
        rc = zcapture(c, nsteps);
        cudaGraphExec_t ge = nsteps == 1 ? c->graph1 : c->graphK;
        if (rc == CTM_OK && ge) {
            if (cudaGraphLaunch(ge, c->stream) != cudaSuccess) rc = CTM_ECUDA;
            CTM_COUNT_LAUNCH(nsteps == 1 ? c->graph1_kernels : c->graphK_kernels);
            done = (rc == CTM_OK);
            if (done) c->steps_done += nsteps;
        }
        c->stream = user;
        ZK(cudaEventRecord(c->ev_out, c->own));
        ZK(cudaStreamWaitEvent(user, c->ev_out, 0));
        if (rc != CTM_OK) return rc;
    }
    for (int i = 0; i < nsteps && !done; ++i)
        if ((rc = zstep(c, i == nsteps - 1)) != CTM_OK) return rc;
    if ((rc = zread_status(c)) != CTM_OK) return rc;
    if (delta_host) {
        ZK(cudaMemcpyAsync(delta_host, c->delta, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        ZK(cudaStreamSynchronize(c->stream));
        if (!isfinite(*delta_host)) return CTM_ENONFINITE;
        return zcheck_env_finite(c);
    }
    return CTM_OK;
}

// Chunks of k steps from the two pipelined graphs on the private stream, as in the real
// path: a second chunk queued while the newest delta read is above 100 tol, queueing
// stopped once it is below tol, and the last executed step's own spectrum at the end.
static int zconverge_pipelined(ctm_complex_ctx *c, int k, int budget, double tol, int *ran, double *delta)
{
    *ran = 0;
    if (budget < k) return CTM_OK;
    int rc = zcapture_pipe(c, k);
    if (rc != CTM_OK || c->pipe_steps != k) return rc;
    int queue[2], nq = 0, next = 0, launched = 0, chunks_read = 0;
    bool stop = false;
    double newest = INFINITY;
    for (;;) {
        while (!stop && nq < (newest > 100.0 * tol ? 2 : 1) && launched + k <= budget) {
            const int h = next;
            next ^= 1;
            ZK(cudaGraphLaunch(c->pipe[h], c->stream));
            CTM_COUNT_LAUNCH(c->pipe_kernels);
            ZK(cudaEventRecord(c->pipe_done[h], c->stream));
            queue[nq++] = h;
            launched += k;
        }
        if (nq == 0) break;
        const int h = queue[0];
        queue[0] = queue[1];
        --nq;
        ZK(cudaEventSynchronize(c->pipe_done[h]));
        c->steps_done += k;
        *ran += k;
        const double *dh = c->ring_h + (size_t)h * c->ring_cap;
        const int first = chunks_read++ == 0 ? 1 : 0;   // slot 0 of the first chunk: no information
        bool finite = true;
        for (int i = first; i < k; ++i) finite = finite && isfinite(dh[i]);
        if (c->ring_err_h[h] || !finite) {
            ZK(cudaStreamSynchronize(c->stream));
            c->steps_done += nq * k;
            *ran += nq * k;
            *delta = NAN;
            return c->ring_err_h[h] ? CTM_ETIMEOUT : CTM_ENONFINITE;
        }
        if (k - 1 >= first) {
            newest = dh[k - 1];
            stop = newest < tol;
        }
    }
    // the last step's own spectrum
    if ((rc = zspectrum(c, c->C, c->stream)) != CTM_OK) return rc;
    ZK(cudaMemcpyAsync(delta, c->delta, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if ((rc = zread_status(c)) != CTM_OK) return rc;
    return isfinite(*delta) ? CTM_OK : CTM_ENONFINITE;
}

// A fresh context's first step runs eagerly; then pipelined chunks of check_every steps
// while that many are left, single steps otherwise (see ctm_converge).
int ctm_complex_converge(ctm_complex_ctx *c, int max_steps, double tol, int check_every, int *steps_out,
                         double *delta_out)
{
    if (!c) return CTM_EINVAL;
    if (max_steps <= 0) max_steps = c->cfg.max_steps;
    if (tol <= 0.0) tol = c->cfg.tol;
    if (check_every < 1) check_every = 1;
    if (max_steps <= 0) return CTM_EINVAL;
    int done = 0, rc = CTM_OK;
    double delta = INFINITY;
    while (!(delta < tol) && done < max_steps) {
        int ran = 0;
        if (c->steps_done > 0 && !c->graph_failed) {
            cudaStream_t user = c->stream;
            ZK(cudaEventRecord(c->ev_in, user));
            ZK(cudaStreamWaitEvent(c->own, c->ev_in, 0));
            c->stream = c->own;
            rc = zconverge_pipelined(c, check_every, max_steps - done, tol, &ran, &delta);
            c->stream = user;
            ZK(cudaEventRecord(c->ev_out, c->own));
            ZK(cudaStreamWaitEvent(user, c->ev_out, 0));
            done += ran;
            if (rc != CTM_OK) break;
        }
        if (ran == 0) {
            rc = ctm_complex_step(c, 1, &delta);
            ++done;
            if (rc != CTM_OK) break;
        }
    }
    if (steps_out) *steps_out = done;
    if (delta_out) *delta_out = delta;
    if (rc != CTM_OK) return rc;
    if ((rc = zcheck_env_finite(c)) != CTM_OK) return rc;
    return delta < tol ? CTM_OK : CTM_ENOTCONVERGED;
}

int ctm_complex_energy(ctm_complex_ctx *c, const double *h_dev, double *e_bond_host, double *e_site_host,
                       double *rho_host)
{
    if (!c || !h_dev) return CTM_EINVAL;
    const int chi = c->chi, D2 = c->D2, d = c->d, dd = d * d;
    const long long n = c->n, D3 = (long long)D2 * D2 * D2;
    int rc;
    if (dd > ZRHO_MAX_DD) return CTM_EUNSUPPORTED;
    // the rotated bond operators h'_a = W_a^H h_a W_a, W_x = U^2 (x) U^2, W_y = U (x) U, W_z = I:
    // the x and y bonds are the z bond of the rotated tensor (App. A, the C3 symmetry)
    double hh[3 * 2 * ZRHO_MAX_DD * ZRHO_MAX_DD];
    ZK(cudaMemcpyAsync(hh, h_dev, sizeof(double) * 3 * 2 * dd * dd, cudaMemcpyDeviceToHost, c->stream));
    ZK(cudaStreamSynchronize(c->stream));
    {
        HMat U = hm_zero(d);
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) U.v[i][j] = Cx{c->U[i][j][0], c->U[i][j][1]};
        const HMat U2 = hm_mul(U, U);
        double hr[3 * 2 * ZRHO_MAX_DD * ZRHO_MAX_DD];
        for (int a = 0; a < 3; ++a) {
            const HMat &V = a == 0 ? U2 : U;
            auto Wel = [&](int r, int q) -> Cx {   // (V (x) V)[r][q], r = (s, t)
                if (a == 2) return Cx{r == q ? 1.0 : 0.0, 0.0};
                return cmul(V.v[r / d][q / d], V.v[r % d][q % d]);
            };
            for (int r = 0; r < dd; ++r)
                for (int q = 0; q < dd; ++q) {
                    Cx acc{0.0, 0.0};
                    for (int i = 0; i < dd; ++i)
                        for (int j = 0; j < dd; ++j) {
                            const double *hv = hh + 2 * ((size_t)a * dd * dd + i * dd + j);
                            acc = cadd(acc, cmul(cmul(cconj(Wel(i, r)), Cx{hv[0], hv[1]}), Wel(j, q)));
                        }
                    hr[2 * ((size_t)a * dd * dd + r * dd + q)] = acc.re;
                    hr[2 * ((size_t)a * dd * dd + r * dd + q) + 1] = acc.im;
                }
        }
        ZK(cudaMemcpyAsync(c->hrot, hr, sizeof(double) * 3 * 2 * dd * dd, cudaMemcpyHostToDevice, c->stream));
        ZK(cudaStreamSynchronize(c->stream));
    }
    // projector of one more step and Ch = sym(Q^H M Q)/|.|
    if ((rc = zenlarged_corner(c)) != CTM_OK) return rc;
    if ((rc = zprojector(c)) != CTM_OK) return rc;
    if ((rc = zcorner(c, c->Cn)) != CTM_OK) return rc;
    // P5 = Ch^5 (the last product into P5b's five planes)
    const double *src = c->Cn;
    double *bufs[2] = {c->P5a, c->P5b};
    const long long DD = (long long)D2 * D2;
    for (int p = 0; p < 4; ++p) {
        double *dst = bufs[p & 1];
        ZGemm z{chi, chi, chi, src, c->PC, p == 0, idx_lin(chi), idx_lin(1), 0, c->Cn, c->PC, idx_lin(chi), idx_lin(1),
                0, dst, c->PC, p == 3, idx_lin(chi), idx_lin(1)};
        if ((rc = zgemm(c, z)) != CTM_OK) return rc;
        src = dst;
    }
    ZLAUNCH(zc_complete_kernel, zgrid((long long)chi * chi), 256, (long long)chi * chi, c->P5b,
            zlay_stacked((long long)chi * chi, 5));
    // F = Q P5 (n x chi) into W; E'[(a,b)][(x,y)] = E[(b,x),(a,y)], E = F Q^H, into H
    ZGemm z{(int)n, chi, chi, c->Qn, c->PQ, 1, idx_lin(chi), idx_lin(1), 0, c->P5b, c->PC, idx_lin(chi), idx_lin(1), 0,
            c->W, chi, 0, idx_lin(2LL * chi), idx_lin(1)};
    if ((rc = zgemm(c, z)) != CTM_OK) return rc;
    z = ZGemm{(int)n, (int)n, chi, c->W, chi, 0, idx_lin(2LL * chi), idx_lin(1), 0, c->Qn, c->PQ, idx_lin(1),
              idx_lin(chi), 1, c->H, c->PM, 0, idx_split(D2, DD, D2), idx_split(D2, (long long)chi * DD, 1)};
    if ((rc = zgemm(c, z)) != CTM_OK) return rc;
    // open layers: the outer site B with its legs as they are, the apex site A with z first
    CTM_COUNT_LAUNCH(2);
    zc_open_layers_kernel<<<zgrid(D3 * dd), 256, 0, c->stream>>>(d, c->D, c->A, c->PA, 0, c->bB);
    zc_open_layers_kernel<<<zgrid(D3 * dd), 256, 0, c->stream>>>(d, c->D, c->A, c->PA, 1, c->bA);
    ZK(cudaGetLastError());
    // Y1o[(a,b)][(pB,z)] = sum_{u,l} X'[(a,b),(u,l)] bB[pB][u][l][z]
    z = ZGemm{chi * chi, dd * D2, D2 * D2, c->X, DD, 0, idx_lin(2 * DD), idx_lin(1), 0, c->bB, c->Pb, idx_lin(D2),
              idx_split(D2, D3, 1), 0, c->Y1o, c->PYo, 0, idx_lin((long long)dd * D2), idx_lin(1)};
    if ((rc = zgemm(c, z)) != CTM_OK) return rc;
    // G2[(a,b)][(pA,z)] = sum_{x,y} E'[(a,b),(x,y)] bA[pA][z][x][y]
    z = ZGemm{chi * chi, dd * D2, D2 * D2, c->H, c->PM, 0, idx_lin(DD), idx_lin(1), 0, c->bA, c->Pb, idx_lin(1),
              idx_split(D2, D3, DD), 0, c->G2, c->PYo, 0, idx_lin((long long)dd * D2), idx_lin(1)};
    if ((rc = zgemm(c, z)) != CTM_OK) return rc;
    ZLAUNCH(zc_rho_partial_kernel, ZRHO_BLOCKS, 256, (long long)chi * chi, dd, D2, c->Y1o, c->G2, c->PYo,
            c->rho_part);
    ZLAUNCH(zc_energy_kernel, 1, 32, d, ZRHO_BLOCKS, c->rho_part, c->hrot, c->eout);
    double host[4 + 2 * ZRHO_MAX_DD * ZRHO_MAX_DD];
    ZK(cudaMemcpyAsync(host, c->eout, sizeof(double) * (4 + 2 * dd * dd), cudaMemcpyDeviceToHost, c->stream));
    if ((rc = zread_status(c)) != CTM_OK) return rc;
    for (int i = 0; i < 4 + 2 * dd * dd; ++i)
        if (!isfinite(host[i])) return CTM_ENONFINITE;
    if (e_bond_host)
        for (int i = 0; i < 3; ++i) e_bond_host[i] = host[i];
    if (e_site_host) *e_site_host = host[3];
    if (rho_host)
        for (int i = 0; i < 2 * dd * dd; ++i) rho_host[i] = host[4 + i];
    return CTM_OK;
}

int ctm_complex_get_env(const ctm_complex_ctx *c, double *C_dev, double *T_dev, double *Q_dev)
{
    if (!c) return CTM_EINVAL;
    cudaStream_t st = c->stream;
    auto out = [&](const double *src, long long cnt, ZLay L, double *dst) -> bool {
        CTM_COUNT_LAUNCH(1);
        zc_interleave_kernel<<<zgrid(cnt), 256, 0, st>>>(cnt, src, L, dst);
        return cudaGetLastError() == cudaSuccess;
    };
    if (C_dev && !out(c->C, c->PC, zlay_stacked(c->PC, 5), C_dev)) return CTM_ECUDA;
    if (T_dev && !out(c->T, c->PT, lay_T(c), T_dev)) return CTM_ECUDA;
    if (Q_dev && !out(c->Q, c->PQ, zlay_stacked(c->PQ, 5), Q_dev)) return CTM_ECUDA;
    ZK(cudaStreamSynchronize(st));
    return CTM_OK;
}

int ctm_complex_set_env(ctm_complex_ctx *c, const double *C_dev, const double *T_dev, const double *Q_dev)
{
    if (!c || !C_dev || !T_dev || !Q_dev) return CTM_EINVAL;
    cudaStream_t st = c->stream;
    CTM_COUNT_LAUNCH(3);
    zc_load_kernel<<<zgrid(c->PC), 256, 0, st>>>(c->PC, C_dev, c->C, zlay_stacked(c->PC, 5));
    zc_load_kernel<<<zgrid(c->PT), 256, 0, st>>>(c->PT, T_dev, c->T, lay_T(c));
    zc_load_kernel<<<zgrid(c->PQ), 256, 0, st>>>(c->PQ, Q_dev, c->Q, zlay_stacked(c->PQ, 5));
    ZK(cudaGetLastError());
    // the spectrum of the new corner becomes the reference for the next delta
    if (zspectrum(c, c->C, st) != CTM_OK) return CTM_ECUDA;
    ZK(cudaStreamSynchronize(st));
    return CTM_OK;
}

int ctm_complex_get_intermediate(const ctm_complex_ctx *c, int which, double *dst, size_t count)
{
    if (!c || !dst) return CTM_EINVAL;
    const long long chi = c->chi, D2 = c->D2, n = c->n;
    cudaStream_t st = c->stream;
    const double *src = nullptr;
    long long cnt = 0;
    ZLay L;
    switch (which) {
    case 0: src = c->M; cnt = n * n; L = zlay_rows(n, 2); break;
    case 1: src = c->Y; cnt = n * chi; L = zlay_stacked(c->PY, 2); break;
    case 2: src = c->R; cnt = chi * chi; L = zlay_stacked(c->PC, 2); break;
    case 3: src = c->Q; cnt = n * chi; L = zlay_stacked(c->PQ, 5); break;
    case 4: {   // the corner spectrum (real)
        if (count < (size_t)chi) return CTM_EINVAL;
        ZK(cudaMemcpyAsync(dst, c->s, sizeof(double) * chi, cudaMemcpyDeviceToDevice, st));
        ZK(cudaStreamSynchronize(st));
        return CTM_OK;
    }
    case 5: src = c->A; cnt = c->PA; L = zlay_stacked(c->PA, 2); break;
    case 6: src = c->a; cnt = D2 * D2 * D2; L = zlay_stacked(c->Pa, 5); break;
    case 7: src = c->C; cnt = chi * chi; L = zlay_stacked(c->PC, 5); break;
    case 8: src = c->T; cnt = chi * D2 * chi; L = lay_T(c); break;
    default: return CTM_EINVAL;
    }
    if (count < (size_t)(2 * cnt)) return CTM_EINVAL;
    CTM_COUNT_LAUNCH(1);
    zc_interleave_kernel<<<zgrid(cnt), 256, 0, st>>>(cnt, src, L, dst);
    ZK(cudaGetLastError());
    ZK(cudaStreamSynchronize(st));
    return CTM_OK;
}

void ctm_complex_destroy(ctm_complex_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    if (c->graph1) cudaGraphExecDestroy(c->graph1);
    if (c->graphK) cudaGraphExecDestroy(c->graphK);
    if (c->own) {
        cudaStreamSynchronize(c->own);
        cudaStreamDestroy(c->own);
    }
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
    }
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    for (int h = 0; h < 2; ++h) {
        if (c->pipe[h]) cudaGraphExecDestroy(c->pipe[h]);
        if (c->pipe_done[h]) cudaEventDestroy(c->pipe_done[h]);
    }
    if (c->ring_h) cudaFreeHost(c->ring_h);
    if (c->ring_err_h) cudaFreeHost(c->ring_err_h);
    delete c;
}

size_t ctm_complex_transfer_workspace_bytes(const ctm_complex_ctx *c, int nev)
{
    if (!c || nev < 2 || 2 * nev + 5 > SUBSPACE_MAXV) return 0;
    double *Vq, *Tp;
    void *sub;
    return ztransfer_layout(c, 2 * nev + 5, nullptr, &Vq, &Tp, &sub);
}

int ctm_complex_transfer_spectrum(ctm_complex_ctx *c, int nev, int max_iter, double tol, void *tws, size_t tws_bytes,
                                  double *lambda_host, double *xi_host, double *gap_host, int *iters_out)
{
    if (!c || !tws || !lambda_host || nev < 2 || 2 * nev + 5 > SUBSPACE_MAXV || max_iter < 1) return CTM_EINVAL;
    if ((uintptr_t)tws % 256 != 0) return CTM_EINVAL;
    if (tws_bytes < ctm_complex_transfer_workspace_bytes(c, nev)) return CTM_ENOMEM;
    if (tol <= 0.0) tol = 1e-12;
    if (c->side_pending) {
        ZK(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
        c->side_pending = 0;
    }
    const int m = 2 * nev + 5;
    const long long N = (long long)c->chi * c->D2 * c->chi;
    double *Vq, *Tp;
    void *sub;
    ztransfer_layout(c, m, (char *)tws, &Vq, &Tp, &sub);
    ZLAUNCH(zc_tr_unblock_kernel, zgrid(5 * N), 256, N, c->chi, c->T, Tp);
    SubspaceWork sw{c->stream, c->splitk, c->splitk_elems, c->err};
    int rc = subspace_spectrum(
        sw, 2 * N, m, nev, 2, max_iter, tol, sub,
        [c, Vq, Tp](const double *v, double *out) {
            return ztransfer_apply(c, v, out, Vq, Tp) == CTM_OK ? cudaSuccess : cudaErrorUnknown;
        },
        lambda_host, iters_out);
    if (rc != CTM_OK && rc != CTM_ENOTCONVERGED) return rc;
    if (xi_host) *xi_host = lambda_host[1] > 0.0 ? -1.0 / log(lambda_host[1]) : 0.0;
    if (gap_host) *gap_host = (nev >= 3 && lambda_host[2] > 0.0) ? log(lambda_host[1] / lambda_host[2]) : INFINITY;
    return rc;
}

}  // extern "C"
