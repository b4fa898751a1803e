// C ABI of libctm: context, workspace layout and the launch sequence of one
// QR-based C3v CTMRG step (Sec. II.B, Fig. 3) and of the bond-energy
// evaluation (Sec. II.C, Eq. 1).  See include/ctm.h for the contract.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "ctm_ctx.h"

namespace {

// ---------------------------------------------------------------- rho reduction
// raw[pB][pA] = sum_{ab, z} Y1o[ab][pB][z] * G2[ab][pA][z]  (dd = d^2 <= 9)
constexpr int RHO_MAX_DD = 9;

__global__ void rho_partial_kernel(long long nab, int dd, int D2, const double *Y1o, const double *G2,
                                   double *partials)
{
    __shared__ double red[RHO_MAX_DD * RHO_MAX_DD][8];
    double acc[RHO_MAX_DD * RHO_MAX_DD];
    for (int i = 0; i < dd * dd; ++i) acc[i] = 0.0;
    const long long row = (long long)dd * D2;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nab * D2;
         t += (long long)gridDim.x * blockDim.x) {
        long long ab = t / D2;
        int z = (int)(t - ab * D2);
        const double *y = Y1o + ab * row + z;
        const double *g = G2 + ab * row + z;
        for (int pb = 0; pb < dd; ++pb) {
            double yv = y[(size_t)pb * D2];
            for (int pa = 0; pa < dd; ++pa) acc[pb * dd + pa] = fma(yv, g[(size_t)pa * D2], acc[pb * dd + pa]);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = 0; i < dd * dd; ++i) {
        double v = acc[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[i][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < dd * dd) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
        partials[(size_t)blockIdx.x * dd * dd + threadIdx.x] = s;
    }
}

__global__ void rho_final_kernel(int nblocks, int dd, const double *partials, double *raw)
{
    int i = threadIdx.x;
    if (i >= dd * dd) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partials[(size_t)b * dd * dd + i];
    raw[i] = s;
}

constexpr int RHO_BLOCKS = 256;
constexpr int NORM_BLOCKS = 256;


}  // namespace


namespace ctmi {

struct Shape {
    int M, N, K;
};

// (M, N, K) of the eleven contractions of one step, in launch order.
std::vector<Shape> step_shapes(const ctm_ctx *c)
{
    const int chi = c->chi, D2 = c->D2, n = (int)c->n;
    return {{n, chi, chi},         {n, n, chi},   {chi * chi, D2, D2 * D2}, {chi * chi, D2 * D2, D2},
            {n, chi, n},           {n, chi, n},   {chi, chi, n},            {n, n, chi},
            {chi * chi, D2, D2 * D2}, {chi * chi, D2 * D2, D2}, {chi, n, n}};
}

// Carve the workspace.  With base == nullptr only the size is computed.
size_t layout(ctm_ctx *c, char *base)
{
    const long long chi = c->chi, D2 = c->D2, n = c->n, d = c->d;
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off += align_up(bytes);
        return p;
    };
    auto td = [&](long long count) -> double * { return (double *)take(sizeof(double) * (size_t)count); };
    c->Araw = td(d * c->D * c->D * c->D);
    c->A = td(d * c->D * c->D * c->D);
    c->a = td(D2 * D2 * D2);
    c->C = td(chi * chi);
    c->Cn = td(chi * chi);
    c->Cr = td(chi * chi);
    c->Cspec = td(chi * chi);
    c->T = td(chi * D2 * chi);
    c->Tn = td(chi * D2 * chi);
    c->Q = td(n * chi);
    c->Qn = td(n * chi);
    c->Qs = td(n * chi);
    c->Y = td(n * chi);
    c->W = td(n * chi);
    c->MQ = td(n * chi);
    c->R = td(chi * chi);
    c->M = td(n * n);
    c->X = td(n * n);
    c->H = td(n * n);
    c->Y1 = td(chi * chi * D2);
    c->s = td(chi);
    c->s_new = td(chi);
    c->delta = td(8);
    c->spec_work = td((long long)spectrum_work_doubles((int)chi));
    // split-K scratch: the largest ksplit * M * N over the step's GEMMs
    size_t sk = 0;
    auto need = [&](long long M, long long N, long long K) {
        int s = gemm_f64_pick_split((int)M, (int)N, (int)K);
        if (s > 1 && (size_t)(s * M * N) > sk) sk = (size_t)(s * M * N);
    };
    need(n, chi, chi);
    need(n, n, chi);
    need(chi * chi, D2, D2 * D2);
    need(chi * chi, D2 * D2, D2);
    need(n, chi, n);
    need(chi, chi, n);
    need(n, D2 * chi, chi);
    need(chi, D2 * chi, n);
    need(chi, chi, chi);
    need(chi * chi, d * d * D2, D2 * D2);
    c->splitk_elems = sk;
    c->splitk = td((long long)sk + 1);
    c->qr_sbuf = td((long long)qr_scratch_doubles((int)chi));
    c->qr_rowbuf = td((long long)qr_rowbuf_doubles((int)chi));
    c->qr_wy = td((long long)qr_wy_doubles((int)n, (int)chi));
    c->qr_slab_elems = qr_slab_doubles((int)n, (int)chi, c->qr_force_slab);
    c->qr_slab = c->qr_slab_elems ? td((long long)c->qr_slab_elems) : nullptr;
    if (c->cfg.deterministic) {
        c->qr_gmax = qr_det_gmax((int)n);
        c->qr_gpart = td((long long)qr_det_gram_doubles((int)chi, c->qr_gmax));
        c->qr_spart = td((long long)qr_det_s_doubles((int)chi, c->qr_gmax));
    }
    c->qr_bar = (unsigned *)take(64);
    c->err = (int *)take(64);
    c->flag = (int *)take(64);
    c->norm_part = td(NORM_BLOCKS);
    c->norm_part2 = td(NORM_BLOCKS);
    c->b = td(d * d * D2 * D2 * D2);
    c->Y1o = td(chi * chi * d * d * D2);
    c->G2 = td(chi * chi * d * d * D2);
    c->P5a = td(chi * chi);
    c->P5b = td(chi * chi);
    c->rho_part = td((long long)RHO_BLOCKS * d * d * d * d);
    c->rho_raw = td(d * d * d * d);
    c->eout = td(4 + d * d * d * d);
    c->h = td(3 * d * d * d * d);
    if (c->tf32_T > 0) {
        // packed TF32 slices, exponents and the split-K FP64 accumulator for the largest
        // operand of the step's, the energy's and the transfer spectrum's contractions
        size_t ap = 0, bp = 0, pp = 0;
        long long ecap = 0;
        std::vector<Shape> shapes = step_shapes(c);
        shapes.push_back({(int)n, (int)n, (int)chi});
        shapes.push_back({(int)(chi * chi), (int)(d * d * D2), (int)(D2 * D2)});
        for (const auto &sh : shapes) {
            SplitPlan pl = tf32_plan_caps(sh.M, sh.N, sh.K, c->tf32_T);
            if (pl.a_pack_bytes > ap) ap = pl.a_pack_bytes;
            if (pl.b_pack_bytes > bp) bp = pl.b_pack_bytes;
            if (pl.partial_bytes > pp) pp = pl.partial_bytes;
            if (sh.M > ecap) ecap = sh.M;
            if (sh.N > ecap) ecap = sh.N;
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
        c->sw.autotune = 0;
        // the corner update (lane2) and the edge update run concurrently after the first
        // step: the corner lane gets its own B pack, exponents and split-K buffer, the
        // edge lane its own A pack and exponents
        c->sw_c = c->sw;
        c->sw_c.Bpk = (unsigned char *)take(bp);
        c->sw_c.eB = (int *)take(sizeof(int) * (size_t)ecap);
        c->sw_c.partial = (void *)take(pp + 8);
        c->sw_e = c->sw;
        c->sw_e.Apk = (unsigned char *)take(ap);
        c->sw_e.eA = (int *)take(sizeof(int) * (size_t)ecap);
    }
    if (c->split_T > 0) {
        // packed digit slices, exponents and the split-K integer accumulator for the
        // largest operand of the step's contractions
        size_t ap = 0, bp = 0, pp = 0;
        long long ecap = 0;
        std::vector<Shape> shapes = step_shapes(c);
        // the energy's large contractions (E = W Q^T and the two open-layer contractions)
        shapes.push_back({(int)n, (int)n, (int)chi});
        shapes.push_back({(int)(chi * chi), (int)(d * d * D2), (int)(D2 * D2)});
        for (const auto &sh : shapes) {
            SplitPlan pl = split_plan_caps(sh.M, sh.N, sh.K, c->split_T);
            if (pl.a_pack_bytes > ap) ap = pl.a_pack_bytes;
            if (pl.b_pack_bytes > bp) bp = pl.b_pack_bytes;
            if (pl.partial_bytes > pp) pp = pl.partial_bytes;
            if (sh.M > ecap) ecap = sh.M;
            if (sh.N > ecap) ecap = sh.N;
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
        c->sw.autotune = 1;   // the first eager call of each contraction shape times its plans
        // the two lanes of the corner / edge updates (see enqueue_step)
        c->sw_c = c->sw;
        c->sw_c.Bpk = (unsigned char *)take(bp);
        c->sw_c.eB = (int *)take(sizeof(int) * (size_t)ecap);
        c->sw_c.partial = (void *)take(pp + 8);
        c->sw_e = c->sw;
        c->sw_e.Apk = (unsigned char *)take(ap);
        c->sw_e.eA = (int *)take(sizeof(int) * (size_t)ecap);
        const Shape ash[2] = {{(int)(chi * chi), (int)D2, (int)(D2 * D2)}, {(int)(chi * chi), (int)(D2 * D2), (int)D2}};
        for (int sl = 0; sl < 2; ++sl) {
            SplitPlan pl = split_plan_caps(ash[sl].M, ash[sl].N, ash[sl].K, c->split_T);
            c->apk[sl] = (unsigned char *)take(pl.b_pack_bytes);
            c->apk_cap[sl] = pl.b_pack_bytes;
            c->ape[sl] = (int *)take(sizeof(int) * (size_t)ash[sl].N);
            c->apk_state[sl] = 0;
        }
        // A packs kept for a second contraction: T (n x chi) and Q^T (chi x n)
        const Shape csh[2] = {{(int)n, (int)chi, (int)chi}, {(int)chi, (int)chi, (int)n}};
        for (int sl = 0; sl < 2; ++sl) {
            SplitPlan pl = split_plan_caps(csh[sl].M, csh[sl].N, csh[sl].K, c->split_T);
            c->ack[sl] = (unsigned char *)take(pl.a_pack_bytes);
            c->ack_cap[sl] = pl.a_pack_bytes;
            c->ace[sl] = (int *)take(sizeof(int) * (size_t)csh[sl].M);
            c->ack_valid[sl] = 0;
        }
    }
    return off;
}

int tf32_slices(int precision)
{
    return precision == CTM_SPLIT_TF32 ? 2 : (precision == CTM_FP32_TF32 ? 1 : 0);
}

bool config_ok(const ctm_config *cfg)
{
    if (!cfg) return false;
    if (cfg->d < 1 || cfg->d > 3) return false;
    if (cfg->D < 1 || cfg->D > 12) return false;
    if (cfg->chi < 1 || cfg->chi > 512) return false;   // the QR's and the corner spectrum's limit
    if (cfg->precision != CTM_FP64 && cfg->precision != CTM_SPLIT_BF16 && cfg->precision != CTM_SPLIT_TF32 &&
        cfg->precision != CTM_FP32_TF32)
        return false;
    if (cfg->precision == CTM_SPLIT_BF16 && !split_supported_T(cfg->n_split)) return false;
    if (cfg->corner_mode != 0 && cfg->corner_mode != 1) return false;
    if (cfg->deterministic != 0 && cfg->deterministic != 1) return false;
    long long n = (long long)cfg->chi * cfg->D * cfg->D;
    if (n > 20000) return false;
    return true;
}

// The step's contractions: FP64 GEMM, or the split-BF16 tcgen05 engine.
cudaError_t run_gemm(ctm_ctx *c, const GemmF64 &g, int hint, int lane)
{
    cudaEvent_t *ev = nullptr;
    if (c->prof_on && c->prof_n + 3 <= CTM_PROF_EVENTS) {
        ev = c->prof_ev + c->prof_n;
        c->prof_n += 3;
    }
    if (c->tf32_T > 0) {
        const SplitWork &w = lane == 1 ? c->sw_c : (lane == 2 ? c->sw_e : c->sw);
        return gemm_tf32(g, c->tf32_T, w, lane == 1 ? c->lane2 : c->stream, ev);
    }
    if (c->split_T > 0) {
        SplitOpts o{};
        if (hint == GEMM_REUSE_A) o.reuse_a = 1;
        if (hint == GEMM_B_IS_A_LZ || hint == GEMM_B_IS_A_ZX) {
            const int slot = hint == GEMM_B_IS_A_LZ ? 0 : 1;
            o.b_pk = c->apk[slot];
            o.b_e = c->ape[slot];
            o.b_cap = c->apk_cap[slot];
            o.b_state = &c->apk_state[slot];
        }
        int fill_slot = -1;
        if (hint >= GEMM_A_FILL_T && hint <= GEMM_A_USE_Q) {
            const int slot = (hint == GEMM_A_FILL_T || hint == GEMM_A_USE_T) ? 0 : 1;
            const bool use = (hint == GEMM_A_USE_T || hint == GEMM_A_USE_Q) && c->ack_valid[slot];
            o.a_pk = c->ack[slot];
            o.a_e = c->ace[slot];
            o.a_cap = c->ack_cap[slot];
            o.a_fill = use ? 0 : 1;
            if (!use) fill_slot = slot;
        }
        const SplitWork &w = lane == 1 ? c->sw_c : (lane == 2 ? c->sw_e : c->sw);
        cudaError_t e = gemm_split(g, c->split_T, w, lane == 1 ? c->lane2 : c->stream, ev, &o);
        if (fill_slot >= 0) c->ack_valid[fill_slot] = (e == cudaSuccess);
        return e;
    }
    if (ev) {
        cudaEventRecord(ev[2], c->stream);   // no pre-pass in FP64
        cudaEventRecord(ev[0], c->stream);
    }
    cudaError_t e = gemm_f64(g, gemm_f64_pick_split(g.M, g.N, g.K), c->splitk, c->splitk_elems, c->stream);
    if (ev) cudaEventRecord(ev[1], c->stream);
    return e;
}

#define CK(expr)                                          \
    do {                                                  \
        cudaError_t _e = (expr);                          \
        if (_e != cudaSuccess) return CTM_ECUDA;          \
    } while (0)

// ---------------------------------------------------------------- enlarged corner
// Fig. 3(c): X'[a][b][u][l] = sum_{g,h} T[a,u,g] C[g,h] T[b,l,h];
// Y1[(a,b)][z] = sum_{u,l} X' aB[u,l,z]; M[(a,y)][(b,x)] = sum_z Y1 aA[z,x,y].
int enqueue_enlarged_corner(ctm_ctx *c)
{
    const int chi = c->chi, D2 = c->D2;
    const long long n = c->n;
    GemmF64 g;
    // W = T C (T's packed digits are kept for H1' = T Q of the edge update)
    g = GemmF64{(int)n, chi, chi, c->T, idx_lin(chi), idx_lin(1), c->C, idx_lin(chi), idx_lin(1),
                c->W, idx_lin(chi), idx_lin(1), 1.0, 0.0};
    c->ack_valid[0] = 0;
    CK(run_gemm(c, g, GEMM_A_FILL_T));
    // X'[a][b][u][l] = W[(a,u),h] T[(b,l),h]
    g = GemmF64{(int)n, (int)n, chi, c->W, idx_lin(chi), idx_lin(1), c->T, idx_lin(1), idx_lin(chi),
                c->X, idx_split(D2, (long long)chi * D2 * D2, D2), idx_split(D2, (long long)D2 * D2, 1), 1.0, 0.0};
    CK(run_gemm(c, g));
    // Y1 = X' a   (chi^2 x D2^2) (D2^2 x D2)
    g = GemmF64{chi * chi, D2, D2 * D2, c->X, idx_lin((long long)D2 * D2), idx_lin(1), c->a, idx_lin(D2),
                idx_lin(1), c->Y1, idx_lin(D2), idx_lin(1), 1.0, 0.0};
    CK(run_gemm(c, g, GEMM_B_IS_A_LZ));
    // M[(a,y)][(b,x)] = Y1[(a,b), z] a[z, x, y]; the GEMM column index runs over (y, x)
    // with x fastest, so an output tile covers whole contiguous (b, x) runs of M
    g = GemmF64{chi * chi, D2 * D2, D2, c->Y1, idx_lin(D2), idx_lin(1), c->a, idx_lin((long long)D2 * D2),
                idx_split(D2, 1, D2), c->M, idx_split(chi, (long long)D2 * n, D2), idx_split(D2, n, 1), 1.0, 0.0};
    CK(run_gemm(c, g, GEMM_B_IS_A_ZX));
    return CTM_OK;
}

// Fig. 3(d): Y = M Qs, Qs = Q diag(sgn C_jj); Householder QR -> Qout, R.
int enqueue_projector(ctm_ctx *c, double *Qout)
{
    const int chi = c->chi;
    const long long n = c->n;
    cudaStream_t st = c->stream;
    c->ack_valid[1] = 0;   // the QR below writes a new Q
    CK(launch_warm_start((int)n, chi, c->Q, c->C, c->Qs, st));
    GemmF64 g{(int)n, chi, (int)n, c->M, idx_lin(n), idx_lin(1), c->Qs, idx_lin(chi), idx_lin(1),
              c->Y, idx_lin(chi), idx_lin(1), 1.0, 0.0};
    CK(run_gemm(c, g));
    QrScratch qs = qr_scratch(c);
    CK(qr_householder((int)n, chi, c->Y, Qout, c->R, qs, st));
    return CTM_OK;
}

// Fig. 3(a): Cout = sym(Qp^T M Qp) / |.|_F.
// lane 1 (split mode): on lane2, with the corner lane's work buffers.
int enqueue_corner(ctm_ctx *c, const double *Qp, double *Cout, int lane = 0)
{
    const int chi = c->chi;
    const long long n = c->n;
    cudaStream_t st = lane == 1 ? c->lane2 : c->stream;
    // the previous split contraction was Y = M Qs (only the QR in between): M is already packed
    GemmF64 g{(int)n, chi, (int)n, c->M, idx_lin(n), idx_lin(1), Qp, idx_lin(chi), idx_lin(1),
              c->MQ, idx_lin(chi), idx_lin(1), 1.0, 0.0};
    CK(run_gemm(c, g, GEMM_REUSE_A, lane));
    g = GemmF64{chi, chi, (int)n, Qp, idx_lin(1), idx_lin(chi), c->MQ, idx_lin(chi), idx_lin(1),
                c->Cr, idx_lin(chi), idx_lin(1), 1.0, 0.0};
    CK(run_gemm(c, g, (Qp == c->Qn || Qp == c->Q) ? GEMM_A_FILL_Q : GEMM_PLAIN, lane));
    CK(launch_corner_sym_normalize(chi, c->Cr, Cout, lane == 1 ? c->norm_part2 : c->norm_part, st));
    return CTM_OK;
}

// Cheap corner variant: Cout = sym(R S)/|.|_F with S = diag(sgn C_jj) of the corner
// that entered the step (R S = Q^T M Q_prev exactly; = Q^T M Q at a fixed point).
int enqueue_corner_from_r(ctm_ctx *c, double *Cout)
{
    const int chi = c->chi;
    CK(launch_warm_start(chi, chi, c->R, c->C, c->Cr, c->stream));
    CK(launch_corner_sym_normalize(chi, c->Cr, Cout, c->norm_part, c->stream));
    return CTM_OK;
}

// Fig. 3(b): T'[i,x,j] = sum Q[(a,y),i] T[a,u,g] a[u,w,z] a[z,x,y] Q[(g,w),j], normalised.
// lane 2 (split mode): with the edge lane's work buffers, concurrent with a corner
// update on lane2; the last contraction waits for it (it uses the corner's pack of Q^T).
int enqueue_edge(ctm_ctx *c, const double *Qp, double *Tout, int lane = 0)
{
    const int chi = c->chi, D2 = c->D2;
    const long long n = c->n;
    cudaStream_t st = c->stream;
    GemmF64 g;
    // H1'[a][j][u][w] = sum_g T[(a,u),g] Q[(g,w),j]; column index (j, w), w fastest
    g = GemmF64{(int)n, (int)n, chi, c->T, idx_lin(chi), idx_lin(1), Qp, idx_lin(n), idx_split(D2, 1, chi),
                c->X, idx_split(D2, (long long)chi * D2 * D2, D2), idx_split(D2, (long long)D2 * D2, 1), 1.0, 0.0};
    CK(run_gemm(c, g, GEMM_A_USE_T, lane));
    // H2[(a,j)][z] = H1'[(a,j),(u,w)] a[(u,w),z]
    g = GemmF64{chi * chi, D2, D2 * D2, c->X, idx_lin((long long)D2 * D2), idx_lin(1), c->a, idx_lin(D2),
                idx_lin(1), c->Y1, idx_lin(D2), idx_lin(1), 1.0, 0.0};
    CK(run_gemm(c, g, GEMM_B_IS_A_LZ, lane));
    // H3'[a][y][x][j] = H2[(a,j),z] a[z, x, y]; column index (y, x), x fastest
    g = GemmF64{chi * chi, D2 * D2, D2, c->Y1, idx_lin(D2), idx_lin(1), c->a, idx_lin((long long)D2 * D2),
                idx_split(D2, 1, D2), c->H, idx_split(chi, (long long)D2 * D2 * chi, 1),
                idx_split(D2, (long long)D2 * chi, chi), 1.0, 0.0};
    CK(run_gemm(c, g, GEMM_B_IS_A_ZX, lane));
    // T'[i][(x,j)] = sum_{(a,y)} Q[(a,y),i] H3'[(a,y),(x,j)]
    g = GemmF64{chi, (int)n, (int)n, Qp, idx_lin(1), idx_lin(chi), c->H, idx_lin(n), idx_lin(1),
                Tout, idx_lin(n), idx_lin(1), 1.0, 0.0};
    if (lane == 2) CK(cudaStreamWaitEvent(st, c->ev_corner, 0));
    CK(run_gemm(c, g, (Qp == c->Qn || Qp == c->Q) ? GEMM_A_USE_Q : GEMM_PLAIN, lane));
    CK(launch_normalize((long long)chi * D2 * chi, Tout, c->norm_part, NORM_BLOCKS, st));
    return CTM_OK;
}

// The corner spectrum of step t runs on the side stream while the step (in split
// mode from the corner update on) and step t+1 compute; it reads C' (its copy
// Cspec in split mode, else C once handed over at the end of step t) and must
// finish before that buffer is rewritten.  `side_pending` marks spectrum work not
// yet joined into the caller's stream; every public call joins it before returning.
int enqueue_step(ctm_ctx *c)
{
    int rc;
    cudaStream_t st = c->stream;
    const long long chi = c->chi, D2 = c->D2, n = c->n;
    if (c->spec_head) {
        // the deferred spectrum of the corner this step starts from, beside the
        // step; C is rewritten only at the hand-over, which waits for it (below,
        // or through the corner update that waits for ev_join)
        CK(cudaEventRecord(c->ev_fork, st));
        CK(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
        CK(launch_spectrum((int)chi, c->C, c->s_new, c->s, c->delta, c->spec_work, c->side, c->qr_rows_min <= 1));
        CK(cudaMemcpyAsync(c->s, c->s_new, sizeof(double) * chi, cudaMemcpyDeviceToDevice, c->side));
        if (c->delta_head)
            CK(cudaMemcpyAsync(c->delta_head, c->delta, sizeof(double), cudaMemcpyDeviceToHost, c->side));
        CK(cudaEventRecord(c->ev_join, c->side));
        c->side_pending = 1;
    }
    // Split mode after the first step (whose eager contractions time their plans
    // one at a time): the corner and edge updates both need only Q, so the corner
    // update runs on lane2 beside the edge update.  This path also writes the new
    // environment in place: C, T and Q are not read after the QR except by their
    // own updates (the warm start and the enlarged corner come before it; the edge
    // update reads T in its first contraction, before its last one writes T'), so
    // no hand-over copies are needed.
    const bool lanes = (c->split_T > 0 || c->tf32_T > 0) && c->steps_done > 0 && c->cfg.corner_mode == 0;
    if ((rc = enqueue_enlarged_corner(c)) != CTM_OK) return rc;
    if ((rc = enqueue_projector(c, lanes ? c->Q : c->Qn)) != CTM_OK) return rc;
    if (lanes) {
        CK(cudaEventRecord(c->ev_q, st));
        CK(cudaStreamWaitEvent(c->lane2, c->ev_q, 0));
        // the previous step's spectrum (reading C or Cspec) is done before C or Cspec is rewritten
        if (c->side_pending) CK(cudaStreamWaitEvent(c->lane2, c->ev_join, 0));
        if ((rc = enqueue_corner(c, c->Q, c->C, 1)) != CTM_OK) return rc;
        if (!c->spec_skip)
            CK(cudaMemcpyAsync(c->Cspec, c->C, sizeof(double) * chi * chi, cudaMemcpyDeviceToDevice, c->lane2));
        CK(cudaEventRecord(c->ev_corner, c->lane2));
        // this step's corner spectrum starts from its private copy of C' as soon as the
        // corner update is done, beside the edge update and the next step's first
        // phases; only the next such step rewrites the copy, after waiting for it
        if (!c->spec_skip) {
            CK(cudaStreamWaitEvent(c->side, c->ev_corner, 0));
            CK(launch_spectrum((int)chi, c->Cspec, c->s_new, c->s, c->delta, c->spec_work, c->side,
                               c->qr_rows_min <= 1));
            CK(cudaMemcpyAsync(c->s, c->s_new, sizeof(double) * chi, cudaMemcpyDeviceToDevice, c->side));
            if (c->delta_dst)
                CK(cudaMemcpyAsync(c->delta_dst, c->delta, sizeof(double), cudaMemcpyDeviceToHost, c->side));
            CK(cudaEventRecord(c->ev_join, c->side));
            c->side_pending = 1;
        }
        // the last edge contraction waits for the corner update (whose pack of Q^T it
        // reuses), which waited for the previous spectrum
        if ((rc = enqueue_edge(c, c->Q, c->T, 2)) != CTM_OK) return rc;
        return CTM_OK;
    }
    if ((rc = c->cfg.corner_mode ? enqueue_corner_from_r(c, c->Cn) : enqueue_corner(c, c->Qn, c->Cn)) != CTM_OK)
        return rc;
    if ((rc = enqueue_edge(c, c->Qn, c->Tn)) != CTM_OK) return rc;
    if (c->side_pending) CK(cudaStreamWaitEvent(st, c->ev_join, 0));
    CK(cudaMemcpyAsync(c->C, c->Cn, sizeof(double) * chi * chi, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(c->T, c->Tn, sizeof(double) * chi * D2 * chi, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(c->Q, c->Qn, sizeof(double) * n * chi, cudaMemcpyDeviceToDevice, st));
    if (c->spec_skip) return CTM_OK;
    CK(cudaEventRecord(c->ev_fork, st));
    CK(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    CK(launch_spectrum((int)chi, c->C, c->s_new, c->s, c->delta, c->spec_work, c->side, c->qr_rows_min <= 1));
    CK(cudaMemcpyAsync(c->s, c->s_new, sizeof(double) * chi, cudaMemcpyDeviceToDevice, c->side));
    if (c->delta_dst) CK(cudaMemcpyAsync(c->delta_dst, c->delta, sizeof(double), cudaMemcpyDeviceToHost, c->side));
    CK(cudaEventRecord(c->ev_join, c->side));
    c->side_pending = 1;
    return CTM_OK;
}

int join_side(ctm_ctx *c)
{
    if (c->side_pending) {
        CK(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
        c->side_pending = 0;
    }
    return CTM_OK;
}

// One step with CUDA events between its phases (same launches as enqueue_step).
int enqueue_step_profiled(ctm_ctx *c, cudaEvent_t *ev)
{
    int rc;
    cudaStream_t st = c->stream;
    const long long chi = c->chi, D2 = c->D2, n = c->n;
    CK(cudaEventRecord(ev[0], st));
    if ((rc = enqueue_enlarged_corner(c)) != CTM_OK) return rc;
    CK(cudaEventRecord(ev[1], st));
    c->ack_valid[1] = 0;   // the QR below writes a new Q
    CK(launch_warm_start((int)n, (int)chi, c->Q, c->C, c->Qs, st));
    {
        GemmF64 g{(int)n, (int)chi, (int)n, c->M, idx_lin(n), idx_lin(1), c->Qs, idx_lin(chi), idx_lin(1),
                  c->Y, idx_lin(chi), idx_lin(1), 1.0, 0.0};
        CK(run_gemm(c, g));
    }
    CK(cudaEventRecord(ev[2], st));
    {
        QrScratch qs = qr_scratch(c);
        CK(qr_householder((int)n, (int)chi, c->Y, c->Qn, c->R, qs, st));
    }
    CK(cudaEventRecord(ev[3], st));
    if ((rc = c->cfg.corner_mode ? enqueue_corner_from_r(c, c->Cn) : enqueue_corner(c, c->Qn, c->Cn)) != CTM_OK)
        return rc;
    CK(cudaEventRecord(ev[4], st));
    if ((rc = enqueue_edge(c, c->Qn, c->Tn)) != CTM_OK) return rc;
    CK(cudaEventRecord(ev[5], st));
    if (c->side_pending) CK(cudaStreamWaitEvent(st, c->ev_join, 0));
    CK(cudaEventRecord(ev[6], st));
    CK(cudaMemcpyAsync(c->C, c->Cn, sizeof(double) * chi * chi, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(c->T, c->Tn, sizeof(double) * chi * D2 * chi, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(c->Q, c->Qn, sizeof(double) * n * chi, cudaMemcpyDeviceToDevice, st));
    CK(cudaEventRecord(ev[7], st));
    CK(cudaStreamWaitEvent(c->side, ev[7], 0));
    CK(cudaEventRecord(ev[8], c->side));
    CK(launch_spectrum((int)chi, c->C, c->s_new, c->s, c->delta, c->spec_work, c->side, c->qr_rows_min <= 1));
    CK(cudaMemcpyAsync(c->s, c->s_new, sizeof(double) * chi, cudaMemcpyDeviceToDevice, c->side));
    CK(cudaEventRecord(ev[9], c->side));
    CK(cudaEventRecord(c->ev_join, c->side));
    c->side_pending = 1;
    return CTM_OK;
}

int read_status(ctm_ctx *c)
{
    int err = 0;
    CK(cudaMemcpyAsync(&err, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (err) return CTM_ETIMEOUT;
    return CTM_OK;
}

int check_env_finite(ctm_ctx *c)
{
    cudaStream_t st = c->stream;
    CK(cudaMemsetAsync(c->flag, 0, sizeof(int), st));
    CK(launch_check_finite((long long)c->chi * c->chi, c->C, c->flag, st));
    CK(launch_check_finite((long long)c->chi * c->D2 * c->chi, c->T, c->flag, st));
    int f = 0;
    CK(cudaMemcpyAsync(&f, c->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return f ? CTM_ENONFINITE : CTM_OK;
}

// Capture `nsteps` steps (spectrum fork/join included) on the private stream
// c->own; the caller has switched c->stream to c->own.  Kernel launches counted
// during the capture are what one replay launches.  The result replaces what
// *exec held; a launch that cannot be captured leaves graph_failed set and the
// caller runs eagerly.  half >= 0 captures the pipelined form, whose corner
// spectra are shifted by one step: the first step also computes the spectrum of
// the corner it starts from (the previous graph's last step), the last step
// leaves its own to the next graph, and ring half `half` (pinned host memory)
// receives the deltas -- slot 0 that of the step before the graph, slot i that
// of step i (1 <= i < nsteps) -- and, at the end, the error flag.
static int capture_into(ctm_ctx *c, int nsteps, cudaGraphExec_t *exec, unsigned long long *kernels, int half = -1)
{
    if (*exec) {
        cudaGraphExecDestroy(*exec);
        *exec = nullptr;
    }
    if (c->graph_failed) return CTM_OK;
    cudaGraph_t g = nullptr;
    const unsigned long long l0 = g_ctm_launches;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int rc = CTM_OK;
    for (int i = 0; i < nsteps && rc == CTM_OK; ++i) {
        double *ring = half >= 0 ? c->ring_h + (size_t)half * c->ring_cap : nullptr;
        c->spec_head = half >= 0 && i == 0;
        c->delta_head = c->spec_head ? ring : nullptr;
        c->spec_skip = half >= 0 && i == nsteps - 1;
        c->delta_dst = (half >= 0 && !c->spec_skip) ? ring + i + 1 : nullptr;
        rc = enqueue_step(c);
    }
    c->delta_dst = c->delta_head = nullptr;
    c->spec_head = c->spec_skip = 0;
    if (rc == CTM_OK) rc = join_side(c);
    if (rc == CTM_OK && half >= 0 &&
        cudaMemcpyAsync(c->ring_err_h + half, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        rc = CTM_ECUDA;
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (rc == CTM_OK && e == cudaSuccess && g) e = cudaGraphInstantiate(exec, g, 0);
    if (g) cudaGraphDestroy(g);
    c->side_pending = 0;
    if (rc != CTM_OK || e != cudaSuccess || !*exec) {
        cudaGetLastError();
        *exec = nullptr;
        c->graph_failed = 1;
    } else {
        *kernels = g_ctm_launches - l0;
    }
    g_ctm_launches = l0;   // nothing ran yet: replays add the captured kernel count
    return CTM_OK;
}

int capture_steps(ctm_ctx *c, int nsteps)
{
    if (nsteps == 1) return c->graph1 ? CTM_OK : capture_into(c, 1, &c->graph1, &c->graph1_kernels);
    if (c->graph && c->graph_steps == nsteps) return CTM_OK;
    int rc = capture_into(c, nsteps, &c->graph, &c->graph_kernels);
    if (c->graph) c->graph_steps = nsteps;
    return rc;
}

// Replay the captured graph of nsteps steps (capture_steps first).
int graph_launch(ctm_ctx *c, int nsteps)
{
    cudaGraphExec_t ge = nsteps == 1 ? c->graph1 : c->graph;
    CK(cudaGraphLaunch(ge, c->stream));
    CTM_COUNT_LAUNCH(nsteps == 1 ? c->graph1_kernels : c->graph_kernels);
    return CTM_OK;
}

// Forget every captured graph (they hold launch arguments and the packed operand
// state of the moment they were captured); the next calls capture again.
void drop_graphs(ctm_ctx *c)
{
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->graph1) cudaGraphExecDestroy(c->graph1);
    c->graph = nullptr;
    c->graph1 = nullptr;
    c->graph_steps = 0;
    for (int h = 0; h < 2; ++h) {
        if (c->pipe[h]) cudaGraphExecDestroy(c->pipe[h]);
        c->pipe[h] = nullptr;
    }
    c->pipe_steps = 0;
}

// The two pipelined graphs of k steps (ring halves 0 and 1), the pinned ring grown
// to k deltas per half first.  Leaves pipe_steps = 0 if capturing failed.
static int capture_pipe(ctm_ctx *c, int k)
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
        CK(cudaHostAlloc((void **)&c->ring_h, sizeof(double) * 2 * (size_t)k, cudaHostAllocDefault));
        c->ring_cap = k;
    }
    if (!c->ring_err_h) CK(cudaHostAlloc((void **)&c->ring_err_h, 2 * sizeof(int), cudaHostAllocDefault));
    for (int h = 0; h < 2; ++h) {
        if (!c->pipe_done[h]) CK(cudaEventCreateWithFlags(&c->pipe_done[h], cudaEventDisableTiming));
        int rc = capture_into(c, k, &c->pipe[h], &c->pipe_kernels, h);
        if (rc != CTM_OK) return rc;
        if (!c->pipe[h]) return CTM_OK;
    }
    c->pipe_steps = k;
    return CTM_OK;
}

// One step with its delta read back (synchronous): the one-step graph once the
// context has stepped in its configured mode, else eagerly.
static int step_and_read(ctm_ctx *c, double *delta)
{
    const int cfg_T = (c->cfg.precision == CTM_SPLIT_BF16) ? c->cfg.n_split : 0;
    bool replayed = false;
    int rc;
    if (c->steps_done > 0 && c->split_T == cfg_T) {
        if ((rc = capture_steps(c, 1)) != CTM_OK) return rc;
        if (c->graph1) {
            if ((rc = graph_launch(c, 1)) != CTM_OK) return rc;
            replayed = true;
        }
    }
    if (!replayed) {
        if ((rc = enqueue_step(c)) != CTM_OK) return rc;
        if (join_side(c) != CTM_OK) return CTM_ECUDA;
    }
    c->steps_done++;
    CK(cudaMemcpyAsync(delta, c->delta, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if ((rc = read_status(c)) != CTM_OK) return rc;
    return isfinite(*delta) ? CTM_OK : CTM_ENONFINITE;
}

// The spectrum of the current corner C against the last one computed, on the
// step's stream (the step whose spectrum the pipelined graphs deferred); delta read
// back (synchronous).
static int spectrum_now(ctm_ctx *c, double *delta)
{
    if (join_side(c) != CTM_OK) return CTM_ECUDA;
    CK(launch_spectrum(c->chi, c->C, c->s_new, c->s, c->delta, c->spec_work, c->stream));
    CK(cudaMemcpyAsync(c->s, c->s_new, sizeof(double) * c->chi, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(delta, c->delta, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    int rc = read_status(c);
    if (rc != CTM_OK) return rc;
    return isfinite(*delta) ? CTM_OK : CTM_ENONFINITE;
}

// Chunks of k steps from the two pipelined graphs while at least k steps are left;
// each chunk's last spectrum runs at the head of the next chunk.  While the newest
// delta read is above 100 tol (or none is known yet) a second chunk is queued
// behind the one whose deltas the host is reading, so the GPU does not wait for
// the host; closer to tol only one chunk is in flight, so that few steps run past
// convergence.  Queueing stops once the newest delta read is below tol; a chunk
// already queued still runs (each step moves the environment closer to the fixed
// point), and the last executed step's own spectrum then gives *delta.  Returns
// with *ran = 0 when no chunk fits.
static int converge_pipelined(ctm_ctx *c, int k, int budget, double tol, int *ran, double *delta)
{
    *ran = 0;
    if (budget < k) return CTM_OK;
    int rc = capture_pipe(c, k);
    if (rc != CTM_OK || c->pipe_steps != k) return rc;
    int queue[2], nq = 0, next = 0, launched = 0, chunks_read = 0;
    bool stop = false;
    double newest = INFINITY;
    for (;;) {
        while (!stop && nq < (newest > 100.0 * tol ? 2 : 1) && launched + k <= budget) {
            const int h = next;
            next ^= 1;
            CK(cudaGraphLaunch(c->pipe[h], c->stream));
            CTM_COUNT_LAUNCH(c->pipe_kernels);
            CK(cudaEventRecord(c->pipe_done[h], c->stream));
            queue[nq++] = h;
            launched += k;
        }
        if (nq == 0) break;
        const int h = queue[0];
        queue[0] = queue[1];
        --nq;
        CK(cudaEventSynchronize(c->pipe_done[h]));
        c->steps_done += k;
        *ran += k;
        const double *dh = c->ring_h + (size_t)h * c->ring_cap;
        // slot 0 of the first chunk repeats the delta of a step whose spectrum was
        // already taken (the recomputation gives 0): no information
        const int first = chunks_read++ == 0 ? 1 : 0;
        bool finite = true;
        for (int i = first; i < k; ++i) finite = finite && isfinite(dh[i]);
        if (c->ring_err_h[h] || !finite) {
            // let a queued chunk finish before reporting
            CK(cudaStreamSynchronize(c->stream));
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
    return spectrum_now(c, delta);
}

// A fresh context's first step runs eagerly (its launches time the plans); then
// pipelined chunks of check_every steps while that many are left (see
// converge_pipelined), and single steps otherwise or when graphs are unavailable.
int converge_on_own(ctm_ctx *c, int max_steps, double tol, int check_every, int *steps_out, double *delta_out)
{
    const int cfg_T = (c->cfg.precision == CTM_SPLIT_BF16) ? c->cfg.n_split : 0;
    int done = 0, rc = CTM_OK;
    double delta = INFINITY;
    while (!(delta < tol) && done < max_steps) {
        int ran = 0;
        if (c->steps_done > 0 && c->split_T == cfg_T && !c->graph_failed) {
            rc = converge_pipelined(c, check_every, max_steps - done, tol, &ran, &delta);
            done += ran;
            if (rc != CTM_OK) break;
        }
        if (ran == 0) {
            if ((rc = step_and_read(c, &delta)) != CTM_OK) break;
            ++done;
        }
    }
    if (steps_out) *steps_out = done;
    if (delta_out) *delta_out = delta;
    if (rc != CTM_OK) return rc;
    if ((rc = check_env_finite(c)) != CTM_OK) return rc;
    return (delta < tol) ? CTM_OK : CTM_ENOTCONVERGED;
}

cudaError_t rho_reduce(ctm_ctx *c)
{
    const int dd = c->d * c->d;
    CTM_COUNT_LAUNCH(2);
    rho_partial_kernel<<<RHO_BLOCKS, 256, 0, c->stream>>>((long long)c->chi * c->chi, dd, c->D2, c->Y1o, c->G2,
                                                         c->rho_part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    rho_final_kernel<<<1, 128, 0, c->stream>>>(RHO_BLOCKS, dd, c->rho_part, c->rho_raw);
    return cudaGetLastError();
}

}  // namespace ctmi

using namespace ctmi;

extern "C" {

size_t ctm_workspace_bytes(const ctm_config *cfg)
{
    if (!config_ok(cfg)) return 0;
    ctm_ctx c;
    memset(&c, 0, sizeof(c));
    c.cfg = *cfg;
    c.d = cfg->d;
    c.D = cfg->D;
    c.D2 = cfg->D * cfg->D;
    c.chi = cfg->chi;
    c.n = (long long)c.chi * c.D2;
    c.split_T = (cfg->precision == CTM_SPLIT_BF16) ? cfg->n_split : 0;
    c.tf32_T = tf32_slices(cfg->precision);
    c.qr_force_slab = qr_force_slab_from_env();
    return layout(&c, nullptr);
}

int ctm_init(const ctm_config *cfg, const double *A_dev, void *workspace, size_t ws_bytes, void *stream,
             ctm_ctx **out)
{
    if (!out) return CTM_EINVAL;
    *out = nullptr;
    if (!cfg || !A_dev || !workspace) return CTM_EINVAL;
    if (!config_ok(cfg)) return CTM_EINVAL;
    if ((uintptr_t)workspace % 256 != 0) return CTM_EINVAL;
    // the QR's per-CTA scratch must fit shared memory (its row blocks may go to the slab)
    if (!qr_supported(cfg->chi * cfg->D * cfg->D, cfg->chi)) return CTM_EUNSUPPORTED;
    ctm_ctx *c = new (std::nothrow) ctm_ctx;
    if (!c) return CTM_ENOMEM;
    memset(c, 0, sizeof(*c));
    c->cfg = *cfg;
    c->d = cfg->d;
    c->D = cfg->D;
    c->D2 = cfg->D * cfg->D;
    c->chi = cfg->chi;
    c->n = (long long)c->chi * c->D2;
    c->split_T = (cfg->precision == CTM_SPLIT_BF16) ? cfg->n_split : 0;
    c->tf32_T = tf32_slices(cfg->precision);
    c->qr_rows_min = 1;
    c->qr_force_slab = qr_force_slab_from_env();
    c->stream = (cudaStream_t)stream;
    if (!qr_supported((int)c->n, c->chi)) {
        delete c;
        return CTM_EUNSUPPORTED;
    }
    size_t need = layout(c, nullptr);
    if (ws_bytes < need) {
        delete c;
        return CTM_ENOMEM;
    }
    layout(c, (char *)workspace);
    cudaStream_t st = c->stream;
    int rc = CTM_OK;
    do {
        if (qr_prepare() != cudaSuccess || spectrum_prepare() != cudaSuccess || split_prepare() != cudaSuccess ||
            tf32_prepare() != cudaSuccess) {
            rc = CTM_ECUDA;
            break;
        }
        // the corner spectrum overlaps the next step on the side stream; lowest priority,
        // so the step's own pending CTAs are scheduled first
        int prio_least = 0, prio_greatest = 0;
        cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
        if (cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_least) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
            cudaStreamCreateWithPriority(&c->lane2, cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_q, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_corner, cudaEventDisableTiming) != cudaSuccess) {
            rc = CTM_ECUDA;
            break;
        }
        if (cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess) {
            rc = CTM_ECUDA;
            break;
        }
        if (cudaMemsetAsync(c->err, 0, sizeof(int), st) != cudaSuccess) { rc = CTM_ECUDA; break; }
        if (cudaMemcpyAsync(c->Araw, A_dev, sizeof(double) * c->d * c->D * c->D * c->D, cudaMemcpyDeviceToDevice,
                            st) != cudaSuccess) {
            rc = CTM_ECUDA;
            break;
        }
        if (launch_c3v_project_normalize(c->d, c->D, A_dev, c->A, cfg->symmetrize ? 1 : 0, st) != cudaSuccess) {
            rc = CTM_ECUDA;
            break;
        }
        if (launch_double_layer(c->d, c->D, c->A, c->A, c->a, st) != cudaSuccess) { rc = CTM_ECUDA; break; }
        if (launch_init_env(c->chi, c->D, c->a, c->C, c->T, c->Q, st) != cudaSuccess) { rc = CTM_ECUDA; break; }
        if (launch_spectrum_init(c->chi, c->s, st) != cudaSuccess) { rc = CTM_ECUDA; break; }
        if (cudaMemsetAsync(c->flag, 0, sizeof(int), st) != cudaSuccess) { rc = CTM_ECUDA; break; }
        if (launch_check_finite((long long)c->d * c->D * c->D * c->D, c->A, c->flag, st) != cudaSuccess) {
            rc = CTM_ECUDA;
            break;
        }
        int f = 0;
        if (cudaMemcpyAsync(&f, c->flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = CTM_ECUDA;
            break;
        }
        if (f) rc = CTM_ENONFINITE;
    } while (0);
    if (rc != CTM_OK) {
        ctm_destroy(c);
        return rc;
    }
    *out = c;
    return CTM_OK;
}

int ctm_step(ctm_ctx *c, int nsteps, double *delta_host)
{
    if (!c || nsteps < 0) return CTM_EINVAL;
    bool done = false;
    // the captured graphs hold the context's configured contractions; a caller that
    // switches the mode for a while (the adjoint's tracked FP64 steps) runs eagerly
    const int cfg_T = (c->cfg.precision == CTM_SPLIT_BF16) ? c->cfg.n_split : 0;
    if (nsteps >= 1 && c->steps_done > 0 && c->split_T == cfg_T) {
        // steps after the first eager one (whose launches ran the autotuners):
        // replay them as one captured graph (one for a single step, one for the
        // last multi-step count), ordered after the caller's stream
        cudaStream_t user = c->stream;
        CK(cudaEventRecord(c->ev_in, user));
        CK(cudaStreamWaitEvent(c->own, c->ev_in, 0));
        c->stream = c->own;
        int rc = capture_steps(c, nsteps);
        if (rc == CTM_OK && (nsteps == 1 ? c->graph1 : c->graph)) {
            rc = graph_launch(c, nsteps);
            done = (rc == CTM_OK);
        }
        c->stream = user;
        if (cudaEventRecord(c->ev_out, c->own) != cudaSuccess) return CTM_ECUDA;
        if (cudaStreamWaitEvent(user, c->ev_out, 0) != cudaSuccess) return CTM_ECUDA;
        if (rc != CTM_OK) return rc;
        if (done) c->steps_done += nsteps;
    }
    for (int i = 0; i < nsteps && !done; ++i) {
        int rc = enqueue_step(c);
        if (rc != CTM_OK) return rc;
        c->steps_done++;
    }
    if (join_side(c) != CTM_OK) return CTM_ECUDA;
    if (delta_host) {
        CK(cudaMemcpyAsync(delta_host, c->delta, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        int rc = read_status(c);
        if (rc != CTM_OK) return rc;
        if (!isfinite(*delta_host)) return CTM_ENONFINITE;
        return check_env_finite(c);
    }
    return CTM_OK;
}

int ctm_converge(ctm_ctx *c, int max_steps, double tol, int check_every, int *steps_out, double *delta_out)
{
    if (!c) return CTM_EINVAL;
    if (max_steps <= 0) max_steps = c->cfg.max_steps;
    if (tol <= 0.0) tol = c->cfg.tol;
    if (check_every < 1) check_every = 1;
    if (max_steps <= 0) return CTM_EINVAL;
    // work is replayed on the private stream, ordered after the caller's stream
    cudaStream_t user = c->stream;
    CK(cudaEventRecord(c->ev_in, user));
    CK(cudaStreamWaitEvent(c->own, c->ev_in, 0));
    c->stream = c->own;
    int rc = converge_on_own(c, max_steps, tol, check_every, steps_out, delta_out);
    c->stream = user;
    if (cudaEventRecord(c->ev_out, c->own) != cudaSuccess) return CTM_ECUDA;
    if (cudaStreamWaitEvent(user, c->ev_out, 0) != cudaSuccess) return CTM_ECUDA;
    return rc;
}

int ctm_energy(ctm_ctx *c, const double *h_dev, double *e_bond_host, double *e_site_host, double *rho_host)
{
    if (!c || !h_dev) return CTM_EINVAL;
    if (join_side(c) != CTM_OK) return CTM_ECUDA;
    const int chi = c->chi, D2 = c->D2, d = c->d, dd = d * d;
    const long long n = c->n;
    cudaStream_t st = c->stream;
    int rc;
    if (dd > RHO_MAX_DD) return CTM_EUNSUPPORTED;
    // projector of one more step and Ch = sym(Q^T M Q)/|.|
    if ((rc = enqueue_enlarged_corner(c)) != CTM_OK) return rc;
    if ((rc = enqueue_projector(c, c->Qn)) != CTM_OK) return rc;
    if ((rc = enqueue_corner(c, c->Qn, c->Cn)) != CTM_OK) return rc;
    // P5 = Ch^5
    GemmF64 g;
    const double *src = c->Cn;
    double *bufs[2] = {c->P5a, c->P5b};
    for (int p = 0; p < 4; ++p) {
        double *dst = bufs[p & 1];
        g = GemmF64{chi, chi, chi, src, idx_lin(chi), idx_lin(1), c->Cn, idx_lin(chi), idx_lin(1), dst,
                    idx_lin(chi), idx_lin(1), 1.0, 0.0};
        CK(gemm_f64(g, gemm_f64_pick_split(g.M, g.N, g.K), c->splitk, c->splitk_elems, st));
        src = dst;
    }
    // E = Q P5 Q^T  (n x n, symmetric) into H
    g = GemmF64{(int)n, chi, chi, c->Qn, idx_lin(chi), idx_lin(1), src, idx_lin(chi), idx_lin(1), c->W,
                idx_lin(chi), idx_lin(1), 1.0, 0.0};
    CK(gemm_f64(g, gemm_f64_pick_split(g.M, g.N, g.K), c->splitk, c->splitk_elems, st));
    // (this and the two open-layer contractions below go through run_gemm: the split-BF16
    // engine in split mode, whose error at T = 5 is far below the energy's tolerance)
    g = GemmF64{(int)n, (int)n, chi, c->W, idx_lin(chi), idx_lin(1), c->Qn, idx_lin(1), idx_lin(chi), c->H,
                idx_lin(n), idx_lin(1), 1.0, 0.0};
    CK(run_gemm(c, g));
    // open layers b[p][..] = A[s] (x) A[t], p = s*d + t
    CK(launch_open_layers(d, c->D, c->A, c->b, st));
    const long long D3 = (long long)D2 * D2 * D2;
    // Y1o[(a,b)][(pB,z)] = sum_{u,l} X'[(a,b),(u,l)] b[pB][u][l][z]
    g = GemmF64{chi * chi, dd * D2, D2 * D2, c->X, idx_lin((long long)D2 * D2), idx_lin(1), c->b, idx_lin(D2),
                idx_split(D2, D3, 1), c->Y1o, idx_lin((long long)dd * D2), idx_lin(1), 1.0, 0.0};
    CK(run_gemm(c, g));
    // G2[(a,b)][(pA,z)] = sum_{x,y} E[(a,y),(b,x)] b[pA][z][x][y]
    g = GemmF64{chi * chi, dd * D2, D2 * D2, c->H, idx_split(chi, (long long)D2 * n, D2), idx_split(D2, 1, n),
                c->b, idx_lin(1), idx_split(D2, D3, (long long)D2 * D2), c->G2, idx_lin((long long)dd * D2),
                idx_lin(1), 1.0, 0.0};
    CK(run_gemm(c, g));
    CTM_COUNT_LAUNCH(1);
    CK(rho_reduce(c));

    CK(launch_bond_energy(d, c->rho_raw, h_dev, c->eout, st));
    double host[4 + RHO_MAX_DD * RHO_MAX_DD];
    CK(cudaMemcpyAsync(host, c->eout, sizeof(double) * (4 + dd * dd), cudaMemcpyDeviceToHost, st));
    if ((rc = read_status(c)) != CTM_OK) return rc;
    for (int i = 0; i < 4 + dd * dd; ++i)
        if (!isfinite(host[i])) return CTM_ENONFINITE;
    if (e_bond_host)
        for (int i = 0; i < 3; ++i) e_bond_host[i] = host[i];
    if (e_site_host) *e_site_host = host[3];
    if (rho_host)
        for (int i = 0; i < dd * dd; ++i) rho_host[i] = host[4 + i];
    return CTM_OK;
}

int ctm_get_env(const ctm_ctx *c, double *C_dev, double *T_dev, double *Q_dev)
{
    if (!c) return CTM_EINVAL;
    const long long chi = c->chi, D2 = c->D2, n = c->n;
    if (C_dev) CK(cudaMemcpyAsync(C_dev, c->C, sizeof(double) * chi * chi, cudaMemcpyDeviceToDevice, c->stream));
    if (T_dev)
        CK(cudaMemcpyAsync(T_dev, c->T, sizeof(double) * chi * D2 * chi, cudaMemcpyDeviceToDevice, c->stream));
    if (Q_dev) CK(cudaMemcpyAsync(Q_dev, c->Q, sizeof(double) * n * chi, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return CTM_OK;
}

int ctm_set_env(ctm_ctx *c, const double *C_dev, const double *T_dev, const double *Q_dev)
{
    if (!c || !C_dev || !T_dev || !Q_dev) return CTM_EINVAL;
    if (join_side(c) != CTM_OK) return CTM_ECUDA;
    const long long chi = c->chi, D2 = c->D2, n = c->n;
    cudaStream_t st = c->stream;
    CK(cudaMemcpyAsync(c->C, C_dev, sizeof(double) * chi * chi, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(c->T, T_dev, sizeof(double) * chi * D2 * chi, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(c->Q, Q_dev, sizeof(double) * n * chi, cudaMemcpyDeviceToDevice, st));
    // the spectrum of the new corner becomes the reference for the next delta
    CK(launch_spectrum((int)chi, c->C, c->s, c->s, c->delta, c->spec_work, st));
    CK(cudaStreamSynchronize(st));
    return CTM_OK;
}

int ctm_get_intermediate(const ctm_ctx *c, int which, double *dst, size_t count)
{
    if (!c || !dst) return CTM_EINVAL;
    const long long chi = c->chi, D2 = c->D2, n = c->n;
    const double *src = nullptr;
    size_t cnt = 0;
    switch (which) {
    case 0: src = c->M; cnt = (size_t)(n * n); break;
    case 1: src = c->Y; cnt = (size_t)(n * chi); break;
    case 2: src = c->R; cnt = (size_t)(chi * chi); break;
    case 3: src = c->Q; cnt = (size_t)(n * chi); break;
    case 4: src = c->s; cnt = (size_t)chi; break;
    case 5: src = c->A; cnt = (size_t)c->d * c->D * c->D * c->D; break;
    case 6: src = c->a; cnt = (size_t)(D2 * D2 * D2); break;
    default: return CTM_EINVAL;
    }
    if (count < cnt) return CTM_EINVAL;
    CK(cudaMemcpyAsync(dst, src, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return CTM_OK;
}

void ctm_destroy(ctm_ctx *c)
{
    if (!c) return;
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->graph1) cudaGraphExecDestroy(c->graph1);
    for (int h = 0; h < 2; ++h) {
        if (c->pipe[h]) cudaGraphExecDestroy(c->pipe[h]);
        if (c->pipe_done[h]) cudaEventDestroy(c->pipe_done[h]);
    }
    if (c->own) {
        cudaStreamSynchronize(c->own);
        cudaStreamDestroy(c->own);
    }
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
    }
    if (c->lane2) {
        cudaStreamSynchronize(c->lane2);
        cudaStreamDestroy(c->lane2);
    }
    if (c->ev_q) cudaEventDestroy(c->ev_q);
    if (c->ev_corner) cudaEventDestroy(c->ev_corner);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->prof_ev[0])
        for (int i = 0; i < CTM_PROF_EVENTS; ++i) cudaEventDestroy(c->prof_ev[i]);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    if (c->ring_h) cudaFreeHost(c->ring_h);
    if (c->ring_err_h) cudaFreeHost(c->ring_err_h);
    delete c;
}

const char *ctm_status_str(int s)
{
    switch (s) {
    case CTM_OK: return "CTM_OK";
    case CTM_EINVAL: return "CTM_EINVAL: invalid argument";
    case CTM_ENOMEM: return "CTM_ENOMEM: workspace too small";
    case CTM_ECUDA: return "CTM_ECUDA: CUDA runtime error";
    case CTM_ENOTCONVERGED: return "CTM_ENOTCONVERGED: step limit reached";
    case CTM_ENONFINITE: return "CTM_ENONFINITE: NaN or Inf";
    case CTM_ETIMEOUT: return "CTM_ETIMEOUT: bounded device wait expired";
    case CTM_EUNSUPPORTED: return "CTM_EUNSUPPORTED: unsupported shape or mode";
    default: return "unknown status";
    }
}

int ctm_step_profiled(ctm_ctx *c, double *phase_ms, int nphase)
{
    if (!c || !phase_ms || nphase < 7) return CTM_EINVAL;
    cudaEvent_t ev[10];
    for (int i = 0; i < 10; ++i)
        if (cudaEventCreate(&ev[i]) != cudaSuccess) return CTM_ECUDA;
    if (!c->prof_ev[0])
        for (int i = 0; i < CTM_PROF_EVENTS; ++i)
            if (cudaEventCreate(&c->prof_ev[i]) != cudaSuccess) return CTM_ECUDA;
    c->prof_on = 1;
    c->prof_n = 0;
    int rc = enqueue_step_profiled(c, ev);
    c->prof_on = 0;
    if (rc == CTM_OK) {
        c->steps_done++;
        if (cudaEventSynchronize(ev[7]) != cudaSuccess || cudaEventSynchronize(ev[9]) != cudaSuccess) rc = CTM_ECUDA;
    }
    if (rc == CTM_OK && join_side(c) != CTM_OK) rc = CTM_ECUDA;
    if (rc == CTM_OK) rc = read_status(c);
    if (rc == CTM_OK)
        for (int i = 0; i < 7; ++i) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) != cudaSuccess) rc = CTM_ECUDA;
            phase_ms[i] = ms;
        }
    if (rc == CTM_OK && nphase >= 8) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev[8], ev[9]) != cudaSuccess) rc = CTM_ECUDA;
        phase_ms[7] = ms;
    }
    if (rc == CTM_OK && nphase >= 9) {
        double tot = 0.0, pre = 0.0;
        for (int i = 0; i + 2 < c->prof_n; i += 3) {
            float ms = 0.f, mp = 0.f;
            if (cudaEventElapsedTime(&ms, c->prof_ev[i], c->prof_ev[i + 1]) != cudaSuccess) rc = CTM_ECUDA;
            if (cudaEventElapsedTime(&mp, c->prof_ev[i + 2], c->prof_ev[i]) != cudaSuccess) rc = CTM_ECUDA;
            tot += ms;
            pre += mp;
        }
        phase_ms[8] = tot;
        if (nphase >= 10) phase_ms[9] = pre;
    }
    for (int i = 0; i < 10; ++i) cudaEventDestroy(ev[i]);
    return rc;
}

unsigned long long ctm_kernel_launches(void) { return g_ctm_launches; }

int ctm_set_site(ctm_ctx *c, const double *A_dev, int reset_env)
{
    if (!c || !A_dev) return CTM_EINVAL;
    if (join_side(c) != CTM_OK) return CTM_ECUDA;
    cudaStream_t st = c->stream;
    const long long nA = (long long)c->d * c->D * c->D * c->D;
    CK(cudaMemcpyAsync(c->Araw, A_dev, sizeof(double) * nA, cudaMemcpyDeviceToDevice, st));
    CK(launch_c3v_project_normalize(c->d, c->D, c->Araw, c->A, c->cfg.symmetrize ? 1 : 0, st));
    CK(launch_double_layer(c->d, c->D, c->A, c->A, c->a, st));
    // the packed digits of the old double layer and the graphs that assumed them are stale
    c->apk_state[0] = c->apk_state[1] = 0;
    drop_graphs(c);
    if (reset_env) {
        CK(launch_init_env(c->chi, c->D, c->a, c->C, c->T, c->Q, st));
        CK(launch_spectrum_init(c->chi, c->s, st));
    }
    CK(cudaMemsetAsync(c->flag, 0, sizeof(int), st));
    CK(launch_check_finite(nA, c->A, c->flag, st));
    int f = 0;
    CK(cudaMemcpyAsync(&f, c->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return f ? CTM_ENONFINITE : CTM_OK;
}

int ctm_debug_force_timeout(ctm_ctx *c, int enable)
{
    if (!c) return CTM_EINVAL;
    if (join_side(c) != CTM_OK) return CTM_ECUDA;
    CK(cudaStreamSynchronize(c->stream));
    c->force_timeout = enable ? 1 : 0;
    // captured graphs hold the QR's launch arguments: capture again with the new ones
    drop_graphs(c);
    return CTM_OK;
}

size_t ctm_gemm_workspace_bytes(int M, int N, int K, int precision, int n_split)
{
    if (M <= 0 || N <= 0 || K <= 0) return 0;
    if (precision == CTM_FP64) {
        int s = gemm_f64_pick_split(M, N, K);
        return align_up(64) + align_up(sizeof(double) * (size_t)(s > 1 ? s : 0) * M * N + 8);
    }
    if (tf32_slices(precision) > 0) {
        SplitPlan p = tf32_plan_caps(M, N, K, tf32_slices(precision));
        int ec = M > N ? M : N;
        return align_up(64) + align_up(p.a_pack_bytes) + align_up(p.b_pack_bytes) + 2 * align_up(sizeof(int) * ec) +
               align_up(p.partial_bytes + 8);
    }
    if (precision != CTM_SPLIT_BF16 || !split_supported_T(n_split)) return 0;
    SplitPlan p = split_plan(M, N, K, n_split);
    int ec = M > N ? M : N;
    return align_up(64) + align_up(p.a_pack_bytes) + align_up(p.b_pack_bytes) + 2 * align_up(sizeof(int) * ec) +
           align_up(p.partial_bytes + 8);
}

int ctm_gemm(int M, int N, int K, const double *A, const double *B, double *C, int precision, int n_split,
             void *workspace, size_t ws_bytes, void *stream)
{
    if (M <= 0 || N <= 0 || K <= 0 || !A || !B || !C || !workspace) return CTM_EINVAL;
    size_t need = ctm_gemm_workspace_bytes(M, N, K, precision, n_split);
    if (need == 0) return CTM_EINVAL;
    if (ws_bytes < need) return CTM_ENOMEM;
    if ((uintptr_t)workspace % 256 != 0) return CTM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    char *base = (char *)workspace;
    int *err = (int *)base;
    size_t off = align_up(64);
    GemmF64 g{M, N, K, A, idx_lin(K), idx_lin(1), B, idx_lin(N), idx_lin(1), C, idx_lin(N), idx_lin(1), 1.0, 0.0};
    CK(cudaMemsetAsync(err, 0, sizeof(int), st));
    if (precision == CTM_FP64) {
        CK(gemm_f64(g, gemm_f64_pick_split(M, N, K), (double *)(base + off), (ws_bytes - off) / sizeof(double), st));
    } else {
        if (split_prepare() != cudaSuccess || tf32_prepare() != cudaSuccess) return CTM_ECUDA;
        const int tT = tf32_slices(precision);
        SplitPlan p = tT > 0 ? tf32_plan_caps(M, N, K, tT) : split_plan(M, N, K, n_split);
        int ec = M > N ? M : N;
        SplitWork w;
        w.Apk = (unsigned char *)(base + off);
        off += align_up(p.a_pack_bytes);
        w.a_pack_cap = p.a_pack_bytes;
        w.Bpk = (unsigned char *)(base + off);
        off += align_up(p.b_pack_bytes);
        w.b_pack_cap = p.b_pack_bytes;
        w.eA = (int *)(base + off);
        off += align_up(sizeof(int) * ec);
        w.eB = (int *)(base + off);
        off += align_up(sizeof(int) * ec);
        w.e_cap = ec;
        w.partial = base + off;
        w.partial_cap = p.partial_bytes;
        w.err = err;
        w.autotune = 0;
        if (tT > 0) CK(gemm_tf32(g, tT, w, st, nullptr));
        else CK(gemm_split(g, n_split, w, st, nullptr));
    }
    int e = 0;
    CK(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return e ? CTM_ETIMEOUT : CTM_OK;
}

const char *ctm_version(void) { return "libctm sm_103a fp64+bf16split+tf32split"; }

}  // extern "C"
