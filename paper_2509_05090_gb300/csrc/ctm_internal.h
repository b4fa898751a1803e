// Internal declarations shared by the libctm translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <functional>

#include "../../include/ctm.h"

// Two-level index map: off(i) = (i / div) * s1 + (i % div) * s2.  A plain
// strided dimension is {div = 1 << 30, s1 = 0, s2 = stride}.  All tensor
// contractions of the step are GEMMs whose operands and outputs are 4-index
// tensors; splitting each GEMM dimension into two indices lets one kernel read
// and write every permuted layout directly.
struct Idx2 {
    int div;
    long long s1, s2;
};

static inline Idx2 idx_lin(long long stride) { return Idx2{1 << 30, 0, stride}; }
static inline Idx2 idx_split(int div, long long s_hi, long long s_lo) { return Idx2{div, s_hi, s_lo}; }

// C(m,n) = alpha * sum_k A(m,k) B(k,n) + beta * C(m,n), FP64.
struct GemmF64 {
    int M, N, K;
    const double *A;
    Idx2 Am, Ak;
    const double *B;
    Idx2 Bk, Bn;
    double *C;
    Idx2 Cm, Cn;
    double alpha, beta;
};

// Launch a FP64 GEMM; split-K (ksplit > 1) uses `scratch` of scratch_elems doubles
// (the split is reduced so that ksplit*M*N fits).
cudaError_t gemm_f64(const GemmF64 &g, int ksplit, double *scratch, size_t scratch_elems, cudaStream_t st);
// Number of K-splits gemm_f64 picks for this shape (1 = none) and the scratch it needs.
int gemm_f64_pick_split(int M, int N, int K);

// ---------------------------------------------------------------- split-BF16 engine
// C = A B evaluated as sum_{i+j<T} A_i B_j of BF16 digit slices on tcgen05 (see gemm_split.cu).
struct SplitPlan {
    int NT, mTiles, nTiles, kTiles, chunks_per_split, ksplit;
    size_t a_pack_bytes, b_pack_bytes, partial_bytes;
    int deep;      // the 48-wide tile with one CTA per SM and a deep A ring (plan code 148)
};
struct SplitWork {
    unsigned char *Apk, *Bpk;
    size_t a_pack_cap, b_pack_cap;
    int *eA, *eB;
    int e_cap;
    void *partial;
    size_t partial_cap;
    int *err;
    int autotune;      // time the candidate tile shapes / K-splits of a new shape once (eager only)
};
// nt_override: 48, 64, 96, or 148 (the 48-wide tile with a deep A ring); ks_override: > 0 a
// K split, 0 automatic.
SplitPlan split_plan(int M, int N, int K, int T, int nt_override = 0, int ks_override = 0);
// Operand reuse: reuse_a = the A operand (same pointer and maps) was packed by the
// previous split call and is unchanged; b_cache = a constant B operand packed once
// into caller-owned buffers (re-packed if the plan's N tile changes).
struct SplitOpts {
    int reuse_a;
    unsigned char *b_pk;
    int *b_e;
    size_t b_cap;
    int *b_state;     // host: N tile of the cached pack, 0 = empty
    // A operand held in caller-owned buffers (a matrix packed once, used by two
    // contractions): a_fill = 1 packs it there, 0 uses the pack as it is
    unsigned char *a_pk;
    int *a_e;
    size_t a_cap;
    int a_fill;
};
// Largest pack / accumulator sizes over every plan the autotuner may pick.
SplitPlan split_plan_caps(int M, int N, int K, int T);
int split_supported_T(int T);
cudaError_t split_prepare();
// ev (may be null): three events, recorded around the contraction kernel (ev[0] before,
// ev[1] after) and before its operand pre-pass (ev[2]).
cudaError_t gemm_split(const GemmF64 &g, int T, SplitWork w, cudaStream_t st, cudaEvent_t *ev,
                       const SplitOpts *opt = nullptr);

// ---------------------------------------------------------------- split-TF32 engine
// C = A B from TF32 hi/lo slices (T = 2: A_hi B_hi + A_hi B_lo + A_lo B_hi; T = 1: A_hi B_hi)
// on tcgen05.mma.kind::tf32 with FP32 accumulation (gemm_split.cu); the same work buffers
// as the BF16 engine, sized by tf32_plan_caps.  ev as for gemm_split.
SplitPlan tf32_plan_caps(int M, int N, int K, int T);
int tf32_supported_T(int T);
cudaError_t tf32_prepare();
cudaError_t gemm_tf32(const GemmF64 &g, int T, SplitWork w, cudaStream_t st, cudaEvent_t *ev);

// ---------------------------------------------------------------- QR
// Householder QR of Y (n x k row-major, n >= k) with diag(R) >= 0.  Q (n x k)
// and R (k x k) row-major.  One cooperative kernel: the blocked factorisation (one
// grid barrier per panel), then Q in compact-WY form and the sign gauge (two more
// grid barriers).
// Subspace iteration for the leading eigenvalue magnitudes of a matrix-free real operator
// (transfer.cu; the transfer-matrix spectra of the real and the complex path): the
// stream, the FP64 GEMM's split-K scratch and a device error flag read at each check.
struct SubspaceWork {
    cudaStream_t stream;
    double *splitk;
    size_t splitk_elems;
    const int *err;
};
constexpr int SUBSPACE_MAXV = 12;   // vectors in the subspace
size_t subspace_workspace_bytes(long long N, int m);
// apply(v, out): out = Op v for device vectors of length N, enqueued on s.stream.  pairs
// = 1: the magnitudes as they come; 2: Op is the real form of a complex operator whose
// spectrum is closed under conjugation, so every magnitude appears twice and every
// second one is kept.  mags (host, nev) gets the leading magnitudes over the largest;
// returns CTM_OK when they moved by less than tol between checks (else
// CTM_ENOTCONVERGED with the last estimates).
int subspace_spectrum(const SubspaceWork &s, long long N, int m, int nev, int pairs, int max_iter, double tol,
                      void *tws, const std::function<cudaError_t(const double *, double *)> &apply, double *mags,
                      int *iters_out);

struct QrScratch {
    double *sbuf;      // qr_scratch_doubles(k): rotating column-sum accumulators
    double *rowbuf;    // qr_rowbuf_doubles(k): published panel rows
    unsigned *bar;     // 2 (count, generation)
    int *err;          // 1
    int rows_min;      // fewest rows per CTA (batched instances use small grids so they overlap)
    double *V;         // k x k: the first k rows of the reflectors
    double *S, *W;     // k x k each: V^T V and T V_top^T
    double *ta;        // 2 x k (unused)
    double *sk;        // unused
    size_t sk_elems;
    unsigned bar_extra;      // arrivals the grid barrier waits for beyond the grid (0; > 0 only to force a timeout)
    long long spin_limit;    // polls before a barrier wait gives up (0: the default, about a second)
    // deterministic mode (null: FP64 atomics): per-CTA partial-sum slots for up to gmax CTAs
    double *gpart;           // qr_det_gram_doubles(k, gmax)
    double *spart;           // qr_det_s_doubles(k, gmax)
    int gmax;
    // row blocks too tall for shared memory (qr_slab_doubles(n, k) > 0): a global slab
    double *yslab;
    size_t yslab_elems;
    bool force_slab;   // the slab for every shape (CTM_QR_SLAB=1 at init: a check of that path)
};
size_t qr_wy_doubles(int n, int k);   // V + S + W + ta + split-K scratch
size_t qr_sk_doubles(int n, int k);   // the split-K scratch part
size_t qr_scratch_doubles(int k);
// deterministic QR: slots of partial sums for up to qr_det_gmax(n) CTAs
size_t qr_det_gram_doubles(int k, int gmax);
size_t qr_det_s_doubles(int k, int gmax);
int qr_det_gmax(int n);
size_t qr_rowbuf_doubles(int k);
// doubles of the global slab that holds the QR's row blocks where one SM's share of the
// rows does not fit shared memory (0 where it does)
size_t qr_slab_doubles(int n, int k, bool force = false);
// CTM_QR_SLAB=1 in the environment: contexts created from then on keep the QR's row blocks
// in the slab for every shape (the same factorisation; a check of that path at small sizes)
bool qr_force_slab_from_env();
cudaError_t qr_householder(int n, int k, const double *Y, double *Q, double *R, QrScratch s,
                           cudaStream_t st);
int qr_supported(int n, int k);

// ---------------------------------------------------------------- small kernels
cudaError_t launch_c3v_project_normalize(int d, int D, const double *Ain, double *Aout, int symmetrize,
                                         cudaStream_t st);
cudaError_t launch_double_layer(int d, int D, const double *K, const double *B, double *a, cudaStream_t st);
cudaError_t launch_init_env(int chi, int D, const double *a, double *C, double *T, double *Q, cudaStream_t st);
cudaError_t launch_warm_start(int n, int chi, const double *Q, const double *C, double *Qs, cudaStream_t st);
// partials: CORNER_NORM_BLOCKS doubles of scratch
constexpr int CORNER_NORM_BLOCKS = 64;
cudaError_t launch_corner_sym_normalize(int chi, const double *Cr, double *Cn, double *partials, cudaStream_t st);
cudaError_t launch_normalize(long long count, double *x, double *partials, int nblocks, cudaStream_t st);
cudaError_t launch_spectrum(int chi, const double *C, double *s_new, const double *s_old, double *delta,
                            double *work, cudaStream_t st, bool reserve_sm = false);
cudaError_t launch_spectrum_init(int chi, double *s, cudaStream_t st);
// The last two phases of launch_spectrum for a real symmetric tridiagonal matrix already in
// `work` (diagonal d in work[0, chi), squared off-diagonal e^2 in work[chi, 2 chi)).
cudaError_t launch_spectrum_from_tridiag(int chi, double *work, double *s_new, const double *s_old, double *delta,
                                        cudaStream_t st);
// The spectrum of a Hermitian chi x chi corner through its real symmetric 2chi x 2chi
// embedding E = [[Re, -Im], [Im, Re]] (every eigenvalue twice): the real reduction and
// bisection on E, then every second sorted magnitude.  work: spectrum_work_doubles(2 chi).
cudaError_t launch_spectrum_pairs(int chi, const double *E, double *s_new, const double *s_old, double *delta,
                                  double *work, cudaStream_t st);
cudaError_t launch_bond_energy(int d, const double *rho_raw, const double *h, double *out, cudaStream_t st);
cudaError_t launch_open_layers(int d, int D, const double *A, double *b, cudaStream_t st);
cudaError_t launch_check_finite(long long count, const double *x, int *flag, cudaStream_t st);
size_t spectrum_work_doubles(int chi);

int device_sm_count();
// Optional persistent autotuning decisions (CTM_AUTOTUNE_CACHE=<file>, see tune_cache.cu).
bool tune_cache_lookup(const char *tag, const int *key, int nkey, int *val, int nval);
void tune_cache_store(const char *tag, const int *key, int nkey, const int *val, int nval);
// Host-side count of kernel launches the library has enqueued (graph replays excluded).
extern unsigned long long g_ctm_launches;
#define CTM_COUNT_LAUNCH(nl) (g_ctm_launches += (unsigned long long)(nl))
cudaError_t qr_prepare();
cudaError_t spectrum_prepare();
