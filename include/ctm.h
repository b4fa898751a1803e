/*
 * ctm.h -- C ABI of libctm, a GB300 (sm_103a) implementation of one QR-based,
 * C3v-symmetric CTMRG renormalisation step for a honeycomb-lattice iPEPS and of
 * the nearest-neighbour bond energies evaluated from its environment
 * (Yang & Corboz, "Efficient iPEPS Simulation on the Honeycomb Lattice via
 * QR-based CTMRG", arXiv 2509.05090).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - All tensors are row-major double (FP64) arrays.  "_dev" pointers are CUDA
 *    device pointers on the current device; "_host" pointers are host memory.
 *  - d = physical dimension, D = virtual bond dimension, D2 = D*D (double-layer
 *    bond), chi = environment bond dimension, n = chi*D2.
 *  - A[s][i][j][k] (d x D x D x D) is the site tensor of the uniform ansatz
 *    (Sec. II.A, Fig. 1a).  The three virtual legs are the three bonds of a
 *    honeycomb site.
 *  - C[g][h] (chi x chi) is the corner of one 60-degree sector and
 *    T[a][u][g] (chi x D2 x chi) its edge: a = outer side (the bonds crossing
 *    the sector boundary), u = the end leg toward the apex, g = the side facing
 *    the corner (Sec. II.B, Fig. 3a,b).
 *  - Q[r][j] (n x chi) is the isometric projector of the last step
 *    (Fig. 3d); its row index r = a*D2 + y fuses the chi index (slow) with a
 *    double-layer leg.
 *  - The caller owns all device memory: it allocates one workspace of
 *    ctm_workspace_bytes() bytes (for example a uint8 torch tensor) and passes
 *    it to ctm_init.  No call allocates device memory after ctm_init.
 *  - Work is enqueued on the stream given to ctm_init (a cudaStream_t passed
 *    as void*; NULL = legacy default stream).  Calls that return "_host"
 *    results synchronise that stream; the others are asynchronous unless stated.
 *  - No C++ exception crosses this interface.  Every call returns a status; a
 *    non-OK status leaves the context valid (it can be destroyed or
 *    re-initialised) but its environment undefined.  A context is not
 *    thread-safe.
 */
#ifndef CTM_H
#define CTM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ctm_ctx ctm_ctx;

typedef enum {
    CTM_OK = 0,
    CTM_EINVAL = 1,          /* bad argument (null pointer, size out of range) */
    CTM_ENOMEM = 2,          /* workspace too small */
    CTM_ECUDA = 3,           /* a CUDA runtime call failed */
    CTM_ENOTCONVERGED = 4,   /* max_steps reached with delta >= tol (outputs still filled) */
    CTM_ENONFINITE = 5,      /* NaN or Inf in the environment or the input tensor */
    CTM_ETIMEOUT = 6,        /* a bounded device-side wait gave up */
    CTM_EUNSUPPORTED = 7     /* shape or mode not supported by this build */
} ctm_status;

typedef enum {
    CTM_FP64 = 0,            /* every contraction in FP64 */
    CTM_SPLIT_BF16 = 1,      /* contractions as split-BF16 tcgen05 products (FP32 accumulate,
                                FP64 recombination); QR, normalisation and the
                                convergence test stay FP64 */
    CTM_SPLIT_TF32 = 2,      /* contractions as A_hi B_hi + A_hi B_lo + A_lo B_hi of TF32 hi/lo
                                slices on tcgen05 (kind::tf32), FP32 accumulation: about FP32
                                accuracy (n_split ignored); QR etc. FP64 */
    CTM_FP32_TF32 = 3        /* contractions as one TF32 product A_hi B_hi (FP32 inputs rounded
                                to TF32), FP32 accumulation; QR etc. FP64 */
} ctm_precision;

typedef struct {
    int d, D, chi;           /* physical, virtual and environment bond dimensions */
    int precision;           /* ctm_precision */
    int n_split;             /* BF16 slices per operand in CTM_SPLIT_BF16 (2..5); ignored in FP64 */
    double tol;              /* convergence threshold on delta (Sec. II.B: "desired precision") */
    int max_steps;           /* step limit of ctm_converge when its argument is <= 0 */
    int symmetrize;          /* 1: project A onto the C3v A1 subspace and normalise (App. A) */
    int corner_mode;         /* 0: C' = sym(Q^T M Q)/|.| (Fig. 3a); 1: C' = sym(R S)/|.| from the QR
                                factor R of the reduced corner Y = M Q_prev S (S = diag(sgn C_ii)),
                                which equals Q^T M Q_prev and so Q^T M Q at a fixed point: skips the
                                two corner contractions (a cheap variant, Sec. II.B, Fig. 3d) */
    int deterministic;       /* 1: the QR's cross-CTA sums (Gram rows, V^T V) are written per CTA and
                                added in CTA order instead of with FP64 atomics, so with FP64 or
                                split-BF16 contractions a replayed step gives the same bits every
                                time (the split-K partials of the TF32 modes still meet through
                                FP64 atomics); costs workspace for per-CTA partial sums and about
                                14 % of the QR's time (5 % of a step at D = 6, chi = 72) */
} ctm_config;

/* Bytes of device workspace ctm_init needs for this configuration (0 on a bad
 * config: d <= 3, D <= 12, chi <= 512, n = chi D^2 <= 20000, n_split 2..5 for
 * CTM_SPLIT_BF16; ctm_init also returns CTM_EUNSUPPORTED when the QR's per-CTA
 * scratch would not fit shared memory on the device).  Where one SM's share of the
 * QR's rows does not fit shared memory, the row blocks go to a slab of about
 * n (chi + 1) doubles in this workspace; for chi > 224 the corner spectrum keeps
 * C's lower triangle in it too.  Dominated by the n x n FP64 intermediates
 * (enlarged corner and edge-chain buffers). */
size_t ctm_workspace_bytes(const ctm_config *cfg);

/* Sec. II.A-B: set up one instance.  A_dev: raw site tensor [s][i][j][k]
 * (device).  With cfg->symmetrize the tensor is averaged over the six leg
 * permutations (the C3v group for the A1 irrep, U_g = I; App. A) and
 * normalised to unit Frobenius norm; then the double layer
 * a[(ii')][(jj')][(kk')] = sum_s A[s,i,j,k] A[s,i',j',k'] is formed (Fig. 1b),
 * and the environment starts from C = I, T[a][u][b] = delta_ab t_u with
 * t_u = sum_{v,w} a[u][(vv)][(ww)], and Q = the first chi columns of I_n.
 * The workspace must stay valid until ctm_destroy.  On success *out owns a
 * host-side context. */
int ctm_init(const ctm_config *cfg, const double *A_dev, void *workspace, size_t ws_bytes,
             void *stream, ctm_ctx **out);

/* Autotuning (no counterpart in the paper).  The first eager call of each
 * contraction shape in split mode times its candidate tile plans, and the first
 * QR of each shape its grid size; the choices are kept for the process.  With
 * the environment variable CTM_AUTOTUNE_CACHE=<file> they are also read from and
 * appended to that text file, so another process runs the same plans.
 * CTM_QR_SLAB=1 in the environment when ctm_init (and ctm_workspace_bytes) run
 * keeps the QR's row blocks in the global slab for every shape, the layout taken
 * where one SM's share of the rows does not fit shared memory: the same
 * factorisation, a check of that path at small sizes. */

/* Sec. II.B, Fig. 3: run nsteps CTMRG steps.  One step builds the enlarged
 * corner M from (C, T, a), the reduced corner Y = M Q diag(sgn C_ii),
 * Householder QR Y = Q R with diag(R) >= 0, C' = sym(Q^T M Q)/|.|,
 * T' = Q^T (T a a) Q/|.|, and delta = |s(C') - s(C)|_2 of the unit-norm
 * descending singular values.  delta_host (may be NULL) receives the last
 * delta and makes the call synchronous.  Returns CTM_ENONFINITE if the new
 * environment holds NaN/Inf (checked only when delta_host is given).
 * Once the context has run a step, a call replays its nsteps steps as one
 * CUDA graph: a one-step graph for nsteps = 1 (captured on the first such call
 * and kept), and one for the last nsteps >= 2 requested (re-captured when that
 * count changes); the work is the same. */
int ctm_step(ctm_ctx *ctx, int nsteps, double *delta_host);

/* Sec. II.B: repeat steps until delta < tol (tol <= 0: cfg->tol) or max_steps
 * (<= 0: cfg->max_steps).  A fresh context's first step runs eagerly; then
 * chunks of check_every (>= 1) steps are replayed from two captured CUDA graphs
 * that copy every step's delta into pinned host memory.  Each chunk's last
 * corner spectrum runs at the head of the next chunk (beside its steps), and
 * while the newest delta is above 100 tol a second chunk is queued behind the
 * one the host is reading; so the host learns a step's delta one chunk late,
 * and up to one chunk (two far from tol) more steps run after the first chunk
 * whose newest delta is below tol.  The run ends with the last step's own
 * spectrum: *delta_out is the delta of the last executed step, *steps_out the
 * number of steps this call ran (at most max_steps; fewer than check_every
 * left run one at a time).  Synchronous.  The ring of deltas is pinned host
 * memory the context allocates on first use (2 x check_every doubles plus two
 * flags; cudaHostAlloc) and frees in ctm_destroy; no device memory is allocated.
 * Returns CTM_ENOTCONVERGED (outputs filled) if the limit was hit with
 * delta >= tol. */
int ctm_converge(ctm_ctx *ctx, int max_steps, double tol, int check_every,
                 int *steps_out, double *delta_out);

/* Eq. (1), Fig. 5b: nearest-neighbour bond energies from the current
 * environment.  With Q from one more QR step and Ch = sym(Q^T M Q)/|.|, the
 * reduced density matrix of the apex bond is
 * rho = tr(Ch^5 Q^T M_oo Q) / tr(Ch^6), where M_oo opens the physical legs of
 * the apex dimer.  h_dev: 3 bond operators (x, y, z) of size d^2 x d^2,
 * h[a][(s t)][(s' t')] = <s t| h_a |s' t'> (device).  e_bond_host[a] =
 * tr(rho h_a); e_site_host = (1/2) sum_a e_bond[a] (Eq. 4 Hamiltonian per
 * site).  rho_host (may be NULL) receives rho (d^2 x d^2).  Synchronous;
 * does not change the environment. */
int ctm_energy(ctm_ctx *ctx, const double *h_dev, double *e_bond_host, double *e_site_host,
               double *rho_host);

/* Sec. II.D: energy gradient by a hand-written adjoint.  From the current
 * environment, run `warmup` steps (treated as constants), then k_tracked steps
 * whose inputs are checkpointed, both in the context's precision (on a
 * CTM_SPLIT_BF16 context: split-BF16 contractions with the FP64 QR), then the
 * energy of ctm_energy.  The adjoint recomputes each tracked step from its
 * checkpoint in FP64 and back-propagates through every contraction, the Householder
 * QR (Y-bar = (Q-bar + Q copyltu(-Q-bar^T Q)) R^{-T}, the triangular solve
 * regularised as R_ii / (R_ii^2 + (1e-13 R_00)^2)), the corner and edge
 * normalisations, the double and open layers, and the C3v projection and
 * normalisation of ctm_init.  The environment entering the tracked steps is
 * held fixed (its dependence on A is not differentiated); the warm-start sign
 * diag(sgn C_ii) is piecewise constant.  h_dev as in ctm_energy.  dA_dev
 * (device, layout of A) receives dE_site/dA for the raw tensor passed to
 * ctm_init; energy_host (may be NULL) the energy.  gws: device workspace of
 * ctm_grad_workspace_bytes(ctx, k_tracked) bytes (256-byte aligned).  On
 * return the context holds the environment after the tracked steps.
 * Synchronous. */
size_t ctm_grad_workspace_bytes(const ctm_ctx *ctx, int k_tracked);
int ctm_grad(ctm_ctx *ctx, int warmup, int k_tracked, const double *h_dev, void *gws, size_t gws_bytes,
             double *energy_host, double *dA_dev);

/* Sec. II.C, Fig. 4a, Eq. 3: leading eigenvalues of the transfer matrix of the
 * current environment.  With each sector a quadrant of radial dimers
 * d[u,w,x,y] = sum_z a[u,w,z] a[z,x,y], one column of the plane (an edge, a
 * dimer, the opposite edge) is
 *   TM[(a,y,b),(g,w,h)] = sum_{u,x} T[a,u,g] d[u,w,x,y] T[b,x,h],
 * (chi D2 chi square), which advances one Bravais vector along the edge.  It is
 * applied matrix-free through the context's contraction engine (FP64 or
 * split-BF16); nev + 5 vectors (at most 12) are iterated and orthonormalised in
 * FP64, and the eigenvalues of their Rayleigh quotient are found on the device
 * every 5 iterations until the nev leading magnitudes, normalised by the largest,
 * change by less than tol (absolute; <= 0: 1e-12) or max_iter iterations ran
 * (CTM_ENOTCONVERGED, outputs filled).  lambda_host[0..nev) receives |lambda_i| / |lambda_0| (descending),
 * xi_host (may be NULL) the correlation length -1 / ln lambda_1 in Bravais
 * vectors, gap_host (may be NULL) ln(lambda_1 / lambda_2) of the finite
 * correlation length extrapolation (nev >= 3), iters_out (may be NULL) the
 * iterations used.  2 <= nev <= 10.  tws: device workspace of
 * ctm_transfer_workspace_bytes bytes (256-byte aligned).  Overwrites the
 * step's scratch intermediates (not C, T, Q or M).  Synchronous. */
size_t ctm_transfer_workspace_bytes(const ctm_ctx *ctx, int nev);
int ctm_transfer_spectrum(ctm_ctx *ctx, int nev, int max_iter, double tol, void *tws, size_t tws_bytes,
                          double *lambda_host, double *xi_host, double *gap_host, int *iters_out);

/* Replace the site tensor of a context (Sec. II.D: an optimiser's next trial
 * tensor) without reallocating: A_dev (raw, as for ctm_init) is projected and
 * normalised under the context's symmetrize setting and its double layer formed;
 * the environment is kept as the warm start of the next steps (reset_env = 0) or
 * reset to the initial environment of ctm_init (reset_env != 0).  Captured step
 * graphs are dropped and captured again on the next call.  CTM_ENONFINITE if the
 * tensor holds NaN/Inf.  Synchronous. */
int ctm_set_site(ctm_ctx *ctx, const double *A_dev, int reset_env);

/* Copy the current environment out / in (device pointers; parity checks and
 * resume).  C: chi x chi, T: chi x D2 x chi, Q: n x chi. */
int ctm_get_env(const ctm_ctx *ctx, double *C_dev, double *T_dev, double *Q_dev);
int ctm_set_env(ctm_ctx *ctx, const double *C_dev, const double *T_dev, const double *Q_dev);

/* Intermediates of the most recent step (device copies; parity checks):
 * which = 0: enlarged corner M (n x n), 1: reduced corner Y (n x chi),
 * 2: R (chi x chi), 3: the projector Q used (n x chi), 4: corner spectrum s
 * (chi, descending, unit norm), 5: the prepared site tensor A (d x D^3),
 * 6: the double layer a (D2^3).  Returns CTM_EINVAL for an unknown id and
 * CTM_EUNSUPPORTED for an intermediate the current precision does not keep. */
int ctm_get_intermediate(const ctm_ctx *ctx, int which, double *dst_dev, size_t count);

/* One step (as ctm_step) with CUDA events recorded on the context's stream
 * between its phases; synchronous.  phase_ms (nphase >= 7) receives the
 * milliseconds of: [0] enlarged corner, [1] warm start + reduced corner
 * Y = M Qs, [2] Householder QR, [3] corner renormalisation, [4] edge
 * renormalisation, [5] wait for the previous step's corner spectrum,
 * [6] environment hand-over, and (nphase >= 8) [7] this step's corner
 * spectrum and delta, which run on a second stream and overlap the next step
 * (here they are waited for before returning), and (nphase >= 9) [8] the
 * summed time of the contraction-engine kernels alone (events around each
 * launch: the FP64 GEMM with its split-K reduction, or the tcgen05 kernel
 * without its operand pre-pass), and (nphase >= 10) [9] the summed time of the
 * split engine's operand pre-pass (exponents and digit packing; 0 in FP64). */
int ctm_step_profiled(ctm_ctx *ctx, double *phase_ms, int nphase);

/* Measured FP64 peak of the device (no counterpart in the paper; the roofline
 * denominator of the FP64 contractions): a grid of 4 CTAs per SM, each thread
 * running 16 independent chains of dependent DFMAs, timed with CUDA events after a
 * warm-up launch.  *tflops_host receives 2 x DFMAs / second / 1e12.  Synchronous
 * on `stream`. */
int ctm_probe_fp64_peak(void *stream, double *tflops_host);

/* Failure-detection test hook (no counterpart in the paper).  With enable != 0
 * the context's next Householder QR runs with a grid barrier that waits for one
 * arrival more than the grid provides and gives up after a short bounded spin
 * (about a millisecond): every CTA raises the context's error flag and returns,
 * and the step reports CTM_ETIMEOUT, exactly as an expired device wait does.
 * Nothing faults or hangs.  The environment is undefined afterwards; destroy the
 * context.  enable = 0 restores normal waits.  Synchronous. */
int ctm_debug_force_timeout(ctm_ctx *ctx, int enable);

/* Number of kernel launches the library has enqueued since it was loaded
 * (host-side count; a replay of a captured graph adds the kernels it holds). */
unsigned long long ctm_kernel_launches(void);

/* The contraction engine on its own (Sec. II.B: every update of Fig. 3 is a
 * chain of such products).  C = A B for row-major FP64 matrices A (M x K),
 * B (K x N), C (M x N), all device pointers.  precision CTM_FP64 runs the FP64
 * GEMM; CTM_SPLIT_BF16 splits every row of A and column of B into n_split
 * (2..5) BF16 digit slices on a per-row / per-column power-of-two grid and
 * sums the slice products of total order < n_split on tcgen05 tensor cores,
 * exactly in FP32 per 256-deep K chunk, recombined in 64-bit integers
 * (relative error ~ n_split 2^(-8 n_split) of the row/column maxima).  The
 * caller supplies ctm_gemm_workspace_bytes() bytes of device workspace
 * (256-byte aligned).  Synchronous.  CTM_ETIMEOUT if a bounded device wait
 * expired. */
size_t ctm_gemm_workspace_bytes(int M, int N, int K, int precision, int n_split);
int ctm_gemm(int M, int N, int K, const double *A_dev, const double *B_dev, double *C_dev, int precision,
             int n_split, void *workspace, size_t ws_bytes, void *stream);

/* Allocation-free ctm_gemm, for callers that cannot allocate device memory
 * (a plugin whose host framework owns every device allocation, a
 * latency-critical loop that cannot afford an allocation or its failure
 * mid-run, a service with a device-memory budget fixed at start-up).  The
 * paper has no counterpart; this is a library convenience.  Same operands,
 * precisions and result as ctm_gemm, but the scratch lives in a file-scope
 * device array of CTM_NOALLOC_SCRATCH_BYTES that every GPU loading the
 * library holds until exit.  A shape whose scratch (ctm_gemm_workspace_bytes)
 * exceeds that size returns CTM_ENOMEM.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress, with that device current)
 * and caches it, so make that first call before any stream capture.  All
 * calls share the array: each call clears what must start at zero, and calls
 * that overlap on the GPU race, so serialise them.  Synchronous. */
#define CTM_NOALLOC_SCRATCH_BYTES (32u << 20)
int ctm_gemm_noalloc(int M, int N, int K, const double *A_dev, const double *B_dev, double *C_dev, int precision,
                     int n_split, void *stream);

/* Ragged batch of independent instances (Sec. III.B's slicing and a
 * parameter sweep run side by side): count configurations (D, chi may
 * differ) with site tensors A_dev[i].  Each instance owns a context, a slice
 * of the caller's workspace (ctm_batch_workspace_bytes) and a stream.
 * ctm_batch_step advances every instance by nsteps steps: the first call runs
 * one step eagerly, timing the split engine's candidate tile shapes for every
 * contraction shape of the batch (autotuner, cached per shape), then captures
 * one batched step -- all instances' kernels, concurrent across their
 * streams -- as a CUDA graph, so each further batched step is one graph
 * launch.  max_delta_host (may be NULL) receives the largest delta and makes
 * the call synchronous.  ctm_batch_ctx exposes instance i's context (after
 * synchronising the batch) for ctm_energy, ctm_get_env and the like; it stays
 * owned by the batch. */
typedef struct ctm_batch ctm_batch;
size_t ctm_batch_workspace_bytes(const ctm_config *cfgs, int count);
int ctm_batch_init(const ctm_config *cfgs, int count, const double *const *A_dev, void *workspace, size_t ws_bytes,
                   void *stream, ctm_batch **out);
int ctm_batch_step(ctm_batch *batch, int nsteps, double *max_delta_host);
int ctm_batch_ctx(ctm_batch *batch, int i, ctm_ctx **ctx);
void ctm_batch_destroy(ctm_batch *batch);

/* ---------------------------------------------------------------------------
 * Complex tensors (App. A, Sec. III.C): the same step for a complex site tensor
 * made symmetric under a complex representation of C3v on the physical leg.
 *
 *  - Complex arrays are interleaved (re, im) pairs of doubles, row-major in the
 *    complex elements (a torch.complex128 tensor's storage), on the device.
 *  - irrep CTM_IRREP_E: the rotation U_C3 = (-1)^(d-1) e^{i 2pi/3}
 *    exp(i 2pi/3 n.S), n = (1,1,1)/sqrt 3, acts with the leg cycle
 *    A[s; i, j, k] -> sum_t U[s,t] A[t; k, i, j]; the reflection through the
 *    plane with spin-space normal m_1 = (1,-1,0)/sqrt 2 acts as the anti-unitary
 *    K-hat C exp(i pi m_1.S) (K-hat: +1, -1, ... on the anti-diagonal; C: complex
 *    conjugation of the whole tensor) with the exchange of the x and y legs; the
 *    other four elements follow by composition.  cfg->symmetrize averages A over
 *    the six and normalises it.  CTM_IRREP_A1: U = I, no conjugation (then the
 *    path reproduces the real one).  d = 2 or 3 for E.
 *  - The double layer a[(ii')][(jj')][(kk')] = sum_s A[s,i,j,k] conj(A[s,i',j',k'])
 *    obeys a[l][u][z] = conj(a[u][l][z]) under each reflection (Fig. 2b), so with
 *    a Hermitian corner and the column edge the conjugate of the row edge the
 *    enlarged corner M[(a,y)][(b,x)] = sum T[a,u,g] C[g,h] conj(T[b,l,h])
 *    a[u,l,z] a[z,x,y] is Hermitian; a step forms Y = M Q diag(sgn Re C_jj),
 *    Y = Q R with diag(R) real and >= 0, C' = sym(Q^H M Q)/|.| (Hermitian part),
 *    T'[i,x,j] = sum conj(Q[(a,y),i]) T[a,u,g] a[u,w,z] a[z,x,y] Q[(g,w),j] /|.|,
 *    and delta from the eigenvalue magnitudes of C'.
 *  - Precisions as for ctm_init (FP64, split BF16, split TF32, one TF32 product):
 *    every real product of a complex contraction runs on the chosen engine.
 *  - Limits: chi <= 256 (beyond 112 the corner spectrum runs on the real 2chi x 2chi
 *    embedding [[Re, -Im], [Im, Re]] of the Hermitian corner), n = chi D^2 <= 12000,
 *    D <= 10.  corner_mode 1 gives the cheap
 *    variant C' = sym(R S)/|.| with S = diag(sgn Re C_jj) (R S = Q^H M Q_prev).
 *  - The caller owns the workspace (ctm_complex_workspace_bytes), as for ctm_init.
 *    Errors as for the real calls. */
typedef struct ctm_complex_ctx ctm_complex_ctx;
enum { CTM_IRREP_A1 = 0, CTM_IRREP_E = 1 };
size_t ctm_complex_workspace_bytes(const ctm_config *cfg, int irrep);

/* App. A, Sec. II.A-B: A_dev = raw complex site tensor [s][i][j][k]
 * (d x D x D x D, interleaved); projection, normalisation, double layer and the
 * environment C = I, T[a][u][b] = delta_ab t_u, Q = [I; 0] as for ctm_init. */
int ctm_complex_init(const ctm_config *cfg, int irrep, const double *A_dev, void *workspace, size_t ws_bytes,
                     void *stream, ctm_complex_ctx **out);

/* Sec. II.B: nsteps steps; delta_host (may be NULL) as for ctm_step.  Synchronous. */
int ctm_complex_step(ctm_complex_ctx *ctx, int nsteps, double *delta_host);

/* Sec. II.B: steps until delta < tol, as for ctm_converge. */
int ctm_complex_converge(ctm_complex_ctx *ctx, int max_steps, double tol, int check_every, int *steps_out,
                         double *delta_out);

/* Eq. 1: bond energies as for ctm_energy, h_dev = 3 complex d^2 x d^2 bond
 * operators (interleaved).  The density matrix rho of the apex bond is formed
 * for the z bond (the apex bond is the z leg of both sites); the x and y bonds
 * are the z bond of the tensor rotated by the C3 element, so
 * e_x = Re tr(rho (W^H h_x W)) with W = U^2 (x) U^2, e_y likewise with
 * W = U (x) U (U = U_C3, or I for A1), e_z = Re tr(rho h_z).  rho_host (may be
 * NULL): the z-bond rho, d^2 x d^2 complex interleaved. */
int ctm_complex_energy(ctm_complex_ctx *ctx, const double *h_dev, double *e_bond_host, double *e_site_host,
                       double *rho_host);

/* C (chi x chi), T (chi x D2 x chi), Q (n x chi), complex interleaved (device).
 * get: any pointer may be NULL; set: the corner's spectrum becomes the
 * reference of the next delta.  Synchronous. */
int ctm_complex_get_env(const ctm_complex_ctx *ctx, double *C_dev, double *T_dev, double *Q_dev);
int ctm_complex_set_env(ctm_complex_ctx *ctx, const double *C_dev, const double *T_dev, const double *Q_dev);

/* Intermediates of the last step, complex interleaved into dst (device,
 * count = doubles available): 0 M (n x n), 1 Y (n x chi), 2 R (chi x chi),
 * 3 Q (n x chi), 4 the corner spectrum s (chi doubles, real), 5 the projected
 * site tensor, 6 the double layer (D2^3), 7 C, 8 T.  Synchronous. */
int ctm_complex_get_intermediate(const ctm_complex_ctx *ctx, int which, double *dst_dev, size_t count);

/* Sec. II.C for complex environments: the leading eigenvalue magnitudes of the column
 * transfer matrix TM[(a,y,b),(g,w,h)] = sum T[a,u,g] aB[u,w,z] aA[z,x,y] conj(T[b,x,h])
 * (the opposite edge is the mirror image of T), normalised by the largest, with
 * xi = -1/ln lambda_1 and ln(lambda_1/lambda_2) as for ctm_transfer_spectrum.  The
 * subspace iteration of the real path runs on the operator's real form (vectors
 * [Re v | Im v]); the spectrum is closed under conjugation, so each magnitude appears
 * twice there and every second one is kept.  nev: 2 or 3.  tws: device workspace of
 * ctm_complex_transfer_workspace_bytes bytes (256-byte aligned).  Overwrites the
 * step's scratch intermediates.  Synchronous. */
size_t ctm_complex_transfer_workspace_bytes(const ctm_complex_ctx *ctx, int nev);
int ctm_complex_transfer_spectrum(ctm_complex_ctx *ctx, int nev, int max_iter, double tol, void *tws,
                                  size_t tws_bytes, double *lambda_host, double *xi_host, double *gap_host,
                                  int *iters_out);

void ctm_complex_destroy(ctm_complex_ctx *ctx);

/* Release the host context (the caller frees the workspace). */
void ctm_destroy(ctm_ctx *ctx);

/* Human-readable name of a status code. */
const char *ctm_status_str(int status);

/* Library build identifier, e.g. "libctm sm_103a fp64+bf16split". */
const char *ctm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CTM_H */
