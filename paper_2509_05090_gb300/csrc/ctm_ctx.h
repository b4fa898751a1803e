// The context behind the C ABI's opaque ctm_ctx, shared by the translation
// units that enqueue work for it (ctm_api.cu: the step and the energy;
// ctm_grad.cu: the adjoint).
#pragma once

#include "ctm_internal.h"

inline size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr int CTM_PROF_EVENTS = 96;

struct ctm_ctx {
    ctm_config cfg;
    int d, D, D2, chi;
    long long n;
    cudaStream_t stream;      // the caller's stream
    cudaStream_t own;         // private stream used for graph capture and replay
    cudaEvent_t ev_in, ev_out;
    cudaStream_t side;        // corner spectrum runs here, overlapped with the edge update
    cudaEvent_t ev_fork, ev_join;
    // split mode: the corner update (M Q, Q^T (M Q), normalisation) runs on lane2
    // while the edge update runs on the step's stream; ev_q = Q is ready,
    // ev_corner = the corner update (and its pack of Q^T) is done
    cudaStream_t lane2;
    cudaEvent_t ev_q, ev_corner;
    // FP64 buffers (device, inside the caller's workspace)
    double *Araw, *A, *a;
    double *C, *Cn, *Cr;
    double *Cspec;            // split mode: the copy of C' the side-stream spectrum reads
    double *T, *Tn;
    double *Q, *Qn, *Qs, *Y, *W, *MQ;
    double *R;
    double *M, *X, *H;
    double *Y1;
    double *s, *s_new, *delta, *spec_work;
    double *splitk;
    size_t splitk_elems;
    int split_T;              // 0: FP64 contractions; 2..5: split-BF16 slices per operand
    int tf32_T;               // 1, 2: TF32 slices per operand (FP32_TF32, SPLIT_TF32); 0 otherwise
    SplitWork sw;
    SplitWork sw_c;           // corner lane: M's pack read from sw; own B pack, exponents, split-K buffer
    SplitWork sw_e;           // edge lane: own A pack and exponents; B pack and split-K buffer of sw
    // the double layer a is a constant B operand of four contractions per step:
    // its packed digit slices are kept (slot 0: a as [(u,l)][z], slot 1: a as [z][(x,y)])
    unsigned char *apk[2];
    int *ape[2];
    size_t apk_cap[2];
    int apk_state[2];
    // split mode: A packs used twice per step (slot 0: T as the A operand of W = T C
    // and H1' = T Q; slot 1: Q^T for C_r = Q^T (M Q) and T' = Q^T H3'), and whether
    // the pack matches the current T / Q
    unsigned char *ack[2];
    int *ace[2];
    size_t ack_cap[2];
    int ack_valid[2];
    double *qr_sbuf, *qr_rowbuf, *qr_wy;
    double *qr_gpart, *qr_spart;   // deterministic mode: per-CTA partial sums (else null)
    double *qr_slab;               // the QR's row blocks where they do not fit shared memory (else null)
    size_t qr_slab_elems;
    bool qr_force_slab;            // CTM_QR_SLAB=1 when the context was created
    int qr_gmax;
    unsigned *qr_bar;
    int *err, *flag;
    double *norm_part, *norm_part2;
    // energy
    double *b, *Y1o, *G2, *P5a, *P5b, *rho_part, *rho_raw, *eout, *h;
    // graph of `graph_steps` steps (captured on the private stream), and how many
    // kernels one replay launches
    cudaGraphExec_t graph;
    int graph_steps;
    int graph_failed;
    unsigned long long graph_kernels;
    // one step, for ctm_step(1) after the first step (a user's step-by-step loop)
    cudaGraphExec_t graph1;
    unsigned long long graph1_kernels;
    int side_pending;
    // pipelined ctm_converge: two graphs of pipe_steps steps that also copy each
    // step's delta, and at the end the error flag, into pinned host memory (ring
    // half 0 and half 1), so the host reads one half while the other graph runs
    cudaGraphExec_t pipe[2];
    int pipe_steps;
    unsigned long long pipe_kernels;
    cudaEvent_t pipe_done[2];
    double *ring_h;           // pinned: 2 x ring_cap deltas
    int *ring_err_h;          // pinned: one error flag per half
    int ring_cap;
    double *delta_dst;        // while capturing those graphs: where this step's delta goes
    // while capturing them, also: spec_head = this step first computes the spectrum
    // of the corner it starts from (the previous step's, whose own spectrum was
    // deferred), its delta to delta_head; spec_skip = this step defers its own
    int spec_head, spec_skip;
    double *delta_head;
    // kernel timing (ctm_step_profiled): events around each contraction launch
    int prof_on, prof_n;
    int qr_rows_min;          // 1 for a lone instance; larger inside a batch
    int force_timeout;        // ctm_debug_force_timeout: the QR grid barrier waits for an arrival that never comes
    cudaEvent_t prof_ev[CTM_PROF_EVENTS];   // three per contraction: kernel start, kernel end, pre-pass start
    int steps_done;
};

namespace ctmi {
// QR scratch views of the context's workspace
inline QrScratch qr_scratch(ctm_ctx *c)
{
    const long long n = c->n, k = c->chi;
    QrScratch q;
    q.sbuf = c->qr_sbuf;
    q.rowbuf = c->qr_rowbuf;
    q.bar = c->qr_bar;
    q.err = c->err;
    q.rows_min = c->qr_rows_min;
    q.V = c->qr_wy;
    q.S = q.V + k * k;
    q.W = q.S + k * k;
    q.ta = q.W + k * k;
    q.sk = nullptr;
    q.sk_elems = 0;
    q.bar_extra = c->force_timeout ? 1u : 0u;
    q.spin_limit = c->force_timeout ? 20000 : 0;
    q.gpart = c->qr_gpart;
    q.spart = c->qr_spart;
    q.gmax = c->qr_gmax;
    q.yslab = c->qr_slab;
    q.yslab_elems = c->qr_slab_elems;
    q.force_slab = c->qr_force_slab;
    return q;
}
enum {
    GEMM_PLAIN = 0,
    GEMM_REUSE_A = 1,
    GEMM_B_IS_A_LZ = 2,
    GEMM_B_IS_A_ZX = 3,
    GEMM_A_FILL_T = 4,
    GEMM_A_USE_T = 5,
    GEMM_A_FILL_Q = 6,
    GEMM_A_USE_Q = 7
};
// lane 0: the step's stream and work buffers; 1: the corner lane; 2: the edge lane
cudaError_t run_gemm(ctm_ctx *c, const GemmF64 &g, int hint = GEMM_PLAIN, int lane = 0);
int enqueue_enlarged_corner(ctm_ctx *c);
int enqueue_step(ctm_ctx *c);
int join_side(ctm_ctx *c);
int read_status(ctm_ctx *c);
void drop_graphs(ctm_ctx *c);   // forget captured graphs (launch arguments or packed state changed)
cudaError_t rho_reduce(ctm_ctx *c);   // raw[pB][pA] = sum Y1o G2 (energy contraction)
}  // namespace ctmi
