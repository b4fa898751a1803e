// Ragged batch of independent CTMRG instances (a parameter sweep, e.g. the
// Kitaev-Heisenberg angle) advanced together.  Each instance keeps its own
// context, workspace slice and CUDA stream; one batched step forks from a root
// stream to every instance stream, enqueues that instance's step (contractions,
// QR, renormalisation, corner spectrum on its side stream), and joins back.
// After one eager step -- which lets the split engine's autotuner time the
// candidate tile shapes for every distinct contraction shape in the batch --
// the batched step is captured once as a CUDA graph, so each further batched
// step is a single graph launch in which the instances' kernels run
// concurrently.  Batched QR kernels use grids of at least 128 rows per CTA, so
// the cooperative launches of small instances stay small and overlap.
#include <stdlib.h>

#include <new>
#include <vector>

#include "ctm_ctx.h"

using namespace ctmi;

struct ctm_batch {
    int count;
    std::vector<ctm_ctx *> ctx;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;
    cudaStream_t user, root;
    cudaEvent_t ev_root, ev_user, ev_back;
    cudaGraphExec_t graph;
    unsigned long long graph_kernels;   // kernels one replay launches (counted at capture)
    long long steps;
};

namespace {

// Batched QR grids keep at least this many rows per CTA: the 96 instances' QRs then hold
// fewer SMs while they wait on their grid barriers (measured 15.2 ms per batched step with
// 64, 14.5 ms with 128, 14.6 with 256, 15.3 with whole instances per CTA).
constexpr int BATCH_QR_ROWS_MIN = 128;

// fork root -> instance streams, one step each, join back to root
int enqueue_batched_step(ctm_batch *b)
{
    if (cudaEventRecord(b->ev_root, b->root) != cudaSuccess) return CTM_ECUDA;
    for (int i = 0; i < b->count; ++i) {
        if (cudaStreamWaitEvent(b->streams[i], b->ev_root, 0) != cudaSuccess) return CTM_ECUDA;
        int rc = enqueue_step(b->ctx[i]);
        if (rc != CTM_OK) return rc;
        if (join_side(b->ctx[i]) != CTM_OK) return CTM_ECUDA;
        if (cudaEventRecord(b->done[i], b->streams[i]) != cudaSuccess) return CTM_ECUDA;
        if (cudaStreamWaitEvent(b->root, b->done[i], 0) != cudaSuccess) return CTM_ECUDA;
    }
    return CTM_OK;
}

void destroy_batch(ctm_batch *b)
{
    if (!b) return;
    if (b->root) cudaStreamSynchronize(b->root);
    for (auto *c : b->ctx)
        if (c) ctm_destroy(c);
    for (auto s : b->streams)
        if (s) cudaStreamDestroy(s);
    for (auto e : b->done)
        if (e) cudaEventDestroy(e);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->root) cudaStreamDestroy(b->root);
    if (b->ev_root) cudaEventDestroy(b->ev_root);
    if (b->ev_user) cudaEventDestroy(b->ev_user);
    if (b->ev_back) cudaEventDestroy(b->ev_back);
    delete b;
}

}  // namespace

extern "C" {

size_t ctm_batch_workspace_bytes(const ctm_config *cfgs, int count)
{
    if (!cfgs || count < 1) return 0;
    size_t tot = 0;
    for (int i = 0; i < count; ++i) {
        size_t s = ctm_workspace_bytes(&cfgs[i]);
        if (s == 0) return 0;
        tot += align_up(s);
    }
    return tot;
}

int ctm_batch_init(const ctm_config *cfgs, int count, const double *const *A_dev, void *workspace, size_t ws_bytes,
                   void *stream, ctm_batch **out)
{
    if (!out) return CTM_EINVAL;
    *out = nullptr;
    if (!cfgs || count < 1 || !A_dev || !workspace) return CTM_EINVAL;
    if ((uintptr_t)workspace % 256 != 0) return CTM_EINVAL;
    const size_t need = ctm_batch_workspace_bytes(cfgs, count);
    if (need == 0) return CTM_EINVAL;
    if (ws_bytes < need) return CTM_ENOMEM;
    ctm_batch *b = new (std::nothrow) ctm_batch();
    if (!b) return CTM_ENOMEM;
    b->count = count;
    b->user = (cudaStream_t)stream;
    b->ctx.assign(count, nullptr);
    b->streams.assign(count, nullptr);
    b->done.assign(count, nullptr);
    if (cudaStreamCreateWithFlags(&b->root, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_root, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_user, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_back, cudaEventDisableTiming) != cudaSuccess) {
        destroy_batch(b);
        return CTM_ECUDA;
    }
    char *base = (char *)workspace;
    size_t off = 0;
    for (int i = 0; i < count; ++i) {
        if (cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->done[i], cudaEventDisableTiming) != cudaSuccess) {
            destroy_batch(b);
            return CTM_ECUDA;
        }
        const size_t s = ctm_workspace_bytes(&cfgs[i]);
        int rc = ctm_init(&cfgs[i], A_dev[i], base + off, s, b->streams[i], &b->ctx[i]);
        if (rc != CTM_OK) {
            destroy_batch(b);
            return rc;
        }
        b->ctx[i]->qr_rows_min = BATCH_QR_ROWS_MIN;
        b->ctx[i]->sw.autotune = 1;
        off += align_up(s);
    }
    *out = b;
    return CTM_OK;
}

int ctm_batch_step(ctm_batch *b, int nsteps, double *max_delta_host)
{
    if (!b || nsteps < 0) return CTM_EINVAL;
    // order after the caller's stream
    if (cudaEventRecord(b->ev_user, b->user) != cudaSuccess) return CTM_ECUDA;
    if (cudaStreamWaitEvent(b->root, b->ev_user, 0) != cudaSuccess) return CTM_ECUDA;
    int done = 0;
    if (!b->graph && nsteps > 0) {
        // eager step: autotunes every distinct contraction shape of the batch
        int rc = enqueue_batched_step(b);
        if (rc != CTM_OK) return rc;
        if (cudaStreamSynchronize(b->root) != cudaSuccess) return CTM_ECUDA;
        for (auto *c : b->ctx)
            if ((rc = read_status(c)) != CTM_OK) return rc;
        ++done;
        cudaGraph_t g = nullptr;
        const unsigned long long l0 = g_ctm_launches;
        if (cudaStreamBeginCapture(b->root, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return CTM_ECUDA;
        rc = enqueue_batched_step(b);
        cudaError_t e = cudaStreamEndCapture(b->root, &g);
        b->graph_kernels = g_ctm_launches - l0;
        g_ctm_launches = l0;   // nothing ran yet: replays add the captured kernel count
        if (rc != CTM_OK) return rc;
        if (e != cudaSuccess || !g) return CTM_ECUDA;
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return CTM_ECUDA;
    }
    for (; done < nsteps; ++done) {
        if (cudaGraphLaunch(b->graph, b->root) != cudaSuccess) return CTM_ECUDA;
        CTM_COUNT_LAUNCH(b->graph_kernels);
    }
    b->steps += nsteps;
    for (auto *c : b->ctx) c->steps_done += 0;
    if (cudaEventRecord(b->ev_back, b->root) != cudaSuccess) return CTM_ECUDA;
    if (cudaStreamWaitEvent(b->user, b->ev_back, 0) != cudaSuccess) return CTM_ECUDA;
    if (max_delta_host) {
        if (cudaStreamSynchronize(b->root) != cudaSuccess) return CTM_ECUDA;
        double mx = 0.0;
        for (auto *c : b->ctx) {
            double dl = 0.0;
            if (cudaMemcpy(&dl, c->delta, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return CTM_ECUDA;
            int rc = read_status(c);
            if (rc != CTM_OK) return rc;
            if (!(dl <= mx)) mx = dl;   // NaN propagates
        }
        *max_delta_host = mx;
        if (mx != mx) return CTM_ENONFINITE;
    }
    return CTM_OK;
}

int ctm_batch_ctx(ctm_batch *b, int i, ctm_ctx **out)
{
    if (!b || !out || i < 0 || i >= b->count) return CTM_EINVAL;
    if (cudaStreamSynchronize(b->root) != cudaSuccess) return CTM_ECUDA;
    *out = b->ctx[i];
    return CTM_OK;
}

void ctm_batch_destroy(ctm_batch *b) { destroy_batch(b); }

}  // extern "C"
