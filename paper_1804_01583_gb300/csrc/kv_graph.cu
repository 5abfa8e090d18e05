// kv_graph.cu -- many small queries packed under one captured CUDA graph.
//
// A small verification query (a 20 x 20 grid, a CSR system of a few thousand
// rows) is a few dozen tiny kernels whose cost is launch latency, not work.
// kv_graph_create records the whole path of n problems into one CUDA graph by
// stream capture: the context stream forks into up to KV_GRAPH_BRANCHES
// branches, problem k is enqueued on branch k % branches, and the branches
// join at the end, so independent queries run concurrently inside the graph.
// kv_graph_launch replays it with one launch; each problem's completion event
// is recorded after the graph so kv_fetch works as after kv_enqueue.
#include <vector>

#include "kv_internal.h"

struct kv_graph {
    kv_ctx* ctx = nullptr;
    std::vector<kv_prob*> probs;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace kv {
int prepare_for_capture(int device) {
    int rc = expm_prepare(device);
    if (!rc) rc = fused_prepare();
    return rc ? rc : fused64_prepare();
}
}  // namespace kv

extern "C" {

int kv_graph_create(kv_ctx* ctx, kv_prob* const* probs, int32_t n, kv_graph** out) {
    using namespace kv;
    if (!ctx || !probs || n < 1 || !out) {
        set_error("kv_graph_create: bad arguments");
        return KV_EINVAL;
    }
    *out = nullptr;
    for (int k = 0; k < n; ++k) {
        if (!probs[k] || probs[k]->ctx != ctx) {
            set_error("kv_graph_create: problem %d is NULL or belongs to another context", k);
            return KV_EINVAL;
        }
    }
    if (ctx->profiling) {
        set_error("kv_graph_create: disable per-kernel profiling before capturing");
        return KV_EINVAL;
    }
    KV_WITH_DEVICE(ctx->device);
    int rc = prepare_for_capture(ctx->device);
    if (rc) return rc;
    KV_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
    const int nb = n < KV_GRAPH_BRANCHES ? n : KV_GRAPH_BRANCHES;
    std::vector<cudaStream_t> br(nb);
    std::vector<cudaEvent_t> join(nb);
    cudaEvent_t fork = nullptr;
    for (int b = 0; b < nb; ++b) {
        KV_CHECK_CUDA(cudaStreamCreateWithFlags(&br[b], cudaStreamNonBlocking));
        KV_CHECK_CUDA(cudaEventCreateWithFlags(&join[b], cudaEventDisableTiming));
    }
    KV_CHECK_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    cudaStream_t origin = ctx->stream;
    kv_graph* g = new kv_graph();
    g->ctx = ctx;
    g->probs.assign(probs, probs + n);
    // enqueueing under capture marks a problem as run; until the graph is
    // launched its results are those of its previous runs, if any
    std::vector<bool> ran_before(n);
    for (int k = 0; k < n; ++k) ran_before[k] = probs[k]->ran;
    ctx->capturing = true;  // plain launches inside the graph
    cudaError_t e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaEventRecord(fork, origin);
    for (int b = 0; b < nb && e == cudaSuccess; ++b) e = cudaStreamWaitEvent(br[b], fork, 0);
    for (int k = 0; k < n && e == cudaSuccess && rc == KV_OK; ++k) {
        ctx->stream = br[k % nb];
        rc = kv_enqueue(probs[k]);
    }
    ctx->stream = origin;
    for (int k = 0; k < n; ++k) probs[k]->ran = ran_before[k];
    for (int b = 0; b < nb && e == cudaSuccess; ++b) {
        e = cudaEventRecord(join[b], br[b]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, join[b], 0);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(origin, &graph);
    ctx->capturing = false;
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess && rc == KV_OK) e = cudaGraphInstantiate(&g->exec, graph, 0);
    g->graph = graph;
    for (int b = 0; b < nb; ++b) {
        cudaStreamDestroy(br[b]);
        cudaEventDestroy(join[b]);
    }
    cudaEventDestroy(fork);
    if (e != cudaSuccess || rc != KV_OK) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        if (rc != KV_OK) return rc;
        set_error("kv_graph_create: capture failed: %s", cudaGetErrorString(e));
        return KV_ECUDA;
    }
    *out = g;
    return KV_OK;
}

int kv_graph_launch(kv_graph* g) {
    using namespace kv;
    if (!g) {
        set_error("kv_graph_launch: NULL graph");
        return KV_EINVAL;
    }
    KV_WITH_DEVICE(g->ctx->device);
    KV_CHECK_CUDA(cudaGraphLaunch(g->exec, g->ctx->stream));
    g->ctx->launches += 1;
    for (kv_prob* p : g->probs) {
        KV_CHECK_CUDA(cudaEventRecord(p->done_ev, g->ctx->stream));
        p->ran = true;
    }
    return KV_OK;
}

int kv_graph_destroy(kv_graph* g) {
    if (!g) return KV_OK;
    ::kv::DeviceGuard kv_device_guard_(g->ctx->device);
    cudaStreamSynchronize(g->ctx->stream);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return KV_OK;
}

}  // extern "C"
