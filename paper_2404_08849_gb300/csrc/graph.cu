// graph.cu - whole-step CUDA graphs: the calls of one model step (dycore
// steps, tracer steps, sums, or any other stream-ordered work on the same
// stream) recorded once by stream capture and replayed as a single graph
// launch, so a step costs one launch on the host instead of one per kernel.
// No counterpart in the paper (a GPU execution device).
#include <new>

#include "common.cuh"

struct grist_graph_s {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" int grist_capture_begin(void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (!st) return GRIST_EINVAL;   // the legacy default stream cannot be captured
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return GRIST_ECUDA;
    if (cs != cudaStreamCaptureStatusNone) return GRIST_EINVAL;
    return cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess ? GRIST_OK : GRIST_ECUDA;
}

extern "C" int grist_capture_end(void *stream, grist_graph *out) {
    if (!stream || !out) return GRIST_EINVAL;
    *out = nullptr;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture((cudaStream_t)stream, &g);
    if (e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return GRIST_ECUDA;
    }
    cudaGraphExec_t x = nullptr;
    if (cudaGraphInstantiate(&x, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        cudaGetLastError();
        return GRIST_ECUDA;
    }
    grist_graph_s *h = new (std::nothrow) grist_graph_s();
    if (!h) {
        cudaGraphExecDestroy(x);
        cudaGraphDestroy(g);
        return GRIST_ENOMEM;
    }
    h->graph = g;
    h->exec = x;
    *out = h;
    return GRIST_OK;
}

extern "C" int grist_graph_launch(grist_graph g, void *stream) {
    if (!g) return GRIST_EINVAL;
    return cudaGraphLaunch(g->exec, (cudaStream_t)stream) == cudaSuccess ? GRIST_OK : GRIST_ECUDA;
}

extern "C" int grist_graph_destroy(grist_graph g) {
    if (!g) return GRIST_OK;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return GRIST_OK;
}
