// graph.cu -- a branch decided on the device inside a captured CUDA graph: a
// conditional (IF) node whose body runs only when a device word is non-zero
// when the replay reaches it.  A Verlet step uses it for its rebuild: the
// displacement test writes the gate word, and a step that needs no rebuild
// skips the rebuild kernels instead of launching them to exit at once.
#include "fpm_common.cuh"

namespace fpm {

__global__ void k_set_condition(cudaGraphConditionalHandle h, const uint32_t *flag)
{
    cudaGraphSetConditional(h, *flag != 0u ? 1u : 0u);
}

static fpm_status cuda_fail(cudaError_t e, const char *what)
{
    return fpm_fail(FPM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace fpm

using namespace fpm;

extern "C" fpm_status fpm_graph_if_begin(const uint32_t *d_flag, fpm_stream stream, fpm_stream body_stream,
                                         int32_t *capturing)
{
    if (!d_flag || !capturing) return fpm_fail(FPM_ERR_INVALID, "fpm_graph_if_begin: null pointer");
    *capturing = 0;
    cudaStream_t s = (cudaStream_t)stream, b = (cudaStream_t)body_stream;
    if (s == b) return fpm_fail(FPM_ERR_INVALID, "fpm_graph_if_begin: the body stream must differ from stream");
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return cuda_fail(e, "fpm_graph_if_begin");
    if (cs != cudaStreamCaptureStatusActive) return FPM_OK;  // not capturing: the caller runs the work gated
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edges = nullptr;
    size_t nd = 0;
    e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edges, &nd);
    if (e != cudaSuccess) return cuda_fail(e, "fpm_graph_if_begin (capture info)");
    cudaGraphConditionalHandle h;
    e = cudaGraphConditionalHandleCreate(&h, g, 0u, 0u);
    if (e != cudaSuccess) return cuda_fail(e, "fpm_graph_if_begin (handle)");
    k_set_condition<<<1, 1, 0, s>>>(h, d_flag);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fpm_graph_if_begin (set kernel)");
    e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edges, &nd);
    if (e != cudaSuccess) return cuda_fail(e, "fpm_graph_if_begin (capture info)");
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeIf;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, deps, edges, nd, &p);
    if (e != cudaSuccess) return cuda_fail(e, "fpm_graph_if_begin (conditional node)");
    e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) return cuda_fail(e, "fpm_graph_if_begin (dependencies)");
    e = cudaStreamBeginCaptureToGraph(b, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return cuda_fail(e, "fpm_graph_if_begin (body capture)");
    *capturing = 1;
    return FPM_OK;
}

extern "C" fpm_status fpm_graph_if_end(fpm_stream body_stream)
{
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture((cudaStream_t)body_stream, &g);
    if (e != cudaSuccess) return cuda_fail(e, "fpm_graph_if_end");
    return FPM_OK;
}
